// Batched ICCG: many systems of uneven size, several right-hand sides each,
// in one cooperative launch (the PCG loop lives inside the kernel; the launch
// is replayed as a CUDA graph).  Each system is the block-multicolor ICCG of
// the single-system path (Alg. 1 for the substitutions, standard PCG around
// it) applied to all of its right-hand sides at once.
//
// Layout.  Per system, every n-vector is stored row-major over the
// right-hand sides: v[i * kp + j] (kp = nrhs rounded up to a power of two
// <= 32), so the values of one row for all right-hand sides are one
// contiguous line.  A "chain" of kp lanes (lane j = right-hand side j) walks
// rows; a matrix or factor entry is loaded once per chain and broadcast to
// its lanes, and every vector access of the chain is one coalesced line.
//
// Schedule.  The grid is split into per-system CTA ranges (proportional to
// the system's rows, at least one CTA each); a system's CTAs synchronise
// only among themselves (a bounded-wait barrier per system), so systems
// progress independently.  Per iteration and system: p update | SpMV and
// <p,q> | forward colors (x / r update fused, the last color's backward
// sweep fused) | backward colors | reduction, with a barrier after each
// phase (2 n_c + 2).  A chain owns a whole block at a time: its rows are
// resolved in order (Alg. 1), the block's earlier (later) results in the
// chain's shared-memory scratch.  Reductions are per right-hand side, per
// CTA, summed in a fixed order by every CTA of the system after a barrier.
// A right-hand side that converged (or met a non-finite value) is frozen.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "iccg_internal.h"

namespace iccg {
namespace {

constexpr int kBatchMaxBlock = 64;   // rows of a block (a chain's scratch in shared memory)
constexpr long long kBatchSpinLimit = 1ll << 27;

struct BatchSys {
  int32_t n, nc, cta0, cta1;
  const int32_t *arp, *acol;
  const double *aval;
  const int32_t *lrp, *lcol, *urp, *ucol;
  const double *lv64, *uv64, *dv64;
  const float *lv32, *uv32, *dv32;
  const int32_t *cblk;     // [nc + 1] first block of each color
  const int32_t *bptr;     // [nb + 1] first row of each block
  const int32_t *perm;     // row -> original row
  double *x, *r, *p, *q;   // [n][kp]
  void *y, *z;             // [n][kp], precision of the preconditioner
  const double *bin;       // [k][n], original numbering (staging)
  double *xio;             // [k][n], original numbering: x0 in, x out (staging)
  double *part;            // [CTAs of the system][4][kp] partial sums
  double *hist;            // [maxit + 1][kp]
  int32_t *iters;          // [kp]
  int32_t *status;         // [kp] per right-hand side
  GridBar *bar;
  unsigned long long wait_ns;   // bounded barrier wait (ns)
};

template <typename PT> __device__ __forceinline__ const PT *b_lv(const BatchSys &S);
template <> __device__ __forceinline__ const double *b_lv<double>(const BatchSys &S) { return S.lv64; }
template <> __device__ __forceinline__ const float *b_lv<float>(const BatchSys &S) { return S.lv32; }
template <typename PT> __device__ __forceinline__ const PT *b_uv(const BatchSys &S);
template <> __device__ __forceinline__ const double *b_uv<double>(const BatchSys &S) { return S.uv64; }
template <> __device__ __forceinline__ const float *b_uv<float>(const BatchSys &S) { return S.uv32; }
template <typename PT> __device__ __forceinline__ const PT *b_dv(const BatchSys &S);
template <> __device__ __forceinline__ const double *b_dv<double>(const BatchSys &S) { return S.dv64; }
template <> __device__ __forceinline__ const float *b_dv<float>(const BatchSys &S) { return S.dv32; }

__device__ __forceinline__ unsigned b_ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long b_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Barrier over the nct CTAs of one system, with a bounded wait (false for
// the whole CTA when this or another CTA of the system gave up).
__device__ __forceinline__ bool sys_sync(GridBar *bar, unsigned nct, unsigned &gen, int *flag,
                                         unsigned long long wait_ns) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    const unsigned arrived = atomicAdd(&bar->count, 1u);
    if (arrived == nct - 1) {
      atomicExch(&bar->count, 0u);
      __threadfence();
      atomicExch(&bar->gen, gen + 1);
    } else {
      const unsigned long long t0 = b_ns();
      // the clock is read on every poll (a short limit must take effect at
      // the first poll); the error word of other CTAs every 64 polls
      for (long long k = 1; b_ld_acquire(&bar->gen) == gen; ++k) {
        if (b_ns() - t0 > wait_ns || k > kBatchSpinLimit ||
            ((k & 63) == 0 && b_ld_acquire(&bar->err) != 0u)) {
          atomicExch(&bar->err, 1u);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    gen = gen + 1;
    *flag = ok && b_ld_acquire(&bar->err) == 0u;
  }
  __syncthreads();
  return *flag != 0;
}

// Per-right-hand-side CTA sum: every lane holds v for its (chain, j); the
// sums over the CTA's chains (fixed order) go to part[lc][slot][j].
__device__ __forceinline__ void cta_rhs_sum(double v, double *red, int kp, int nchain, double *part_slot) {
  const int j = threadIdx.x % kp, ch = threadIdx.x / kp;
  __syncthreads();
  red[ch * kp + j] = v;
  __syncthreads();
  if (threadIdx.x < kp) {
    double s = 0.0;
    for (int c = 0; c < nchain; ++c) s += red[c * kp + threadIdx.x];
    part_slot[threadIdx.x] = s;
  }
}

// Sum over the system's CTAs of part[.][slot][j] (fixed order) into
// out[j], j < kp; every CTA computes the same values.
__device__ __forceinline__ void sys_rhs_sum(const double *part, int nct, int kp, int slot, double *out) {
  __syncthreads();
  if (threadIdx.x < kp) {
    double s = 0.0;
    for (int c = 0; c < nct; ++c) s += __ldcg(part + (size_t(c) * 4 + slot) * kp + threadIdx.x);
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// One substitution pass of a system (UPDATE: with the x / r update in front
// of the forward sweep).  A chain owns a block at a time; w is the chain's
// scratch (block rows x kp).
template <typename PT, bool UPDATE>
__device__ __forceinline__ bool batch_precond(const BatchSys &S, PT *w, int kp, int j, int gc, int total,
                                              double alpha, bool act, double &rr, double &rz, unsigned nct,
                                              unsigned &gen, int *flag) {
  const PT *lv = b_lv<PT>(S), *uv = b_uv<PT>(S), *dv = b_dv<PT>(S);
  PT *y = reinterpret_cast<PT *>(S.y);
  PT *z = reinterpret_cast<PT *>(S.z);
  const int nc = S.nc;
  for (int c = 0; c < nc; ++c) {
    const bool last = c == nc - 1;
    const int b1 = __ldg(S.cblk + c + 1);
    for (int blk = __ldg(S.cblk + c) + gc; blk < b1; blk += total) {
      const int r0 = __ldg(S.bptr + blk), r1 = __ldg(S.bptr + blk + 1);
      for (int i = r0; i < r1; ++i) {
        double ri = __ldcg(S.r + size_t(i) * kp + j);
        if (UPDATE && act) {
          ri -= alpha * __ldcg(S.q + size_t(i) * kp + j);
          S.r[size_t(i) * kp + j] = ri;
          S.x[size_t(i) * kp + j] = __ldcg(S.x + size_t(i) * kp + j) + alpha * __ldcg(S.p + size_t(i) * kp + j);
          rr += ri * ri;
        }
        PT acc = PT(ri);
        const int e1 = __ldg(S.lrp + i + 1);
        for (int e = __ldg(S.lrp + i); e < e1; ++e) {
          const int col = __ldg(S.lcol + e);
          const PT v = __ldg(lv + e);
          const PT yc = col >= r0 ? w[(col - r0) * kp + j] : __ldcg(y + size_t(col) * kp + j);
          acc -= v * yc;
        }
        const PT yi = acc * __ldg(dv + i);
        w[(i - r0) * kp + j] = yi;
        if (!last) y[size_t(i) * kp + j] = yi;
      }
      if (last) {
        // the last color: backward sweep of the same block at once (no
        // later colors), y in the scratch
        for (int i = r1 - 1; i >= r0; --i) {
          PT acc = w[(i - r0) * kp + j];
          const int e1 = __ldg(S.urp + i + 1);
          for (int e = __ldg(S.urp + i); e < e1; ++e) acc -= __ldg(uv + e) * w[(__ldg(S.ucol + e) - r0) * kp + j];
          const PT zi = acc * __ldg(dv + i);
          w[(i - r0) * kp + j] = zi;
          z[size_t(i) * kp + j] = zi;
          rz += __ldcg(S.r + size_t(i) * kp + j) * double(zi);
        }
      }
    }
    // every color's results (for the last color: its z) complete before the
    // next color reads them
    if (!sys_sync(S.bar, nct, gen, flag, S.wait_ns)) return false;
  }
  for (int c = nc - 2; c >= 0; --c) {
    const int b1 = __ldg(S.cblk + c + 1);
    for (int blk = __ldg(S.cblk + c) + gc; blk < b1; blk += total) {
      const int r0 = __ldg(S.bptr + blk), r1 = __ldg(S.bptr + blk + 1);
      for (int i = r1 - 1; i >= r0; --i) {
        PT acc = __ldcg(y + size_t(i) * kp + j);
        const int e1 = __ldg(S.urp + i + 1);
        for (int e = __ldg(S.urp + i); e < e1; ++e) {
          const int col = __ldg(S.ucol + e);
          const PT zc = col < r1 ? w[(col - r0) * kp + j] : __ldcg(z + size_t(col) * kp + j);
          acc -= __ldg(uv + e) * zc;
        }
        const PT zi = acc * __ldg(dv + i);
        w[(i - r0) * kp + j] = zi;
        z[size_t(i) * kp + j] = zi;
        rz += __ldcg(S.r + size_t(i) * kp + j) * double(zi);
      }
    }
    if (c > 0 && !sys_sync(S.bar, nct, gen, flag, S.wait_ns)) return false;
  }
  return true;
}

// R: rows per chain and pass of the SpMV and the p update (1, 2 or 4)
template <typename PT, int R>
__global__ void __launch_bounds__(kMaxWarpsPerCta * kWarp, 1)
batch_kernel(const BatchSys *sys, const int32_t *cta_sys, int k, int kp, int smax, int maxit, double tol) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ BatchSys S;
  __shared__ int flag;
  __shared__ double sv[4][32];    // per right-hand side: bb / rr / pq / rz sums
  __shared__ double st_rz[32], st_beta[32], st_bn[32];
  __shared__ int st_act[32];
  __shared__ int any_act;
  if (threadIdx.x == 0) S = sys[cta_sys[blockIdx.x]];
  __syncthreads();
  const int nchain = blockDim.x / kp;
  const int ch = threadIdx.x / kp, j = threadIdx.x % kp;
  const int lc = blockIdx.x - S.cta0;
  const unsigned nct = unsigned(S.cta1 - S.cta0);
  const int gc = lc * nchain + ch, total = int(nct) * nchain;
  PT *w = reinterpret_cast<PT *>(smem) + size_t(ch) * smax * kp;
  double *red = reinterpret_cast<double *>(smem + size_t(nchain) * smax * kp * sizeof(PT));
  double *mypart = S.part + size_t(lc) * 4 * kp;
  const int n = S.n;
  unsigned gen = 0;
  bool ok = true;
  const bool real = j < k;

  // solve start: x, b (in r) in the internal numbering; p = 0; <b,b>
  double acc = 0.0;
  for (int i = gc; i < n; i += total) {
    const int o = __ldg(S.perm + i);
    const double bi = real ? __ldcg(S.bin + size_t(j) * n + o) : 0.0;
    S.x[size_t(i) * kp + j] = real ? __ldcg(S.xio + size_t(j) * n + o) : 0.0;
    S.r[size_t(i) * kp + j] = bi;
    S.p[size_t(i) * kp + j] = 0.0;
    acc += bi * bi;
  }
  cta_rhs_sum(acc, red, kp, nchain, mypart + 0 * kp);
  ok = sys_sync(S.bar, nct, gen, &flag, S.wait_ns);
  // r0 = b - A x0, <r0, r0> (a row's b is read and r written by its own lane)
  if (ok) {
    acc = 0.0;
    for (int i = gc; i < n; i += total) {
      double s = 0.0;
      const int e1 = __ldg(S.arp + i + 1);
      for (int e = __ldg(S.arp + i); e < e1; ++e)
        s += __ldg(S.aval + e) * __ldcg(S.x + size_t(__ldg(S.acol + e)) * kp + j);
      const double ri = __ldcg(S.r + size_t(i) * kp + j) - s;
      S.r[size_t(i) * kp + j] = ri;
      acc += ri * ri;
    }
    cta_rhs_sum(acc, red, kp, nchain, mypart + 1 * kp);
    ok = sys_sync(S.bar, nct, gen, &flag, S.wait_ns);
  }
  // z0 = M^-1 r0, <r0, z0>
  double rr = 0.0, rz = 0.0;
  if (ok) ok = batch_precond<PT, false>(S, w, kp, j, gc, total, 0.0, false, rr, rz, nct, gen, &flag);
  if (ok) {
    cta_rhs_sum(rz, red, kp, nchain, mypart + 3 * kp);
    ok = sys_sync(S.bar, nct, gen, &flag, S.wait_ns);
  }
  int it = 0;
  if (ok) {
    sys_rhs_sum(S.part, int(nct), kp, 0, sv[0]);
    sys_rhs_sum(S.part, int(nct), kp, 1, sv[1]);
    sys_rhs_sum(S.part, int(nct), kp, 3, sv[3]);
    if (threadIdx.x < kp) {
      const int t = threadIdx.x;
      const double bn = sqrt(sv[0][t]);
      st_bn[t] = bn;
      st_rz[t] = sv[3][t];
      st_beta[t] = 0.0;
      int a = 0, status = ICCG_OK;
      double rn = 0.0;
      if (t < k && bn > 0.0) {
        rn = sqrt(sv[1][t]) / bn;
        if (!isfinite(rn) || !isfinite(sv[3][t])) status = ICCG_ERR_NONFINITE;
        else if (rn <= tol) status = ICCG_OK;
        else if (maxit <= 0) status = ICCG_NOT_CONVERGED;
        else a = 1;
      }
      st_act[t] = a;
      if (lc == 0) {
        S.hist[t] = rn;
        S.iters[t] = 0;
        S.status[t] = a ? ICCG_NOT_CONVERGED : status;
      }
    }
    if (threadIdx.x == 0) {
      int a = 0;
      for (int t = 0; t < kp; ++t) a |= st_act[t];
      any_act = a;
    }
    __syncthreads();
  }
  while (ok && any_act) {
    const bool act = st_act[j] != 0;
    const double beta = st_beta[j];
    // p = z + beta p
    const PT *z = reinterpret_cast<const PT *>(S.z);
    // R consecutive rows per chain and pass: their loads are issued together
    if (act && R == 1) {
      for (int i = gc; i < n; i += total)
        S.p[size_t(i) * kp + j] = double(__ldcg(z + size_t(i) * kp + j)) + beta * __ldcg(S.p + size_t(i) * kp + j);
    } else if (act) {
      for (int i0 = gc * R; i0 < n; i0 += total * R) {
        double zz[R], pp[R];
#pragma unroll
        for (int u = 0; u < R; ++u)
          if (i0 + u < n) {
            zz[u] = double(__ldcg(z + size_t(i0 + u) * kp + j));
            pp[u] = __ldcg(S.p + size_t(i0 + u) * kp + j);
          }
#pragma unroll
        for (int u = 0; u < R; ++u)
          if (i0 + u < n) S.p[size_t(i0 + u) * kp + j] = zz[u] + beta * pp[u];
      }
    }
    if (!(ok = sys_sync(S.bar, nct, gen, &flag, S.wait_ns))) break;
    // q = A p, <p, q>
    acc = 0.0;
    if (act && R == 1) {
      for (int i = gc; i < n; i += total) {
        double s = 0.0;
        const int e1 = __ldg(S.arp + i + 1);
        for (int e = __ldg(S.arp + i); e < e1; ++e)
          s += __ldg(S.aval + e) * __ldcg(S.p + size_t(__ldg(S.acol + e)) * kp + j);
        S.q[size_t(i) * kp + j] = s;
        acc += __ldcg(S.p + size_t(i) * kp + j) * s;
      }
    } else if (act) {
      for (int i0 = gc * R; i0 < n; i0 += total * R) {
        int e0[R], e1[R];
        double sq[R];
        int len = 0;
#pragma unroll
        for (int u = 0; u < R; ++u) {
          const bool v = i0 + u < n;
          e0[u] = v ? __ldg(S.arp + i0 + u) : 0;
          e1[u] = v ? __ldg(S.arp + i0 + u + 1) : 0;
          sq[u] = 0.0;
          len = max(len, e1[u] - e0[u]);
        }
        // the rows' t-th entries together (each row's sum in entry order)
        for (int t = 0; t < len; ++t) {
#pragma unroll
          for (int u = 0; u < R; ++u)
            if (e0[u] + t < e1[u])
              sq[u] += __ldg(S.aval + e0[u] + t) * __ldcg(S.p + size_t(__ldg(S.acol + e0[u] + t)) * kp + j);
        }
#pragma unroll
        for (int u = 0; u < R; ++u)
          if (i0 + u < n) {
            S.q[size_t(i0 + u) * kp + j] = sq[u];
            acc += __ldcg(S.p + size_t(i0 + u) * kp + j) * sq[u];
          }
      }
    }
    cta_rhs_sum(acc, red, kp, nchain, mypart + 2 * kp);
    if (!(ok = sys_sync(S.bar, nct, gen, &flag, S.wait_ns))) break;
    sys_rhs_sum(S.part, int(nct), kp, 2, sv[2]);
    const double alpha = act ? st_rz[j] / sv[2][j] : 0.0;
    // x / r update, z = M^-1 r, <r,r>, <r,z>
    rr = 0.0;
    rz = 0.0;
    if (!(ok = batch_precond<PT, true>(S, w, kp, j, gc, total, alpha, act, rr, rz, nct, gen, &flag))) break;
    cta_rhs_sum(rr, red, kp, nchain, mypart + 1 * kp);
    cta_rhs_sum(rz, red, kp, nchain, mypart + 3 * kp);
    if (!(ok = sys_sync(S.bar, nct, gen, &flag, S.wait_ns))) break;
    sys_rhs_sum(S.part, int(nct), kp, 1, sv[1]);
    sys_rhs_sum(S.part, int(nct), kp, 3, sv[3]);
    ++it;
    if (threadIdx.x < kp) {
      const int t = threadIdx.x;
      if (st_act[t]) {
        const double rn = sqrt(sv[1][t]) / st_bn[t];
        int a = 1, status = ICCG_NOT_CONVERGED;
        if (!isfinite(rn) || !isfinite(sv[3][t])) { a = 0; status = ICCG_ERR_NONFINITE; }
        else if (rn <= tol) { a = 0; status = ICCG_OK; }
        else if (it >= maxit) { a = 0; status = ICCG_NOT_CONVERGED; }
        else {
          st_beta[t] = sv[3][t] / st_rz[t];
          st_rz[t] = sv[3][t];
        }
        if (lc == 0) {
          S.hist[size_t(it) * kp + t] = rn;
          S.iters[t] = it;
          S.status[t] = status;
        }
        st_act[t] = a;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int a = 0;
      for (int t = 0; t < kp; ++t) a |= st_act[t];
      any_act = a;
    }
    __syncthreads();
  }
  if (ok) {
    for (int i = gc; i < n; i += total)
      if (real) S.xio[size_t(j) * n + __ldg(S.perm + i)] = st_bn[j] > 0.0 ? __ldcg(S.x + size_t(i) * kp + j) : 0.0;
  } else if (lc == 0 && threadIdx.x < kp) {
    S.status[threadIdx.x] = ICCG_ERR_TIMEOUT;
  }
}

int pow2_at_least(int k) {
  int p = 1;
  while (p < k) p <<= 1;
  return p;
}

// allow dynamic shared memory up to the opt-in limit minus the kernel's
// static shared memory
template <typename K>
cudaError_t allow_smem_b(K kernel) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              optin - int(fa.sharedSizeBytes) - 256);
}

using BatchKernel = void (*)(const BatchSys *, const int32_t *, int, int, int, int, double);

template <typename PT>
BatchKernel batch_kernel_of(int R) {
  return R == 4 ? batch_kernel<PT, 4> : (R == 2 ? batch_kernel<PT, 2> : batch_kernel<PT, 1>);
}

}  // namespace
}  // namespace iccg

using namespace iccg;

struct iccg_batch {
  int device = 0;
  cudaStream_t stream = nullptr;
  int nsys = 0, k = 0, kp = 0, smax = 1;
  bool fp32 = false;
  std::vector<iccg_ctx *> ctxs;
  std::vector<int32_t> n;
  std::vector<void *> allocs;
  // per system device buffers
  std::vector<double *> x, r, p, q, bin, xio, part, hist;
  std::vector<void *> y, z;
  std::vector<int32_t *> iters, status, cblk, bptr;
  GridBar *bars = nullptr;
  BatchSys *d_sys = nullptr;
  int32_t *d_cta_sys = nullptr;
  int hist_cap = 0;
  // launch shape
  int W = 8, cps = 1, grid = 0, smem = 0, max_part_ctas = 0;
  int R = 1;             // rows per chain and pass (SpMV, p update)
  double wexp = 1.0;     // CTAs per system proportional to n^wexp
  std::vector<int32_t> cta0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int graph_maxit = -1;
  double graph_tol = -1.0;
  bool direct = false;   // the runtime refused to capture the cooperative launch: launch it directly
  unsigned long long wait_ns = kDefaultWaitNs;   // barrier wait limit of the batched kernel
  std::string err_msg;
};

namespace {

cudaError_t b_alloc(iccg_batch *b, void **p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes + 64);
  if (e != cudaSuccess) return e;
  b->allocs.push_back(*p);
  return cudaMemsetAsync(*p, 0, bytes + 64, b->stream);
}

int batch_smem(const iccg_batch *b, int W) {
  const int nchain = W * kWarp / b->kp;
  const int elem = b->fp32 ? 4 : 8;
  return nchain * b->smax * b->kp * elem + nchain * b->kp * 8;
}

int batch_occupancy(const iccg_batch *b, int W, int smem) {
  int nb = 0;
  const cudaError_t e =
      b->fp32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_kernel_of<float>(b->R), W * kWarp, size_t(smem))
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_kernel_of<double>(b->R), W * kWarp, size_t(smem));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}

void destroy_batch_graph(iccg_batch *b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->gexec = nullptr;
  b->graph = nullptr;
}

// CTA ranges per system (>= 1 each) for a grid of G CTAs, proportional to
// n^wexp: wexp = 1 spreads rows evenly, wexp = 4/3 weights rows by an
// iteration count that grows with the grid side (CG on a discretised
// elliptic operator needs O(sqrt kappa) = O(side) iterations); returns false
// when G < nsys.
bool assign_ctas(iccg_batch *b, int G) {
  if (G < b->nsys) return false;
  double tot = 0.0;
  std::vector<double> wt(b->nsys);
  for (int s = 0; s < b->nsys; ++s) {
    wt[s] = std::pow(double(b->n[s]), b->wexp);
    tot += wt[s];
  }
  std::vector<int32_t> c(b->nsys, 1);
  int used = b->nsys;
  // largest remainder over the CTAs beyond one per system
  std::vector<double> want(b->nsys);
  for (int s = 0; s < b->nsys; ++s) want[s] = double(G) * wt[s] / tot;
  for (int s = 0; s < b->nsys; ++s) {
    const int extra = std::max(0, int(want[s]) - 1);
    c[s] += extra;
    used += extra;
  }
  while (used > G) {
    int best = -1;
    for (int s = 0; s < b->nsys; ++s)
      if (c[s] > 1 && (best < 0 || double(c[s]) - want[s] > double(c[best]) - want[best])) best = s;
    if (best < 0) break;
    c[best]--;
    used--;
  }
  while (used < G) {
    int best = 0;
    for (int s = 1; s < b->nsys; ++s)
      if (want[s] - double(c[s]) > want[best] - double(c[best])) best = s;
    c[best]++;
    used++;
  }
  b->cta0.assign(b->nsys + 1, 0);
  for (int s = 0; s < b->nsys; ++s) b->cta0[s + 1] = b->cta0[s] + c[s];
  b->grid = b->cta0[b->nsys];
  return true;
}

iccg_status upload_plan(iccg_batch *b, int maxit) {
  // per-system descriptors for the current CTA assignment and history size
  std::vector<BatchSys> hs(b->nsys);
  std::vector<int32_t> cs(b->grid);
  for (int s = 0; s < b->nsys; ++s) {
    const iccg_ctx *c = b->ctxs[s];
    const Params &P = c->P;
    BatchSys &S = hs[s];
    std::memset(&S, 0, sizeof(S));
    S.n = b->n[s];
    S.nc = c->H.n_c;
    S.cta0 = b->cta0[s];
    S.cta1 = b->cta0[s + 1];
    S.arp = P.arp; S.acol = P.acol; S.aval = P.aval;
    S.lrp = P.lrp; S.lcol = P.lcol; S.urp = P.urp; S.ucol = P.ucol;
    S.lv64 = P.lval; S.uv64 = P.uval; S.dv64 = P.invd;
    S.lv32 = P.lval32; S.uv32 = P.uval32; S.dv32 = P.invd32;
    S.cblk = b->cblk[s];
    S.bptr = b->bptr[s];
    S.perm = P.perm;
    S.x = b->x[s]; S.r = b->r[s]; S.p = b->p[s]; S.q = b->q[s];
    S.y = b->y[s]; S.z = b->z[s];
    S.bin = b->bin[s];
    S.xio = b->xio[s];
    S.part = b->part[s];
    S.hist = b->hist[s];
    S.iters = b->iters[s];
    S.status = b->status[s];
    S.bar = b->bars + s;
    S.wait_ns = b->wait_ns;
    for (int g = S.cta0; g < S.cta1; ++g) cs[g] = s;
  }
  if (cudaMemcpyAsync(b->d_sys, hs.data(), sizeof(BatchSys) * hs.size(), cudaMemcpyHostToDevice, b->stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(b->d_cta_sys, cs.data(), sizeof(int32_t) * cs.size(), cudaMemcpyHostToDevice, b->stream) !=
          cudaSuccess) {
    b->err_msg = std::string("batch plan upload: ") + cudaGetErrorString(cudaGetLastError());
    return ICCG_ERR_CUDA;
  }
  (void)maxit;
  return ICCG_OK;
}

cudaError_t batch_launch(iccg_batch *b, cudaStream_t s, int maxit, double tol) {
  cudaError_t e = cudaMemsetAsync(b->bars, 0, sizeof(GridBar) * size_t(b->nsys), s);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(b->grid));
  cfg.blockDim = dim3(unsigned(b->W * kWarp));
  cfg.dynamicSmemBytes = size_t(b->smem);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const BatchSys *sys = b->d_sys;
  const int32_t *cts = b->d_cta_sys;
  if (b->fp32) return cudaLaunchKernelEx(&cfg, batch_kernel_of<float>(b->R), sys, cts, b->k, b->kp, b->smax, maxit, tol);
  return cudaLaunchKernelEx(&cfg, batch_kernel_of<double>(b->R), sys, cts, b->k, b->kp, b->smax, maxit, tol);
}

iccg_status set_shape(iccg_batch *b, int W, int cps, int sms) {
  const int smem = batch_smem(b, W);
  const int occ = batch_occupancy(b, W, smem);
  if (occ <= 0) {
    b->err_msg = "batched kernel does not fit an SM with this shape";
    return ICCG_ERR_ARG;
  }
  const int c = cps <= 0 ? occ : std::min(cps, occ);
  if (!assign_ctas(b, sms * c)) {
    b->err_msg = "more systems than resident CTAs";
    return ICCG_ERR_ARG;
  }
  if (b->grid > b->max_part_ctas) {
    b->err_msg = "CTA count above the partial-sum capacity";
    return ICCG_ERR_ARG;
  }
  b->W = W;
  b->cps = c;
  b->smem = smem;
  destroy_batch_graph(b);
  return ICCG_OK;
}

iccg_status ensure_hist(iccg_batch *b, int maxit) {
  if (maxit + 1 <= b->hist_cap) return ICCG_OK;
  const int cap = std::max(maxit + 1, 1024);
  for (int s = 0; s < b->nsys; ++s) {
    void *h = nullptr;
    if (b_alloc(b, &h, sizeof(double) * size_t(cap) * size_t(b->kp)) != cudaSuccess) {
      b->err_msg = "history allocation failed";
      return ICCG_ERR_CUDA;
    }
    b->hist[s] = static_cast<double *>(h);
  }
  b->hist_cap = cap;
  destroy_batch_graph(b);
  return ICCG_OK;
}

iccg_status run(iccg_batch *b, int maxit, double tol) {
  if (b->direct) {
    iccg_status st = upload_plan(b, maxit);
    if (st != ICCG_OK) return st;
    const cudaError_t e = batch_launch(b, b->stream, maxit, tol);
    if (e != cudaSuccess) {
      b->err_msg = std::string("batched launch: ") + cudaGetErrorString(e);
      return ICCG_ERR_CUDA;
    }
    return ICCG_OK;
  }
  if (!b->gexec || b->graph_maxit != maxit || b->graph_tol != tol) {
    destroy_batch_graph(b);
    iccg_status st = upload_plan(b, maxit);
    if (st != ICCG_OK) return st;
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
      b->err_msg = "capture stream";
      return ICCG_ERR_CUDA;
    }
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    cudaError_t el = e == cudaSuccess ? batch_launch(b, cs, maxit, tol) : e;
    cudaGraph_t g = nullptr;
    cudaError_t ee = e == cudaSuccess ? cudaStreamEndCapture(cs, &g) : e;
    cudaStreamDestroy(cs);
    if (el != cudaSuccess || ee != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      b->direct = true;
      return run(b, maxit, tol);
    }
    b->graph = g;
    if (cudaGraphInstantiate(&b->gexec, g, 0) != cudaSuccess) {
      b->err_msg = "batched graph instantiate";
      destroy_batch_graph(b);
      return ICCG_ERR_CUDA;
    }
    b->graph_maxit = maxit;
    b->graph_tol = tol;
  }
  if (cudaGraphLaunch(b->gexec, b->stream) != cudaSuccess) {
    b->err_msg = std::string("batched graph launch: ") + cudaGetErrorString(cudaGetLastError());
    return ICCG_ERR_CUDA;
  }
  return ICCG_OK;
}

}  // namespace

extern "C" {

iccg_status iccg_batch_create(iccg_batch **out, iccg_ctx *const *ctxs, int32_t nsys, int32_t nrhs,
                              const iccg_batch_opts *opts) {
  if (!out) return ICCG_ERR_ARG;
  *out = nullptr;
  if (!ctxs || nsys < 1 || nrhs < 1 || nrhs > 32) return ICCG_ERR_ARG;
  iccg_batch_opts o{};
  if (opts) o = *opts;
  for (int k = 0; k < 4; ++k)
    if (o.reserved[k] != 0) return ICCG_ERR_ARG;
  if (o.warps_per_cta < 0 || o.warps_per_cta > kMaxWarpsPerCta || o.ctas_per_sm < 0) return ICCG_ERR_ARG;
  if (o.rows_per_thread != 0 && o.rows_per_thread != 1 && o.rows_per_thread != 2 && o.rows_per_thread != 4)
    return ICCG_ERR_ARG;
  for (int s = 0; s < nsys; ++s) {
    const iccg_ctx *c = ctxs[s];
    if (!c || !c->factored || c->H.n < 1) return ICCG_ERR_STATE;
    if (c->H.tile_colors != 0 || c->H.unit_colors != 0) return ICCG_ERR_ARG;   // set up with lane_block_max = -1
    if (c->device != ctxs[0]->device || c->fp32 != ctxs[0]->fp32) return ICCG_ERR_ARG;
    for (int j = 0; j < c->H.n_b; ++j)
      if (c->H.block_ptr[j + 1] - c->H.block_ptr[j] > kBatchMaxBlock) return ICCG_ERR_ARG;
  }
  iccg_batch *b = new iccg_batch();
  *out = b;
  b->device = ctxs[0]->device;
  b->stream = ctxs[0]->stream;
  b->nsys = nsys;
  b->k = nrhs;
  b->kp = pow2_at_least(nrhs);
  b->fp32 = ctxs[0]->fp32;
  b->ctxs.assign(ctxs, ctxs + nsys);
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != b->device) cudaSetDevice(b->device);
  cudaError_t e = cudaSuccess;
  for (int R : {1, 2, 4}) {
    if (e == cudaSuccess) e = b->fp32 ? allow_smem_b(batch_kernel_of<float>(R)) : allow_smem_b(batch_kernel_of<double>(R));
  }
  const size_t pe = b->fp32 ? 4 : 8;
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  b->max_part_ctas = sms * 32;
  b->x.resize(nsys); b->r.resize(nsys); b->p.resize(nsys); b->q.resize(nsys);
  b->bin.resize(nsys); b->xio.resize(nsys); b->part.resize(nsys); b->hist.resize(nsys);
  b->y.resize(nsys); b->z.resize(nsys);
  b->iters.resize(nsys); b->status.resize(nsys); b->cblk.resize(nsys); b->bptr.resize(nsys);
  for (int s = 0; s < nsys && e == cudaSuccess; ++s) {
    const iccg_ctx *c = ctxs[s];
    const size_t n = size_t(c->H.n), kp = size_t(b->kp);
    b->n.push_back(c->H.n);
    for (int j = 0; j < c->H.n_b; ++j) b->smax = std::max(b->smax, c->H.block_ptr[j + 1] - c->H.block_ptr[j]);
    void *v = nullptr;
    if (e == cudaSuccess && (e = b_alloc(b, &v, 8 * n * kp)) == cudaSuccess) b->x[s] = static_cast<double *>(v);
    if (e == cudaSuccess && (e = b_alloc(b, &v, 8 * n * kp)) == cudaSuccess) b->r[s] = static_cast<double *>(v);
    if (e == cudaSuccess && (e = b_alloc(b, &v, 8 * n * kp)) == cudaSuccess) b->p[s] = static_cast<double *>(v);
    if (e == cudaSuccess && (e = b_alloc(b, &v, 8 * n * kp)) == cudaSuccess) b->q[s] = static_cast<double *>(v);
    if (e == cudaSuccess && (e = b_alloc(b, &v, pe * n * kp)) == cudaSuccess) b->y[s] = v;
    if (e == cudaSuccess && (e = b_alloc(b, &v, pe * n * kp)) == cudaSuccess) b->z[s] = v;
    if (e == cudaSuccess && (e = b_alloc(b, &v, 8 * n * size_t(b->k))) == cudaSuccess) b->bin[s] = static_cast<double *>(v);
    if (e == cudaSuccess && (e = b_alloc(b, &v, 8 * n * size_t(b->k))) == cudaSuccess) b->xio[s] = static_cast<double *>(v);
    if (e == cudaSuccess && (e = b_alloc(b, &v, 8 * size_t(b->max_part_ctas) * 4 * kp)) == cudaSuccess)
      b->part[s] = static_cast<double *>(v);
    if (e == cudaSuccess && (e = b_alloc(b, &v, 4 * kp)) == cudaSuccess) b->iters[s] = static_cast<int32_t *>(v);
    if (e == cudaSuccess && (e = b_alloc(b, &v, 4 * kp)) == cudaSuccess) b->status[s] = static_cast<int32_t *>(v);
    if (e == cudaSuccess && (e = b_alloc(b, &v, 4 * c->H.color_ptr.size())) == cudaSuccess) {
      b->cblk[s] = static_cast<int32_t *>(v);
      e = cudaMemcpyAsync(v, c->H.color_ptr.data(), 4 * c->H.color_ptr.size(), cudaMemcpyHostToDevice, b->stream);
    }
    if (e == cudaSuccess && (e = b_alloc(b, &v, 4 * c->H.block_ptr.size())) == cudaSuccess) {
      b->bptr[s] = static_cast<int32_t *>(v);
      e = cudaMemcpyAsync(v, c->H.block_ptr.data(), 4 * c->H.block_ptr.size(), cudaMemcpyHostToDevice, b->stream);
    }
  }
  void *v = nullptr;
  if (e == cudaSuccess && (e = b_alloc(b, &v, sizeof(GridBar) * size_t(nsys))) == cudaSuccess)
    b->bars = static_cast<GridBar *>(v);
  if (e == cudaSuccess && (e = b_alloc(b, &v, sizeof(BatchSys) * size_t(nsys))) == cudaSuccess)
    b->d_sys = static_cast<BatchSys *>(v);
  if (e == cudaSuccess && (e = b_alloc(b, &v, sizeof(int32_t) * size_t(b->max_part_ctas))) == cudaSuccess)
    b->d_cta_sys = static_cast<int32_t *>(v);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
  if (e != cudaSuccess) {
    b->err_msg = std::string("batch allocation: ") + cudaGetErrorString(e);
    return ICCG_ERR_CUDA;
  }
  int coop = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, b->device);
  if (!coop) {
    b->err_msg = "cooperative launch not supported";
    return ICCG_ERR_CUDA;
  }
  b->R = o.rows_per_thread > 0 ? o.rows_per_thread : 1;
  iccg_status st = set_shape(b, o.warps_per_cta > 0 ? o.warps_per_cta : 8, o.ctas_per_sm, sms);
  if (st != ICCG_OK) return st;
  if (o.autotune) {
    st = iccg_batch_tune(b, nullptr, 0.0, 0, nullptr);
    if (st != ICCG_OK) return st;
  }
  return ICCG_OK;
}

iccg_status iccg_batch_solve(iccg_batch *b, const double *const *B, double *const *X, double tol, int32_t maxit,
                             int32_t *iters, int32_t *status, double *const *res_hist) {
  if (!b || !B || !X || tol < 0 || !(tol == tol) || maxit < 0) return ICCG_ERR_ARG;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != b->device) cudaSetDevice(b->device);
  struct Restore {
    int p, d;
    ~Restore() { if (p >= 0 && p != d) cudaSetDevice(p); }
  } rs{prev, b->device};
  iccg_status st = ensure_hist(b, maxit);
  if (st != ICCG_OK) return st;
  cudaStream_t s = b->stream;
  for (int i = 0; i < b->nsys; ++i) {
    const size_t bytes = sizeof(double) * size_t(b->n[i]) * size_t(b->k);
    if (!B[i] || !X[i]) return ICCG_ERR_ARG;
    if (cudaMemcpyAsync(b->bin[i], B[i], bytes, cudaMemcpyDefault, s) != cudaSuccess ||
        cudaMemcpyAsync(b->xio[i], X[i], bytes, cudaMemcpyDefault, s) != cudaSuccess) {
      b->err_msg = "copy of B / X0";
      return ICCG_ERR_CUDA;
    }
  }
  st = run(b, maxit, tol);
  if (st != ICCG_OK) return st;
  std::vector<int32_t> it(size_t(b->kp)), stv(size_t(b->kp));
  std::vector<double> h;
  iccg_status worst = ICCG_OK;
  for (int i = 0; i < b->nsys; ++i) {
    const size_t bytes = sizeof(double) * size_t(b->n[i]) * size_t(b->k);
    if (cudaMemcpyAsync(X[i], b->xio[i], bytes, cudaMemcpyDefault, s) != cudaSuccess ||
        cudaMemcpyAsync(it.data(), b->iters[i], 4 * size_t(b->kp), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(stv.data(), b->status[i], 4 * size_t(b->kp), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      b->err_msg = std::string("batched solve: ") + cudaGetErrorString(cudaGetLastError());
      return ICCG_ERR_CUDA;
    }
    for (int j = 0; j < b->k; ++j) {
      if (iters) iters[size_t(i) * b->k + j] = it[j];
      if (status) status[size_t(i) * b->k + j] = stv[j];
      const iccg_status sj = static_cast<iccg_status>(stv[j]);
      if (sj != ICCG_OK && (worst == ICCG_OK || sj != ICCG_NOT_CONVERGED)) worst = sj;
    }
    if (res_hist && res_hist[i]) {
      int mx = 0;
      for (int j = 0; j < b->k; ++j) mx = std::max(mx, it[j]);
      h.assign(size_t(mx + 1) * b->kp, 0.0);
      if (cudaMemcpy(h.data(), b->hist[i], sizeof(double) * h.size(), cudaMemcpyDeviceToHost) != cudaSuccess) {
        b->err_msg = "history copy";
        return ICCG_ERR_CUDA;
      }
      // res_hist[i]: [maxit + 1][nrhs]; entries past a right-hand side's
      // iteration count are 0
      for (int t = 0; t <= maxit; ++t)
        for (int j = 0; j < b->k; ++j)
          res_hist[i][size_t(t) * b->k + j] = (t <= it[j] && t <= mx) ? h[size_t(t) * b->kp + j] : 0.0;
    }
  }
  if (worst == ICCG_ERR_TIMEOUT) b->err_msg = "a barrier wait of the batched solve gave up";
  return worst;
}

iccg_status iccg_batch_tune(iccg_batch *b, const double *const *B, double tol, int32_t maxit, double *best_ms) {
  if (!b || (B && (tol < 0 || !(tol == tol) || maxit < 0))) return ICCG_ERR_ARG;
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  // every candidate shape solves the given right-hand sides from x0 = 0 to
  // (tol, maxit), or, without B, random right-hand sides for a fixed 20
  // iterations (tol 0); the fastest shape is kept
  std::vector<std::vector<double>> hb(b->nsys), hx(b->nsys);
  std::vector<const double *> Bp(b->nsys);
  std::vector<double *> X(b->nsys);
  uint64_t st = 0x9e3779b97f4a7c15ull;
  for (int s = 0; s < b->nsys; ++s) {
    hx[s].assign(size_t(b->n[s]) * b->k, 0.0);
    X[s] = hx[s].data();
    if (B) {
      Bp[s] = B[s];
      if (!B[s]) return ICCG_ERR_ARG;
      continue;
    }
    hb[s].resize(size_t(b->n[s]) * b->k);
    for (double &v : hb[s]) {
      st ^= st << 13; st ^= st >> 7; st ^= st << 17;
      v = double(st >> 11) * (1.0 / 9007199254740992.0) - 0.5;
    }
    Bp[s] = hb[s].data();
  }
  const double ttol = B ? tol : 0.0;
  const int tmax = B ? maxit : 20;
  const int Ws[3] = {4, 8, 16};
  const double Es[2] = {1.0, 4.0 / 3.0};
  double best = 1e300, bE = b->wexp;
  int bW = b->W, bC = b->cps;
  for (double E : Es)
  for (int W : Ws) {
    const int occ = batch_occupancy(b, W, batch_smem(b, W));
    for (int cps = 1; cps <= std::min(occ, 4); cps *= 2) {
      b->wexp = E;
      if (set_shape(b, W, cps, sms) != ICCG_OK) continue;
      for (auto &x : hx) std::fill(x.begin(), x.end(), 0.0);
      // the first call captures the graph; the second is timed
      if (iccg_batch_solve(b, Bp.data(), X.data(), ttol, tmax, nullptr, nullptr, nullptr) == ICCG_ERR_CUDA) continue;
      for (auto &x : hx) std::fill(x.begin(), x.end(), 0.0);
      const auto t0 = std::chrono::steady_clock::now();
      const iccg_status r = iccg_batch_solve(b, Bp.data(), X.data(), ttol, tmax, nullptr, nullptr, nullptr);
      const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      if (r == ICCG_ERR_CUDA || r == ICCG_ERR_TIMEOUT) continue;
      if (ms < best) { best = ms; bW = W; bC = cps; bE = E; }
    }
  }
  // rows per thread at the best shape
  b->wexp = bE;
  int bR = b->R;
  const int R0 = b->R;
  for (int R : {1, 2, 4}) {
    if (R == R0) continue;
    b->R = R;   // the shape's occupancy is that of this R's kernel
    if (set_shape(b, bW, bC, sms) != ICCG_OK) continue;
    for (auto &x : hx) std::fill(x.begin(), x.end(), 0.0);
    if (iccg_batch_solve(b, Bp.data(), X.data(), ttol, tmax, nullptr, nullptr, nullptr) == ICCG_ERR_CUDA) continue;
    for (auto &x : hx) std::fill(x.begin(), x.end(), 0.0);
    const auto t0 = std::chrono::steady_clock::now();
    const iccg_status r = iccg_batch_solve(b, Bp.data(), X.data(), ttol, tmax, nullptr, nullptr, nullptr);
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (r == ICCG_ERR_CUDA || r == ICCG_ERR_TIMEOUT) continue;
    if (ms < best) { best = ms; bR = R; }
  }
  b->R = bR;
  if (best_ms) *best_ms = best;
  return set_shape(b, bW, bC, sms);
}

iccg_status iccg_batch_set_wait_limit(iccg_batch *b, uint64_t wait_ns) {
  if (!b) return ICCG_ERR_ARG;
  b->wait_ns = wait_ns ? wait_ns : kDefaultWaitNs;
  destroy_batch_graph(b);   // the next solve uploads the descriptors again
  return ICCG_OK;
}

iccg_status iccg_batch_info(const iccg_batch *b, int32_t out[7]) {
  if (!b || !out) return ICCG_ERR_ARG;
  out[0] = b->W;
  out[1] = b->cps;
  out[2] = b->grid;
  out[3] = b->kp;
  out[4] = b->smax;
  out[5] = int32_t(b->wexp * 3.0 + 0.5);   // 3 x the CTA-split exponent (3: rows, 4: rows^(4/3))
  out[6] = b->R;
  return ICCG_OK;
}

iccg_status iccg_batch_last_error(const iccg_batch *b, const char **msg) {
  if (!b) return ICCG_ERR_ARG;
  if (msg) *msg = b->err_msg.c_str();
  return ICCG_OK;
}

void iccg_batch_destroy(iccg_batch *b) {
  if (!b) return;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != b->device) cudaSetDevice(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  destroy_batch_graph(b);
  for (void *p : b->allocs) cudaFree(p);
  if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
  delete b;
}

}  // extern "C"
