// Device kernels of block-multicolor ICCG for sm_103a.
//
// One PCG iteration is 2*n_c launches (n_c = number of block colors):
//   spmv                 q = A (z + beta p_old), p_new = z + beta p_old, <p,q>;
//                        its last group sets alpha = (r,z)/(p,q)
//   fwd color 0..n_c-2   x += alpha p, r -= alpha q, <r,r>, then the forward
//                        substitution L y = r for the rows of that color
//                        (Alg. 1: colors in sequence, blocks of a color in
//                        parallel, rows of a block in order)
//   fused color n_c-1    the same, followed at once by the backward sweep of
//                        the last color (its rows have no later-color
//                        dependencies), <r,z>
//   bwd color n_c-2..0   backward substitution L^T z = y (the reverse sweep
//                        described after Alg. 1), <r,z>; the last group of the
//                        color-0 launch reduces <r,r>, <r,z>, records the
//                        residual history, tests ||r||/||b|| <= tol and sets
//                        the CUDA-graph WHILE condition.
//
// Work mapping: one warp per task (a run of whole small blocks of one color,
// or one large block walked tile by tile); every launch has one warp per task
// or per 32R-row SpMV tile, so latency is hidden by the number of resident
// warps.  A tile's CSR segment of L, U or A (values and column indices) is
// copied into the warp's shared memory with cp.async (16-byte, L2 only, all
// copies in flight at once) while the row pointers and 1/L_ii load into
// registers.  Kernels are launched with programmatic dependent launch: each
// lets its successor start at once (griddepcontrol.launch_dependents), and
// every kernel issues these static loads before it waits
// (griddepcontrol.wait) for data its predecessor produces (r, q, x, p, y, z,
// scalars, reduction slots).
//
// Within a tile every lane owns rows r0 + lane + 32k.  The entries that point
// outside the tile are gathered first (y or z written by earlier colors or
// earlier tiles); the in-tile entries (a contiguous run of each CSR row,
// since columns are sorted) are cached in registers and the in-tile
// dependencies are resolved by repeated sweeps over the tile (depth + 1
// sweeps; after sweep k every row of level <= k is final).
//
// Reductions are deterministic and two-level: every CTA writes its partial;
// the last CTA of each group of kGroup CTAs (arrival ticket) sums the group's
// partials in index order; the last group of the launch runs the epilogue.
#include <cstdio>
#include <type_traits>

#include "iccg_internal.h"

namespace iccg {

namespace {

constexpr int kVecThreads = 256;
constexpr int kChunk = 4;    // row entries processed per predicated batch
constexpr int kCacheInt = 4; // in-tile entries per row kept in registers
enum StepMode { M_FWD = 0, M_BWD = 1, M_FUSED = 2 };

__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of one value per thread; result valid in thread 0.  Fixed order.
__device__ __forceinline__ double cta_sum(double v, double *red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < nw; ++k) s += red[k];
  return s;
}

// Deterministic sum of p[0..count) by the whole CTA (result in thread 0);
// optionally clears the entries.
__device__ __forceinline__ double cta_sum_array(double *p, int count, double *red, bool clear) {
  double s = 0.0;
  for (int k = threadIdx.x; k < count; k += blockDim.x) {
    s += __ldcg(p + k);
    if (clear) p[k] = 0.0;
  }
  return cta_sum(s, red);
}

// Arrival on a counter by thread 0 after a fence; true (for the whole CTA)
// for the last of `expected` arrivals, which also resets the counter.
__device__ __forceinline__ bool arrive_last(uint32_t *ticket, uint32_t expected, int *flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const uint32_t t = atomicAdd(ticket, 1u);
    *flag = (t == expected - 1) ? 1 : 0;
    if (*flag) {
      *ticket = 0;
      __threadfence();
    }
  }
  __syncthreads();
  return *flag != 0;
}

// First level: each CTA publishes (a, b); the last CTA of the group returns
// true with the group sums in thread 0's ga / gb.
__device__ __forceinline__ bool group_reduce(const Params &P, double a, double b, bool two, double *red, int *flag,
                                             double &ga, double &gb) {
  const int g = blockIdx.x / kGroup;
  const int g0 = g * kGroup;
  const int gs = min(kGroup, int(gridDim.x) - g0);
  if (threadIdx.x == 0) {
    P.part0[blockIdx.x] = a;
    if (two) P.part1[blockIdx.x] = b;
  }
  if (!arrive_last(P.gticket + g, uint32_t(gs), flag)) return false;
  const double va = threadIdx.x < gs ? __ldcg(P.part0 + g0 + threadIdx.x) : 0.0;
  ga = cta_sum(va, red);
  gb = 0.0;
  if (two) {
    const double vb = threadIdx.x < gs ? __ldcg(P.part1 + g0 + threadIdx.x) : 0.0;
    gb = cta_sum(vb, red);
  }
  return true;
}

// Second level: the last group of the launch.
__device__ __forceinline__ bool launch_last(const Params &P, int *flag) {
  const uint32_t ng = (gridDim.x + kGroup - 1) / kGroup;
  return arrive_last(&P.sc->ticket, ng, flag);
}

// A CSR segment [e0, e1): staged in shared memory (entry e at sv[e - bv],
// sc[e - bc]) when its 16-byte-aligned cover fits the buffer, else read from
// global memory.
template <typename VT>
struct Seg {
  const VT *sv;
  const int32_t *sc;
  const VT *gv;
  const int32_t *gc;
  int bv, bc;
  bool staged;
  __device__ __forceinline__ VT v(int e) const { return staged ? sv[e - bv] : __ldg(gv + e); }
  __device__ __forceinline__ int32_t c(int e) const { return staged ? sc[e - bc] : __ldg(gc + e); }
};

// Start the asynchronous copy of a segment into (sv, sc) and commit it as one
// cp.async group.  Device arrays carry 64 bytes of padding, so the aligned
// cover stays inside the allocation.
template <typename VT>
__device__ __forceinline__ Seg<VT> stage_async(const VT *gv, const int32_t *gc, int e0, int e1, VT *sv,
                                               int32_t *sc, int cap, int lane) {
  Seg<VT> s;
  s.sv = sv; s.sc = sc; s.gv = gv; s.gc = gc;
  constexpr int EV = 16 / sizeof(VT);
  const int a0v = e0 & ~(EV - 1), a1v = (e1 + EV - 1) & ~(EV - 1);
  const int a0c = e0 & ~3, a1c = (e1 + 3) & ~3;
  s.bv = a0v; s.bc = a0c;
  s.staged = (a1v - a0v <= cap) && (a1c - a0c <= cap);
  if (s.staged) {
    const int nv = (a1v - a0v) / EV;
    for (int k = lane; k < nv; k += kWarp) cp_async16(sv + k * EV, gv + a0v + k * EV);
    const int nc = (a1c - a0c) / 4;
    for (int k = lane; k < nc; k += kWarp) cp_async16(sc + k * 4, gc + a0c + k * 4);
  }
  cp_commit();
  return s;
}

// acc -= sum of v_e * x(c_e) over the entries e in [rb, re); entries in
// ascending order, kChunk at a time with predicated loads so a chunk's loads
// are in flight together.
template <typename VT, typename AT, typename Load>
__device__ __forceinline__ AT row_sub(const Seg<VT> &S, int rb, int re, AT acc, Load x) {
  for (int e0 = rb; e0 < re; e0 += kChunk) {
    int cc[kChunk];
    VT vv[kChunk];
#pragma unroll
    for (int j = 0; j < kChunk; ++j) {
      const bool ok = e0 + j < re;
      cc[j] = ok ? S.c(e0 + j) : -1;
      vv[j] = ok ? S.v(e0 + j) : VT(0);
    }
    AT xx[kChunk];
#pragma unroll
    for (int j = 0; j < kChunk; ++j) xx[j] = cc[j] >= 0 ? AT(x(cc[j])) : AT(0);
#pragma unroll
    for (int j = 0; j < kChunk; ++j) acc -= AT(vv[j]) * xx[j];
  }
  return acc;
}

// number of entries of [rb, re) whose column is below `bound` (columns sorted)
template <typename VT>
__device__ __forceinline__ int count_below(const Seg<VT> &S, int rb, int re, int bound) {
  int n = 0;
  for (int e = rb; e < re; ++e) n += S.c(e) < bound ? 1 : 0;
  return n;
}

template <typename PT> __device__ __forceinline__ const PT *lvals(const Params &P);
template <> __device__ __forceinline__ const double *lvals<double>(const Params &P) { return P.lval; }
template <> __device__ __forceinline__ const float *lvals<float>(const Params &P) { return P.lval32; }
template <typename PT> __device__ __forceinline__ const PT *uvals(const Params &P);
template <> __device__ __forceinline__ const double *uvals<double>(const Params &P) { return P.uval; }
template <> __device__ __forceinline__ const float *uvals<float>(const Params &P) { return P.uval32; }
template <typename PT> __device__ __forceinline__ const PT *invds(const Params &P);
template <> __device__ __forceinline__ const double *invds<double>(const Params &P) { return P.invd; }
template <> __device__ __forceinline__ const float *invds<float>(const Params &P) { return P.invd32; }

// Per-warp shared memory: one staging buffer [vals cap][cols cap] and the
// tile's in-flight y / z values [32R].  Sizes are rounded to 16 bytes.
__host__ __device__ __forceinline__ int warp_bytes1(int cap, int R, int elem) {
  return ((cap * elem + 15) & ~15) + ((cap * 4 + 15) & ~15) + ((kWarp * R * elem + 15) & ~15);
}

template <typename VT>
__device__ __forceinline__ void warp_bufs(unsigned char *base, int cap, int R, VT *&sv, int32_t *&sc, VT *&ysh) {
  const int bytes_v = (cap * int(sizeof(VT)) + 15) & ~15;
  const int bytes_c = (cap * 4 + 15) & ~15;
  unsigned char *mine = base + (threadIdx.x >> 5) * warp_bytes1(cap, R, int(sizeof(VT)));
  sv = reinterpret_cast<VT *>(mine);
  sc = reinterpret_cast<int32_t *>(mine + bytes_v);
  ysh = reinterpret_cast<VT *>(mine + bytes_v + bytes_c);
}

__device__ __forceinline__ TileDesc load_desc(const TileDesc *d) {
  const int4 a = __ldg(reinterpret_cast<const int4 *>(d));
  const int4 b = __ldg(reinterpret_cast<const int4 *>(d) + 1);
  TileDesc t;
  t.r0 = a.x; t.r1 = a.y; t.rounds = a.z; t.pad = a.w;
  t.l0 = b.x; t.l1 = b.y; t.u0 = b.z; t.u1 = b.w;
  return t;
}

__device__ __forceinline__ void load_task(const TaskDesc *t, TileDesc &first, int &tile0, int &ntiles) {
  first = load_desc(&t->first);
  const int4 c = __ldg(reinterpret_cast<const int4 *>(t) + 2);
  tile0 = c.x;
  ntiles = c.y;
}

// Everything of one tile step that no earlier kernel writes.
template <typename PT, int R>
struct Step {
  int r0, r1, rounds;
  Seg<PT> S;
  int rb[R], re[R];
  PT dv[R];
};

template <typename PT, int R>
__device__ __forceinline__ void step_load(const Params &P, const TileDesc &d, bool upper, PT *sv, int32_t *sc, int cap,
                                          int lane, Step<PT, R> &st) {
  st.r0 = d.r0;
  st.r1 = d.r1;
  st.rounds = upper ? (d.rounds >> 16) : (d.rounds & 0xffff);
  st.S = upper ? stage_async<PT>(uvals<PT>(P), P.ucol, d.u0, d.u1, sv, sc, cap, lane)
               : stage_async<PT>(lvals<PT>(P), P.lcol, d.l0, d.l1, sv, sc, cap, lane);
  const int32_t *rp = upper ? P.urp : P.lrp;
  const PT *idv = invds<PT>(P);
#pragma unroll
  for (int k = 0; k < R; ++k) {
    const int i = d.r0 + lane + kWarp * k;
    const bool ok = i < d.r1;
    st.rb[k] = ok ? __ldg(rp + i) : 0;
    st.re[k] = ok ? __ldg(rp + i + 1) : 0;
    st.dv[k] = ok ? __ldg(idv + i) : PT(0);
  }
}

// One tile of the forward (UPPER = false, L rows: out-of-tile entries are a
// prefix of each row) or backward (UPPER = true, U rows: out-of-tile entries
// are a suffix) substitution.  `src` is r (forward) or y (backward); `ext` is
// the vector gathered for out-of-tile columns (y or z); the result goes to
// `dst` (y or z).  UPDATE fuses x += alpha p, r -= alpha q, <r,r> in front.
template <typename PT, int R, bool UPPER, bool UPDATE>
__device__ __forceinline__ void tile_step(const Params &P, const Step<PT, R> &st, PT *ysh, int lane, double alpha,
                                          const double *pn, double &rr_acc, double &rz_acc) {
  const PT *ext = reinterpret_cast<const PT *>(UPPER ? P.z : P.y);
  PT *dst = reinterpret_cast<PT *>(UPPER ? P.z : P.y);
  const int r0 = st.r0, r1 = st.r1;
  PT tv[R];
  int ib[R], ie[R];   // in-tile entry range of each row
  int lo[R][kCacheInt];
  PT lv[R][kCacheInt];
#pragma unroll
  for (int k = 0; k < R; ++k) {
    const int i = r0 + lane + kWarp * k;
    tv[k] = PT(0);
    ib[k] = ie[k] = 0;
    if (i < r1) {
      PT src;
      if (UPPER) {
        src = reinterpret_cast<const PT *>(P.y)[i];
      } else {
        double ri = P.r[i];
        if (UPDATE) {
          ri -= alpha * P.q[i];
          P.r[i] = ri;
          P.xh[i] += alpha * pn[i];
          rr_acc += ri * ri;
        }
        src = PT(ri);
      }
      // L row: [rb, split) outside (c < r0), [split, re) inside
      // U row: [rb, split) inside (c < r1), [split, re) outside
      const int split = st.rb[k] + count_below(st.S, st.rb[k], st.re[k], UPPER ? r1 : r0);
      const int xb = UPPER ? split : st.rb[k], xe = UPPER ? st.re[k] : split;
      ib[k] = UPPER ? st.rb[k] : split;
      ie[k] = UPPER ? split : st.re[k];
      tv[k] = row_sub<PT, PT>(st.S, xb, xe, src, [&](int c) { return ext[c]; });
    }
#pragma unroll
    for (int j = 0; j < kCacheInt; ++j) {
      const int e = ib[k] + j;
      const bool ok = e < ie[k];
      lo[k][j] = ok ? st.S.c(e) - r0 : 0;
      lv[k][j] = ok ? st.S.v(e) : PT(0);
    }
    if (i < r1) ysh[lane + kWarp * k] = tv[k] * st.dv[k];
  }
  // overflow of the register cache is rare (wide in-tile rows); warp-uniform
  bool spill = false;
#pragma unroll
  for (int k = 0; k < R; ++k) spill |= (ie[k] - ib[k]) > kCacheInt;
  spill = __any_sync(0xffffffffu, spill);
  for (int rd = 1; rd < st.rounds; ++rd) {
    __syncwarp();
    PT yn[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
      PT acc = tv[k];
#pragma unroll
      for (int j = 0; j < kCacheInt; ++j) acc -= lv[k][j] * ysh[lo[k][j]];
      if (spill && ie[k] - ib[k] > kCacheInt)
        acc = row_sub<PT, PT>(st.S, ib[k] + kCacheInt, ie[k], acc, [&](int c) { return ysh[c - r0]; });
      yn[k] = acc * st.dv[k];
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < R; ++k)
      if (r0 + lane + kWarp * k < r1) ysh[lane + kWarp * k] = yn[k];
  }
  __syncwarp();
#pragma unroll
  for (int k = 0; k < R; ++k) {
    const int i = r0 + lane + kWarp * k;
    if (i < r1) {
      const PT v = ysh[lane + kWarp * k];
      dst[i] = v;
      if (UPPER) rz_acc += P.r[i] * double(v);
    }
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------
// epilogues run by the last group of a launch
// ---------------------------------------------------------------------------
__device__ void set_condition(const Scalars *s, int keep_going) {
  if (s->use_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)s->cond_handle, keep_going ? 1u : 0u);
}

// After the backward sweep of iteration k: residual history, stop test, beta.
__device__ void finish_iteration(const Params &P, double *red) {
  const double rr = cta_sum_array(P.acc_rr, P.ngroup, red, true);
  const double rz = cta_sum_array(P.acc_rz, P.ngroup, red, true);
  if (threadIdx.x == 0) {
    Scalars *s = P.sc;
    const int k = s->iter;
    const double rn = sqrt(rr) / s->bnorm;
    P.hist[k + 1] = rn;
    s->iter = k + 1;
    s->rr = rr;
    int done = 0;
    if (!isfinite(rn) || !isfinite(rz)) { s->status = ICCG_ERR_NONFINITE; done = 1; }
    else if (rn <= s->tol) { s->status = ICCG_OK; done = 1; }
    else if (k + 1 >= s->maxit) { s->status = ICCG_NOT_CONVERGED; done = 1; }
    else { s->beta = rz / s->rz; s->rz = rz; }
    s->done = done;
    set_condition(s, !done);
  }
}

// After r0 = b - A x0 and z0 = M^-1 r0: ||b||, history[0], stop test.
// init_bb holds <b,b> partials, gpq the <r0,r0> group sums.
__device__ void finish_init(const Params &P, double *red) {
  const double bb = cta_sum_array(P.init_bb, P.nbb, red, true);
  const double rr = cta_sum_array(P.gpq, P.ngroup, red, true);
  const double rz = cta_sum_array(P.acc_rz, P.ngroup, red, true);
  cta_sum_array(P.acc_rr, P.ngroup, red, true);
  if (threadIdx.x == 0) {
    Scalars *s = P.sc;
    const double bn = sqrt(bb);
    s->bb = bb;
    s->bnorm = bn;
    s->iter = 0;
    s->beta = 0.0;
    s->rz = rz;
    s->rr = rr;
    int done = 0;
    if (bn == 0.0) { P.hist[0] = 0.0; s->status = ICCG_OK; done = 1; }
    else {
      const double rn = sqrt(rr) / bn;
      P.hist[0] = rn;
      if (!isfinite(rn) || !isfinite(rz)) { s->status = ICCG_ERR_NONFINITE; done = 1; }
      else if (rn <= s->tol) { s->status = ICCG_OK; done = 1; }
      else if (s->maxit <= 0) { s->status = ICCG_NOT_CONVERGED; done = 1; }
      else s->status = ICCG_NOT_CONVERGED;
    }
    s->done = done;
    set_condition(s, !done);
  }
}

enum Fin { FIN_NONE = 0, FIN_ITER = 1, FIN_INIT = 2 };

// ---------------------------------------------------------------------------
// color kernel: MODE = forward sweep of one color, backward sweep of one
// color, or both for the last color (fused)
// ---------------------------------------------------------------------------
template <typename PT, int R, int MODE, bool UPDATE>
__global__ void __launch_bounds__(kMaxWarpsPerCta * kWarp)
color_kernel(Params P, int task0, int task1, int cap, int fin) {
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[kMaxWarpsPerCta];
  __shared__ int flag;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
  PT *sv; int32_t *sc; PT *ysh;
  warp_bufs<PT>(smem, cap, R, sv, sc, ysh);
  double rr_acc = 0.0, rz_acc = 0.0;
  const int task = task0 + blockIdx.x * W + warp;
  if (task < task1) {
    TileDesc d;
    int tile0, ntiles;
    load_task(P.tasks + task, d, tile0, ntiles);
    const int nsteps = MODE == M_FUSED ? 2 * ntiles : ntiles;
    double alpha = 0.0;
    const double *pn = nullptr;
    for (int s = 0; s < nsteps; ++s) {
      bool upper;
      int tl;
      if (MODE == M_FWD) { tl = tile0 + s; upper = false; }
      else if (MODE == M_BWD) { tl = tile0 + ntiles - 1 - s; upper = true; }
      else if (s < ntiles) { tl = tile0 + s; upper = false; }
      else { tl = tile0 + 2 * ntiles - 1 - s; upper = true; }
      if (s > 0 || MODE == M_BWD) {
        if (!(s == 0 && ntiles == 1)) d = load_desc(P.tdesc + tl);
      }
      Step<PT, R> st;
      step_load<PT, R>(P, d, upper, sv, sc, cap, lane, st);
      cp_wait_all();
      __syncwarp();
      if (s == 0) {
        pdl_wait();
        if (UPDATE) {
          alpha = __ldcg(&P.sc->alpha);
          pn = ((__ldcg(&P.sc->iter) + 1) & 1) ? P.p1 : P.p0;
        }
      }
      if (upper) tile_step<PT, R, true, false>(P, st, ysh, lane, 0.0, nullptr, rr_acc, rz_acc);
      else tile_step<PT, R, false, UPDATE>(P, st, ysh, lane, alpha, pn, rr_acc, rz_acc);
    }
  } else {
    pdl_wait();
  }
  if (MODE == M_FWD && !UPDATE) return;
  const bool two = MODE == M_FUSED && UPDATE;
  const double a = MODE == M_BWD ? rz_acc : (MODE == M_FUSED && !UPDATE ? rz_acc : rr_acc);
  const double b = rz_acc;
  double ga, gb;
  if (group_reduce(P, cta_sum(a, red), two ? cta_sum(b, red) : 0.0, two, red, &flag, ga, gb)) {
    if (threadIdx.x == 0) {
      // slot g was last written by an earlier launch on another SM: read it
      // from L2, not from this SM's L1
      const int g = blockIdx.x / kGroup;
      if (MODE == M_FWD) P.acc_rr[g] = __ldcg(P.acc_rr + g) + ga;
      else if (MODE == M_BWD || !UPDATE) P.acc_rz[g] = __ldcg(P.acc_rz + g) + ga;
      else {
        P.acc_rr[g] = __ldcg(P.acc_rr + g) + ga;
        P.acc_rz[g] = __ldcg(P.acc_rz + g) + gb;
      }
    }
    if (fin != FIN_NONE && launch_last(P, &flag)) {
      if (fin == FIN_ITER) finish_iteration(P, red);
      else finish_init(P, red);
    }
  }
}

// ---------------------------------------------------------------------------
// SpMV-shaped kernel over 32R-row tiles of A_hat, one warp per tile
// ---------------------------------------------------------------------------
// mode 0: q = A (z + beta p_old), p_new = z + beta p_old, <p_new, q>; last group: alpha
// mode 1: r = b_hat - A x_hat, <r, r> group sums into gpq (solve start)
// mode 2: q = A x_hat (plain SpMV)
template <typename ZT, int R, int MODE>
__global__ void __launch_bounds__(kMaxWarpsPerCta * kWarp)
spmv_kernel(Params P, int cap) {
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[kMaxWarpsPerCta];
  __shared__ int flag;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
  double *sv; int32_t *sc; double *unused;
  warp_bufs<double>(smem, cap, 0, sv, sc, unused);
  const int T = kWarp * R;
  const int t0 = (blockIdx.x * W + warp) * T;
  double acc = 0.0;
  if (t0 < P.n) {
    const int t1 = min(P.n, t0 + T);
    int rb[R], re[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int i = t0 + lane + kWarp * k;
      rb[k] = i < t1 ? __ldg(P.arp + i) : 0;
      re[k] = i < t1 ? __ldg(P.arp + i + 1) : 0;
    }
    const int e0 = __shfl_sync(0xffffffffu, rb[0], 0);
    const int e1 = __ldg(P.arp + t1);
    const Seg<double> S = stage_async<double>(P.aval, P.acol, e0, e1, sv, sc, cap, lane);
    cp_wait_all();
    __syncwarp();
    pdl_wait();
    const ZT *z = reinterpret_cast<const ZT *>(P.z);
    double beta = 0.0;
    const double *pold = P.p0;
    double *pnew = P.p1;
    if (MODE == 0) {
      beta = __ldcg(&P.sc->beta);
      const int it = __ldcg(&P.sc->iter);
      pold = (it & 1) ? P.p1 : P.p0;
      pnew = (it & 1) ? P.p0 : P.p1;
    }
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int i = t0 + lane + kWarp * k;
      if (i < t1) {
        if (MODE == 0) {
          const double s = -row_sub<double, double>(S, rb[k], re[k], 0.0,
                                                    [&](int c) { return double(z[c]) + beta * pold[c]; });
          const double pi = double(z[i]) + beta * pold[i];
          pnew[i] = pi;
          P.q[i] = s;
          acc += pi * s;
        } else {
          const double s = -row_sub<double, double>(S, rb[k], re[k], 0.0, [&](int c) { return P.xh[c]; });
          if (MODE == 1) {
            const double ri = P.bh[i] - s;
            P.r[i] = ri;
            acc += ri * ri;
          } else {
            P.q[i] = s;
          }
        }
      }
    }
  } else {
    pdl_wait();
  }
  if (MODE == 2) return;
  double ga, gb;
  if (group_reduce(P, cta_sum(acc, red), 0.0, false, red, &flag, ga, gb)) {
    if (threadIdx.x == 0) P.gpq[blockIdx.x / kGroup] = ga;
    if (MODE == 0 && launch_last(P, &flag)) {
      const double pq = cta_sum_array(P.gpq, P.ngroup, red, true);
      if (threadIdx.x == 0) {
        P.sc->pq = pq;
        P.sc->alpha = P.sc->rz / pq;
      }
    }
  }
}

// b_hat = b[perm], x_hat = x0[perm], <b, b> partials into init_bb
__global__ void __launch_bounds__(kVecThreads) perm_in_kernel(Params P) {
  __shared__ double red[kMaxWarpsPerCta];
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
    const int o = P.perm[i];
    const double b = P.bin[o];
    P.bh[i] = b;
    P.xh[i] = P.xin[o];
    acc += b * b;
  }
  const double tot = cta_sum(acc, red);
  if (threadIdx.x == 0) P.init_bb[blockIdx.x] = tot;
}

// x[perm[i]] = x_hat[i] (x = 0 when b = 0)
__global__ void __launch_bounds__(kVecThreads) perm_out_kernel(Params P) {
  const bool zero = P.sc->bnorm == 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x)
    P.xout[P.perm[i]] = zero ? 0.0 : P.xh[i];
}

__global__ void __launch_bounds__(kVecThreads) permute_kernel(const double *src, double *dst, const int32_t *perm,
                                                              int n, int gather) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (gather) dst[i] = src[perm[i]];
    else dst[perm[i]] = src[i];
  }
}

__global__ void __launch_bounds__(kVecThreads) widen_kernel(const float *src, double *dst, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = double(src[i]);
}

// ---------------------------------------------------------------------------
// IC(0) (up-looking, one row per lane, rows of a tile level by level)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void factor_row(const Params &P, int i) {
  const int rb = P.lrp[i], re = P.lrp[i + 1];
  double d = P.adiag[i];
  for (int p = rb; p < re; ++p) {
    const int j = P.lcol[p];
    double s = P.ainit[p];
    int a = rb, b = P.lrp[j];
    const int be = P.lrp[j + 1];
    while (a < p && b < be) {
      const int ca = P.lcol[a], cb = P.lcol[b];
      if (ca == cb) { s -= P.lval[a] * P.lval[b]; ++a; ++b; }
      else if (ca < cb) ++a;
      else ++b;
    }
    const double lij = s / P.ldiag[j];
    P.lval[p] = lij;
    d -= lij * lij;
  }
  if (!(d > 0.0) || !isfinite(d)) {
    atomicMin(P.err_row, (unsigned long long)i);
    d = 1.0;
  }
  P.ldiag[i] = sqrt(d);
}

__global__ void __launch_bounds__(kMaxWarpsPerCta * kWarp) factor_color_kernel(Params P, int task0, int task1) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
  const int task = task0 + blockIdx.x * W + warp;
  if (task >= task1) return;
  const TaskDesc t = P.tasks[task];
  for (int tl = t.tile0; tl < t.tile0 + t.ntiles; ++tl) {
    const TileDesc d = P.tdesc[tl];
    const int rounds = d.rounds & 0xffff;
    for (int lv = 0; lv < rounds; ++lv) {
      for (int i = d.r0 + lane; i < d.r1; i += kWarp)
        if (P.lev[i] == lv) factor_row(P, i);
      __syncwarp();
    }
  }
}

// invd = 1/L_ii, U values mirrored from L, FP32 copies
__global__ void __launch_bounds__(kVecThreads) factor_finish_kernel(Params P, int nL) {
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += stride) {
    const double iv = 1.0 / P.ldiag[i];
    P.invd[i] = iv;
    P.invd32[i] = float(iv);
  }
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < nL; u += stride) {
    const double lv = P.lval[P.umap[u]];
    P.uval[u] = lv;
    P.uval32[u] = float(lv);
    P.lval32[u] = float(P.lval[u]);
  }
}

// ---------------------------------------------------------------------------
// launch helpers
// ---------------------------------------------------------------------------
template <typename... KArgs, typename... Args>
cudaError_t launch(void (*kernel)(KArgs...), int grid, int threads, int smem, const Plan &L, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(grid));
  cfg.blockDim = dim3(unsigned(threads));
  cfg.dynamicSmemBytes = size_t(smem);
  cfg.stream = L.stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = L.pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <typename PT, int R>
cudaError_t launch_fwd(const Params &P, const Plan &L, int c, bool update, bool fused, int fin) {
  const int threads = L.W * kWarp;
  const int cap = fused ? max(P.cap_l, P.cap_u) : P.cap_l;
  const int smem = fused ? L.smem_fused : L.smem_fwd;
  const int g = L.grid_c[c], t0 = L.task0[c], t1 = L.task1[c];
  if (update) {
    if (fused) return launch(color_kernel<PT, R, M_FUSED, true>, g, threads, smem, L, P, t0, t1, cap, fin);
    return launch(color_kernel<PT, R, M_FWD, true>, g, threads, smem, L, P, t0, t1, cap, fin);
  }
  if (fused) return launch(color_kernel<PT, R, M_FUSED, false>, g, threads, smem, L, P, t0, t1, cap, fin);
  return launch(color_kernel<PT, R, M_FWD, false>, g, threads, smem, L, P, t0, t1, cap, fin);
}

template <typename PT, int R>
cudaError_t launch_bwd(const Params &P, const Plan &L, int c, int fin) {
  return launch(color_kernel<PT, R, M_BWD, false>, L.grid_c[c], L.W * kWarp, L.smem_bwd, L, P, L.task0[c],
                L.task1[c], P.cap_u, fin);
}

// Forward sweep (with or without the x/r update), fused last color, backward
// sweep.  fin_last: the epilogue run by the last launch.
template <typename PT, int R>
cudaError_t sweep(const Params &P, const Plan &L, bool update, int fin_last, PhaseHook h, void *u) {
  cudaError_t e = cudaSuccess;
  const int nc = L.n_c;
  for (int c = 0; c < nc - 1 && e == cudaSuccess; ++c) {
    if (h) h(u, PH_FWD, 1);
    e = launch_fwd<PT, R>(P, L, c, update, false, FIN_NONE);
    if (h) h(u, PH_FWD, 0);
  }
  if (e != cudaSuccess) return e;
  if (h) h(u, PH_FUSED, 1);
  e = launch_fwd<PT, R>(P, L, nc - 1, update, true, nc == 1 ? fin_last : FIN_NONE);
  if (h) h(u, PH_FUSED, 0);
  for (int c = nc - 2; c >= 0 && e == cudaSuccess; --c) {
    if (h) h(u, PH_BWD, 1);
    e = launch_bwd<PT, R>(P, L, c, c == 0 ? fin_last : FIN_NONE);
    if (h) h(u, PH_BWD, 0);
  }
  return e;
}

template <typename ZT, int R, int MODE>
cudaError_t launch_spmv(const Params &P, const Plan &L) {
  return launch(spmv_kernel<ZT, R, MODE>, L.grid_a, L.W * kWarp, L.smem_a, L, P, P.cap_a);
}

template <typename F>
cudaError_t by_R(int R, F &&f) {
  switch (R) {
    case 1: return f(std::integral_constant<int, 1>());
    case 2: return f(std::integral_constant<int, 2>());
    case 4: return f(std::integral_constant<int, 4>());
    default: return cudaErrorInvalidValue;
  }
}

template <typename K>
cudaError_t allow_smem(K kernel) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - 1024);
}

template <typename PT, int R>
cudaError_t configure_pr() {
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = allow_smem(color_kernel<PT, R, M_FUSED, true>);
  if (e == cudaSuccess) e = allow_smem(color_kernel<PT, R, M_FWD, true>);
  if (e == cudaSuccess) e = allow_smem(color_kernel<PT, R, M_FUSED, false>);
  if (e == cudaSuccess) e = allow_smem(color_kernel<PT, R, M_FWD, false>);
  if (e == cudaSuccess) e = allow_smem(color_kernel<PT, R, M_BWD, false>);
  if (e == cudaSuccess) e = allow_smem(spmv_kernel<PT, R, 0>);
  if (e == cudaSuccess) e = allow_smem(spmv_kernel<PT, R, 1>);
  if (e == cudaSuccess) e = allow_smem(spmv_kernel<PT, R, 2>);
  return e;
}

}  // namespace

int warp_smem_bytes(int cap, int R, int elem) { return warp_bytes1(cap, R, elem); }

cudaError_t configure_kernels() {
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = configure_pr<double, 1>();
  if (e == cudaSuccess) e = configure_pr<double, 2>();
  if (e == cudaSuccess) e = configure_pr<double, 4>();
  if (e == cudaSuccess) e = configure_pr<float, 1>();
  if (e == cudaSuccess) e = configure_pr<float, 2>();
  if (e == cudaSuccess) e = configure_pr<float, 4>();
  return e;
}

cudaError_t launch_factor(const Params &P, const Plan &L, int nL) {
  for (int c = 0; c < L.n_c; ++c) {
    factor_color_kernel<<<L.grid_c[c], L.W * kWarp, 0, L.stream>>>(P, L.task0[c], L.task1[c]);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  factor_finish_kernel<<<L.grid_v, kVecThreads, 0, L.stream>>>(P, nL);
  return cudaGetLastError();
}

cudaError_t launch_solve_init(const Params &P, const Plan &L, bool fp32, PhaseHook h, void *u) {
  if (h) h(u, PH_INIT, 1);
  cudaError_t e = cudaMemsetAsync(P.acc_rr, 0, sizeof(double) * size_t(P.ngroup), L.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(P.acc_rz, 0, sizeof(double) * size_t(P.ngroup), L.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(P.gpq, 0, sizeof(double) * size_t(P.ngroup), L.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(P.gticket, 0, sizeof(uint32_t) * size_t(P.ngroup), L.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(P.p0, 0, sizeof(double) * size_t(P.n > 0 ? P.n : 1), L.stream);
  if (e == cudaSuccess) {
    perm_in_kernel<<<L.grid_v, kVecThreads, 0, L.stream>>>(P);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = by_R(L.R, [&](auto RC) { return launch_spmv<double, decltype(RC)::value, 1>(P, L); });
  if (h) h(u, PH_INIT, 0);
  if (e != cudaSuccess) return e;
  if (h) h(u, PH_INIT, 1);
  if (fp32) e = by_R(L.R, [&](auto RC) { return sweep<float, decltype(RC)::value>(P, L, false, FIN_INIT, nullptr, nullptr); });
  else e = by_R(L.R, [&](auto RC) { return sweep<double, decltype(RC)::value>(P, L, false, FIN_INIT, nullptr, nullptr); });
  if (h) h(u, PH_INIT, 0);
  return e;
}

cudaError_t launch_solve_body(const Params &P, const Plan &L, bool fp32, PhaseHook h, void *u) {
  cudaError_t e;
  if (h) h(u, PH_SPMV, 1);
  if (fp32) e = by_R(L.R, [&](auto RC) { return launch_spmv<float, decltype(RC)::value, 0>(P, L); });
  else e = by_R(L.R, [&](auto RC) { return launch_spmv<double, decltype(RC)::value, 0>(P, L); });
  if (h) h(u, PH_SPMV, 0);
  if (e != cudaSuccess) return e;
  if (fp32) return by_R(L.R, [&](auto RC) { return sweep<float, decltype(RC)::value>(P, L, true, FIN_ITER, h, u); });
  return by_R(L.R, [&](auto RC) { return sweep<double, decltype(RC)::value>(P, L, true, FIN_ITER, h, u); });
}

cudaError_t launch_solve_final(const Params &P, const Plan &L) {
  perm_out_kernel<<<L.grid_v, kVecThreads, 0, L.stream>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_precond(const Params &P, const Plan &L, bool fp32) {
  if (fp32) return by_R(L.R, [&](auto RC) { return sweep<float, decltype(RC)::value>(P, L, false, FIN_NONE, nullptr, nullptr); });
  return by_R(L.R, [&](auto RC) { return sweep<double, decltype(RC)::value>(P, L, false, FIN_NONE, nullptr, nullptr); });
}

cudaError_t launch_spmv_plain(const Params &P, const Plan &L) {
  return by_R(L.R, [&](auto RC) { return launch_spmv<double, decltype(RC)::value, 2>(P, L); });
}

cudaError_t launch_permute(const double *src, double *dst, const int32_t *perm, int32_t n, bool gather,
                           int32_t grid, cudaStream_t s) {
  permute_kernel<<<grid, kVecThreads, 0, s>>>(src, dst, perm, n, gather ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_widen(const float *src, double *dst, int32_t n, int32_t grid, cudaStream_t s) {
  widen_kernel<<<grid, kVecThreads, 0, s>>>(src, dst, n);
  return cudaGetLastError();
}

}  // namespace iccg
