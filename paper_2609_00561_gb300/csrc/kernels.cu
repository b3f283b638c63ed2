// Device kernels of block-multicolor ICCG for sm_103a.
//
// One PCG iteration is 2*n_c + 1 launches (n_c = number of block colors):
//   p update             p = z + beta p
//   spmv                 q = A p, <p,q>; its last group sets alpha = (r,z)/(p,q)
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
// Substitution work mapping.  One warp owns a group: consecutive whole blocks
// of one color (at most 32R rows), or one block larger than that.  Blocks of
// one color share no edge, so the group's rows depend on earlier colors and
// on earlier rows of their own block only.  The warp works in two phases:
//   A  every row at once, one row per lane: the entries that point to earlier
//      colors (y or z gathers) and the fused x / r update;
//   B  the in-block dependencies, level by level: the rows of all the group's
//      blocks are listed by their depth in their block's dependency DAG, and
//      each level is processed with the rows packed across lanes, so every row
//      is computed exactly once and the FP64 lanes are mostly busy.  The
//      per-row arithmetic is the row of Alg. 1 (earlier-color terms first).
// GB300's FP64 FMA rate is 2 lanes/cycle/SM, so a DFMA issued with idle lanes
// costs as much as a full one; this packing is what keeps the FP64 pipe from
// becoming the bound.
//
// Memory: a fitting group's CSR segment of L or U, its row pointers, 1/L_ii,
// schedule and level pointers are copied into the warp's shared memory with
// cp.async (16-byte, L2 only, all in flight at once) before the kernel waits
// on its predecessor (programmatic dependent launch: griddepcontrol.wait), so
// this static traffic overlaps the previous launch.  A group too large for the
// shared-memory plan reads the same data from global memory.
//
// Vectors that other CTAs write during a solve (r, q, x, p, y, z) are read
// with L2 loads (ld.global.cg), so no SM ever sees a stale L1 line of them.
//
// Reductions are deterministic and two-level: every CTA writes its partial;
// the last CTA of each group of kGroup CTAs (arrival ticket) sums the group's
// partials in index order; the last group of the launch runs the epilogue.
#include <algorithm>
#include <cstdio>
#include <type_traits>

#include "iccg_internal.h"

namespace iccg {

namespace {

constexpr int kVecThreads = 256;
constexpr int kChunk = 4;    // row entries processed per predicated batch
enum StepMode { M_FWD = 0, M_BWD = 1, M_FUSED = 2 };

__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
// 4- and 8-byte copies (.ca: cached in L1 as well)
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
}
template <typename PT>
__device__ __forceinline__ void cp_async_elem(PT *smem, const PT *gmem);
template <> __device__ __forceinline__ void cp_async_elem<double>(double *smem, const double *gmem) {
  cp_async8(smem, gmem);
}
template <> __device__ __forceinline__ void cp_async_elem<float>(float *smem, const float *gmem) {
  cp_async4(smem, gmem);
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
// all but the most recently committed group
__device__ __forceinline__ void cp_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// sum over the warp, valid in lane 0: each step adds on the lower half of
// the lanes still in play (16, 8, 4, 2, 1), since FP64 adds are the scarce
// resource on this GPU
__device__ __forceinline__ double warp_sum(double v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double u = __shfl_down_sync(0xffffffffu, v, o);
    // a predicated add (the compiler would otherwise add on every lane and select)
    asm("{\n\t.reg .pred p;\n\tsetp.lt.s32 p, %1, %2;\n\t@p add.rn.f64 %0, %0, %3;\n\t}"
        : "+d"(v)
        : "r"(lane), "r"(o), "d"(u));
  }
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

// A CSR segment: staged in shared memory (entry e at sv[e - bv], sc[e - bc])
// or read from global memory.
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

// Issue the cp.async copies of the 16-byte-aligned cover of g[a, b) into s;
// returns the index of s[0] in g.  Device arrays carry 64 bytes of padding,
// so the cover stays inside the allocation; s needs (b - a) + 2 * (16 /
// sizeof(T)) elements.
template <typename T>
__device__ __forceinline__ int stage_cover(const T *g, int a, int b, T *s, int tid, int nthr) {
  constexpr int EV = 16 / sizeof(T);
  const int a0 = a & ~(EV - 1), a1 = (b + EV - 1) & ~(EV - 1);
  const int nv = (a1 - a0) / EV;
  for (int k = tid; k < nv; k += nthr) cp_async16(s + k * EV, g + a0 + k * EV);
  return a0;
}

// count of entries of [rb, re) whose column is below `bound` (columns sorted)
template <typename VT>
__device__ __forceinline__ int count_below(const Seg<VT> &S, int rb, int re, int bound) {
  int n = 0;
  for (int e = rb; e < re; ++e) n += S.c(e) < bound ? 1 : 0;
  return n;
}

// acc -= sum of v_e * x(c_e) over the entries e in [rb, re), ascending;
// loads in predicated batches of kChunk, then the FMAs of the batch.
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
    for (int j = 0; j < kChunk; ++j)
      if (cc[j] >= 0) acc -= AT(vv[j]) * xx[j];
  }
  return acc;
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

// ---------------------------------------------------------------------------
// per-CTA shared memory of the substitution kernels (one CTA per group)
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ int r16(int bytes) { return (bytes + 15) & ~15; }

struct GroupSmemPlan {
  int o_sv, o_sc, o_rp, o_dv, o_sch, o_lp, o_w, o_spl, total;
};

__host__ __device__ __forceinline__ GroupSmemPlan group_smem_plan(int cap, int rows, int levs, int elem) {
  GroupSmemPlan p;
  int o = 0;
  p.o_sv = o; o += r16((cap + 8) * elem);
  p.o_sc = o; o += r16((cap + 8) * 4);
  p.o_rp = o; o += r16((rows + 9) * 4);
  p.o_dv = o; o += r16((rows + 8) * elem);
  p.o_sch = o; o += r16((rows + 8) * 4);
  p.o_lp = o; o += r16((levs + 9) * 4);
  p.o_w = o; o += r16(rows * elem);
  p.o_spl = o; o += r16(rows * 4);
  p.total = o;
  return p;
}

template <typename PT>
struct GroupSmem {
  PT *sv;
  int32_t *sc, *rp, *sch, *lp, *spl;
  PT *dv, *w;
};

template <typename PT>
__device__ __forceinline__ GroupSmem<PT> group_smem(unsigned char *base, const GroupSmemPlan &p) {
  unsigned char *m = base;
  GroupSmem<PT> s;
  s.sv = reinterpret_cast<PT *>(m + p.o_sv);
  s.sc = reinterpret_cast<int32_t *>(m + p.o_sc);
  s.rp = reinterpret_cast<int32_t *>(m + p.o_rp);
  s.dv = reinterpret_cast<PT *>(m + p.o_dv);
  s.sch = reinterpret_cast<int32_t *>(m + p.o_sch);
  s.lp = reinterpret_cast<int32_t *>(m + p.o_lp);
  s.w = reinterpret_cast<PT *>(m + p.o_w);
  s.spl = reinterpret_cast<int32_t *>(m + p.o_spl);
  return s;
}

__device__ __forceinline__ GroupDesc load_group(const GroupDesc *g) {
  const int4 *p = reinterpret_cast<const int4 *>(g);
  const int4 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
  GroupDesc d;
  d.r0 = a.x; d.r1 = a.y; d.l0 = a.z; d.l1 = a.w;
  d.u0 = b.x; d.u1 = b.y; d.lf = b.z; d.lb = b.w;
  d.nlf = c.x; d.nlb = c.y; d.fit = c.z;
  return d;
}

// Where the static data of one sweep over a group lives (shared memory for a
// fitting group, global memory otherwise).
template <typename PT>
struct Sweep {
  Seg<PT> S;
  bool fit;
  int rpb, dvb, schb, lpb;       // index of the first staged element
  const int32_t *grp, *gsch;     // global row pointers / schedule
  const PT *gdv;
  int lev0, nlev;                // level pointers at levp[lev0 ..]
  __device__ __forceinline__ int rp(const GroupSmem<PT> &m, int i) const { return fit ? m.rp[i - rpb] : __ldg(grp + i); }
  __device__ __forceinline__ PT dv(const GroupSmem<PT> &m, int i) const { return fit ? m.dv[i - dvb] : __ldg(gdv + i); }
};

// index of the first element of the 16-byte-aligned cover that stage_cover copies
template <typename T>
__device__ __forceinline__ int cover_base(int a) { return a & ~(int(16 / sizeof(T)) - 1); }

// Describe where the static data of a forward (upper = false) or backward
// (upper = true) sweep over group d lives once sweep_issue's copies landed.
template <typename PT>
__device__ __forceinline__ Sweep<PT> sweep_desc(const Params &P, const GroupDesc &d, bool upper,
                                                const GroupSmem<PT> &m) {
  Sweep<PT> sw;
  sw.fit = d.fit != 0;
  sw.grp = upper ? P.urp : P.lrp;
  sw.gsch = upper ? P.sched_b : P.sched_f;
  sw.gdv = invds<PT>(P);
  sw.lev0 = upper ? d.lb : d.lf;
  sw.nlev = upper ? d.nlb : d.nlf;
  sw.S.gv = upper ? uvals<PT>(P) : lvals<PT>(P);
  sw.S.gc = upper ? P.ucol : P.lcol;
  sw.S.sv = m.sv;
  sw.S.sc = m.sc;
  sw.S.staged = sw.fit;
  sw.S.bv = sw.S.bc = 0;
  sw.rpb = sw.dvb = sw.schb = sw.lpb = 0;
  if (sw.fit) {
    const int e0 = upper ? d.u0 : d.l0;
    sw.S.bv = cover_base<PT>(e0);
    sw.S.bc = cover_base<int32_t>(e0);
    sw.rpb = cover_base<int32_t>(d.r0);
    sw.dvb = cover_base<PT>(d.r0);
    sw.schb = cover_base<int32_t>(d.r0);
    sw.lpb = cover_base<int32_t>(sw.lev0);
  }
  return sw;
}

// Issue (without committing) the cp.async copies of a fitting group's static
// sweep data into m; nothing for a group that reads global memory.
template <typename PT>
__device__ __forceinline__ void sweep_issue(const Params &P, const GroupDesc &d, bool upper, const GroupSmem<PT> &m,
                                            int tid, int nthr) {
  if (!d.fit) return;
  const int e0 = upper ? d.u0 : d.l0, e1 = upper ? d.u1 : d.l1;
  const int lev0 = upper ? d.lb : d.lf, nlev = upper ? d.nlb : d.nlf;
  stage_cover<PT>(upper ? uvals<PT>(P) : lvals<PT>(P), e0, e1, m.sv, tid, nthr);
  stage_cover<int32_t>(upper ? P.ucol : P.lcol, e0, e1, m.sc, tid, nthr);
  stage_cover<int32_t>(upper ? P.urp : P.lrp, d.r0, d.r1 + 1, m.rp, tid, nthr);
  stage_cover<PT>(invds<PT>(P), d.r0, d.r1, m.dv, tid, nthr);
  stage_cover<int32_t>(upper ? P.sched_b : P.sched_f, d.r0, d.r1, m.sch, tid, nthr);
  stage_cover<int32_t>(P.levp, lev0, lev0 + nlev + 1, m.lp, tid, nthr);
}

// Stage and describe the static data of one sweep; commits the copies, the
// caller waits.
template <typename PT>
__device__ __forceinline__ Sweep<PT> sweep_static(const Params &P, const GroupDesc &d, bool upper,
                                                  const GroupSmem<PT> &m, int tid, int nthr) {
  sweep_issue<PT>(P, d, upper, m, tid, nthr);
  cp_commit();
  return sweep_desc<PT>(P, d, upper, m);
}

// One sweep over a group.  UPPER = false: forward, L rows (entries to earlier
// colors are a prefix of each row, in-block entries the rest); the source is
// r (with the x / r update when UPDATE) and the result y.  UPPER = true:
// backward, U rows (in-block entries a prefix, later colors the rest); the
// source is y (from `ysrc`: shared memory when the fused kernel keeps y of a
// fitting group there) and the result z, with <r, z>.
// Fitting groups keep t / y / z in m.w; other groups work in place in the
// global result vector.
template <typename PT, bool UPPER, bool UPDATE>
__device__ __forceinline__ void group_sweep(const Params &P, const GroupDesc &d, const Sweep<PT> &sw,
                                            const GroupSmem<PT> &m, int tid, int nthr, double alpha,
                                            const double *pn, bool y_in_smem, bool store_result, double &rr_acc,
                                            double &rz_acc) {
  PT *yv = reinterpret_cast<PT *>(P.y);
  PT *zv = reinterpret_cast<PT *>(P.z);
  PT *res = UPPER ? zv : yv;        // global result vector
  const PT *ext = UPPER ? zv : yv;  // gathered for out-of-group columns
  const int r0 = d.r0, r1 = d.r1, nrows = r1 - r0;
  const bool fit = sw.fit;
  // phase A: out-of-group entries, all rows at once (one row per thread)
  for (int l = tid; l < nrows; l += nthr) {
    const int i = r0 + l;
    const int rb = sw.rp(m, i), re = sw.rp(m, i + 1);
    PT src;
    if (UPPER) {
      src = y_in_smem ? m.w[l] : __ldcg(yv + i);
    } else {
      double ri = __ldcg(P.r + i);
      if (UPDATE) {
        ri -= alpha * __ldcg(P.q + i);
        P.r[i] = ri;
        P.xh[i] = __ldcg(P.xh + i) + alpha * __ldcg(pn + i);
        rr_acc += ri * ri;
      }
      src = PT(ri);
    }
    const int split = rb + count_below(sw.S, rb, re, UPPER ? r1 : r0);
    const int xb = UPPER ? split : rb, xe = UPPER ? re : split;
    const PT t = row_sub<PT, PT>(sw.S, xb, xe, src, [&](int c) { return __ldcg(ext + c); });
    if (fit) {
      m.w[l] = t;
      m.spl[l] = split;
    } else {
      res[i] = t;
    }
  }
  __syncthreads();
  // phase B: in-block entries, level by level; a level's rows go to the
  // first threads, so only as many warps as the level needs issue FP64 work
  for (int lv = 0; lv < sw.nlev; ++lv) {
    const int p0 = fit ? m.lp[sw.lev0 + lv - sw.lpb] : __ldg(P.levp + sw.lev0 + lv);
    const int p1 = fit ? m.lp[sw.lev0 + lv + 1 - sw.lpb] : __ldg(P.levp + sw.lev0 + lv + 1);
    for (int p = p0 + tid; p < p1; p += nthr) {
      const int l = fit ? m.sch[r0 + p - sw.schb] : __ldg(sw.gsch + r0 + p);
      const int i = r0 + l;
      const int rb = sw.rp(m, i), re = sw.rp(m, i + 1);
      int ib, ie;
      PT acc;
      if (fit) {
        acc = m.w[l];
        ib = UPPER ? rb : m.spl[l];
        ie = UPPER ? m.spl[l] : re;
        acc = row_sub<PT, PT>(sw.S, ib, ie, acc, [&](int c) { return m.w[c - r0]; });
        m.w[l] = acc * sw.dv(m, i);
      } else {
        acc = __ldcg(res + i);
        const int split = rb + count_below(sw.S, rb, re, UPPER ? r1 : r0);
        ib = UPPER ? rb : split;
        ie = UPPER ? split : re;
        acc = row_sub<PT, PT>(sw.S, ib, ie, acc, [&](int c) { return __ldcg(res + c); });
        res[i] = acc * sw.dv(m, i);
      }
    }
    __syncthreads();
  }
  // results: fitting groups store from shared memory (coalesced)
  for (int l = tid; l < nrows; l += nthr) {
    const int i = r0 + l;
    const PT v = fit ? m.w[l] : __ldcg(res + i);
    if (fit && store_result) res[i] = v;
    if (UPPER) rz_acc += __ldcg(P.r + i) * double(v);
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// epilogues run by the last group of a launch
// ---------------------------------------------------------------------------
__device__ void set_condition(const Scalars *s, int keep_going) {
  if (s->use_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)s->cond_handle, keep_going ? 1u : 0u);
}

// After the backward sweep of iteration k: residual history, stop test, beta.
// rr, rz valid in thread 0.
__device__ void finish_iteration(const Params &P, double rr, double rz) {
  if (threadIdx.x == 0) {
    Scalars *s = P.sc;
    const int k = s->iter;
    const double rn = sqrt(rr) / s->bnorm;
    P.hist[k + 1] = rn;
    s->iter = k + 1;
    s->rr = rr;
    int done = 0;
    // a bounded wait of this iteration gave up (a cooperative launch of the
    // sweep): the solve stops with that status
    if (s->status == ICCG_ERR_TIMEOUT) done = 1;
    else if (!isfinite(rn) || !isfinite(rz)) { s->status = ICCG_ERR_NONFINITE; done = 1; }
    else if (rn <= s->tol) { s->status = ICCG_OK; done = 1; }
    else if (k + 1 >= s->maxit) { s->status = ICCG_NOT_CONVERGED; done = 1; }
    else { s->beta = rz / s->rz; s->rz = rz; }
    s->done = done;
    set_condition(s, !done);
  }
}

// After r0 = b - A x0 and z0 = M^-1 r0: ||b||, history[0], stop test.
// init_bb holds <b,b> partials, part_a the <r0,r0> partials; rz valid in
// thread 0.
__device__ void finish_init(const Params &P, double rz, double *red) {
  const double bb = cta_sum_array(P.init_bb, P.nbb, red, false);
  const double rr = cta_sum_array(P.part_a, P.npart_a, red, false);
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
    if (s->status == ICCG_ERR_TIMEOUT) done = 1;
    else if (bn == 0.0) { P.hist[0] = 0.0; s->status = ICCG_OK; done = 1; }
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
// color, or both for the last color (fused); one CTA per group
// ---------------------------------------------------------------------------
struct SlotArgs {
  int off_rr, off_rz;     // this launch's slot regions
  int last_rr, last_rz;   // slots of earlier launches (final launch only)
};

// End of a color launch: this CTA's <r,r> / <r,z> partials.  A non-final
// launch stores one partial per CTA in its slot region (plain stores: the
// iteration's last launch sums them).  The last launch of the iteration:
// every CTA sums a fixed chunk of the earlier launches' slots (complete:
// griddepcontrol.wait before) plus its own partial; then groups of CTAs, then
// the last group runs the epilogue.
__device__ __forceinline__ void launch_epilogue(const Params &P, int fin, const SlotArgs &sa, bool has_rr,
                                                bool has_rz, double rr_acc, double rz_acc, double *red, int *flag) {
  if (!has_rr && !has_rz) return;
  if (fin == FIN_NONE) {
    const double rr_c = has_rr ? cta_sum(rr_acc, red) : 0.0;
    const double rz_c = has_rz ? cta_sum(rz_acc, red) : 0.0;
    if (threadIdx.x == 0) {
      if (has_rr) P.slot_rr[sa.off_rr + blockIdx.x] = rr_c;
      if (has_rz) P.slot_rz[sa.off_rz + blockIdx.x] = rz_c;
    }
    return;
  }
  // the final launch: this CTA's share of the earlier launches' slots joins
  // the threads' own partial sums, then one CTA sum per quantity
  const int nb = gridDim.x;
  const int crr = (sa.last_rr + nb - 1) / nb, crz = (sa.last_rz + nb - 1) / nb;
  double a = has_rr ? rr_acc : 0.0, b = has_rz ? rz_acc : 0.0;
  for (int k = threadIdx.x; k < crr; k += blockDim.x) {
    const int idx = blockIdx.x * crr + k;
    if (idx < sa.last_rr) a += __ldcg(P.slot_rr + idx);
  }
  for (int k = threadIdx.x; k < crz; k += blockDim.x) {
    const int idx = blockIdx.x * crz + k;
    if (idx < sa.last_rz) b += __ldcg(P.slot_rz + idx);
  }
  // a quantity that only the first warp holds (slots alone, at most 32 per
  // CTA) is summed by that warp
  if (!has_rr && crr <= kWarp) {
    if (threadIdx.x < kWarp) a = warp_sum(a);
  } else {
    a = cta_sum(a, red);
  }
  if (!has_rz && crz <= kWarp) {
    if (threadIdx.x < kWarp) b = warp_sum(b);
  } else {
    b = cta_sum(b, red);
  }
  double ga, gb;
  if (group_reduce(P, a, b, true, red, flag, ga, gb)) {
    if (threadIdx.x == 0) {
      P.gsum0[blockIdx.x / kGroup] = ga;
      P.gsum1[blockIdx.x / kGroup] = gb;
    }
    if (launch_last(P, flag)) {
      const int ng = (nb + kGroup - 1) / kGroup;
      const double rr = cta_sum_array(P.gsum0, ng, red, false);
      const double rz = cta_sum_array(P.gsum1, ng, red, false);
      if (fin == FIN_ITER) finish_iteration(P, rr, rz);
      else finish_init(P, rz, red);
    }
  }
}

template <typename PT, int MODE, bool UPDATE>
__global__ void __launch_bounds__(kMaxWarpsPerCta * kWarp)
color_kernel(Params P, int g0, int g1, GroupSmemPlan plan, int fin, SlotArgs sa) {
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[kMaxWarpsPerCta];
  __shared__ int flag;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const GroupSmem<PT> m = group_smem<PT>(smem, plan);
  double rr_acc = 0.0, rz_acc = 0.0;
  const int g = g0 + blockIdx.x;
  if (g < g1) {
    const GroupDesc d = load_group(P.groups + g);
    const Sweep<PT> sw = sweep_static<PT>(P, d, MODE == M_BWD, m, tid, nthr);
    cp_wait_all();
    __syncthreads();
    pdl_wait();
    if (MODE == M_BWD) {
      group_sweep<PT, true, false>(P, d, sw, m, tid, nthr, 0.0, nullptr, false, true, rr_acc, rz_acc);
    } else {
      double alpha = 0.0;
      const double *pn = P.p0;
      if (UPDATE) alpha = __ldcg(&P.sc->alpha);
      group_sweep<PT, false, UPDATE>(P, d, sw, m, tid, nthr, alpha, pn, false, MODE == M_FWD || !sw.fit,
                                     rr_acc, rz_acc);
      if (MODE == M_FUSED) {
        // the last color: y of a fitting group stays in shared memory; the
        // backward sweep restages the U side (the schedule changes, 1/L_ii
        // stays)
        const bool keep = sw.fit;
        const Sweep<PT> su = sweep_static<PT>(P, d, true, m, tid, nthr);
        cp_wait_all();
        __syncthreads();
        group_sweep<PT, true, false>(P, d, su, m, tid, nthr, 0.0, nullptr, keep, true, rr_acc, rz_acc);
      }
    }
  } else {
    pdl_wait();
  }
  launch_epilogue(P, fin, sa, MODE != M_BWD && UPDATE, MODE != M_FWD, rr_acc, rz_acc, red, &flag);
}

// ---------------------------------------------------------------------------
// lane-tile kernels: one CTA per tile of up to 32 blocks of one color, one
// block per lane (Alg. 1: blocks of a color in parallel, rows of a block in
// sequence).  Step k of the tile is the k-th row of every block; its 32 rows
// are consecutive.
//   A  all warps, steps in parallel: the x / r update, the entries to other
//      colors (gathers of y or z), 1/L_ii and the step's in-block entries
//      into shared memory;
//   B  one warp: the in-block recurrence, step after step, every lane on its
//      own block, shared memory only (no barrier inside);
//   C  all warps: results to global memory, <r,z>.
// ---------------------------------------------------------------------------
template <typename PT> __device__ __forceinline__ const PT *slv(const Params &P);
template <> __device__ __forceinline__ const double *slv<double>(const Params &P) { return P.sl_val; }
template <> __device__ __forceinline__ const float *slv<float>(const Params &P) { return P.sl_val32; }
template <typename PT> __device__ __forceinline__ const PT *suv(const Params &P);
template <> __device__ __forceinline__ const double *suv<double>(const Params &P) { return P.su_val; }
template <> __device__ __forceinline__ const float *suv<float>(const Params &P) { return P.su_val32; }
template <typename PT> __device__ __forceinline__ const PT *siv(const Params &P);
template <> __device__ __forceinline__ const double *siv<double>(const Params &P) { return P.si_val; }
template <> __device__ __forceinline__ const float *siv<float>(const Params &P) { return P.si_val32; }
template <typename PT> __device__ __forceinline__ const PT *uiv(const Params &P);
template <> __device__ __forceinline__ const double *uiv<double>(const Params &P) { return P.ui_val; }
template <> __device__ __forceinline__ const float *uiv<float>(const Params &P) { return P.ui_val32; }

__device__ __forceinline__ TileDesc load_tile(const TileDesc *t) {
  const int4 *p = reinterpret_cast<const int4 *>(t);
  const int4 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2), d = __ldg(p + 3);
  TileDesc r;
  r.row0 = a.x; r.nrows = a.y; r.nsteps = a.z; r.step0 = a.w;
  r.lo0 = b.x; r.lo1 = b.y; r.li0 = b.z; r.li1 = b.w;
  r.uo0 = c.x; r.uo1 = c.y; r.ui0 = c.z; r.ui1 = c.w;
  r.wl = d.x; r.wu = d.y; r.lw0 = d.z; r.uw0 = d.w;
  return r;
}

// One staged buffer of a tile: step descriptors, 1/L_ii (index row - bdv),
// in-block entries of the first and second set (index entry - base).
template <typename PT>
struct TileBuf {
  const StepDesc *st;
  const PT *dv;
  const int32_t *ic, *ic2;
  const PT *iv, *iv2;
  const int32_t *oc;     // other-color entries (cap_o > 0)
  const PT *ov;
  const double *vec;     // four row vectors of (cap_r + 8) doubles each
  int vstride;
};

template <typename PT>
__device__ __forceinline__ TileBuf<PT> tile_buf(unsigned char *smem, const TilePlan &pl, int size, int k) {
  unsigned char *b = smem + k * size;
  TileBuf<PT> t;
  t.st = reinterpret_cast<const StepDesc *>(b + pl.o_steps);
  t.dv = reinterpret_cast<const PT *>(b + pl.o_dv);
  t.ic = reinterpret_cast<const int32_t *>(b + pl.o_ic);
  t.iv = reinterpret_cast<const PT *>(b + pl.o_iv);
  t.ic2 = reinterpret_cast<const int32_t *>(b + pl.o_ic2);
  t.iv2 = reinterpret_cast<const PT *>(b + pl.o_iv2);
  t.oc = reinterpret_cast<const int32_t *>(b + pl.o_oc);
  t.ov = reinterpret_cast<const PT *>(b + pl.o_ov);
  t.vec = reinterpret_cast<const double *>(b + pl.o_vec);
  t.vstride = r16b((pl.cap_r + 8) * 8) / 8;
  return t;
}

// Whether tile t's other-color entries and row vectors are (to be) staged
__device__ __forceinline__ bool ext_staged(const TilePlan &pl, const TileDesc &t, bool upper) {
  const int n = upper ? t.uo1 - t.uo0 : t.lo1 - t.lo0;
  return pl.cap_o > 0 && n <= pl.cap_o && t.nrows <= pl.cap_r;
}

// Issue (no commit) the copies of tile t's static data into buffer tb:
// steps, 1/L_ii, in-block entries of L (FIRST_UPPER = false) or U, and of U
// as the second set when TWO; an in-block range larger than the capacity
// stays in global memory.
template <typename PT, bool FIRST_UPPER, bool TWO>
__device__ __forceinline__ void tile_stage(const Params &P, const TileDesc &t, const TileBuf<PT> &tb,
                                           const TilePlan &pl, int tid, int nthr) {
  const int cap_i = pl.cap_i, cap_i2 = pl.cap_i2;
  int4 *st = reinterpret_cast<int4 *>(const_cast<StepDesc *>(tb.st));
  const int4 *gs = reinterpret_cast<const int4 *>(P.steps + t.step0);
  for (int k = tid; k < t.nsteps * 3; k += nthr) cp_async16(st + k, gs + k);
  stage_cover<PT>(invds<PT>(P), t.row0, t.row0 + t.nrows, const_cast<PT *>(tb.dv), tid, nthr);
  // entries to other colors of the first sweep (static, like the above)
  if (ext_staged(pl, t, FIRST_UPPER)) {
    const int o0 = FIRST_UPPER ? t.uo0 : t.lo0, o1 = FIRST_UPPER ? t.uo1 : t.lo1;
    if (o1 > o0) {
      stage_cover<int32_t>(FIRST_UPPER ? P.su_col : P.sl_col, o0, o1, const_cast<int32_t *>(tb.oc), tid, nthr);
      stage_cover<PT>(FIRST_UPPER ? suv<PT>(P) : slv<PT>(P), o0, o1, const_cast<PT *>(tb.ov), tid, nthr);
    }
  }
  // a set is copied only into a region the launch has (capacity > 0) and
  // only when non-empty (the cover of an empty range is still 16 bytes)
  const int i0 = FIRST_UPPER ? t.ui0 : t.li0, i1 = FIRST_UPPER ? t.ui1 : t.li1;
  if (i1 > i0 && i1 - i0 <= cap_i) {
    stage_cover<int32_t>(FIRST_UPPER ? P.ui_col : P.si_col, i0, i1, const_cast<int32_t *>(tb.ic), tid, nthr);
    stage_cover<PT>(FIRST_UPPER ? uiv<PT>(P) : siv<PT>(P), i0, i1, const_cast<PT *>(tb.iv), tid, nthr);
  }
  if (TWO && t.ui1 > t.ui0 && t.ui1 - t.ui0 <= cap_i2) {
    stage_cover<int32_t>(P.ui_col, t.ui0, t.ui1, const_cast<int32_t *>(tb.ic2), tid, nthr);
    stage_cover<PT>(uiv<PT>(P), t.ui0, t.ui1, const_cast<PT *>(tb.iv2), tid, nthr);
  }
}

// Issue (no commit) the copies of the row vectors tile t's first sweep reads
// (r, q, x, p forward; y, r backward) when its entries are staged.  They come
// from earlier launches, so the first tile's are issued after
// griddepcontrol.wait; each tile's rows are written by that tile alone.
template <typename PT, bool FIRST_UPPER, bool UPD>
__device__ __forceinline__ void tile_stage_vec(const Params &P, const TileDesc &t, const TileBuf<PT> &tb,
                                               const TilePlan &pl, int tid, int nthr) {
  if (!ext_staged(pl, t, FIRST_UPPER)) return;
  double *v = const_cast<double *>(tb.vec);
  const int r0 = t.row0, r1 = t.row0 + t.nrows, vs = tb.vstride;
  if (FIRST_UPPER) {
    stage_cover<PT>(reinterpret_cast<const PT *>(P.y), r0, r1, reinterpret_cast<PT *>(v), tid, nthr);
    stage_cover<double>(P.r, r0, r1, v + vs, tid, nthr);
  } else {
    stage_cover<double>(P.r, r0, r1, v, tid, nthr);
    if (UPD) {
      stage_cover<double>(P.q, r0, r1, v + vs, tid, nthr);
      stage_cover<double>(P.xh, r0, r1, v + 2 * vs, tid, nthr);
      stage_cover<double>(P.p0, r0, r1, v + 3 * vs, tid, nthr);
    }
  }
}

// The in-block entries a tile's chain reads: staged (index entry - base) or
// the global arrays.
template <typename PT>
struct InBlock {
  const int32_t *ic;
  const PT *iv;
};

template <typename PT>
__device__ __forceinline__ InBlock<PT> in_block(const int32_t *sc, const PT *sv, const int32_t *gc, const PT *gv,
                                               int i0, int i1, int cap_i) {
  if (i1 > i0 && i1 - i0 <= cap_i) return InBlock<PT>{sc - cover_base<int32_t>(i0), sv - cover_base<PT>(i0)};
  return InBlock<PT>{gc, gv};
}

// acc -= sum over a step's sliced-ELL entries to other colors of v * g[col]
// (coalesced loads of the entries, then the gathers; FMAs only for the
// step's real width, a warp-uniform count; padding entries are (kPadCol, 0))
// (NC: col / val in global memory, read through the read-only path; else
// shared-memory copies, plain loads)
template <typename PT, bool NC = true>
__device__ __forceinline__ PT ext_sub(const int32_t *col, const PT *val, int e, int stride, int width, PT acc,
                                      const PT *g) {
  for (int j0 = 0; j0 < width; j0 += kChunk) {
    const int nj = min(kChunk, width - j0);
    int cc[kChunk];
    PT vv[kChunk], xx[kChunk];
#pragma unroll
    for (int j = 0; j < kChunk; ++j) {
      if (NC) {
        cc[j] = j < nj ? __ldg(col + e + (j0 + j) * stride) : kPadCol;
        vv[j] = j < nj ? __ldg(val + e + (j0 + j) * stride) : PT(0);
      } else {
        cc[j] = j < nj ? col[e + (j0 + j) * stride] : kPadCol;
        vv[j] = j < nj ? val[e + (j0 + j) * stride] : PT(0);
      }
    }
#pragma unroll
    for (int j = 0; j < kChunk; ++j) xx[j] = cc[j] == kPadCol ? PT(0) : __ldcg(g + cc[j]);
#pragma unroll
    for (int j = 0; j < kChunk; ++j)
      if (j < nj) acc -= vv[j] * xx[j];
  }
  return acc;
}

// Phase A: forward (UPPER = false; source r with the x / r update when
// UPDATE, gathers of y) or backward (source y from w or global memory,
// gathers of z); the partial row value goes to w[step][lane].
template <typename PT, bool UPPER, bool UPDATE>
__device__ __forceinline__ void tile_phase_a(const Params &P, const TileDesc &t, const TileBuf<PT> &tb, PT *w,
                                             double alpha, const double *pn, bool y_in_smem, bool staged,
                                             double &rr_acc, int warp, int W) {
  const int lane = threadIdx.x & 31;
  PT *yv = reinterpret_cast<PT *>(P.y);
  const PT *zv = reinterpret_cast<const PT *>(P.z);
  // entries to other colors and row vectors: the staged copies (indexed by
  // global entry / row) or global memory
  const int o0 = UPPER ? t.uo0 : t.lo0;
  const int32_t *oc_s = tb.oc - cover_base<int32_t>(o0), *oc_g = UPPER ? P.su_col : P.sl_col;
  const PT *ov_s = tb.ov - cover_base<PT>(o0), *ov_g = UPPER ? suv<PT>(P) : slv<PT>(P);
  const int vs = tb.vstride;
  const double *v0 = tb.vec - cover_base<double>(t.row0);
  const PT *ys = reinterpret_cast<const PT *>(tb.vec) - cover_base<PT>(t.row0);
  for (int k = warp; k < t.nsteps; k += W) {
    const StepDesc &s = tb.st[k];
    const int cnt = s.cnt;
    if (lane < cnt) {
      const int i = s.row + lane;
      PT acc;
      if (UPPER) {
        PT src;
        if (y_in_smem) src = w[k * kWarp + lane];
        else if (staged) src = ys[i];
        else src = __ldcg(yv + i);
        if (staged) acc = ext_sub<PT, false>(oc_s, ov_s, s.uo + lane, cnt, s.uw, src, zv);
        else acc = ext_sub<PT>(oc_g, ov_g, s.uo + lane, cnt, s.uw, src, zv);
      } else {
        double ri;
        if (staged) {
          ri = v0[i];
          if (UPDATE) {
            ri -= alpha * v0[vs + i];
            P.r[i] = ri;
            P.xh[i] = v0[2 * vs + i] + alpha * v0[3 * vs + i];
            rr_acc += ri * ri;
          }
          acc = ext_sub<PT, false>(oc_s, ov_s, s.lo + lane, cnt, s.lw, PT(ri), yv);
        } else {
          ri = __ldcg(P.r + i);
          if (UPDATE) {
            ri -= alpha * __ldcg(P.q + i);
            P.r[i] = ri;
            P.xh[i] = __ldcg(P.xh + i) + alpha * __ldcg(pn + i);
            rr_acc += ri * ri;
          }
          acc = ext_sub<PT>(oc_g, ov_g, s.lo + lane, cnt, s.lw, PT(ri), yv);
        }
      }
      w[k * kWarp + lane] = acc;
    }
  }
}

// Phase B: warp 0 resolves the in-block recurrence, steps ascending (forward)
// or descending (backward), from shared memory only; a lane reads only its
// own block's values.  In-block padding entries are (step 0, value 0).
template <typename PT, bool UPPER>
__device__ __forceinline__ void tile_phase_b(const TileDesc &t, const StepDesc *st, const PT *dv,
                                             const int32_t *ic, const PT *iv, PT *w, int lane) {
  for (int kk = 0; kk < t.nsteps; ++kk) {
    const int k = UPPER ? t.nsteps - 1 - kk : kk;
    const StepDesc &s = st[k];
    const int cnt = s.cnt, wi = UPPER ? s.uiw : s.liw, e = (UPPER ? s.ui : s.li) + lane;
    if (lane < cnt) {
      PT acc = w[k * kWarp + lane];
      for (int j = 0; j < wi; ++j) acc -= iv[e + j * cnt] * w[ic[e + j * cnt] * kWarp + lane];
      w[k * kWarp + lane] = acc * dv[s.row + lane];
    }
  }
}

// Phase C: the tile's results to global memory (y or z), <r,z> (backward)
template <typename PT, bool UPPER>
__device__ __forceinline__ void tile_phase_c(const Params &P, const TileDesc &t, const StepDesc *st, const PT *w,
                                             bool store, const double *rs, double &rz_acc, int warp, int W) {
  const int lane = threadIdx.x & 31;
  PT *res = reinterpret_cast<PT *>(UPPER ? P.z : P.y);
  for (int k = warp; k < t.nsteps; k += W) {
    const StepDesc &s = st[k];
    if (lane < s.cnt) {
      const int i = s.row + lane;
      const PT v = w[k * kWarp + lane];
      if (store) res[i] = v;
      if (UPPER) {
        double ri;
        if (rs) ri = rs[i];
        else ri = __ldcg(P.r + i);
        rz_acc += ri * double(v);
      }
    }
  }
}

// A lane-tile launch: CTAs walk the color's tiles grid-stride; the static
// data of the next tile is copied into the other buffer while the current one
// is computed (the first tile's before griddepcontrol.wait); one <r,r> /
// <r,z> reduction per CTA at the end.
template <typename PT, int MODE, bool UPDATE>
__global__ void __launch_bounds__(kMaxWarpsPerCta * kWarp)
tile_kernel(Params P, int t0, int t1, TilePlan pl, int fin, SlotArgs sa) {
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[kMaxWarpsPerCta];
  __shared__ int flag;
  constexpr bool FU = MODE == M_BWD, TWO = MODE == M_FUSED;
  const int bsize = TWO && pl.cap_i2 > 0 ? pl.buf2 : pl.buf1;
  const int nbuf = pl.nbuf;
  PT *w = reinterpret_cast<PT *>(smem + nbuf * bsize);
  double rr_acc = 0.0, rz_acc = 0.0;
  int t = t0 + int(blockIdx.x), buf = 0;
  const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  TileDesc td = load_tile(P.tiles + min(t, t1 - 1));
  if (t < t1) tile_stage<PT, FU, TWO>(P, td, tile_buf<PT>(smem, pl, bsize, 0), pl, threadIdx.x, blockDim.x);
  pdl_wait();
  if (t < t1) tile_stage_vec<PT, FU, UPDATE>(P, td, tile_buf<PT>(smem, pl, bsize, 0), pl, threadIdx.x, blockDim.x);
  cp_commit();
  const double alpha = UPDATE ? __ldcg(&P.sc->alpha) : 0.0;
  for (; t < t1; t += gridDim.x) {
    const int tn = t + int(gridDim.x);
    TileDesc tdn = td;
    if (tn < t1) tdn = load_tile(P.tiles + tn);
    if (tn < t1 && nbuf == 2) {
      tile_stage<PT, FU, TWO>(P, tdn, tile_buf<PT>(smem, pl, bsize, buf ^ 1), pl, threadIdx.x, blockDim.x);
      tile_stage_vec<PT, FU, UPDATE>(P, tdn, tile_buf<PT>(smem, pl, bsize, buf ^ 1), pl, threadIdx.x, blockDim.x);
    }
    cp_commit();
    cp_wait_prev();
    __syncthreads();
    const TileBuf<PT> tb = tile_buf<PT>(smem, pl, bsize, buf);
    const PT *dv = tb.dv - cover_base<PT>(td.row0);
    const InBlock<PT> ul = in_block<PT>(tb.ic, tb.iv, P.ui_col, uiv<PT>(P), td.ui0, td.ui1, pl.cap_i);
    const InBlock<PT> ll = in_block<PT>(tb.ic, tb.iv, P.si_col, siv<PT>(P), td.li0, td.li1, pl.cap_i);
    const bool stg = ext_staged(pl, td, MODE == M_BWD);
    if (MODE == M_BWD) {
      tile_phase_a<PT, true, false>(P, td, tb, w, 0.0, nullptr, false, stg, rr_acc, wid, nw);
      __syncthreads();
      if (wid == 0) tile_phase_b<PT, true>(td, tb.st, dv, ul.ic, ul.iv, w, threadIdx.x);
      __syncthreads();
      tile_phase_c<PT, true>(P, td, tb.st, w, true, stg ? tb.vec + tb.vstride - cover_base<double>(td.row0) : nullptr,
                             rz_acc, wid, nw);
    } else {
      tile_phase_a<PT, false, UPDATE>(P, td, tb, w, alpha, P.p0, false, stg, rr_acc, wid, nw);
      __syncthreads();
      if (wid == 0) tile_phase_b<PT, false>(td, tb.st, dv, ll.ic, ll.iv, w, threadIdx.x);
      __syncthreads();
      if (MODE == M_FWD) {
        tile_phase_c<PT, false>(P, td, tb.st, w, true, nullptr, rz_acc, wid, nw);
      } else {
        // the last color: y stays in shared memory for the backward sweep
        // (its entries to other colors from global memory: the staged set is L's)
        const InBlock<PT> u2 = in_block<PT>(tb.ic2, tb.iv2, P.ui_col, uiv<PT>(P), td.ui0, td.ui1, pl.cap_i2);
        tile_phase_a<PT, true, false>(P, td, tb, w, 0.0, nullptr, true, false, rr_acc, wid, nw);
        __syncthreads();
        if (wid == 0) tile_phase_b<PT, true>(td, tb.st, dv, u2.ic, u2.iv, w, threadIdx.x);
        __syncthreads();
        tile_phase_c<PT, true>(P, td, tb.st, w, true, nullptr, rz_acc, wid, nw);
      }
    }
    __syncthreads();   // buffer buf and w are reused by the next tile
    if (nbuf == 1) {
      // one buffer: the next tile's copies start now (waited on by the next
      // pass's cp_wait_prev, which leaves only its own empty group pending)
      if (tn < t1) {
        tile_stage<PT, FU, TWO>(P, tdn, tile_buf<PT>(smem, pl, bsize, 0), pl, threadIdx.x, blockDim.x);
        tile_stage_vec<PT, FU, UPDATE>(P, tdn, tile_buf<PT>(smem, pl, bsize, 0), pl, threadIdx.x, blockDim.x);
      }
      cp_commit();
    } else {
      buf ^= 1;
    }
    td = tdn;
  }
  cp_wait_all();
  launch_epilogue(P, fin, sa, MODE != M_BWD && UPDATE, MODE != M_FWD, rr_acc, rz_acc, red, &flag);
}

// ---------------------------------------------------------------------------
// warp-tile kernels: one warp per lane tile, all of the tile's steps in order
// by that warp (Alg. 1 again: a lane per block, the block's rows in
// sequence).  For colors of many tiles with few steps (blocks of a few rows)
// this keeps every warp of a CTA busy where the CTA-per-tile kernel spreads
// the steps of one tile over its warps; no barrier, and a lane's in-block
// values stay in its own column of the warp's shared-memory buffer.
// ---------------------------------------------------------------------------
__device__ __forceinline__ StepDesc load_step_g(const StepDesc *s) {
  const int4 *p = reinterpret_cast<const int4 *>(s);
  const int4 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
  StepDesc r;
  r.row = a.x; r.cnt = a.y; r.lo = a.z; r.lw = a.w;
  r.li = b.x; r.liw = b.y; r.uo = b.z; r.uw = b.w;
  r.ui = c.x; r.uiw = c.y; r.pad0 = r.pad1 = 0;
  return r;
}

// One sweep over tile t by one warp.  Forward (UPPER = false): source r (with
// the x / r update when UPDATE), entries to earlier colors gathered from y,
// in-block entries from wv; result y.  Backward: source y (from wv when
// y_in_smem, the fused last color), gathers of z, result z and <r,z>.
// wv[step * 32 + lane] keeps the lane's own values of the tile.
template <typename PT, bool UPPER, bool UPDATE>
__device__ __forceinline__ void wtile_sweep(const Params &P, const TileDesc &t, PT *wv, double alpha,
                                            bool y_in_smem, bool store, double &rr_acc, double &rz_acc, int lane) {
  PT *res = reinterpret_cast<PT *>(UPPER ? P.z : P.y);
  const PT *ext = reinterpret_cast<const PT *>(UPPER ? P.z : P.y);
  const PT *yv = reinterpret_cast<const PT *>(P.y);
  const PT *dvg = invds<PT>(P);
  const int32_t *icol = UPPER ? P.ui_col : P.si_col;
  const PT *ival = UPPER ? uiv<PT>(P) : siv<PT>(P);
  // in-block padding entries are (step 0, value 0): a backward sweep reads
  // step 0 before computing it, so it must hold a finite value (forward
  // sweeps and the fused one have written it by then)
  if (UPPER && !y_in_smem) {
    for (int k = 0; k < t.nsteps; ++k) wv[k * kWarp + lane] = PT(0);
    __syncwarp();
  }
  for (int kk = 0; kk < t.nsteps; ++kk) {
    const int k = UPPER ? t.nsteps - 1 - kk : kk;
    StepDesc s;
    if (t.nsteps == 1) {
      s.row = t.row0; s.cnt = t.nrows; s.lo = t.lo0; s.lw = t.lw0; s.li = t.li0; s.liw = t.wl;
      s.uo = t.uo0; s.uw = t.uw0; s.ui = t.ui0; s.uiw = t.wu;
    } else {
      s = load_step_g(P.steps + t.step0 + k);
    }
    if (lane < s.cnt) {
      const int i = s.row + lane;
      PT acc;
      if (UPPER) {
        const PT src = y_in_smem ? wv[k * kWarp + lane] : __ldcg(yv + i);
        acc = ext_sub<PT>(P.su_col, suv<PT>(P), s.uo + lane, s.cnt, s.uw, src, ext);
      } else {
        double ri = __ldcg(P.r + i);
        if (UPDATE) {
          ri -= alpha * __ldcg(P.q + i);
          P.r[i] = ri;
          P.xh[i] = __ldcg(P.xh + i) + alpha * __ldcg(P.p0 + i);
          rr_acc += ri * ri;
        }
        acc = ext_sub<PT>(P.sl_col, slv<PT>(P), s.lo + lane, s.cnt, s.lw, PT(ri), ext);
      }
      const int wi = UPPER ? s.uiw : s.liw, e = (UPPER ? s.ui : s.li) + lane;
      for (int j = 0; j < wi; ++j) acc -= __ldg(ival + e + j * s.cnt) * wv[__ldg(icol + e + j * s.cnt) * kWarp + lane];
      const PT v = acc * __ldg(dvg + i);
      wv[k * kWarp + lane] = v;
      if (store) res[i] = v;
      if (UPPER) rz_acc += __ldcg(P.r + i) * double(v);
    }
  }
}

// A warp-tile launch: the warps walk the color's tiles grid-stride (tile of
// warp w of CTA b: t0 + b * W + w, then + gridDim.x * W); one <r,r> / <r,z>
// reduction per CTA at the end.  Shared memory: cap_s * 32 values per warp.
#ifndef ICCG_TILE_MAXNREG
#define ICCG_TILE_MAXNREG 64
#endif

template <typename PT, int MODE, bool UPDATE>
__global__ void __maxnreg__(ICCG_TILE_MAXNREG)
wtile_kernel(Params P, int t0, int t1, int cap_s, int fin, SlotArgs sa) {
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[kMaxWarpsPerCta];
  __shared__ int flag;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  PT *wv = reinterpret_cast<PT *>(smem) + size_t(wid) * cap_s * kWarp;
  double rr_acc = 0.0, rz_acc = 0.0;
  int t = t0 + int(blockIdx.x) * nw + wid;
  TileDesc td = load_tile(P.tiles + min(t, t1 - 1));
  pdl_wait();
  const double alpha = UPDATE ? __ldcg(&P.sc->alpha) : 0.0;
  for (; t < t1; t += int(gridDim.x) * nw) {
    const int tn = t + int(gridDim.x) * nw;
    const TileDesc tdn = tn < t1 ? load_tile(P.tiles + tn) : td;
    if (MODE == M_BWD) {
      wtile_sweep<PT, true, false>(P, td, wv, 0.0, false, true, rr_acc, rz_acc, lane);
    } else {
      wtile_sweep<PT, false, UPDATE>(P, td, wv, alpha, false, MODE == M_FWD, rr_acc, rz_acc, lane);
      __syncwarp();
      if (MODE == M_FUSED) wtile_sweep<PT, true, false>(P, td, wv, 0.0, true, true, rr_acc, rz_acc, lane);
    }
    __syncwarp();
    td = tdn;
  }
  launch_epilogue(P, fin, sa, MODE != M_BWD && UPDATE, MODE != M_FWD, rr_acc, rz_acc, red, &flag);
}

// ---------------------------------------------------------------------------
// pair kernels: colors of blocks of one or two rows (tiles of at most two
// steps).  A warp per tile, a lane per block, the block's rows in registers:
// forward
//   y0 = (r0 - sum_j L0j y_j) / L00
//   y1 = (r1 - sum_j L1j y_j - L10 y0) / L11
// (the sums over earlier colors), backward
//   z1 = (y1 - sum_j Lj1 z_j) / L11
//   z0 = (y0 - sum_j Lj0 z_j - L10 z1) / L00
// (the sums over later colors); a one-row block is its step 0 alone.
// Padding entries (kPadCol, 0) add 0 * an element the sweep has already
// written: y_0 (first color) forward, z_{n-1} (last color) backward.
// ---------------------------------------------------------------------------
// a descriptor whose first 16 bytes (first row, block counts) are already
// in registers
__device__ __forceinline__ PairDesc load_pair_rest(const PairDesc *p, int4 a) {
  const int4 *q = reinterpret_cast<const int4 *>(p);
  const int4 b = __ldg(q + 1), c = __ldg(q + 2), d = __ldg(q + 3);
  PairDesc r;
  r.row0 = a.x; r.c0 = a.y; r.c1 = a.z; r.lo = a.w;
  r.lw0 = b.x; r.lw1 = b.y; r.li = b.z; r.liw1 = b.w;
  r.uo = c.x; r.uw0 = c.y; r.uw1 = c.z; r.ui = c.w;
  r.uiw0 = d.x; r.pad0 = r.pad1 = r.pad2 = 0;
  return r;
}
__device__ __forceinline__ int4 pair_head(const PairDesc *p) { return __ldg(reinterpret_cast<const int4 *>(p)); }
__device__ __forceinline__ PairDesc load_pair(const PairDesc *p) { return load_pair_rest(p, pair_head(p)); }

template <typename PT>
__device__ __forceinline__ PT pair_sub(const int32_t *col, const PT *val, int e, int cnt, int w, PT acc,
                                       const PT *g, int pad) {
#pragma unroll 4
  for (int j = 0; j < w; ++j) {
    const int c = __ldg(col + e + j * cnt);
    const PT v = __ldg(val + e + j * cnt);
    acc -= v * __ldcg(g + (c == kPadCol ? pad : c));
  }
  return acc;
}

// backward over one tile from y0 (and y1 when a1): stores z, adds <r,z>
template <typename PT>
__device__ __forceinline__ void pair_bwd(const Params &P, const PairDesc &d, int lane, bool a1, PT y0, PT y1,
                                         PT dv0, PT dv1, double r0, double r1, double &rz_acc) {
  PT *zv = reinterpret_cast<PT *>(P.z);
  const int i0 = d.row0 + lane, i1 = d.row0 + d.c0 + lane;
  // both steps' gathers before any store (a store to z would order the
  // other step's gathers after it)
  PT acc0 = pair_sub<PT>(P.su_col, suv<PT>(P), d.uo + lane, d.c0, d.uw0, y0, zv, P.n - 1);
  PT z1 = PT(0);
  if (a1) z1 = pair_sub<PT>(P.su_col, suv<PT>(P), d.uo + d.uw0 * d.c0 + lane, d.c1, d.uw1, y1, zv, P.n - 1) * dv1;
  for (int j = 0; j < d.uiw0; ++j) acc0 -= __ldg(uiv<PT>(P) + d.ui + j * d.c0 + lane) * z1;
  const PT z0 = acc0 * dv0;
  zv[i0] = z0;
  rz_acc += r0 * double(z0);
  if (a1) {
    zv[i1] = z1;
    rz_acc += r1 * double(z1);
  }
}

// one tile of a pair color, warp-wide (lanes beyond the tile's blocks idle)
template <typename PT, int MODE, bool UPDATE>
__device__ __forceinline__ void pair_tile_h(const Params &P, int t, int4 head, int lane, double alpha,
                                            double &rr_acc, double &rz_acc) {
  PT *yv = reinterpret_cast<PT *>(P.y);
  const PT *dvg = invds<PT>(P);
  const PairDesc d = load_pair_rest(P.pairs + t, head);
  if (lane >= d.c0) return;   // a lane active in step 1 is active in step 0
  const bool a1 = lane < d.c1;
  const int i0 = d.row0 + lane, i1 = d.row0 + d.c0 + lane;
  const PT dv0 = __ldg(dvg + i0), dv1 = a1 ? __ldg(dvg + i1) : PT(0);
  if (MODE == M_BWD) {
    const PT y0 = __ldcg(yv + i0), y1 = a1 ? __ldcg(yv + i1) : PT(0);
    const double r0 = __ldcg(P.r + i0), r1 = a1 ? __ldcg(P.r + i1) : 0.0;
    pair_bwd<PT>(P, d, lane, a1, y0, y1, dv0, dv1, r0, r1, rz_acc);
  } else {
    double r0 = __ldcg(P.r + i0), r1 = a1 ? __ldcg(P.r + i1) : 0.0;
    if (UPDATE) {
      r0 -= alpha * __ldcg(P.q + i0);
      P.r[i0] = r0;
      P.xh[i0] = __ldcg(P.xh + i0) + alpha * __ldcg(P.p0 + i0);
      rr_acc += r0 * r0;
      if (a1) {
        r1 -= alpha * __ldcg(P.q + i1);
        P.r[i1] = r1;
        P.xh[i1] = __ldcg(P.xh + i1) + alpha * __ldcg(P.p0 + i1);
        rr_acc += r1 * r1;
      }
    }
    const PT y0 = pair_sub<PT>(P.sl_col, slv<PT>(P), d.lo + lane, d.c0, d.lw0, PT(r0), yv, 0) * dv0;
    PT y1 = PT(0);
    if (a1) {
      PT acc1 = pair_sub<PT>(P.sl_col, slv<PT>(P), d.lo + d.lw0 * d.c0 + lane, d.c1, d.lw1, PT(r1), yv, 0);
      for (int j = 0; j < d.liw1; ++j) acc1 -= __ldg(siv<PT>(P) + d.li + j * d.c1 + lane) * y0;
      y1 = acc1 * dv1;
    }
    if (MODE == M_FWD) {
      yv[i0] = y0;
      if (a1) yv[i1] = y1;
    } else {
      pair_bwd<PT>(P, d, lane, a1, y0, y1, dv0, dv1, r0, r1, rz_acc);
    }
  }
}

template <typename PT, int MODE, bool UPDATE>
__device__ __forceinline__ void pair_tile(const Params &P, int t, int lane, double alpha, double &rr_acc,
                                          double &rz_acc) {
  pair_tile_h<PT, MODE, UPDATE>(P, t, pair_head(P.pairs + t), lane, alpha, rr_acc, rz_acc);
}

// The staged pair kernel (pair_kernel<.., STAGE = true>, chosen per color
// and sweep on the host) loads each tile's static data ahead of its
// gathers: the descriptor, the pivots' reciprocals and in-block coefficient
// in registers, and the first kPairStage entries of each step (the sums over
// the other colors: lower for the forward sweep, upper for the backward) in
// the warp's shared-memory buffer by cp.async.  The warp's first tile is
// staged before griddepcontrol.wait, so these loads overlap the previous
// launch; after the wait a tile's gathers of both steps and its row vectors
// are in flight together.  Wider steps take their remaining entries from
// global memory.  The unstaged kernel (pair_tile_h) keeps the loads in the
// order the recurrence uses them and serves sweeps with few such entries.
constexpr int kPairStage = 6;   // a 7-point row has at most 6 entries to other blocks

template <typename PT>
struct PairStage {
  int32_t col[2][kPairStage][kWarp];
  PT val[2][kPairStage][kWarp];
};

template <typename PT>
struct PairPre {
  PairDesc d;
  PT dv0, dv1, e;   // 1/L_00, 1/L_11 and the in-block coefficient of the sweep
};

template <typename PT, bool BWD>
__device__ __forceinline__ PairPre<PT> pair_stage(const Params &P, int t, int lane, PairStage<PT> &s) {
  PairPre<PT> q;
  q.d = load_pair(P.pairs + t);
  const PairDesc &d = q.d;
  q.dv0 = q.dv1 = q.e = PT(0);
  if (lane < d.c0) {
    const bool a1 = lane < d.c1;
    const PT *dvg = invds<PT>(P);
    q.dv0 = __ldg(dvg + d.row0 + lane);
    if (a1) q.dv1 = __ldg(dvg + d.row0 + d.c0 + lane);
    const int32_t *col = BWD ? P.su_col : P.sl_col;
    const PT *val = BWD ? suv<PT>(P) : slv<PT>(P);
    const int b0 = BWD ? d.uo : d.lo, w0 = BWD ? d.uw0 : d.lw0, w1 = BWD ? d.uw1 : d.lw1;
    const int n0 = min(w0, kPairStage), n1 = a1 ? min(w1, kPairStage) : 0;
    for (int j = 0; j < n0; ++j) {
      cp_async4(&s.col[0][j][lane], col + b0 + j * d.c0 + lane);
      cp_async_elem<PT>(&s.val[0][j][lane], val + b0 + j * d.c0 + lane);
    }
    const int b1 = b0 + w0 * d.c0;
    for (int j = 0; j < n1; ++j) {
      cp_async4(&s.col[1][j][lane], col + b1 + j * d.c1 + lane);
      cp_async_elem<PT>(&s.val[1][j][lane], val + b1 + j * d.c1 + lane);
    }
    // a block of two rows has at most one in-block entry per row: row 1's
    // to row 0 forward, row 0's to row 1 backward
    if (BWD) {
      if (d.uiw0 > 0) q.e = __ldg(uiv<PT>(P) + d.ui + lane);
    } else {
      if (a1 && d.liw1 > 0) q.e = __ldg(siv<PT>(P) + d.li + lane);
    }
  }
  cp_commit();
  return q;
}

// the staged sums of both steps: every gather issued before the first
// multiply-add; entries past kPairStage from global memory
template <typename PT, bool BWD>
__device__ __forceinline__ void pair_staged_sums(const Params &P, const PairDesc &d, const PairStage<PT> &s,
                                                 int lane, bool a1, PT &acc0, PT &acc1) {
  const PT *g = reinterpret_cast<const PT *>(BWD ? P.z : P.y);
  const int pad = BWD ? P.n - 1 : 0;
  const int w0 = BWD ? d.uw0 : d.lw0, w1 = BWD ? d.uw1 : d.lw1;
  PT g0[kPairStage], g1[kPairStage];
#pragma unroll
  for (int j = 0; j < kPairStage; ++j) {
    g0[j] = PT(0);
    if (j < w0) {
      const int c = s.col[0][j][lane];
      g0[j] = __ldcg(g + (c == kPadCol ? pad : c));
    }
  }
#pragma unroll
  for (int j = 0; j < kPairStage; ++j) {
    g1[j] = PT(0);
    if (a1 && j < w1) {
      const int c = s.col[1][j][lane];
      g1[j] = __ldcg(g + (c == kPadCol ? pad : c));
    }
  }
#pragma unroll
  for (int j = 0; j < kPairStage; ++j)
    if (j < w0) acc0 -= s.val[0][j][lane] * g0[j];
#pragma unroll
  for (int j = 0; j < kPairStage; ++j)
    if (a1 && j < w1) acc1 -= s.val[1][j][lane] * g1[j];
  if (w0 > kPairStage || w1 > kPairStage) {
    const int32_t *col = BWD ? P.su_col : P.sl_col;
    const PT *val = BWD ? suv<PT>(P) : slv<PT>(P);
    const int b0 = BWD ? d.uo : d.lo, b1 = b0 + w0 * d.c0;
    for (int j = kPairStage; j < w0; ++j) {
      const int e = b0 + j * d.c0 + lane, c = __ldg(col + e);
      acc0 -= __ldg(val + e) * __ldcg(g + (c == kPadCol ? pad : c));
    }
    if (a1)
      for (int j = kPairStage; j < w1; ++j) {
        const int e = b1 + j * d.c1 + lane, c = __ldg(col + e);
        acc1 -= __ldg(val + e) * __ldcg(g + (c == kPadCol ? pad : c));
      }
  }
}

template <typename PT, int MODE, bool UPDATE>
__device__ __forceinline__ void pair_tile_staged(const Params &P, const PairPre<PT> &q, const PairStage<PT> &s,
                                                 int lane, double alpha, double &rr_acc, double &rz_acc) {
  const PairDesc &d = q.d;
  if (lane >= d.c0) return;
  const bool a1 = lane < d.c1;
  const int i0 = d.row0 + lane, i1 = d.row0 + d.c0 + lane;
  cp_wait_all();   // the lane's own staged entries (it reads no other lane's)
  if (MODE == M_BWD) {
    const PT *yv = reinterpret_cast<const PT *>(P.y);
    PT acc0 = __ldcg(yv + i0), acc1 = a1 ? __ldcg(yv + i1) : PT(0);
    const double r0 = __ldcg(P.r + i0), r1 = a1 ? __ldcg(P.r + i1) : 0.0;
    pair_staged_sums<PT, true>(P, d, s, lane, a1, acc0, acc1);
    const PT z1 = acc1 * q.dv1;
    acc0 -= q.e * z1;
    for (int j = 1; j < d.uiw0; ++j) acc0 -= __ldg(uiv<PT>(P) + d.ui + j * d.c0 + lane) * z1;
    const PT z0 = acc0 * q.dv0;
    PT *zv = reinterpret_cast<PT *>(P.z);
    zv[i0] = z0;
    rz_acc += r0 * double(z0);
    if (a1) {
      zv[i1] = z1;
      rz_acc += r1 * double(z1);
    }
  } else {
    PT acc0, acc1 = PT(0);
    double r0 = __ldcg(P.r + i0), r1 = a1 ? __ldcg(P.r + i1) : 0.0;
    if (UPDATE) {
      const double q0 = __ldcg(P.q + i0), x0 = __ldcg(P.xh + i0), p0 = __ldcg(P.p0 + i0);
      double q1 = 0.0, x1 = 0.0, p1 = 0.0;
      if (a1) {
        q1 = __ldcg(P.q + i1);
        x1 = __ldcg(P.xh + i1);
        p1 = __ldcg(P.p0 + i1);
      }
      r0 -= alpha * q0;
      rr_acc += r0 * r0;
      if (a1) {
        r1 -= alpha * q1;
        rr_acc += r1 * r1;
      }
      acc0 = PT(r0);
      acc1 = PT(r1);
      pair_staged_sums<PT, false>(P, d, s, lane, a1, acc0, acc1);
      P.r[i0] = r0;
      P.xh[i0] = x0 + alpha * p0;
      if (a1) {
        P.r[i1] = r1;
        P.xh[i1] = x1 + alpha * p1;
      }
    } else {
      acc0 = PT(r0);
      acc1 = PT(r1);
      pair_staged_sums<PT, false>(P, d, s, lane, a1, acc0, acc1);
    }
    const PT y0 = acc0 * q.dv0;
    PT y1 = PT(0);
    if (a1) {
      acc1 -= q.e * y0;
      for (int j = 1; j < d.liw1; ++j) acc1 -= __ldg(siv<PT>(P) + d.li + j * d.c1 + lane) * y0;
      y1 = acc1 * q.dv1;
    }
    PT *yv = reinterpret_cast<PT *>(P.y);
    if (MODE == M_FWD) {
      yv[i0] = y0;
      if (a1) yv[i1] = y1;
    } else {
      pair_bwd<PT>(P, d, lane, a1, y0, y1, q.dv0, q.dv1, r0, r1, rz_acc);
    }
  }
}

template <typename PT>
constexpr int pair_stage_bytes() { return int(sizeof(PairStage<PT>)); }

template <typename PT, int MODE, bool UPDATE, bool STAGE>
__global__ void __launch_bounds__(kMaxWarpsPerCta * kWarp)
pair_kernel(Params P, int t0, int t1, int fin, SlotArgs sa) {
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[kMaxWarpsPerCta];
  __shared__ int flag;
  const int lane = threadIdx.x & 31, wid = int(threadIdx.x >> 5);
  const int nw = int(blockDim.x >> 5), stride = int(gridDim.x) * nw;
  double rr_acc = 0.0, rz_acc = 0.0;
  int t = t0 + int(blockIdx.x) * nw + wid;
  if constexpr (STAGE) {
    PairStage<PT> &st = reinterpret_cast<PairStage<PT> *>(smem)[wid];
    PairPre<PT> q;
    if (t < t1) q = pair_stage<PT, MODE == M_BWD>(P, t, lane, st);
    pdl_wait();
    const double alpha = UPDATE ? __ldcg(&P.sc->alpha) : 0.0;
    while (t < t1) {
      pair_tile_staged<PT, MODE, UPDATE>(P, q, st, lane, alpha, rr_acc, rz_acc);
      t += stride;
      __syncwarp();
      if (t < t1) q = pair_stage<PT, MODE == M_BWD>(P, t, lane, st);
    }
  } else {
    // the next tile's first descriptor word (its rows) loads while the
    // current tile runs, the first tile's before the wait
    int4 hn = make_int4(0, 0, 0, 0);
    if (t < t1) hn = pair_head(P.pairs + t);
    pdl_wait();
    const double alpha = UPDATE ? __ldcg(&P.sc->alpha) : 0.0;
    for (; t < t1; t += stride) {
      const int4 h = hn;
      if (t + stride < t1) hn = pair_head(P.pairs + t + stride);
      pair_tile_h<PT, MODE, UPDATE>(P, t, h, lane, alpha, rr_acc, rz_acc);
    }
  }
  launch_epilogue(P, fin, sa, MODE != M_BWD && UPDATE, MODE != M_FWD, rr_acc, rz_acc, red, &flag);
}

// ---------------------------------------------------------------------------
// warp-unit kernels: colors of blocks of at most 32 rows.  One warp holds 32 / S
// whole blocks, a lane per row (Alg. 1: the blocks of a color in parallel,
// the rows of a block in order).  A sweep over a unit:
//   A  every lane: its source (r with the x / r update, or y) minus its
//      entries to other colors (sliced-ELL over the warp: coalesced);
//   B  the in-block recurrence as a chain of steps: at every step a lane
//      subtracts at most one in-block term, coefficient x t_k, where t_k is
//      the final value of the term's source row k (read from its lane by a
//      shuffle) and the coefficient is the entry divided by the pivot of
//      row k, so the division of Alg. 1 is applied to each row once, at the
//      end.  The host orders each lane's terms by the step their sources
//      become final, so independent terms of different rows share a step:
//      the chain is about as long as the in-block dependency depth or the
//      widest row, not the block size;
//   C  y = t / L_ii (times 1/L_ii), stored; <r,z> for the backward sweep.
// Every static datum of a unit (descriptor, masks, coefficients, 1/L_ii) is
// loaded before the first dependent access (griddepcontrol.wait).  A step at
// which no lane of the warp has a coefficient issues no FP64 instruction.
// ---------------------------------------------------------------------------
template <typename PT> __device__ __forceinline__ const PT *wlv(const Params &P);
template <> __device__ __forceinline__ const double *wlv<double>(const Params &P) { return P.wl_val; }
template <> __device__ __forceinline__ const float *wlv<float>(const Params &P) { return P.wl_val32; }
template <typename PT> __device__ __forceinline__ const PT *wuv(const Params &P);
template <> __device__ __forceinline__ const double *wuv<double>(const Params &P) { return P.wu_val; }
template <> __device__ __forceinline__ const float *wuv<float>(const Params &P) { return P.wu_val32; }

__device__ __forceinline__ WarpUnit load_unit(const WarpUnit *u) {
  const int4 *p = reinterpret_cast<const int4 *>(u);
  const int4 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2), e = __ldg(p + 3);
  WarpUnit r;
  r.blk0 = a.x; r.nblk = a.y; r.lo = a.z; r.lw = a.w;
  r.uo = b.x; r.uw = b.y; r.li = b.z; r.lm = b.w;
  r.ui = c.x; r.um = c.y; r.row0 = c.z; r.nrows = c.w;
  r.ls = e.x; r.us = e.y; r.pad0 = r.pad1 = 0;
  return r;
}

constexpr int kUnitChunk = 8;   // entries to other colors per batch of loads

// acc -= sum over the lane's entries to other colors (width w, stride 32)
template <typename PT>
__device__ __forceinline__ PT unit_ext(const int32_t *col, const PT *val, int e, int w, PT acc, const PT *g) {
  for (int j0 = 0; j0 < w; j0 += kUnitChunk) {
    const int nj = min(kUnitChunk, w - j0);
    int cc[kUnitChunk];
    PT vv[kUnitChunk], xx[kUnitChunk];
#pragma unroll
    for (int j = 0; j < kUnitChunk; ++j) {
      cc[j] = j < nj ? __ldg(col + e + (j0 + j) * kWarp) : kPadCol;
      vv[j] = j < nj ? __ldg(val + e + (j0 + j) * kWarp) : PT(0);
    }
#pragma unroll
    for (int j = 0; j < kUnitChunk; ++j) xx[j] = cc[j] == kPadCol ? PT(0) : __ldcg(g + cc[j]);
#pragma unroll
    for (int j = 0; j < kUnitChunk; ++j)
      if (j < nj) acc -= vv[j] * xx[j];
  }
  return acc;
}

// the lane's chain coefficients by step (0 where its mask has no bit) and the
// source lanes (four bytes a word)
template <typename PT, int S>
__device__ __forceinline__ void unit_coef(const PT *v, const uint32_t *sw, int off, int soff, int M, uint32_t mask,
                                          int lane, PT (&cf)[S], uint32_t (&src)[(S + 3) / 4]) {
  // the lane's terms are stored term-major (its j-th term at off + j * 32 +
  // lane): the term of step k is number popc(mask below k)
#pragma unroll
  for (int k = 0; k < S; ++k)
    cf[k] = ((mask >> k) & 1u) ? __ldg(v + off + __popc(mask & ((1u << k) - 1u)) * kWarp + lane) : PT(0);
#pragma unroll
  for (int w = 0; w < (S + 3) / 4; ++w) src[w] = 4 * w < M ? __ldg(sw + soff + w * kWarp + lane) : 0u;
}

// the lane's chain coefficients into its column of the warp's shared-memory
// buffer (cp.async, only the steps its mask has: no registers held while the
// copies fly) and its source lanes into registers

template <typename PT, int S>
__device__ __forceinline__ void unit_coef_smem(const PT *v, const uint32_t *sw, int off, int soff, int M,
                                               uint32_t mask, int lane, PT *cfs, uint32_t (&src)[(S + 3) / 4]) {
#pragma unroll
  for (int k = 0; k < S; ++k)
    if ((mask >> k) & 1u)
      cp_async_elem<PT>(cfs + k * kWarp + lane, v + off + __popc(mask & ((1u << k) - 1u)) * kWarp + lane);
  asm volatile("cp.async.commit_group;" ::: "memory");
#pragma unroll
  for (int w = 0; w < (S + 3) / 4; ++w) src[w] = 4 * w < M ? __ldg(sw + soff + w * kWarp + lane) : 0u;
}

// phase B with the coefficients in shared memory (the lane's own column)
template <typename PT, int S>
__device__ __forceinline__ PT unit_chain_smem(PT t, int M, uint32_t mask, uint32_t wmask, const PT *cfs, int lane,
                                              const uint32_t (&src)[(S + 3) / 4]) {
  asm volatile("cp.async.wait_group 0;" ::: "memory");
#pragma unroll
  for (int k = 0; k < S; ++k) {
    if (k < M) {
      const int sl = int((src[k / 4] >> (8 * (k % 4))) & 0xffu);
      const PT tk = __shfl_sync(0xffffffffu, t, sl);
      if ((wmask >> k) & 1u) {
        if ((mask >> k) & 1u) t -= cfs[k * kWarp + lane] * tk;
      }
    }
  }
  return t;
}

// phase B of a unit: M chain steps; at step k every lane with a term
// subtracts coefficient x the (final) value of its source lane; wmask = OR
// of the warp's lane masks (a step no lane uses issues no FP64 instruction)
template <typename PT, int S>
__device__ __forceinline__ PT unit_chain(PT t, int M, uint32_t mask, uint32_t wmask, const PT (&cf)[S],
                                         const uint32_t (&src)[(S + 3) / 4]) {
#pragma unroll
  for (int k = 0; k < S; ++k) {
    if (k < M) {
      const int sl = int((src[k / 4] >> (8 * (k % 4))) & 0xffu);
      const PT tk = __shfl_sync(0xffffffffu, t, sl);
      if ((wmask >> k) & 1u) {
        if ((mask >> k) & 1u) t -= cf[k] * tk;
      }
    }
  }
  return t;
}

constexpr int kUnitWarps = 8;   // warps (units in flight) per CTA of the warp-unit kernels

// chain coefficients of segments of at least kUnitSmemS steps sit in shared
// memory (S x 32 values per warp) instead of registers
constexpr int kUnitSmemS = 16;

inline int unit_smem_bytes(int S, int elem) { return S >= kUnitSmemS ? kUnitWarps * S * kWarp * elem : 0; }

template <typename PT, int MODE, bool UPDATE, int S>
__global__ void __launch_bounds__(kUnitWarps * kWarp)
unit_kernel(Params P, int u0, int u1, int fin, SlotArgs sa) {
  pdl_trigger();
  __shared__ double red[kMaxWarpsPerCta];
  __shared__ int flag;
  extern __shared__ __align__(16) unsigned char usm[];
  constexpr bool SM = S >= kUnitSmemS;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  PT *cfs = reinterpret_cast<PT *>(usm) + (SM ? wid * S * kWarp : 0);
  const int step = lane & (S - 1);
  constexpr bool FWD = MODE != M_BWD;
  PT *yv = reinterpret_cast<PT *>(P.y);
  PT *zv = reinterpret_cast<PT *>(P.z);
  const PT *dvg = invds<PT>(P);
  double rr_acc = 0.0, rz_acc = 0.0;
  bool waited = false;
  double alpha = 0.0;
  for (int u = u0 + int(blockIdx.x) * nw + wid; u < u1; u += int(gridDim.x) * nw) {
    // static data of the unit
    const WarpUnit d = load_unit(P.units + u);
    int row = -1;
    if (lane / S < d.nblk) {
      const int b = d.blk0 + lane / S;
      const int r = __ldg(P.bptr + b) + step;
      if (r < __ldg(P.bptr + b + 1)) row = r;
    }
    const bool on = row >= 0;
    const uint32_t mf = FWD ? __ldg(P.wl_mask + size_t(u) * kWarp + lane) : 0u;
    const uint32_t mb = MODE != M_FWD ? __ldg(P.wu_mask + size_t(u) * kWarp + lane) : 0u;
    PT cf[SM ? 1 : S];
    uint32_t src[(S + 3) / 4];
    if constexpr (SM) {
      if (FWD) unit_coef_smem<PT, S>(wlv<PT>(P), P.wl_src, d.li, d.ls, d.lm, mf, lane, cfs, src);
      else unit_coef_smem<PT, S>(wuv<PT>(P), P.wu_src, d.ui, d.us, d.um, mb, lane, cfs, src);
    } else {
      if (FWD) unit_coef<PT, S>(wlv<PT>(P), P.wl_src, d.li, d.ls, d.lm, mf, lane, cf, src);
      else unit_coef<PT, S>(wuv<PT>(P), P.wu_src, d.ui, d.us, d.um, mb, lane, cf, src);
    }
    const PT dv = on ? __ldg(dvg + row) : PT(0);
    if (!waited) {
      pdl_wait();
      waited = true;
      if (UPDATE) alpha = __ldcg(&P.sc->alpha);
    }
    PT t = PT(0);
    if (FWD) {
      // A: source r (with the x / r update), entries to earlier colors
      if (on) {
        double ri = __ldcg(P.r + row);
        if (UPDATE) {
          ri -= alpha * __ldcg(P.q + row);
          P.r[row] = ri;
          P.xh[row] = __ldcg(P.xh + row) + alpha * __ldcg(P.p0 + row);
          rr_acc += ri * ri;
        }
        t = PT(ri);
      }
      t = unit_ext<PT>(P.sl_col, slv<PT>(P), d.lo + lane, d.lw, t, yv);
      // B, C
      if constexpr (SM) t = unit_chain_smem<PT, S>(t, d.lm, mf, __reduce_or_sync(0xffffffffu, mf), cfs, lane, src);
      else t = unit_chain<PT, S>(t, d.lm, mf, __reduce_or_sync(0xffffffffu, mf), cf, src);
      const PT y = t * dv;
      if (MODE == M_FWD) {
        if (on) yv[row] = y;
        continue;
      }
      // the last color: its backward sweep at once (y stays in registers)
      if constexpr (SM) unit_coef_smem<PT, S>(wuv<PT>(P), P.wu_src, d.ui, d.us, d.um, mb, lane, cfs, src);
      else unit_coef<PT, S>(wuv<PT>(P), P.wu_src, d.ui, d.us, d.um, mb, lane, cf, src);
      t = y;
    } else {
      if (on) t = __ldcg(yv + row);
    }
    t = unit_ext<PT>(P.su_col, suv<PT>(P), d.uo + lane, d.uw, t, zv);
    if constexpr (SM) t = unit_chain_smem<PT, S>(t, d.um, mb, __reduce_or_sync(0xffffffffu, mb), cfs, lane, src);
    else t = unit_chain<PT, S>(t, d.um, mb, __reduce_or_sync(0xffffffffu, mb), cf, src);
    const PT z = t * dv;
    if (on) {
      zv[row] = z;
      rz_acc += __ldcg(P.r + row) * double(z);
    }
  }
  if (!waited) pdl_wait();
  launch_epilogue(P, fin, sa, MODE != M_BWD && UPDATE, MODE != M_FWD, rr_acc, rz_acc, red, &flag);
}

// ---------------------------------------------------------------------------
// p = z + beta p (start of an iteration; beta = 0 on the first)
// ---------------------------------------------------------------------------
// (two rows per thread per pass: 16-byte loads of p and, for FP64 z, of z)
template <typename ZT>
__global__ void __launch_bounds__(kVecThreads) pupdate_kernel(Params P) {
  pdl_trigger();
  pdl_wait();
  const double beta = __ldcg(&P.sc->beta);
  const ZT *z = reinterpret_cast<const ZT *>(P.z);
  const int n2 = P.n / 2;
  const int stride = gridDim.x * blockDim.x;
  double2 *p2 = reinterpret_cast<double2 *>(P.p0);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n2; k += stride) {
    const double2 pv = __ldcg(p2 + k);
    double z0, z1;
    if (sizeof(ZT) == 8) {
      const double2 zv = __ldcg(reinterpret_cast<const double2 *>(z) + k);
      z0 = zv.x; z1 = zv.y;
    } else {
      const float2 zv = __ldcg(reinterpret_cast<const float2 *>(z) + k);
      z0 = double(zv.x); z1 = double(zv.y);
    }
    p2[k] = make_double2(z0 + beta * pv.x, z1 + beta * pv.y);
  }
  if ((P.n & 1) && blockIdx.x == 0 && threadIdx.x == 0)
    P.p0[P.n - 1] = double(__ldcg(z + P.n - 1)) + beta * __ldcg(P.p0 + P.n - 1);
}

// ---------------------------------------------------------------------------
// SpMV over the 32-row slices of A_hat's sliced-ELL copy, one row per lane:
// coalesced loads of a slice's columns and values straight into registers,
// then the gathers; a full-occupancy grid walks the slices grid-stride (each
// warp one slice at a time; the resident warps keep the loads in flight).
// Off-diagonal entries in column order, then the diagonal.
// ---------------------------------------------------------------------------
// mode 0: q = A p, <p, q>; the last CTA sets alpha = rz / pq
// mode 1: r = b_hat - A x_hat, <r, r> partials in part_a (solve start)
// mode 2: q = A x_hat (plain SpMV)
constexpr int kSpmvChunk = 6;   // entries per predicated batch of the SpMV

// 6 CTAs of 8 warps per SM (at most 40 registers a thread): measured 1%
// faster per PCG iteration than 4 CTAs at 60 registers
template <int MODE>
__global__ void __launch_bounds__(kSpmvWarps * kWarp, 6)
spmv_kernel(Params P) {
  pdl_trigger();
  __shared__ double red[kMaxWarpsPerCta];
  __shared__ int flag;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
  const int nsl = (P.n + kWarp - 1) / kWarp;
  const double *xin = MODE == 0 ? P.p0 : P.xh;
  double acc = 0.0;
  pdl_wait();
  for (int sl = blockIdx.x * W + warp; sl < nsl; sl += gridDim.x * W) {
    const int e0 = __ldg(P.sa_ptr + sl), w = (__ldg(P.sa_ptr + sl + 1) - e0) >> 5;
    const int i = sl * kWarp + lane;
    const int32_t *col = P.sa_col + e0 + lane;
    const double *val = P.sa_val + e0 + lane;
    double s = 0.0;
    for (int j0 = 0; j0 < w; j0 += kSpmvChunk) {
      int cc[kSpmvChunk];
      double vv[kSpmvChunk], xx[kSpmvChunk];
#pragma unroll
      for (int j = 0; j < kSpmvChunk; ++j) {
        const bool ok = j0 + j < w;
        cc[j] = ok ? __ldg(col + (j0 + j) * kWarp) : 0;
        vv[j] = ok ? __ldg(val + (j0 + j) * kWarp) : 0.0;
      }
#pragma unroll
      for (int j = 0; j < kSpmvChunk; ++j) xx[j] = j0 + j < w ? __ldcg(xin + cc[j]) : 0.0;
#pragma unroll
      for (int j = 0; j < kSpmvChunk; ++j)
        if (j0 + j < w) s += vv[j] * xx[j];
    }
    if (i < P.n) {
      const double xi = __ldcg(xin + i);
      s += __ldg(P.adiag + i) * xi;
      if (MODE == 0) {
        P.q[i] = s;
        acc += xi * s;
      } else if (MODE == 1) {
        const double ri = __ldcg(P.bh + i) - s;
        P.r[i] = ri;
        acc += ri * ri;
      } else {
        P.q[i] = s;
      }
    }
  }
  if (MODE == 2) return;
  const double tot = cta_sum(acc, red);
  if (threadIdx.x == 0) P.part_a[blockIdx.x] = tot;
  if (MODE == 0 && arrive_last(&P.sc->ticket, gridDim.x, &flag)) {
    const double pq = cta_sum_array(P.part_a, gridDim.x, red, false);
    if (threadIdx.x == 0) {
      P.sc->pq = pq;
      P.sc->alpha = __ldcg(&P.sc->rz) / pq;
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
// IC(0) (up-looking, rows of a group level by level, one row per lane)
// ---------------------------------------------------------------------------
// Row i of the up-looking IC(0): for every j < i in the pattern, ascending,
//   L_ij = (a_ij - sum_{k < j, k in pat(i) and pat(j)} L_ik L_jk) / L_jj,
// then L_ii = sqrt(a_ii - sum_j L_ij^2); rows j are final when row i runs.
// A finished row also stores 1/L_ii, and later rows multiply by it.
// General form: the common columns by a merge of the two sorted rows (a
// chain of dependent loads).
__device__ __forceinline__ void factor_row_merge(const Params &P, int i) {
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
    const double lij = s * __ldcg(P.invd + j);
    P.lval[p] = lij;
    d -= lij * lij;
  }
  if (!(d > 0.0) || !isfinite(d)) {
    atomicMin(P.err_row, (unsigned long long)i);
    d = 1.0;
  }
  const double lii = sqrt(d);
  P.ldiag[i] = lii;
  P.invd[i] = 1.0 / lii;
}

// Rows of at most kFacRow strictly-lower entries whose referenced rows have
// at most kFacRow as well: row i's columns and computed values sit in the
// thread's slice of shared memory (sc, sv), each row j is loaded with
// independent loads into registers, and the common columns are found by
// compare-and-select, so no load waits on another.  The terms are
// subtracted in ascending k, as in the general form.
constexpr int kFacRow = 32;
constexpr int kFacThreads = 64;    // small CTAs: a level's rows spread over many SMs' FP64 units

__device__ __forceinline__ void factor_row(const Params &P, int i, int32_t *sc, double *sv) {
  const int rb = P.lrp[i], ni = P.lrp[i + 1] - rb;
  if (ni > kFacRow) { factor_row_merge(P, i); return; }
  // the row's columns and the longest referenced row (all loads issued at once)
  int nmax = 0;
#pragma unroll
  for (int t = 0; t < kFacRow; ++t) {
    if (t < ni) {
      const int j = __ldg(P.lcol + rb + t);
      sc[t] = j;
      nmax = max(nmax, __ldg(P.lrp + j + 1) - __ldg(P.lrp + j));
    }
  }
  if (nmax > kFacRow) { factor_row_merge(P, i); return; }
  double d = P.adiag[i];
  for (int p = 0; p < ni; ++p) {
    const int j = sc[p];
    const int jb = __ldg(P.lrp + j), nj = __ldg(P.lrp + j + 1) - jb;
    int cj[kFacRow];
    double vj[kFacRow];
#pragma unroll
    for (int u = 0; u < kFacRow; ++u) {
      cj[u] = u < nj ? __ldg(P.lcol + jb + u) : -2;
      vj[u] = u < nj ? __ldcg(P.lval + jb + u) : 0.0;
    }
    double s = __ldg(P.ainit + rb + p);
    for (int t = 0; t < p; ++t) {
      const int c = sc[t];
      double v = 0.0;
      bool hit = false;
#pragma unroll
      for (int u = 0; u < kFacRow; ++u) {
        const bool m = cj[u] == c;
        v = m ? vj[u] : v;
        hit = hit || m;
      }
      if (hit) s -= sv[t] * v;
    }
    // times 1/L_jj (one division per row, at its end, instead of one per
    // entry: FP64 division is a multi-instruction sequence on this GPU)
    const double lij = s * __ldcg(P.invd + j);
    sv[p] = lij;
    d -= lij * lij;
  }
  for (int t = 0; t < ni; ++t) P.lval[rb + t] = sv[t];
  if (!(d > 0.0) || !isfinite(d)) {
    atomicMin(P.err_row, (unsigned long long)i);
    d = 1.0;
  }
  const double lii = sqrt(d);
  P.ldiag[i] = lii;
  P.invd[i] = 1.0 / lii;
}

// Row i from its precomputed update pairs (per entry L_ij, the pairs
// (position of k in row i, index of L_jk) for the common columns k < j,
// ascending k).  A level has few rows, so each row's latency is the cost:
// all pair indices and positions of a pass are copied into shared memory
// with cp.async at once, then all pair values L_jk (rows j are final)
// gathered the same way, then every entry takes its own terms from shared
// memory, k ascending as in the general form.  Shared memory is
// thread-interleaved (element q of thread t at q T + t: no bank conflicts).
constexpr int kFacRowThreads = 32;
constexpr int kFacStage = 160;   // pairs per pass

template <typename T>
struct Strided {
  T *base;
  __device__ __forceinline__ T &operator[](int q) const { return base[q * kFacRowThreads]; }
};


struct FacSmem {
  Strided<double> sv, ivj, pv;
  Strided<int32_t> qe, pb;
  Strided<uint32_t> pw;   // fp_pos bytes, as the 4-byte words covering the pass
};

// STAGE: pairs per pass
// The row's static data (its record, pair indices and positions, columns,
// a_ij, pair ends) is read before griddepcontrol.wait, i.e. while the
// previous level's launch still runs; 1/L_jj and the pair values L_jk after.
template <int STAGE>
__device__ __forceinline__ void factor_row_pairs(const Params &P, int4 rec, const FacSmem &m) {
  const int i = rec.x, rb = rec.y, q0 = rec.z, ni = rec.w & 0xff, np = rec.w >> 8;
  if (ni > kFacRow) {
    pdl_wait();
    factor_row_merge(P, i);
    return;
  }
  // the first pass's pair indices and position words, before anything else
  const uint32_t *posw = reinterpret_cast<const uint32_t *>(P.fp_pos);
  {
    const int nq = min(STAGE, np), w0 = q0 >> 2, w1 = (q0 + nq + 3) >> 2;
    for (int q = 0; q < nq; ++q) cp_async4(&m.pb[q], P.fp_b + q0 + q);
    for (int w = w0; w < w1; ++w) cp_async4(&m.pw[w - w0], posw + w);
    cp_commit();
  }
  {
    int col[kFacRow];
#pragma unroll
    for (int p = 0; p < kFacRow; ++p) col[p] = p < ni ? __ldg(P.lcol + rb + p) : 0;
#pragma unroll
    for (int p = 0; p < kFacRow; ++p)
      if (p < ni) {
        m.sv[p] = __ldg(P.ainit + rb + p);
        m.qe[p] = __ldg(P.fp_ptr + rb + p + 1) - q0;
      }
    pdl_wait();
#pragma unroll
    for (int p = 0; p < kFacRow; ++p)
      if (p < ni) m.ivj[p] = __ldcg(P.invd + col[p]);
  }
  double d = P.adiag[i];
  int p = 0;
  double s = 0.0;
  // entries without terms before the first pair
  while (p < ni && m.qe[p] == 0) {
    const double lij = m.sv[p] * m.ivj[p];
    m.sv[p] = lij;
    d -= lij * lij;
    ++p;
  }
  if (p < ni) s = m.sv[p];
  for (int qa = 0; qa < np; qa += STAGE) {
    const int nq = min(STAGE, np - qa);
    // indices and the words holding the positions (the first pass's were
    // issued at the start)
    const int g0 = q0 + qa, w0 = g0 >> 2, w1 = (g0 + nq + 3) >> 2;
    if (qa > 0) {
      for (int q = 0; q < nq; ++q) cp_async4(&m.pb[q], P.fp_b + g0 + q);
      for (int w = w0; w < w1; ++w) cp_async4(&m.pw[w - w0], posw + w);
      cp_commit();
    }
    cp_wait_all();
    // the pair values
    for (int q = 0; q < nq; ++q) cp_async8(&m.pv[q], P.lval + m.pb[q]);
    cp_commit();
    cp_wait_all();
    const int sh = g0 & 3;
    for (int q = 0; q < nq; ++q) {
      const int bq = q + sh;
      const int pos = int((m.pw[bq >> 2] >> (8 * (bq & 3))) & 0xffu);
      s -= m.sv[pos] * m.pv[q];
      // the entry is complete after its last pair; then the following
      // entries up to the next one with pairs left
      while (p < ni && m.qe[p] == qa + q + 1) {
        const double lij = s * m.ivj[p];
        m.sv[p] = lij;
        d -= lij * lij;
        ++p;
        s = p < ni ? m.sv[p] : 0.0;
      }
    }
  }
  cp_wait_all();   // no copy of this row may land in the next row's buffers
  for (int t = 0; t < ni; ++t) P.lval[rb + t] = m.sv[t];
  if (!(d > 0.0) || !isfinite(d)) {
    atomicMin(P.err_row, (unsigned long long)i);
    d = 1.0;
  }
  const double lii = sqrt(d);
  P.ldiag[i] = lii;
  P.invd[i] = 1.0 / lii;
}

constexpr int kFacPosWords = kFacStage / 4 + 2;
constexpr int kFacSmem = kFacRowThreads * (kFacRow * 20 + kFacStage * 12 + kFacPosWords * 4);

// the rows of one in-block level of a lane-tile or warp-unit color, one row
// per thread (dynamic shared memory, thread-interleaved)
__global__ void __launch_bounds__(kFacRowThreads) factor_rows_kernel(Params P, int k0, int k1) {
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char fsm[];
  const int t = threadIdx.x;
  constexpr int T = kFacRowThreads;
  unsigned char *q = fsm;
  FacSmem m;
  m.sv.base = reinterpret_cast<double *>(q) + t;
  q += size_t(T) * kFacRow * 8;
  m.ivj.base = reinterpret_cast<double *>(q) + t;
  q += size_t(T) * kFacRow * 8;
  m.pv.base = reinterpret_cast<double *>(q) + t;
  q += size_t(T) * kFacStage * 8;
  m.qe.base = reinterpret_cast<int32_t *>(q) + t;
  q += size_t(T) * kFacRow * 4;
  m.pb.base = reinterpret_cast<int32_t *>(q) + t;
  q += size_t(T) * kFacStage * 4;
  m.pw.base = reinterpret_cast<uint32_t *>(q) + t;
  for (int k = k0 + int(blockIdx.x * blockDim.x + threadIdx.x); k < k1; k += int(gridDim.x * blockDim.x)) {
    if (P.fac_rec) {
      factor_row_pairs<kFacStage>(P, __ldg(P.fac_rec + k), m);
    } else {
      pdl_wait();
      factor_row_merge(P, __ldg(P.fac_rows + k));
    }
  }
}

// levels of short rows (at most kFacShort lower entries): one row per thread,
// the general form (short merges), no staging, full CTAs
constexpr int kFacShort = 8;
__global__ void __launch_bounds__(kVecThreads) factor_short_kernel(Params P, int k0, int k1) {
  pdl_trigger();
  pdl_wait();
  for (int k = k0 + int(blockIdx.x * blockDim.x + threadIdx.x); k < k1; k += int(gridDim.x * blockDim.x))
    factor_row_merge(P, __ldg(P.fac_rows + k));
}


// group colors: one CTA per group, its rows level by level of the in-group
// schedule (dynamic shared memory: a kFacRow slice per thread)
__global__ void __launch_bounds__(kMaxWarpsPerCta * kWarp) factor_color_kernel(Params P, int g0, int g1) {
  extern __shared__ __align__(16) unsigned char fsm[];
  int32_t *sc = reinterpret_cast<int32_t *>(fsm) + threadIdx.x * kFacRow;
  double *sv = reinterpret_cast<double *>(fsm + size_t(blockDim.x) * kFacRow * 4) + threadIdx.x * kFacRow;
  const int g = g0 + blockIdx.x;
  if (g >= g1) return;
  const GroupDesc d = P.groups[g];
  for (int lv = 0; lv < d.nlf; ++lv) {
    const int p0 = P.levp[d.lf + lv], p1 = P.levp[d.lf + lv + 1];
    for (int p = p0 + int(threadIdx.x); p < p1; p += blockDim.x) factor_row(P, d.r0 + P.sched_f[d.r0 + p], sc, sv);
    __syncthreads();
  }
}

// invd = 1/L_ii, U values mirrored from L, FP32 copies, sliced-ELL values
__global__ void __launch_bounds__(kVecThreads) factor_finish_kernel(Params P, int nL) {
  const int stride = gridDim.x * blockDim.x;
  // 1/L_ii was stored with each row; its FP32 copy
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += stride) P.invd32[i] = float(P.invd[i]);
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < nL; u += stride) {
    const double lv = P.lval[P.umap[u]];
    P.uval[u] = lv;
    P.uval32[u] = float(lv);
    P.lval32[u] = float(P.lval[u]);
  }
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < P.nsl; e += stride) {
    const int m = P.sl_map[e];
    const double v = m >= 0 ? P.lval[m] : 0.0;
    P.sl_val[e] = v;
    P.sl_val32[e] = float(v);
  }
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < P.nsu; e += stride) {
    const int m = P.su_map[e];
    const double v = m >= 0 ? P.lval[m] : 0.0;
    P.su_val[e] = v;
    P.su_val32[e] = float(v);
  }
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < P.nsi; e += stride) {
    const int m = P.si_map[e];
    const double v = m >= 0 ? P.lval[m] : 0.0;
    P.si_val[e] = v;
    P.si_val32[e] = float(v);
  }
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < P.nui; e += stride) {
    const int m = P.ui_map[e];
    const double v = m >= 0 ? P.lval[m] : 0.0;
    P.ui_val[e] = v;
    P.ui_val32[e] = float(v);
  }
  // warp-unit coefficients: the entry divided by the pivot of its source row
  // (times the stored 1/L_kk)
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < P.nwl; e += stride) {
    const int m = P.wl_map[e];
    const double v = m >= 0 ? P.lval[m] * P.invd[P.wl_srow[e]] : 0.0;
    P.wl_val[e] = v;
    P.wl_val32[e] = float(v);
  }
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < P.nwu; e += stride) {
    const int m = P.wu_map[e];
    const double v = m >= 0 ? P.lval[m] * P.invd[P.wu_srow[e]] : 0.0;
    P.wu_val[e] = v;
    P.wu_val32[e] = float(v);
  }
}

// ---------------------------------------------------------------------------
// Persistent solve: the whole PCG solve in one cooperative launch.  The
// phases of an iteration are
//   SpMV     p = z + beta p (into the other p buffer) and q = A p in one pass:
//            a row's q gathers (z_j + beta p_j), the value the owner of row j
//            stores as its new p_j, so no barrier separates the two; <p,q>
//   fwd c    colors 0 .. n_c-2 (x / r update, <r,r>, L y = r)
//   fused    the last color, forward then backward
//   bwd c    colors n_c-2 .. 0 (L^T z = y, <r,z>)
// with one grid barrier after each (2 n_c per iteration).  Every CTA reduces
// the per-CTA partials itself, in index order, right after the barrier that
// completes them, so all CTAs take identical decisions with no broadcast.
// A CTA walks the groups g0_c + blockIdx.x + k * gridDim.x of each color; the
// static data of its next group (next color, next pass) is copied into the
// other of two shared-memory buffers while it computes the current one, and
// across the barriers in between.
// ---------------------------------------------------------------------------

// A barrier wait gives up after P.wait_ns of wall time (default 4 s, settable
// per context) or kSpinLimit polls, whichever comes first: long enough for any
// phase of a solve the shared-memory plan admits, short enough that a missing
// CTA cannot hang the device.
constexpr long long kSpinLimit = 1ll << 27;

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Sense-reversing grid barrier with a bounded wait.  Returns false (for the
// whole CTA) when this CTA or another one gave up; the error word stays set.
__device__ __forceinline__ bool grid_sync(GridBar *bar, unsigned &gen, int *flag, unsigned long long wait_ns) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    const unsigned arrived = atomicAdd(&bar->count, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(&bar->count, 0u);
      __threadfence();
      atomicExch(&bar->gen, gen + 1);
    } else {
      const unsigned long long t0 = global_ns();
      // the clock is read on every poll (a short limit must take effect at
      // the first poll); the error word of other CTAs every 64 polls
      for (long long k = 1; ld_acquire_u32(&bar->gen) == gen; ++k) {
        if (global_ns() - t0 > wait_ns || k > kSpinLimit ||
            ((k & 63) == 0 && ld_acquire_u32(&bar->err) != 0u)) {
          atomicExch(&bar->err, 1u);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    gen = gen + 1;
    *flag = ok && ld_acquire_u32(&bar->err) == 0u;
  }
  __syncthreads();
  return *flag != 0;
}

// Barrier state of one CTA plus the optional phase trace (CTA 0 records the
// time it leaves each barrier, tagged with the phase that barrier ends).
struct GridSync {
  GridBar *bar;
  unsigned gen;
  int *flag;
  unsigned long long *trace;
  int tk, cap;
  unsigned long long wait_ns;
};

__device__ __forceinline__ bool phase_end(GridSync &s, int tag) {
  const bool ok = grid_sync(s.bar, s.gen, s.flag, s.wait_ns);
  if (s.trace && blockIdx.x == 0 && threadIdx.x == 0 && s.tk < s.cap)
    s.trace[s.tk++] = (global_ns() << 4) | unsigned(tag);
  return ok;
}

// sum of arr[0 .. count) (fixed order), broadcast to every thread
__device__ __forceinline__ double cta_sum_bcast(const double *arr, int count, double *red, double *bc) {
  const double s = cta_sum_array(const_cast<double *>(arr), count, red, false);
  if (threadIdx.x == 0) *bc = s;
  __syncthreads();
  const double v = *bc;
  __syncthreads();
  return v;
}

// One pass over all 32-row tiles of A_hat, one row per lane, entries staged
// per warp.  INIT: r = b_hat - A x_hat, returns this thread's share of <r,r>.
// Otherwise: p_new = z + beta p_old, q = A p_new, share of <p_new, q>.
template <bool INIT, typename ZT>
__device__ __forceinline__ double spmv_pass(const Params &P, unsigned char *smem, int cap, double beta,
                                            const double *pold, double *pnew) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
  double *sv = reinterpret_cast<double *>(smem + warp * (r16((cap + 8) * 8) + r16((cap + 8) * 4)));
  int32_t *sc = reinterpret_cast<int32_t *>(reinterpret_cast<unsigned char *>(sv) + r16((cap + 8) * 8));
  const int ntile = (P.n + kWarp - 1) / kWarp;
  const ZT *z = reinterpret_cast<const ZT *>(P.z);
  double acc = 0.0;
  for (int tile = blockIdx.x * W + warp; tile < ntile; tile += gridDim.x * W) {
    const int t0 = tile * kWarp, t1 = min(P.n, t0 + kWarp);
    const int i = t0 + lane;
    const int rb = i < t1 ? __ldg(P.arp + i) : 0;
    const int re = i < t1 ? __ldg(P.arp + i + 1) : 0;
    const int e0 = __shfl_sync(0xffffffffu, rb, 0);
    const int e1 = __ldg(P.arp + t1);
    Seg<double> S;
    S.gv = P.aval; S.gc = P.acol; S.sv = sv; S.sc = sc;
    S.staged = e1 - e0 <= cap;
    S.bv = S.bc = 0;
    if (S.staged) {
      S.bv = stage_cover<double>(P.aval, e0, e1, sv, lane, kWarp);
      S.bc = stage_cover<int32_t>(P.acol, e0, e1, sc, lane, kWarp);
    }
    cp_commit();
    cp_wait_all();
    __syncwarp();
    if (i < t1) {
      if (INIT) {
        const double s = -row_sub<double, double>(S, rb, re, 0.0, [&](int c) { return __ldcg(P.xh + c); });
        const double ri = __ldcg(P.bh + i) - s;
        P.r[i] = ri;
        acc += ri * ri;
      } else {
        const double s = -row_sub<double, double>(
            S, rb, re, 0.0, [&](int c) { return double(__ldcg(z + c)) + beta * __ldcg(pold + c); });
        const double pi = double(__ldcg(z + i)) + beta * __ldcg(pold + i);
        pnew[i] = pi;
        P.q[i] = s;
        acc += pi * s;
      }
    }
    __syncwarp();
  }
  return acc;
}

// ---- the work items of one preconditioner pass ----------------------------
// Phase ph in [0, 2 n_c - 1): ph < n_c is the forward sweep of color ph (the
// last of them fused with its backward sweep), ph >= n_c the backward sweep
// of color 2 n_c - 2 - ph.  An item is one sweep over one group; the fused
// phase has two per group (sub 0 forward, sub 1 backward).
struct Item {
  int ph, g, sub;
  bool ok, wrap;   // wrap: the item belongs to the next pass
};

__device__ __forceinline__ int ph_color(int ph, int nc) { return ph < nc ? ph : 2 * nc - 2 - ph; }

// first item of this CTA at phase >= ph (group g of phase ph, or its first)
__device__ __forceinline__ Item seek_item(const Params &P, int ph, int g) {
  const int nc = P.n_c;
  for (; ph < 2 * nc - 1; ++ph, g = -1) {
    const int c = ph_color(ph, nc);
    if (g < 0) g = __ldg(P.color_group + c) + int(blockIdx.x);
    if (g < __ldg(P.color_group + c + 1)) return Item{ph, g, 0, true, false};
  }
  return Item{0, 0, 0, false, false};
}

__device__ __forceinline__ Item next_item(const Params &P, const Item &it) {
  if (it.ph == P.n_c - 1 && it.sub == 0) return Item{it.ph, it.g, 1, true, false};
  Item n = seek_item(P, it.ph, it.g + int(gridDim.x));
  if (!n.ok) {
    n = seek_item(P, 0, -1);
    n.wrap = true;
  }
  return n;
}

__device__ __forceinline__ bool item_upper(const Item &it, int nc) { return it.ph >= nc || it.sub == 1; }

// Double-buffered group plan: static data of buffer k at k * o_w, the
// row-work arrays (w, spl) shared by both buffers after them.
template <typename PT>
__device__ __forceinline__ GroupSmem<PT> group_smem_buf(unsigned char *base, const GroupSmemPlan &p, int k) {
  GroupSmem<PT> s = group_smem<PT>(base + k * p.o_w, p);
  s.w = reinterpret_cast<PT *>(base + 2 * p.o_w);
  s.spl = reinterpret_cast<int32_t *>(base + p.o_w + p.o_spl);
  return s;
}

// copies of item it's static data into buffer k, committed as one group
// (an empty group when there is no item)
template <typename PT>
__device__ __forceinline__ void stage_item(const Params &P, const Item &it, unsigned char *smem,
                                           const GroupSmemPlan &plan, int k) {
  if (it.ok) {
    const GroupDesc d = load_group(P.groups + it.g);
    sweep_issue<PT>(P, d, item_upper(it, P.n_c), group_smem_buf<PT>(smem, plan, k), threadIdx.x, blockDim.x);
  }
  cp_commit();
}

// One preconditioner pass (forward colors, fused color, backward colors)
// with a barrier after every phase but the last; `cur` (staged in buffer
// `buf`) is this CTA's first item and becomes the first item of the next
// pass.  Accumulates this thread's <r,r> (UPDATE) and <r,z> shares.
template <typename PT, bool UPDATE>
__device__ __forceinline__ bool precond_pass(const Params &P, const GroupSmemPlan &plan, unsigned char *smem,
                                             Item &cur, int &buf, double alpha, const double *pn, double &rr_acc,
                                             double &rz_acc, GridSync &gs) {
  const int nc = P.n_c, nph = 2 * nc - 1;
  const int tid = threadIdx.x, nthr = blockDim.x;
  cur.wrap = false;
  for (int ph = 0; ph < nph; ++ph) {
    while (cur.ok && !cur.wrap && cur.ph == ph) {
      const Item nx = next_item(P, cur);
      stage_item<PT>(P, nx, smem, plan, buf ^ 1);
      cp_wait_prev();
      __syncthreads();
      const GroupSmem<PT> m = group_smem_buf<PT>(smem, plan, buf);
      const GroupDesc d = load_group(P.groups + cur.g);
      const bool fused = ph == nc - 1;
      if (!item_upper(cur, nc)) {
        const Sweep<PT> sw = sweep_desc<PT>(P, d, false, m);
        group_sweep<PT, false, UPDATE>(P, d, sw, m, tid, nthr, alpha, pn, false, !fused || !sw.fit, rr_acc,
                                       rz_acc);
      } else {
        const Sweep<PT> sw = sweep_desc<PT>(P, d, true, m);
        group_sweep<PT, true, false>(P, d, sw, m, tid, nthr, 0.0, nullptr, fused && sw.fit, true, rr_acc, rz_acc);
      }
      buf ^= 1;
      cur = nx;
    }
    if (ph < nph - 1 && !phase_end(gs, ph < nc - 1 ? PH_FWD : (ph == nc - 1 ? PH_FUSED : PH_BWD))) return false;
  }
  return true;
}

// 64 registers a thread: up to 2 CTAs of 16 warps (or 8 of 4) per SM
#ifndef ICCG_PERSIST_MIN_CTAS
#define ICCG_PERSIST_MIN_CTAS 2
#endif

template <typename PT>
__global__ void __launch_bounds__(kMaxWarpsPerCta * kWarp, ICCG_PERSIST_MIN_CTAS)
persistent_kernel(Params P, GroupSmemPlan plan, int cap_a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[kMaxWarpsPerCta];
  __shared__ double bc;
  __shared__ int flag;
  const int tid = threadIdx.x, nthr = blockDim.x, nb = gridDim.x, b = blockIdx.x;
  const int gstride = nb * nthr, gi = b * nthr + tid;
  unsigned char *smem_a = smem + plan.o_w + plan.total;   // SpMV staging
  GridSync gs{P.bar, 0u, &flag, P.trace, 0, P.trace_cap, P.wait_ns};
  Scalars *S = P.sc;
  const double tol = __ldcg(&S->tol);
  const int maxit = __ldcg(&S->maxit);
  double *pp_a = P.part0, *pp_b = P.part1;   // per-CTA partials [gridDim.x]
  int status = ICCG_ERR_TIMEOUT, it = 0;
  bool ok = true;

  // this CTA's first preconditioner item, staged while the solve starts
  int buf = 0;
  Item cur = seek_item(P, 0, -1);
  stage_item<PT>(P, cur, smem, plan, 0);

  // solve start: b_hat, x_hat, p = 0, <b,b>
  double acc = 0.0;
  for (int i = gi; i < P.n; i += gstride) {
    const int o = __ldg(P.perm + i);
    const double bi = __ldcg(P.bin + o);
    P.bh[i] = bi;
    P.xh[i] = __ldcg(P.xin + o);
    P.p0[i] = 0.0;
    acc += bi * bi;
  }
  acc = cta_sum(acc, red);
  if (tid == 0) P.init_bb[b] = acc;
  ok = phase_end(gs, PH_INIT);
  // r0 = b_hat - A x_hat, <r0, r0>
  if (ok) {
    acc = cta_sum(spmv_pass<true, PT>(P, smem_a, cap_a, 0.0, nullptr, nullptr), red);
    if (tid == 0) pp_a[b] = acc;
    ok = phase_end(gs, PH_INIT);
  }
  // z0 = M^-1 r0, <r0, z0>
  double rr_acc = 0.0, rz_acc = 0.0;
  if (ok) ok = precond_pass<PT, false>(P, plan, smem, cur, buf, 0.0, nullptr, rr_acc, rz_acc, gs);
  if (ok) {
    acc = cta_sum(rz_acc, red);
    if (tid == 0) pp_b[b] = acc;
    ok = phase_end(gs, PH_INIT);
  }
  double bnorm = 0.0, rz = 0.0;
  bool done = false;
  if (ok) {
    const double bb = cta_sum_bcast(P.init_bb, nb, red, &bc);
    const double rr0 = cta_sum_bcast(pp_a, nb, red, &bc);
    rz = cta_sum_bcast(pp_b, nb, red, &bc);
    bnorm = sqrt(bb);
    if (bnorm == 0.0) {
      done = true;
      status = ICCG_OK;
      if (b == 0 && tid == 0) P.hist[0] = 0.0;
    } else {
      const double rn = sqrt(rr0) / bnorm;
      if (b == 0 && tid == 0) P.hist[0] = rn;
      if (!isfinite(rn) || !isfinite(rz)) { done = true; status = ICCG_ERR_NONFINITE; }
      else if (rn <= tol) { done = true; status = ICCG_OK; }
      else if (maxit <= 0) { done = true; status = ICCG_NOT_CONVERGED; }
    }
    // pp_a is next written by the SpMV, read after its barrier; pp_b after at
    // least one color barrier: every CTA has read both by then
  }
  double beta = 0.0;
  while (ok && !done) {
    // p_new = z + beta p_old, q = A p_new, <p_new, q>, alpha
    const double *pold = (it & 1) ? P.p1 : P.p0;
    double *pnew = (it & 1) ? P.p0 : P.p1;
    acc = cta_sum(spmv_pass<false, PT>(P, smem_a, cap_a, beta, pold, pnew), red);
    if (tid == 0) pp_a[b] = acc;
    if (!(ok = phase_end(gs, PH_SPMV))) break;
    const double pq = cta_sum_bcast(pp_a, nb, red, &bc);
    const double alpha = rz / pq;
    // x / r update, forward and backward substitution
    rr_acc = 0.0;
    rz_acc = 0.0;
    if (!(ok = precond_pass<PT, true>(P, plan, smem, cur, buf, alpha, pnew, rr_acc, rz_acc, gs))) break;
    const double rrc = cta_sum(rr_acc, red);
    const double rzc = cta_sum(rz_acc, red);
    if (tid == 0) { pp_a[b] = rrc; pp_b[b] = rzc; }
    if (!(ok = phase_end(gs, PH_BWD))) break;
    const double rr = cta_sum_bcast(pp_a, nb, red, &bc);
    const double rz_new = cta_sum_bcast(pp_b, nb, red, &bc);
    ++it;
    const double rn = sqrt(rr) / bnorm;
    if (b == 0 && tid == 0) P.hist[it] = rn;
    if (!isfinite(rn) || !isfinite(rz_new)) { done = true; status = ICCG_ERR_NONFINITE; }
    else if (rn <= tol) { done = true; status = ICCG_OK; }
    else if (it >= maxit) { done = true; status = ICCG_NOT_CONVERGED; }
    else {
      beta = rz_new / rz;
      rz = rz_new;
    }
  }
  cp_wait_all();
  if (ok) {
    for (int i = gi; i < P.n; i += gstride) P.xout[__ldg(P.perm + i)] = bnorm == 0.0 ? 0.0 : __ldcg(P.xh + i);
  }
  if (b == 0 && tid == 0) {
    S->iter = it;
    S->status = ok ? status : ICCG_ERR_TIMEOUT;
    S->bnorm = bnorm;
    S->done = 1;
    if (P.trace && gs.tk < P.trace_cap) P.trace[gs.tk++] = (global_ns() << 4) | unsigned(PH_ALL);
    if (P.trace_len) *P.trace_len = gs.tk;
  }
}

// ---------------------------------------------------------------------------
// Cooperative sweep: a whole preconditioner application in one launch for a
// layout whose colors are all pair tiles (blocks of one or two rows): the
// forward colors, the fused last color and the backward colors (Alg. 1 and
// the reverse sweep) one after another, each color's tiles taken grid-stride
// by every warp of the grid, a bounded grid barrier where a color needs the
// previous one's results; one reduction closes the launch.  It replaces the
// 2 n_c - 1 color launches of the sweep, whose fixed cost (launch, ramp-up,
// tail, per-launch reduction) dominates colors of few rows.
// ---------------------------------------------------------------------------
constexpr int kCoopWarps = 8;

// c_lo > 0: the tail of a sweep (forward colors c_lo .. n_c - 2, the fused
// last color, backward colors n_c - 2 .. c_lo), between per-color launches;
// its <r,r> / <r,z> partials go to the slot regions of those colors (one per
// CTA in the first region of each, zeros in the others), which the
// iteration's last launch sums.
template <typename PT, bool UPDATE>
__global__ void __launch_bounds__(kCoopWarps * kWarp)
coop_sweep_kernel(Params P, int c_lo, int fin, int rr0, int ntail) {
  __shared__ double red[kMaxWarpsPerCta];
  __shared__ int flag;
  const int lane = threadIdx.x & 31;
  const int nw = int(blockDim.x >> 5), gw = int(blockIdx.x) * nw + int(threadIdx.x >> 5);
  const int NW = int(gridDim.x) * nw, nc = P.n_c;
  double rr_acc = 0.0, rz_acc = 0.0;
  pdl_wait();
  const double alpha = UPDATE ? __ldcg(&P.sc->alpha) : 0.0;
  GridSync gs{P.bar, 0u, &flag, nullptr, 0, 0, P.wait_ns};
  bool ok = true;
  for (int c = c_lo; c < nc - 1 && ok; ++c) {
    const int t1 = __ldg(P.ctile + c + 1);
    for (int t = __ldg(P.ctile + c) + gw; t < t1; t += NW) pair_tile<PT, M_FWD, UPDATE>(P, t, lane, alpha, rr_acc, rz_acc);
    ok = phase_end(gs, PH_FWD);
  }
  if (ok) {
    const int t1 = __ldg(P.ctile + nc);
    for (int t = __ldg(P.ctile + nc - 1) + gw; t < t1; t += NW)
      pair_tile<PT, M_FUSED, UPDATE>(P, t, lane, alpha, rr_acc, rz_acc);
  }
  for (int c = nc - 2; c >= c_lo && ok; --c) {
    if (!(ok = phase_end(gs, PH_BWD))) break;
    const int t1 = __ldg(P.ctile + c + 1);
    for (int t = __ldg(P.ctile + c) + gw; t < t1; t += NW) pair_tile<PT, M_BWD, false>(P, t, lane, alpha, rr_acc, rz_acc);
  }
  if (!ok) {
    // a barrier wait gave up: the solve stops with ICCG_ERR_TIMEOUT
    if (threadIdx.x == 0) {
      P.sc->status = ICCG_ERR_TIMEOUT;
      P.sc->done = 1;
      set_condition(P.sc, 0);
    }
    return;
  }
  if (c_lo > 0) {
    const double rr_c = UPDATE ? cta_sum(rr_acc, red) : 0.0;
    const double rz_c = cta_sum(rz_acc, red);
    if (threadIdx.x == 0) {
      const int G = int(gridDim.x), b = int(blockIdx.x);
      for (int k = 0; k < ntail; ++k) {
        if (UPDATE) P.slot_rr[rr0 + k * G + b] = k == 0 ? rr_c : 0.0;
        P.slot_rz[k * G + b] = k == 0 ? rz_c : 0.0;
      }
    }
    return;
  }
  if (fin == FIN_NONE) return;
  launch_epilogue(P, fin, SlotArgs{0, 0, 0, 0}, UPDATE, true, rr_acc, rz_acc, red, &flag);
}

// ---------------------------------------------------------------------------
// launch helpers
// ---------------------------------------------------------------------------
template <typename... KArgs, typename... Args>
cudaError_t launch_coop(void (*kernel)(KArgs...), int grid, int threads, int smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(grid));
  cfg.blockDim = dim3(unsigned(threads));
  cfg.dynamicSmemBytes = size_t(smem);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

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

template <typename PT>
GroupSmemPlan plan_of(const Params &P, bool fused, bool upper) {
  const int cap = fused ? max(P.cap_l, P.cap_u) : (upper ? P.cap_u : P.cap_l);
  return group_smem_plan(cap, P.cap_rows, P.cap_lev, int(sizeof(PT)));
}

template <typename PT>
TilePlan tile_plan_of(const Params &P, bool stage_ext = true) {
  TilePlan p = tile_plan(P.lane_max, P.tcap_r, P.tcap_i, int(sizeof(PT)), stage_ext ? P.tcap_o : 0);
  p.nbuf = P.tnbuf;
  p.cap_i2 = P.tcap_i2;
  return p;
}

template <typename PT>
cudaError_t launch_tile(const Params &P, const Plan &L, int c, int mode, bool update, int fin, const SlotArgs &sa) {
  const TilePlan pl = tile_plan_of<PT>(P, L.stage_ext[c] != 0);
  const int g = L.grid_c[c], t0 = L.tile0[c], t1 = L.tile1[c], th = L.Wt * kWarp;
  const int sm = tile_launch_bytes(pl, mode == M_FUSED);
  if (mode == M_BWD) return launch(tile_kernel<PT, M_BWD, false>, g, th, sm, L, P, t0, t1, pl, fin, sa);
  if (update) {
    if (mode == M_FUSED) return launch(tile_kernel<PT, M_FUSED, true>, g, th, sm, L, P, t0, t1, pl, fin, sa);
    return launch(tile_kernel<PT, M_FWD, true>, g, th, sm, L, P, t0, t1, pl, fin, sa);
  }
  if (mode == M_FUSED) return launch(tile_kernel<PT, M_FUSED, false>, g, th, sm, L, P, t0, t1, pl, fin, sa);
  return launch(tile_kernel<PT, M_FWD, false>, g, th, sm, L, P, t0, t1, pl, fin, sa);
}

template <typename PT>
cudaError_t launch_wtile(const Params &P, const Plan &L, int c, int mode, bool update, int fin, const SlotArgs &sa) {
  const int g = L.grid_c[c], t0 = L.tile0[c], t1 = L.tile1[c], th = L.Ww * kWarp, sm = L.smem_wt, cs = L.cap_ws;
  if (mode == M_BWD) return launch(wtile_kernel<PT, M_BWD, false>, g, th, sm, L, P, t0, t1, cs, fin, sa);
  if (update) {
    if (mode == M_FUSED) return launch(wtile_kernel<PT, M_FUSED, true>, g, th, sm, L, P, t0, t1, cs, fin, sa);
    return launch(wtile_kernel<PT, M_FWD, true>, g, th, sm, L, P, t0, t1, cs, fin, sa);
  }
  if (mode == M_FUSED) return launch(wtile_kernel<PT, M_FUSED, false>, g, th, sm, L, P, t0, t1, cs, fin, sa);
  return launch(wtile_kernel<PT, M_FWD, false>, g, th, sm, L, P, t0, t1, cs, fin, sa);
}

template <typename PT, bool STAGE>
cudaError_t launch_pair_s(const Params &P, const Plan &L, int c, int mode, bool update, int fin,
                          const SlotArgs &sa) {
  const int g = L.grid_c[c], t0 = L.tile0[c], t1 = L.tile1[c], th = L.Wp * kWarp;
  const int sm = STAGE ? L.Wp * pair_stage_bytes<PT>() : 0;
  if (mode == M_BWD) return launch(pair_kernel<PT, M_BWD, false, STAGE>, g, th, sm, L, P, t0, t1, fin, sa);
  if (update) {
    if (mode == M_FUSED) return launch(pair_kernel<PT, M_FUSED, true, STAGE>, g, th, sm, L, P, t0, t1, fin, sa);
    return launch(pair_kernel<PT, M_FWD, true, STAGE>, g, th, sm, L, P, t0, t1, fin, sa);
  }
  if (mode == M_FUSED) return launch(pair_kernel<PT, M_FUSED, false, STAGE>, g, th, sm, L, P, t0, t1, fin, sa);
  return launch(pair_kernel<PT, M_FWD, false, STAGE>, g, th, sm, L, P, t0, t1, fin, sa);
}

template <typename PT>
cudaError_t launch_pair(const Params &P, const Plan &L, int c, int mode, bool update, int fin, const SlotArgs &sa) {
  const bool stage = mode == M_BWD ? L.pstage_b[c] != 0 : L.pstage_f[c] != 0;
  return stage ? launch_pair_s<PT, true>(P, L, c, mode, update, fin, sa)
               : launch_pair_s<PT, false>(P, L, c, mode, update, fin, sa);
}

template <typename PT, int S>
cudaError_t launch_unit_s(const Params &P, const Plan &L, int c, int mode, bool update, int fin, const SlotArgs &sa) {
  const int g = L.grid_c[c], t0 = L.unit0[c], t1 = L.unit1[c], th = kUnitWarps * kWarp;
  const int sm = unit_smem_bytes(S, int(sizeof(PT)));
  if (mode == M_BWD) return launch(unit_kernel<PT, M_BWD, false, S>, g, th, sm, L, P, t0, t1, fin, sa);
  if (update) {
    if (mode == M_FUSED) return launch(unit_kernel<PT, M_FUSED, true, S>, g, th, sm, L, P, t0, t1, fin, sa);
    return launch(unit_kernel<PT, M_FWD, true, S>, g, th, sm, L, P, t0, t1, fin, sa);
  }
  if (mode == M_FUSED) return launch(unit_kernel<PT, M_FUSED, false, S>, g, th, sm, L, P, t0, t1, fin, sa);
  return launch(unit_kernel<PT, M_FWD, false, S>, g, th, sm, L, P, t0, t1, fin, sa);
}

template <typename PT>
cudaError_t launch_unit(const Params &P, const Plan &L, int c, int mode, bool update, int fin, const SlotArgs &sa) {
  switch (L.unit_S[c]) {
    case 1: return launch_unit_s<PT, 1>(P, L, c, mode, update, fin, sa);
    case 2: return launch_unit_s<PT, 2>(P, L, c, mode, update, fin, sa);
    case 4: return launch_unit_s<PT, 4>(P, L, c, mode, update, fin, sa);
    case 8: return launch_unit_s<PT, 8>(P, L, c, mode, update, fin, sa);
    case 16: return launch_unit_s<PT, 16>(P, L, c, mode, update, fin, sa);
    default: return launch_unit_s<PT, 32>(P, L, c, mode, update, fin, sa);
  }
}

template <typename PT>
cudaError_t launch_fwd(const Params &P, const Plan &L, int c, bool update, bool fused, int fin) {
  if (L.unit1[c] > L.unit0[c])
    return launch_unit<PT>(P, L, c, fused ? M_FUSED : M_FWD, update, fin, SlotArgs{L.off_rr[c], L.off_rz[c], 0, 0});
  if (L.tile1[c] > L.tile0[c] && L.wtile[c] == 2)
    return launch_pair<PT>(P, L, c, fused ? M_FUSED : M_FWD, update, fin, SlotArgs{L.off_rr[c], L.off_rz[c], 0, 0});
  if (L.tile1[c] > L.tile0[c] && L.wtile[c])
    return launch_wtile<PT>(P, L, c, fused ? M_FUSED : M_FWD, update, fin, SlotArgs{L.off_rr[c], L.off_rz[c], 0, 0});
  if (L.tile1[c] > L.tile0[c])
    return launch_tile<PT>(P, L, c, fused ? M_FUSED : M_FWD, update, fin, SlotArgs{L.off_rr[c], L.off_rz[c], 0, 0});
  const int threads = L.W * kWarp;
  const GroupSmemPlan pl = plan_of<PT>(P, fused, false);
  const int smem = pl.total;
  const int g = L.grid_c[c], t0 = L.task0[c], t1 = L.task1[c];
  // a final fused launch (one color) has no earlier slots
  const SlotArgs sa{L.off_rr[c], L.off_rz[c], 0, 0};
  if (update) {
    if (fused) return launch(color_kernel<PT, M_FUSED, true>, g, threads, smem, L, P, t0, t1, pl, fin, sa);
    return launch(color_kernel<PT, M_FWD, true>, g, threads, smem, L, P, t0, t1, pl, fin, sa);
  }
  if (fused) return launch(color_kernel<PT, M_FUSED, false>, g, threads, smem, L, P, t0, t1, pl, fin, sa);
  return launch(color_kernel<PT, M_FWD, false>, g, threads, smem, L, P, t0, t1, pl, fin, sa);
}

template <typename PT>
cudaError_t launch_bwd(const Params &P, const Plan &L, int c, int fin) {
  const GroupSmemPlan pl = plan_of<PT>(P, false, true);
  // the final backward launch sums the <r,r> slots only in an iteration (the
  // solve start has no x / r update)
  const SlotArgs sa{0, L.off_rz[c], fin == FIN_ITER ? L.last_rr : 0, L.last_rz};
  if (L.unit1[c] > L.unit0[c]) return launch_unit<PT>(P, L, c, M_BWD, false, fin, sa);
  if (L.tile1[c] > L.tile0[c] && L.wtile[c] == 2) return launch_pair<PT>(P, L, c, M_BWD, false, fin, sa);
  if (L.tile1[c] > L.tile0[c] && L.wtile[c]) return launch_wtile<PT>(P, L, c, M_BWD, false, fin, sa);
  if (L.tile1[c] > L.tile0[c]) return launch_tile<PT>(P, L, c, M_BWD, false, fin, sa);
  return launch(color_kernel<PT, M_BWD, false>, L.grid_c[c], L.W * kWarp, pl.total, L, P, L.task0[c],
                L.task1[c], pl, fin, sa);
}

// Forward sweep (with or without the x/r update), fused last color, backward
// sweep.  fin_last: the epilogue run by the last launch.
template <typename PT>
cudaError_t launch_coop_sweep(const Params &P, const Plan &L, bool update, int fin) {
  cudaError_t e = cudaMemsetAsync(P.bar, 0, sizeof(GridBar), L.stream);
  if (e != cudaSuccess) return e;
  if (update) return launch_coop(coop_sweep_kernel<PT, true>, L.grid_coop, kCoopWarps * kWarp, 0, L.stream, P, 0, fin, 0, 0);
  return launch_coop(coop_sweep_kernel<PT, false>, L.grid_coop, kCoopWarps * kWarp, 0, L.stream, P, 0, fin, 0, 0);
}

// the sweep's tail colors (tail_c .. n_c - 1) in one cooperative launch
template <typename PT>
cudaError_t launch_coop_tail(const Params &P, const Plan &L, bool update) {
  cudaError_t e = cudaMemsetAsync(P.bar, 0, sizeof(GridBar), L.stream);
  if (e != cudaSuccess) return e;
  const int ct = L.tail_c, nt = L.n_c - ct, rr0 = L.off_rr[ct];
  if (update)
    return launch_coop(coop_sweep_kernel<PT, true>, L.grid_tail, kCoopWarps * kWarp, 0, L.stream, P, ct, int(FIN_NONE),
                       rr0, nt);
  return launch_coop(coop_sweep_kernel<PT, false>, L.grid_tail, kCoopWarps * kWarp, 0, L.stream, P, ct, int(FIN_NONE),
                     rr0, nt);
}

template <typename PT>
cudaError_t sweep(const Params &P, const Plan &L, bool update, int fin_last, PhaseHook h, void *u) {
  cudaError_t e = cudaSuccess;
  const int nc = L.n_c;
  if (L.coop) {
    if (h) h(u, PH_FWD, 1);
    e = launch_coop_sweep<PT>(P, L, update, fin_last);
    if (h) h(u, PH_FWD, 0);
    return e;
  }
  if (L.tail_c > 0) {
    for (int c = 0; c < L.tail_c && e == cudaSuccess; ++c) {
      if (h) h(u, PH_FWD, 1);
      e = launch_fwd<PT>(P, L, c, update, false, FIN_NONE);
      if (h) h(u, PH_FWD, 0);
    }
    if (e != cudaSuccess) return e;
    if (h) h(u, PH_FUSED, 1);
    e = launch_coop_tail<PT>(P, L, update);
    if (h) h(u, PH_FUSED, 0);
    for (int c = L.tail_c - 1; c >= 0 && e == cudaSuccess; --c) {
      if (h) h(u, PH_BWD, 1);
      e = launch_bwd<PT>(P, L, c, c == 0 ? fin_last : FIN_NONE);
      if (h) h(u, PH_BWD, 0);
    }
    return e;
  }
  for (int c = 0; c < nc - 1 && e == cudaSuccess; ++c) {
    if (h) h(u, PH_FWD, 1);
    e = launch_fwd<PT>(P, L, c, update, false, FIN_NONE);
    if (h) h(u, PH_FWD, 0);
  }
  if (e != cudaSuccess) return e;
  if (h) h(u, PH_FUSED, 1);
  e = launch_fwd<PT>(P, L, nc - 1, update, true, nc == 1 ? fin_last : FIN_NONE);
  if (h) h(u, PH_FUSED, 0);
  for (int c = nc - 2; c >= 0 && e == cudaSuccess; --c) {
    if (h) h(u, PH_BWD, 1);
    e = launch_bwd<PT>(P, L, c, c == 0 ? fin_last : FIN_NONE);
    if (h) h(u, PH_BWD, 0);
  }
  return e;
}

template <int MODE>
cudaError_t launch_spmv(const Params &P, const Plan &L) {
  return launch(spmv_kernel<MODE>, L.grid_a, L.Wa * kWarp, 0, L, P);
}

template <typename K>
cudaError_t allow_smem(K kernel) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - 1024);
}

template <typename PT>
cudaError_t configure_pt() {
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = allow_smem(color_kernel<PT, M_FUSED, true>);
  if (e == cudaSuccess) e = allow_smem(color_kernel<PT, M_FWD, true>);
  if (e == cudaSuccess) e = allow_smem(color_kernel<PT, M_FUSED, false>);
  if (e == cudaSuccess) e = allow_smem(color_kernel<PT, M_FWD, false>);
  if (e == cudaSuccess) e = allow_smem(color_kernel<PT, M_BWD, false>);
  if (e == cudaSuccess) e = allow_smem(persistent_kernel<PT>);
  if (e == cudaSuccess) e = allow_smem(tile_kernel<PT, M_FUSED, true>);
  if (e == cudaSuccess) e = allow_smem(tile_kernel<PT, M_FWD, true>);
  if (e == cudaSuccess) e = allow_smem(tile_kernel<PT, M_FUSED, false>);
  if (e == cudaSuccess) e = allow_smem(tile_kernel<PT, M_FWD, false>);
  if (e == cudaSuccess) e = allow_smem(tile_kernel<PT, M_BWD, false>);
  if (e == cudaSuccess) e = allow_smem(pair_kernel<PT, M_FUSED, true, true>);
  if (e == cudaSuccess) e = allow_smem(pair_kernel<PT, M_FWD, true, true>);
  if (e == cudaSuccess) e = allow_smem(pair_kernel<PT, M_FUSED, false, true>);
  if (e == cudaSuccess) e = allow_smem(pair_kernel<PT, M_FWD, false, true>);
  if (e == cudaSuccess) e = allow_smem(pair_kernel<PT, M_BWD, false, true>);
  if (e == cudaSuccess) e = allow_smem(wtile_kernel<PT, M_FUSED, true>);
  if (e == cudaSuccess) e = allow_smem(wtile_kernel<PT, M_FWD, true>);
  if (e == cudaSuccess) e = allow_smem(wtile_kernel<PT, M_FUSED, false>);
  if (e == cudaSuccess) e = allow_smem(wtile_kernel<PT, M_FWD, false>);
  if (e == cudaSuccess) e = allow_smem(wtile_kernel<PT, M_BWD, false>);
  if (e == cudaSuccess) e = allow_smem(unit_kernel<PT, M_FWD, true, 32>);
  if (e == cudaSuccess) e = allow_smem(unit_kernel<PT, M_FWD, false, 32>);
  if (e == cudaSuccess) e = allow_smem(unit_kernel<PT, M_FUSED, true, 32>);
  if (e == cudaSuccess) e = allow_smem(unit_kernel<PT, M_FUSED, false, 32>);
  if (e == cudaSuccess) e = allow_smem(unit_kernel<PT, M_BWD, false, 32>);
  return e;
}

}  // namespace

int group_smem_bytes(int cap, int rows, int levs, int elem) { return group_smem_plan(cap, rows, levs, elem).total; }
int spmv_smem_bytes(int cap) { return r16((cap + 8) * 8) + r16((cap + 8) * 4); }

int tile_resident_ctas(bool fp32, int threads, int smem) {
  int nb = 0;
  const cudaError_t e =
      fp32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, tile_kernel<float, M_FUSED, true>, threads, size_t(smem))
           : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, tile_kernel<double, M_FUSED, true>, threads, size_t(smem));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return nb > 0 ? nb : 1;
}

int wtile_resident_ctas(bool fp32, int threads, int smem) {
  int nb = 0;
  const cudaError_t e =
      fp32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, wtile_kernel<float, M_FWD, true>, threads, size_t(smem))
           : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, wtile_kernel<double, M_FWD, true>, threads, size_t(smem));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return nb > 0 ? nb : 1;
}

int pair_resident_ctas(bool fp32, int threads) {
  int nb = 0;
  const cudaError_t e =
      fp32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pair_kernel<float, M_FWD, true, true>, threads,
                                                           size_t(threads / kWarp) * pair_stage_bytes<float>())
           : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pair_kernel<double, M_FWD, true, true>, threads,
                                                           size_t(threads / kWarp) * pair_stage_bytes<double>());
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return nb > 0 ? nb : 1;
}

int coop_sweep_resident_ctas(bool fp32) {
  int nb = 0;
  const cudaError_t e =
      fp32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, coop_sweep_kernel<float, true>, kCoopWarps * kWarp, 0)
           : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, coop_sweep_kernel<double, true>, kCoopWarps * kWarp, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}

int unit_resident_ctas(bool fp32, int S, int threads) {
  int nb = 0;
  cudaError_t e;
  const size_t sm = size_t(unit_smem_bytes(S <= 8 ? 8 : 32, fp32 ? 4 : 8));
  if (fp32) {
    e = S <= 8 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, unit_kernel<float, M_FWD, true, 8>, threads, sm)
               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, unit_kernel<float, M_FWD, true, 32>, threads, sm);
  } else {
    e = S <= 8 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, unit_kernel<double, M_FWD, true, 8>, threads, sm)
               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, unit_kernel<double, M_FWD, true, 32>, threads, sm);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return nb > 0 ? nb : 1;
}

int spmv_resident_ctas(int Wa, int smem) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, spmv_kernel<0>, Wa * kWarp, size_t(smem)) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return nb > 0 ? nb : 1;
}

int persistent_smem_bytes(const Params &P, bool fp32, int W, int budget, int *cap_spmv) {
  const GroupSmemPlan pl = fp32 ? plan_of<float>(P, true, false) : plan_of<double>(P, true, false);
  // two buffers of static group data, the shared row-work arrays, then the
  // SpMV staging; a tile larger than the staging capacity that fits the
  // budget reads global memory instead
  const int groups = pl.o_w + pl.total;
  int cap = P.cap_a;
  while (cap > 4 && W * spmv_smem_bytes(cap) > budget) cap = std::max(4, (cap / 2) & ~3);
  *cap_spmv = cap;
  return groups + W * spmv_smem_bytes(cap);
}

int persistent_resident_ctas(bool fp32, int W, int smem) {
  int nb = 0;
  const cudaError_t e =
      fp32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, persistent_kernel<float>, W * kWarp, size_t(smem))
           : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, persistent_kernel<double>, W * kWarp, size_t(smem));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}

cudaError_t launch_solve_persistent(const Params &P, const Plan &L, bool fp32) {
  cudaError_t e = cudaMemsetAsync(P.bar, 0, sizeof(GridBar), L.stream);
  if (e != cudaSuccess) return e;
  const int threads = L.W * kWarp;
  if (fp32)
    return launch_coop(persistent_kernel<float>, L.grid_p, threads, L.smem_p, L.stream, P,
                       plan_of<float>(P, true, false), L.cap_p);
  return launch_coop(persistent_kernel<double>, L.grid_p, threads, L.smem_p, L.stream, P,
                     plan_of<double>(P, true, false), L.cap_p);
}

cudaError_t configure_kernels() {
  cudaError_t e = cudaFuncSetAttribute(factor_color_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kMaxWarpsPerCta * kWarp * kFacRow * 12);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(factor_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kFacSmem);
  if (e == cudaSuccess) e = configure_pt<double>();
  if (e == cudaSuccess) e = configure_pt<float>();
  return e;
}

cudaError_t launch_factor(const Params &P, const Plan &L, int nL) {
  for (int c = 0; c < L.n_c; ++c) {
    if (L.tile1[c] > L.tile0[c] || L.unit1[c] > L.unit0[c]) {
      // lane-tile and warp-unit colors: one launch per in-block level, a thread per row
      for (int v = 0; v < L.fac_nlev[c]; ++v) {
        const int k0 = L.fac_ptr[size_t(L.fac_lev0[c] + v)], k1 = L.fac_ptr[size_t(L.fac_lev0[c] + v + 1)];
        // consecutive levels overlap through programmatic dependent launch:
        // a level's static loads run while the previous level finishes
        cudaError_t e;
        if (L.fac_wide[size_t(L.fac_lev0[c] + v)] <= kFacShort) {
          const int grid = std::max(1, std::min((k1 - k0 + kVecThreads - 1) / kVecThreads, L.grid_v));
          e = launch(factor_short_kernel, grid, kVecThreads, 0, L, P, k0, k1);
        } else {
          const int grid = std::max(1, std::min((k1 - k0 + kFacRowThreads - 1) / kFacRowThreads, 8 * L.grid_v));
          e = launch(factor_rows_kernel, grid, kFacRowThreads, kFacSmem, L, P, k0, k1);
        }
        if (e != cudaSuccess) return e;
      }
    } else {
      const int threads = L.W * kWarp;
      factor_color_kernel<<<L.grid_c[c], threads, size_t(threads) * kFacRow * 12, L.stream>>>(P, L.task0[c], L.task1[c]);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  factor_finish_kernel<<<L.grid_v, kVecThreads, 0, L.stream>>>(P, nL);
  return cudaGetLastError();
}

cudaError_t launch_solve_init(const Params &P, const Plan &L, bool fp32, PhaseHook h, void *u) {
  if (h) h(u, PH_INIT, 1);
  cudaError_t e = cudaMemsetAsync(P.gticket, 0, sizeof(uint32_t) * size_t(P.ngroup), L.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(P.p0, 0, sizeof(double) * size_t(P.n > 0 ? P.n : 1), L.stream);
  if (e == cudaSuccess) {
    perm_in_kernel<<<L.grid_v, kVecThreads, 0, L.stream>>>(P);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = launch_spmv<1>(P, L);
  if (h) h(u, PH_INIT, 0);
  if (e != cudaSuccess) return e;
  if (h) h(u, PH_INIT, 1);
  e = fp32 ? sweep<float>(P, L, false, FIN_INIT, nullptr, nullptr) : sweep<double>(P, L, false, FIN_INIT, nullptr, nullptr);
  if (h) h(u, PH_INIT, 0);
  return e;
}

cudaError_t launch_spmv_phase(const Params &P, const Plan &L, bool fp32) {
  cudaError_t e = fp32 ? launch(pupdate_kernel<float>, L.grid_v, kVecThreads, 0, L, P)
                       : launch(pupdate_kernel<double>, L.grid_v, kVecThreads, 0, L, P);
  if (e == cudaSuccess) e = launch_spmv<0>(P, L);
  return e;
}

cudaError_t launch_solve_body(const Params &P, const Plan &L, bool fp32, PhaseHook h, void *u) {
  if (h) h(u, PH_SPMV, 1);
  cudaError_t e = launch_spmv_phase(P, L, fp32);
  if (h) h(u, PH_SPMV, 0);
  if (e != cudaSuccess) return e;
  return fp32 ? sweep<float>(P, L, true, FIN_ITER, h, u) : sweep<double>(P, L, true, FIN_ITER, h, u);
}

cudaError_t launch_solve_final(const Params &P, const Plan &L) {
  perm_out_kernel<<<L.grid_v, kVecThreads, 0, L.stream>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_precond(const Params &P, const Plan &L, bool fp32) {
  return fp32 ? sweep<float>(P, L, false, FIN_NONE, nullptr, nullptr) : sweep<double>(P, L, false, FIN_NONE, nullptr, nullptr);
}

cudaError_t launch_spmv_plain(const Params &P, const Plan &L) { return launch_spmv<2>(P, L); }

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
