// C ABI of libiccg: context management, setup, IC(0), the graph-driven PCG
// solve and the per-kernel entry points used by the parity tests.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "iccg_internal.h"

using namespace iccg;


namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

iccg_status cuda_fail(iccg_ctx *c, cudaError_t e, const char *where) {
  if (c) {
    c->err_index = -1;
    c->err_msg = std::string(where) + ": " + cudaGetErrorString(e);
  }
  return ICCG_ERR_CUDA;
}

#define CK(call, where)                          \
  do {                                           \
    cudaError_t e_ = (call);                     \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
  } while (0)

bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename T>
bool host_copy(const T *p, size_t count, std::vector<T> &out, cudaStream_t s) {
  out.resize(count);
  if (count == 0) return true;
  if (is_device_ptr(p)) {
    if (cudaMemcpyAsync(out.data(), p, count * sizeof(T), cudaMemcpyDeviceToHost, s) != cudaSuccess) return false;
    return cudaStreamSynchronize(s) == cudaSuccess;
  }
  std::memcpy(out.data(), p, count * sizeof(T));
  return true;
}

template <typename T>
cudaError_t dev_alloc(iccg_ctx *c, T **p, size_t count) {
  // 64 bytes of padding: 16-byte vector loads of a segment's aligned cover
  // may read up to 15 bytes past the last element.
  void *q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(T) + 64);
  if (e != cudaSuccess) return e;
  c->allocs.push_back(q);
  cudaMemsetAsync(q, 0, count * sizeof(T) + 64, c->stream);
  *p = static_cast<T *>(q);
  return cudaSuccess;
}

template <typename T>
cudaError_t dev_upload(iccg_ctx *c, T **p, const std::vector<T> &v) {
  cudaError_t e = dev_alloc(c, p, v.size());
  if (e != cudaSuccess || v.empty()) return e;
  return cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, c->stream);
}

// copy a caller array (host or device) into a device buffer
cudaError_t copy_in(iccg_ctx *c, double *dst, const double *src, size_t count) {
  if (count == 0) return cudaSuccess;
  cudaMemcpyKind k = is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  return cudaMemcpyAsync(dst, src, count * sizeof(double), k, c->stream);
}

cudaError_t copy_out(iccg_ctx *c, double *dst, const double *src, size_t count) {
  if (count == 0) return cudaSuccess;
  cudaMemcpyKind k = is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  return cudaMemcpyAsync(dst, src, count * sizeof(double), k, c->stream);
}

constexpr int kCapLimit = 4096;          // staged entries per warp (beyond: global reads)
constexpr int kCtaSmemBudget = 64 * 1024;    // per-CTA shared-memory plan, bytes

int cap_of(int seg) {
  int c = (seg + 3) & ~3;
  return std::min(std::max(c, 4), kCapLimit);
}

std::once_flag g_cfg_once[64];
cudaError_t g_cfg_err[64];

void destroy_graph(iccg_ctx *c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->graph) cudaGraphDestroy(c->graph);
  c->gexec = nullptr;
  c->graph = nullptr;
}

}  // namespace

extern "C" {

iccg_status iccg_setup(iccg_ctx **out, int32_t n, int64_t nnz, const int64_t *rowptr, const int32_t *colind,
                       const double *val, const int32_t *perm, const int32_t *block_ptr,
                       const int32_t *color_ptr, int32_t n_b, int32_t n_c, const iccg_opts *opts,
                       iccg_stream_t stream) {
  if (!out) return ICCG_ERR_ARG;
  *out = nullptr;
  if (n < 0 || nnz < 0) return ICCG_ERR_ARG;
  if (!rowptr || (n > 0 && (!colind || !val || !perm || !block_ptr || !color_ptr))) return ICCG_ERR_ARG;
  iccg_opts o{};
  if (opts) o = *opts;
  if (o.tile_mapping < ICCG_TILES_AUTO || o.tile_mapping > ICCG_TILES_UNITS) return ICCG_ERR_ARG;
  if (o.lane_block_max > 32 || o.lane_block_max < -1) return ICCG_ERR_ARG;
  if (o.solver < ICCG_SOLVER_AUTO || o.solver > ICCG_SOLVER_PHASED) return ICCG_ERR_ARG;
  if (o.fuse_sweep < -1 || o.fuse_sweep > 2) return ICCG_ERR_ARG;
  const bool w_auto = o.warps_per_cta == 0;
  if (o.warps_per_cta == 0) o.warps_per_cta = 8;
  if (o.rows_per_thread == 0) o.rows_per_thread = 1;
  if (o.warps_per_cta < 1 || o.warps_per_cta > kMaxWarpsPerCta) return ICCG_ERR_ARG;
  if (o.rows_per_thread < 1 || o.rows_per_thread > 32 || (o.rows_per_thread & (o.rows_per_thread - 1)))
    return ICCG_ERR_ARG;

  iccg_ctx *ctx = new iccg_ctx();
  ctx->opts = o;
  ctx->fp32 = o.precond_fp32 != 0;
  ctx->stream = static_cast<cudaStream_t>(stream);
  *out = ctx;
  // host views of the inputs (device inputs are copied down); all validation
  // happens before the first CUDA call that needs a device
  std::vector<int64_t> hrp;
  std::vector<int32_t> hci, hperm, hbp, hcp;
  std::vector<double> hval;
  if (!host_copy(rowptr, size_t(n) + 1, hrp, ctx->stream)) return cuda_fail(ctx, cudaGetLastError(), "copy rowptr");
  if (hrp[0] != 0 || hrp[n] != nnz) {
    ctx->err_msg = "rowptr[0] must be 0 and rowptr[n] = nnz";
    return ICCG_ERR_ARG;
  }
  if (!host_copy(colind, size_t(nnz), hci, ctx->stream) || !host_copy(val, size_t(nnz), hval, ctx->stream) ||
      !host_copy(perm, size_t(n), hperm, ctx->stream) ||
      !host_copy(block_ptr, size_t(n > 0 ? n_b + 1 : 0), hbp, ctx->stream) ||
      !host_copy(color_ptr, size_t(n > 0 ? n_c + 1 : 0), hcp, ctx->stream))
    return cuda_fail(ctx, cudaGetLastError(), "copy inputs");
  if (n == 0) { hbp.assign(1, 0); hcp.assign(1, 0); }
  const int R = o.rows_per_thread, W = o.warps_per_cta;
  const int G = 32 * W * R;   // rows of a group (one CTA of W warps)
  // lane tiles for colors of small blocks; the persistent kernel runs groups only
  const int lane_max = o.solver == ICCG_SOLVER_PERSISTENT || o.lane_block_max < 0 ? 0
                       : (o.lane_block_max == 0 ? 32 : o.lane_block_max);
  // warp units (one warp per block, a lane per row): automatically for colors
  // of blocks of 5..32 rows (on a GB300 12% faster than lane tiles at 8 rows,
  // 2.7x at 32, 2.5% slower at 4), explicitly for every color of at most 32
  const int32_t unit_min = lane_max <= 0 ? 0
                           : o.tile_mapping == ICCG_TILES_UNITS ? 1
                           : o.tile_mapping == ICCG_TILES_AUTO ? 5 : 0;
  iccg_status st = build_layout(n, nnz, hrp.data(), hci.data(), hval.data(), hperm.data(), hbp.data(),
                                hcp.data(), n_b, n_c, G, lane_max, unit_min, ctx->H, ctx->err_index, ctx->err_msg);
  if (st != ICCG_OK) return st;
  if (cudaGetDevice(&ctx->device) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "cudaGetDevice");
  {
    int dev = ctx->device;
    if (dev < 64) {
      std::call_once(g_cfg_once[dev], [dev] { g_cfg_err[dev] = configure_kernels(); });
      if (g_cfg_err[dev] != cudaSuccess) return cuda_fail(ctx, g_cfg_err[dev], "configure_kernels");
    }
  }
  HostLayout &H = ctx->H;

  // launch plan
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
  Plan &L = ctx->plan;
  L.stream = ctx->stream;
  L.W = W;
  L.R = R;
  L.n_c = n_c;
  L.n = n;
  L.pdl = o.no_pdl == 0;
  const int elem = ctx->fp32 ? 4 : 8;
  // per-CTA shared-memory plan for groups of at most G rows; shrink the entry
  // capacity until the plan fits the budget, then mark the groups that fit it
  // (the others read their data from global memory)
  int cap_l = cap_of(H.seg_l), cap_u = cap_of(H.seg_u);
  const int cap_rows = std::max(H.fit_rows, 1), cap_lev = std::max(H.fit_levels, 1);
  while (group_smem_bytes(std::max(cap_l, cap_u), cap_rows, cap_lev, elem) > kCtaSmemBudget &&
         std::max(cap_l, cap_u) > 64) {
    cap_l = std::min(cap_l, std::max(cap_l, cap_u) / 2);
    cap_u = std::min(cap_u, std::max(cap_l, cap_u) / 2);
  }
  for (GroupDesc &d : H.groups) {
    const int rows = d.r1 - d.r0;
    d.fit = (rows <= std::min(cap_rows, G) && d.l1 - d.l0 <= cap_l && d.u1 - d.u0 <= cap_u &&
             std::max(d.nlf, d.nlb) <= cap_lev) ? 1 : 0;
  }
  const int cap_a = cap_of(H.seg_a);
  const int Wc = W;   // warps per CTA of the color kernels (one CTA per group)
  const int Wa = kSpmvWarps;   // warps per CTA of the SpMV (one warp per 32-row slice)
  L.W = Wc;
  L.Wa = Wa;
  L.smem_fwd = group_smem_bytes(cap_l, cap_rows, cap_lev, elem);
  L.smem_bwd = group_smem_bytes(cap_u, cap_rows, cap_lev, elem);
  L.smem_fused = group_smem_bytes(std::max(cap_l, cap_u), cap_rows, cap_lev, elem);
  L.smem_a = 0;
  // one CTA per group (color kernels), one warp per 32-row tile (SpMV)
  // (a lane-tile color: Wt tiles per CTA)
  L.grid_c.assign(n_c, 0);
  L.task0.assign(n_c, 0);
  L.task1.assign(n_c, 0);
  L.tile0.assign(n_c, 0);
  L.tile1.assign(n_c, 0);
  // lane tiles: one CTA of up to 8 warps per tile (steps shared out in phases
  // A and C)
  L.Wt = std::max(1, std::min(W, H.lane_max));   // warps per lane-tile CTA (one tile at a time)
  {
    // every tile's in-block entries staged: two buffers within
    // kTileSmemBudget, else one buffer within kTileSmemBudget1 (the fused
    // launch's second set may then read global memory); else the capacity
    // shrinks and larger tiles read their in-block entries from global memory
    const int S = std::max(H.lane_max, 1);
    int cap_i = H.tcap_i, nbuf = 2;
    TilePlan tp = tile_plan(S, H.tcap_r, cap_i, elem);
    if (tile_launch_bytes(tp, false) > kTileSmemBudget) {
      nbuf = 1;
      tp.nbuf = 1;
      while (cap_i > 0 && tile_launch_bytes(tp, false) > kTileSmemBudget1) {
        cap_i /= 2;
        tp = tile_plan(S, H.tcap_r, cap_i, elem);
        tp.nbuf = 1;
      }
    }
    L.cap_ti = cap_i;
    L.nbuf_t = nbuf;
    L.smem_tile = tile_launch_bytes(tp, false);
    // the fused launch stages its second set only where both fit
    L.cap_ti2 = tile_launch_bytes(tp, true) <= (nbuf == 2 ? kTileSmemBudget : kTileSmemBudget1) ? cap_i : 0;
    tp.cap_i2 = L.cap_ti2;
    L.smem_tile2 = tile_launch_bytes(tp, true);
    // the entries to other colors and the row vectors as well, where the
    // launch then still fits its budget
    L.cap_to = 0;
    if (H.tcap_o > 0) {
      TilePlan to = tile_plan(S, H.tcap_r, cap_i, elem, H.tcap_o);
      to.nbuf = nbuf;
      to.cap_i2 = L.cap_ti2;
      if (tile_launch_bytes(to, true) <= (nbuf == 2 ? kTileSmemBudget : kTileSmemBudget1)) {
        L.cap_to = H.tcap_o;
        L.smem_tile_x = tile_launch_bytes(to, false);
      }
    }
  }
  // a lane-tile launch: at most the CTAs the device holds at once, each
  // walking tiles grid-stride
  const int tile_full =
      H.tile_colors > 0 ? sms * tile_resident_ctas(ctx->fp32, L.Wt * kWarp, L.smem_tile) : 1;
  const int tile_full_x =
      H.tile_colors > 0 && L.cap_to > 0 ? sms * tile_resident_ctas(ctx->fp32, L.Wt * kWarp, L.smem_tile_x) : 1;
  // warp-tile kernels: W warps per CTA, one tile per warp at a time, a
  // buffer of (largest tile's steps) x 32 values per warp
  L.Ww = W;
  L.cap_ws = std::max(H.lane_max, 1);
  L.smem_wt = L.Ww * L.cap_ws * kWarp * elem;
  const int wt_full =
      H.tile_colors > 0 ? sms * wtile_resident_ctas(ctx->fp32, L.Ww * kWarp, L.smem_wt) : 1;
  // pair kernels: 4 warps per CTA unless set (on a GB300 at 128^3 with two-row
  // blocks 3% faster than 8, 16 slower)
  L.Wp = w_auto ? 4 : W;
  const int pr_full = H.tile_colors > 0 ? sms * pair_resident_ctas(ctx->fp32, L.Wp * kWarp) : 1;
  L.pstage_f.assign(n_c, 0);
  L.pstage_b.assign(n_c, 0);
  L.wtile.assign(n_c, 0);
  L.stage_ext.assign(n_c, 0);
  L.unit0.assign(n_c, 0);
  L.unit1.assign(n_c, 0);
  L.unit_S.assign(n_c, 0);
  L.Wu = 8;
  int32_t gbig = 1;
  for (int c = 0; c < n_c; ++c) {
    L.task0[c] = H.color_group[c];
    L.task1[c] = H.color_group[c + 1];
    L.tile0[c] = H.color_tile[c];
    L.tile1[c] = H.color_tile[c + 1];
    const int nt = L.tile1[c] - L.tile0[c];
    // the color's longest tile, and whether all its blocks have two rows
    int steps = 0;
    bool pairs = true;
    for (int t = L.tile0[c]; t < L.tile1[c]; ++t) {
      const TileDesc &td = H.tiles[t];
      steps = std::max(steps, td.nsteps);
      if (td.nsteps != 2 || H.steps[size_t(td.step0) + 1].cnt != H.steps[size_t(td.step0)].cnt) pairs = false;
    }
    // automatic: colors of two-row blocks only as pair kernels, one CTA per
    // tile otherwise (on a GB300 the pair kernels measured 7% faster for
    // ABMC with blocks of 2 rows, slower where one-row blocks share a tile
    // with two-row ones, and no better for one-row blocks alone)
    L.wtile[c] = 0;
    if (nt > 0 && o.tile_mapping == ICCG_TILES_WARP) L.wtile[c] = 1;
    if (nt > 0 && steps <= 2 && ((pairs && o.tile_mapping == ICCG_TILES_AUTO) || o.tile_mapping == ICCG_TILES_PAIR))
      L.wtile[c] = 2;
    // one-CTA-per-tile colors of short tiles also stage their entries to
    // other colors and row vectors (measured 3% faster in FP64 and 14% in
    // FP32 at blocks of 1-2 rows; slower for tiles of 8 steps)
    L.stage_ext[c] = L.cap_to > 0 && steps <= 2;
    L.unit0[c] = H.color_unit[c];
    L.unit1[c] = H.color_unit[c + 1];
    L.unit_S[c] = H.unit_S[c];
    const int nu = L.unit1[c] - L.unit0[c];
    if (nu > 0) {
      L.wtile[c] = 3;
      const int full = sms * unit_resident_ctas(ctx->fp32, L.unit_S[c], L.Wu * kWarp);
      L.grid_c[c] = std::max(1, std::min((nu + L.Wu - 1) / L.Wu, full));
    } else if (L.wtile[c] == 1) L.grid_c[c] = std::min((nt + L.Ww - 1) / L.Ww, wt_full);
    else if (L.wtile[c] == 2) {
      L.grid_c[c] = std::min((nt + L.Wp - 1) / L.Wp, pr_full);
      // a sweep stages its entries to other colors ahead of the gathers when
      // its tiles have on average at least two (over both steps), and always
      // with the FP32 preconditioner (on a GB300 at 128^3 with two-row blocks:
      // FP64 41.2 ms with this rule against 43.5 with every color staged, where
      // the staged kernel of a color without entries ran 50% longer; FP32 34.0
      // ms with every color staged against 35.8 with this rule)
      int64_t wf = 0, wb = 0;
      for (int t = L.tile0[c]; t < L.tile1[c]; ++t) {
        const PairDesc &d = H.pairs[size_t(t)];
        wf += d.lw0 + d.lw1;
        wb += d.uw0 + d.uw1;
      }
      L.pstage_f[c] = ctx->fp32 || wf >= 2 * int64_t(nt);
      L.pstage_b[c] = ctx->fp32 || wb >= 2 * int64_t(nt);
    }
    else L.grid_c[c] = nt > 0 ? std::min(nt, L.stage_ext[c] ? tile_full_x : tile_full)
                              : std::max(1, L.task1[c] - L.task0[c]);
    gbig = std::max(gbig, L.grid_c[c]);
  }
  // one cooperative launch per sweep when every color is pair tiles (blocks
  // of one or two rows) and every CTA of that launch can be resident
  {
    bool pairs_only = n_c > 0 && H.groups.empty() && H.units.empty();
    for (const TileDesc &td : H.tiles) pairs_only = pairs_only && td.nsteps <= 2;
    for (int c = 0; c < n_c; ++c) pairs_only = pairs_only && L.tile1[c] > L.tile0[c];
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device);
    // on request only: at 128^3 with Leiden CPM 0.5 (8 colors) its grid
    // barriers cost more than the launch boundaries they replace
    const int per_sm = pairs_only && coop && o.fuse_sweep == 1 ? coop_sweep_resident_ctas(ctx->fp32) : 0;
    L.coop = per_sm > 0;
    L.grid_coop = L.coop ? sms * per_sm : 0;
    gbig = std::max(gbig, L.grid_coop);
    // the tail of every sweep (the last colors, together at most n / 32 rows,
    // all of them lane tiles of at most two steps) in one cooperative launch,
    // one CTA per SM
    L.tail_c = 0;
    L.grid_tail = 0;
    if (!L.coop && coop && o.fuse_sweep == 2 && n_c >= 3 && coop_sweep_resident_ctas(ctx->fp32) > 0) {
      int ct = n_c;
      int64_t rows = 0;
      for (int c = n_c - 1; c >= 1; --c) {
        bool short_tiles = L.tile1[c] > L.tile0[c] && L.unit1[c] == L.unit0[c];
        for (int t = L.tile0[c]; t < L.tile1[c] && short_tiles; ++t) short_tiles = H.tiles[t].nsteps <= 2;
        rows += int64_t(H.color_ptr[c + 1] > H.color_ptr[c]
                            ? H.block_ptr[H.color_ptr[c + 1]] - H.block_ptr[H.color_ptr[c]] : 0);
        if (!short_tiles || rows * 32 > int64_t(n)) break;
        ct = c;
      }
      if (ct <= n_c - 2) {
        L.tail_c = ct;
        L.grid_tail = sms;
        for (int c = ct; c < n_c; ++c) L.grid_c[c] = L.grid_tail;
      }
    }
  }
  // slot regions: forward launches in color order (<r,r>), then the fused
  // launch and the backward launches in launch order (<r,z>); the final
  // launch (backward color 0, or the fused launch of a one-color ordering)
  // sums everything written before its own region
  L.off_rr.assign(n_c, 0);
  L.off_rz.assign(n_c, 0);
  int32_t nslot = 0;
  for (int c = 0; c < n_c; ++c) { L.off_rr[c] = nslot; nslot += L.grid_c[c]; }
  int32_t orz = 0;
  if (n_c > 0) { L.off_rz[n_c - 1] = orz; orz += L.grid_c[n_c - 1]; }
  for (int c = n_c - 2; c >= 0; --c) { L.off_rz[c] = orz; orz += L.grid_c[c]; }
  L.last_rr = n_c > 1 ? nslot : 0;
  L.last_rz = n_c > 1 ? L.off_rz[0] : 0;
  const int ntile_a = (n + 31) / 32;
  const int a_full = sms * spmv_resident_ctas(Wa, L.smem_a);
  L.grid_a = std::max(1, std::min(a_full, (ntile_a + Wa - 1) / Wa));
  L.grid_v = std::max(1, std::min((n + 255) / 256, sms * 8));

  // device arrays
  Params &P = ctx->P;
  P.n = n; P.R = R; P.W = Wc; P.n_c = n_c;
  P.cap_l = cap_l; P.cap_u = cap_u; P.cap_a = cap_a;
  P.cap_rows = cap_rows; P.cap_lev = cap_lev;
  // persistent kernel: as many CTAs as fit on the device at once (cooperative
  // launch), but no more than the widest phase can use
  {
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device);
    L.smem_p = persistent_smem_bytes(P, ctx->fp32, Wc, kCtaSmemBudget, &L.cap_p);
    const int per_sm = coop ? persistent_resident_ctas(ctx->fp32, Wc, L.smem_p) : 0;
    const int widest = std::max(gbig, (ntile_a + Wc - 1) / Wc);
    L.grid_p = per_sm > 0 ? std::max(1, std::min(sms * per_sm, widest)) : 0;
    if (o.solver == ICCG_SOLVER_PERSISTENT && L.grid_p == 0) {
      ctx->err_msg = "the persistent solve kernel cannot be made resident on this device";
      return ICCG_ERR_ARG;
    }
    ctx->persistent = o.solver == ICCG_SOLVER_PERSISTENT;
  }
  int32_t *d_arp, *d_acol, *d_lrp, *d_lcol, *d_urp, *d_ucol, *d_umap, *d_perm, *d_sf, *d_sb, *d_levp;
  GroupDesc *d_groups;
  double *d_aval, *d_ainit, *d_adiag;
  CK(dev_upload(ctx, &d_arp, H.arp), "alloc A");
  CK(dev_upload(ctx, &d_acol, H.acol), "alloc A");
  CK(dev_upload(ctx, &d_aval, H.aval), "alloc A");
  {
    int32_t *d_sap, *d_sac;
    double *d_sav;
    CK(dev_upload(ctx, &d_sap, H.sa_ptr), "alloc A");
    CK(dev_upload(ctx, &d_sac, H.sa_col), "alloc A");
    CK(dev_upload(ctx, &d_sav, H.sa_val), "alloc A");
    P.sa_ptr = d_sap; P.sa_col = d_sac; P.sa_val = d_sav;
  }
  CK(dev_upload(ctx, &d_lrp, H.lrp), "alloc L");
  CK(dev_upload(ctx, &d_lcol, H.lcol), "alloc L");
  CK(dev_upload(ctx, &d_ainit, H.ainit), "alloc L");
  CK(dev_upload(ctx, &d_adiag, H.adiag), "alloc L");
  CK(dev_upload(ctx, &d_urp, H.urp), "alloc U");
  CK(dev_upload(ctx, &d_ucol, H.ucol), "alloc U");
  CK(dev_upload(ctx, &d_umap, H.umap), "alloc U");
  CK(dev_upload(ctx, &d_groups, H.groups), "alloc groups");
  CK(dev_upload(ctx, &d_sf, H.sched_f), "alloc groups");
  CK(dev_upload(ctx, &d_sb, H.sched_b), "alloc groups");
  CK(dev_upload(ctx, &d_levp, H.levp), "alloc groups");
  CK(dev_upload(ctx, &d_perm, H.perm), "alloc perm");
  {
    int32_t *d_fr;
    CK(dev_upload(ctx, &d_fr, H.fac_rows), "alloc factor schedule");
    P.fac_rows = d_fr;
    P.fp_ptr = nullptr; P.fp_b = nullptr; P.fp_pos = nullptr; P.fac_rec = nullptr;
    if (!H.fp_ptr.empty()) {
      int32_t *d_fp, *d_fb;
      uint8_t *d_fs;
      CK(dev_upload(ctx, &d_fp, H.fp_ptr), "alloc factor pairs");
      CK(dev_upload(ctx, &d_fb, H.fp_b), "alloc factor pairs");
      CK(dev_upload(ctx, &d_fs, H.fp_pos), "alloc factor pairs");
      P.fp_ptr = d_fp; P.fp_b = d_fb; P.fp_pos = d_fs;
      // one 16-byte record per scheduled row (no dependent index loads in
      // the factor kernels); rows the record cannot describe take the
      // general form (entries field 255)
      std::vector<int4> rec(H.fac_rows.size());
      for (size_t k = 0; k < rec.size(); ++k) {
        const int32_t i = H.fac_rows[k], rb = H.lrp[i], ni = H.lrp[i + 1] - rb;
        const int32_t q0 = H.fp_ptr[size_t(rb)], np = H.fp_ptr[size_t(rb + ni)] - q0;
        const bool ok = ni < 255 && np < (1 << 23);
        rec[k] = make_int4(i, rb, q0, ok ? (ni | (np << 8)) : 255);
      }
      int4 *d_rec;
      CK(dev_upload(ctx, &d_rec, rec), "alloc factor schedule");
      P.fac_rec = d_rec;
    }
    L.fac_ptr = H.fac_ptr;
    L.fac_lev0 = H.fac_lev0;
    L.fac_nlev = H.fac_nlev;
    L.fac_wide = H.fac_wide;
  }
  int32_t *d_cg;
  CK(dev_upload(ctx, &d_cg, H.color_group), "alloc groups");
  P.color_group = d_cg;
  {
    int32_t *d_ct;
    CK(dev_upload(ctx, &d_ct, H.color_tile), "alloc tiles");
    P.ctile = d_ct;
  }
  {
    WarpUnit *d_units;
    uint32_t *d_wlm, *d_wum;
    int32_t *d_wlmap, *d_wlsr, *d_wumap, *d_wusr, *d_bptr;
    CK(dev_upload(ctx, &d_units, H.units), "alloc units");
    CK(dev_upload(ctx, &d_wlm, H.wl_mask), "alloc units");
    CK(dev_upload(ctx, &d_wum, H.wu_mask), "alloc units");
    uint32_t *d_wls, *d_wus;
    CK(dev_upload(ctx, &d_wls, H.wl_src), "alloc units");
    CK(dev_upload(ctx, &d_wus, H.wu_src), "alloc units");
    P.wl_src = d_wls; P.wu_src = d_wus;
    CK(dev_upload(ctx, &d_wlmap, H.wl_map), "alloc units");
    CK(dev_upload(ctx, &d_wlsr, H.wl_srow), "alloc units");
    CK(dev_upload(ctx, &d_wumap, H.wu_map), "alloc units");
    CK(dev_upload(ctx, &d_wusr, H.wu_srow), "alloc units");
    CK(dev_upload(ctx, &d_bptr, H.block_ptr), "alloc units");
    P.units = d_units;
    P.wl_mask = d_wlm; P.wu_mask = d_wum;
    P.wl_map = d_wlmap; P.wl_srow = d_wlsr; P.wu_map = d_wumap; P.wu_srow = d_wusr;
    P.bptr = d_bptr;
    P.nwl = int32_t(H.wl_map.size());
    P.nwu = int32_t(H.wu_map.size());
    CK(dev_alloc(ctx, &P.wl_val, H.wl_map.size()), "alloc units");
    CK(dev_alloc(ctx, &P.wu_val, H.wu_map.size()), "alloc units");
    CK(dev_alloc(ctx, &P.wl_val32, H.wl_map.size()), "alloc units");
    CK(dev_alloc(ctx, &P.wu_val32, H.wu_map.size()), "alloc units");
  }
  {
    TileDesc *d_tiles;
    StepDesc *d_steps;
    int32_t *d_slc, *d_suc, *d_slm, *d_sum, *d_sic, *d_uic, *d_sim, *d_uim;
    CK(dev_upload(ctx, &d_tiles, H.tiles), "alloc tiles");
    PairDesc *d_pairs;
    CK(dev_upload(ctx, &d_pairs, H.pairs), "alloc tiles");
    P.pairs = d_pairs;
    CK(dev_upload(ctx, &d_steps, H.steps), "alloc tiles");
    CK(dev_upload(ctx, &d_slc, H.sl_col), "alloc tiles");
    CK(dev_upload(ctx, &d_suc, H.su_col), "alloc tiles");
    CK(dev_upload(ctx, &d_slm, H.sl_map), "alloc tiles");
    CK(dev_upload(ctx, &d_sum, H.su_map), "alloc tiles");
    CK(dev_upload(ctx, &d_sic, H.si_col), "alloc tiles");
    CK(dev_upload(ctx, &d_uic, H.ui_col), "alloc tiles");
    CK(dev_upload(ctx, &d_sim, H.si_map), "alloc tiles");
    CK(dev_upload(ctx, &d_uim, H.ui_map), "alloc tiles");
    P.tiles = d_tiles; P.steps = d_steps;
    P.sl_col = d_slc; P.su_col = d_suc; P.sl_map = d_slm; P.su_map = d_sum;
    P.si_col = d_sic; P.ui_col = d_uic; P.si_map = d_sim; P.ui_map = d_uim;
    P.nsl = int32_t(H.sl_col.size());
    P.nsu = int32_t(H.su_col.size());
    P.nsi = int32_t(H.si_col.size());
    P.nui = int32_t(H.ui_col.size());
    P.lane_max = std::max(H.lane_max, 1);
    P.wi_max = H.wi_max;
    P.tcap_r = H.tcap_r;
    P.tcap_i = L.cap_ti;
    P.tnbuf = L.nbuf_t;
    P.tcap_i2 = L.cap_ti2;
    P.tcap_o = L.cap_to;
    CK(dev_alloc(ctx, &P.sl_val, H.sl_col.size()), "alloc tiles");
    CK(dev_alloc(ctx, &P.su_val, H.su_col.size()), "alloc tiles");
    CK(dev_alloc(ctx, &P.si_val, H.si_col.size()), "alloc tiles");
    CK(dev_alloc(ctx, &P.ui_val, H.ui_col.size()), "alloc tiles");
    CK(dev_alloc(ctx, &P.sl_val32, H.sl_col.size()), "alloc tiles");
    CK(dev_alloc(ctx, &P.su_val32, H.su_col.size()), "alloc tiles");
    CK(dev_alloc(ctx, &P.si_val32, H.si_col.size()), "alloc tiles");
    CK(dev_alloc(ctx, &P.ui_val32, H.ui_col.size()), "alloc tiles");
  }
  CK(dev_alloc(ctx, &P.bar, 1), "alloc barrier");
  P.wait_ns = kDefaultWaitNs;
  P.arp = d_arp; P.acol = d_acol; P.aval = d_aval;
  P.lrp = d_lrp; P.lcol = d_lcol; P.urp = d_urp; P.ucol = d_ucol; P.umap = d_umap;
  P.ainit = d_ainit; P.adiag = d_adiag;
  P.groups = d_groups;
  P.sched_f = d_sf;
  P.sched_b = d_sb;
  P.levp = d_levp;
  P.perm = d_perm;
  const size_t nL = size_t(H.nL), nn = size_t(n);
  CK(dev_alloc(ctx, &P.lval, nL), "alloc factor");
  CK(dev_alloc(ctx, &P.uval, nL), "alloc factor");
  CK(dev_alloc(ctx, &P.lval32, nL), "alloc factor");
  CK(dev_alloc(ctx, &P.uval32, nL), "alloc factor");
  CK(dev_alloc(ctx, &P.ldiag, nn), "alloc factor");
  CK(dev_alloc(ctx, &P.invd, nn), "alloc factor");
  CK(dev_alloc(ctx, &P.invd32, nn), "alloc factor");
  CK(dev_alloc(ctx, &P.xh, nn), "alloc vectors");
  CK(dev_alloc(ctx, &P.r, nn), "alloc vectors");
  CK(dev_alloc(ctx, &P.q, nn), "alloc vectors");
  CK(dev_alloc(ctx, &P.p0, nn), "alloc vectors");
  CK(dev_alloc(ctx, &P.p1, nn), "alloc vectors");
  CK(dev_alloc(ctx, &P.bh, nn), "alloc vectors");
  double *y, *z;
  CK(dev_alloc(ctx, &y, nn), "alloc vectors");
  CK(dev_alloc(ctx, &z, nn), "alloc vectors");
  P.y = y; P.z = z;
  CK(dev_alloc(ctx, &ctx->bin, nn), "alloc vectors");
  CK(dev_alloc(ctx, &ctx->xin, nn), "alloc vectors");
  CK(dev_alloc(ctx, &ctx->xout, nn), "alloc vectors");
  P.bin = ctx->bin; P.xin = ctx->xin; P.xout = ctx->xout;
  // reduction slots: one per CTA of the widest launch, doubled so the solve
  // start can keep <b,b> and <r0,r0> partials side by side; kept even for
  // 16-byte loads
  P.nslot = std::max(nslot, 1);
  P.npart = std::max(gbig, L.grid_p);
  P.ngroup = (gbig + kGroup - 1) / kGroup;
  P.npart_a = L.grid_a;
  P.nbb = std::max(L.grid_v, L.grid_p);
  CK(dev_alloc(ctx, &P.slot_rr, size_t(P.nslot)), "alloc reductions");
  CK(dev_alloc(ctx, &P.slot_rz, size_t(P.nslot)), "alloc reductions");
  CK(dev_alloc(ctx, &P.part0, size_t(P.npart)), "alloc reductions");
  CK(dev_alloc(ctx, &P.part1, size_t(P.npart)), "alloc reductions");
  CK(dev_alloc(ctx, &P.gsum0, size_t(P.ngroup)), "alloc reductions");
  CK(dev_alloc(ctx, &P.gsum1, size_t(P.ngroup)), "alloc reductions");
  CK(dev_alloc(ctx, &P.part_a, size_t(P.npart_a)), "alloc reductions");
  CK(dev_alloc(ctx, &P.init_bb, size_t(P.nbb)), "alloc reductions");
  CK(dev_alloc(ctx, &P.gticket, size_t(P.ngroup)), "alloc reductions");
  CK(dev_alloc(ctx, &P.sc, 1), "alloc scalars");
  CK(dev_alloc(ctx, &P.err_row, 1), "alloc scalars");
  CK(cudaMallocHost(&ctx->sc_host, sizeof(Scalars)), "pinned");
  std::memset(ctx->sc_host, 0, sizeof(Scalars));
  CK(cudaStreamSynchronize(ctx->stream), "setup sync");
  return ICCG_OK;
}

iccg_status iccg_factor(iccg_ctx *ctx) {
  if (!ctx) return ICCG_ERR_ARG;
  DeviceGuard g(ctx->device);
  ctx->factored = false;
  if (ctx->H.n == 0) { ctx->factored = true; return ICCG_OK; }
  // the factorization's launches (one per in-block level of every color)
  // are captured once into a graph and replayed: no host launch cost per level
  if (ctx->opts.no_graph == 0 && !ctx->fexec && !ctx->fgraph_failed) {
    cudaGraph_t fg = nullptr;
    cudaError_t e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e1 = cudaMemsetAsync(ctx->P.err_row, 0xff, sizeof(unsigned long long), ctx->stream);
      if (e1 == cudaSuccess) e1 = launch_factor(ctx->P, ctx->plan, int(ctx->H.nL));
      e = cudaStreamEndCapture(ctx->stream, &fg);
      if (e == cudaSuccess) e = e1;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ctx->fexec, fg, 0);
    if (fg) cudaGraphDestroy(fg);
    if (e != cudaSuccess) {
      // e.g. the legacy default stream, which cannot be captured
      cudaGetLastError();
      if (ctx->fexec) cudaGraphExecDestroy(ctx->fexec);
      ctx->fexec = nullptr;
      ctx->fgraph_failed = true;
    }
  }
  if (ctx->fexec) {
    CK(cudaGraphLaunch(ctx->fexec, ctx->stream), "factor graph launch");
  } else {
    CK(cudaMemsetAsync(ctx->P.err_row, 0xff, sizeof(unsigned long long), ctx->stream), "factor");
    CK(launch_factor(ctx->P, ctx->plan, int(ctx->H.nL)), "factor launch");
  }
  unsigned long long row = 0;
  CK(cudaMemcpyAsync(&row, ctx->P.err_row, sizeof(row), cudaMemcpyDeviceToHost, ctx->stream), "factor");
  CK(cudaStreamSynchronize(ctx->stream), "factor sync");
  if (row != ~0ULL) {
    ctx->err_index = ctx->H.perm[size_t(row)];
    ctx->err_msg = "IC(0) pivot not positive";
    return ICCG_ERR_BREAKDOWN;
  }
  ctx->factored = true;
  return ICCG_OK;
}

static iccg_status ensure_hist(iccg_ctx *ctx, int32_t maxit) {
  if (maxit + 1 > ctx->hist_cap) {
    int32_t cap = std::max(maxit + 1, 1024);
    double *h = nullptr;
    CK(dev_alloc(ctx, &h, size_t(cap)), "alloc history");
    ctx->hist = h;
    ctx->hist_cap = cap;
    ctx->P.hist = h;
    destroy_graph(ctx);   // the graph captured the old pointer
  }
  if (maxit + 1 > ctx->hist_host_cap) {
    if (ctx->hist_host) cudaFreeHost(ctx->hist_host);
    ctx->hist_host = nullptr;
    int32_t cap = std::max(maxit + 1, 1024);
    CK(cudaMallocHost(&ctx->hist_host, sizeof(double) * size_t(cap)), "pinned history");
    ctx->hist_host_cap = cap;
  }
  return ICCG_OK;
}

static iccg_status build_graph(iccg_ctx *ctx) {
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0), "graph");
  ctx->graph = g;
  cudaGraphConditionalHandle h;
  CK(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault), "graph cond");
  ctx->cond_handle = (unsigned long long)h;
  // capture on a private stream (the legacy default stream cannot capture);
  // the instantiated graph is launched on the context's stream
  cudaStream_t s = nullptr;
  CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "capture stream");
  struct StreamGuard { cudaStream_t s; ~StreamGuard() { cudaStreamDestroy(s); } } sg{s};
  Plan Lc = ctx->plan;
  Lc.stream = s;
  CK(cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal), "capture");
  cudaError_t e = launch_solve_init(ctx->P, Lc, ctx->fp32, nullptr, nullptr);
  cudaGraphNodeParams cp = {};
  cudaGraphNode_t cnode = nullptr;
  if (e == cudaSuccess) {
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    e = cudaStreamGetCaptureInfo(s, &cst, nullptr, nullptr, &deps, nullptr, &ndeps);
    if (e == cudaSuccess) {
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = h;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      e = cudaGraphAddNode(&cnode, g, deps, nullptr, ndeps, &cp);
    }
    if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(s, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e == cudaSuccess) e = launch_solve_final(ctx->P, Lc);
  }
  cudaGraph_t g2 = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(s, &g2);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "capture init");
  if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "end capture");
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  CK(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal), "capture body");
  e = launch_solve_body(ctx->P, Lc, ctx->fp32, nullptr, nullptr);
  e2 = cudaStreamEndCapture(s, &body);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "capture body");
  if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "end capture body");
  CK(cudaGraphInstantiate(&ctx->gexec, g, 0), "instantiate");
  return ICCG_OK;
}

struct ProfileState {
  cudaStream_t s;
  std::vector<cudaEvent_t> ev;
  std::vector<int> phase;
  size_t used = 0;
  double ms[PH_COUNT] = {0};
  int64_t launches[PH_COUNT] = {0};
  void flush() {
    cudaStreamSynchronize(s);
    for (size_t k = 0; k + 1 < used; k += 2) {
      float t = 0.f;
      cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
      ms[phase[k]] += t;
      launches[phase[k]] += 1;
    }
    used = 0;
  }
  static void hook(void *u, int ph, int begin) {
    ProfileState *p = static_cast<ProfileState *>(u);
    if (begin && p->used + 2 > p->ev.size()) p->flush();
    if (p->used >= p->ev.size()) return;
    p->phase[p->used] = ph;
    cudaEventRecord(p->ev[p->used], p->s);
    p->used++;
    (void)begin;
  }
};

static iccg_status solve_impl(iccg_ctx *ctx, const double *b, double *x, double tol, int32_t maxit,
                              int32_t *iters, double *res_hist, ProfileState *prof) {
  if (!ctx || tol < 0 || !(tol == tol) || maxit < 0) return ICCG_ERR_ARG;
  DeviceGuard guard(ctx->device);
  const int32_t n = ctx->H.n;
  if (n > 0 && (!b || !x)) return ICCG_ERR_ARG;
  if (!ctx->factored) { ctx->err_msg = "iccg_solve before a successful iccg_factor"; return ICCG_ERR_STATE; }
  if (n == 0) {
    if (iters) *iters = 0;
    if (res_hist) res_hist[0] = 0.0;
    return ICCG_OK;
  }
  iccg_status st = ensure_hist(ctx, maxit);
  if (st != ICCG_OK) return st;
  cudaStream_t s = ctx->stream;
  const bool persistent = ctx->persistent && prof == nullptr;
  const bool use_graph = !persistent && ctx->opts.no_graph == 0 && prof == nullptr;
  if (use_graph && !ctx->gexec) {
    st = build_graph(ctx);
    if (st != ICCG_OK && (ctx->plan.coop || ctx->plan.tail_c > 0)) {
      // the runtime would not capture the cooperative sweep into the graph:
      // one launch per color instead
      destroy_graph(ctx);
      cudaGetLastError();
      ctx->plan.coop = false;
      ctx->plan.tail_c = 0;
      st = build_graph(ctx);
    }
    if (st != ICCG_OK) { destroy_graph(ctx); return st; }
  }
  CK(copy_in(ctx, ctx->bin, b, size_t(n)), "copy b");
  CK(copy_in(ctx, ctx->xin, x, size_t(n)), "copy x0");
  Scalars *sh = ctx->sc_host;
  std::memset(sh, 0, sizeof(Scalars));
  sh->tol = tol;
  sh->maxit = maxit;
  sh->use_cond = use_graph ? 1 : 0;
  sh->cond_handle = ctx->cond_handle;
  sh->status = ICCG_NOT_CONVERGED;
  CK(cudaMemcpyAsync(ctx->P.sc, sh, sizeof(Scalars), cudaMemcpyHostToDevice, s), "scalars");
  if (persistent) {
    CK(launch_solve_persistent(ctx->P, ctx->plan, ctx->fp32), "persistent launch");
  } else if (use_graph) {
    CK(cudaGraphLaunch(ctx->gexec, s), "graph launch");
  } else {
    CK(launch_solve_init(ctx->P, ctx->plan, ctx->fp32, prof ? ProfileState::hook : nullptr, prof), "init");
    for (;;) {
      CK(cudaMemcpyAsync(sh, ctx->P.sc, sizeof(Scalars), cudaMemcpyDeviceToHost, s), "scalars");
      CK(cudaStreamSynchronize(s), "sync");
      if (sh->done) break;
      CK(launch_solve_body(ctx->P, ctx->plan, ctx->fp32, prof ? ProfileState::hook : nullptr, prof), "body");
    }
    CK(launch_solve_final(ctx->P, ctx->plan), "final");
  }
  CK(copy_out(ctx, x, ctx->xout, size_t(n)), "copy x");
  CK(cudaMemcpyAsync(sh, ctx->P.sc, sizeof(Scalars), cudaMemcpyDeviceToHost, s), "scalars");
  CK(cudaStreamSynchronize(s), "solve sync");
  const int32_t it = sh->iter;
  if (iters) *iters = it;
  if (sh->status == ICCG_ERR_TIMEOUT) {
    ctx->err_index = -1;
    ctx->err_msg = "a grid-barrier wait of the persistent solve gave up (iccg_set_wait_limit)";
  }
  if (res_hist) {
    CK(cudaMemcpyAsync(ctx->hist_host, ctx->hist, sizeof(double) * size_t(it + 1), cudaMemcpyDeviceToHost, s), "history");
    CK(cudaStreamSynchronize(s), "history sync");
    std::memcpy(res_hist, ctx->hist_host, sizeof(double) * size_t(it + 1));
  }
  return static_cast<iccg_status>(sh->status);
}

iccg_status iccg_solve(iccg_ctx *ctx, const double *b, double *x, double tol, int32_t maxit, int32_t *iters,
                       double *res_hist) {
  return solve_impl(ctx, b, x, tol, maxit, iters, res_hist, nullptr);
}

// Persistent solver: CTA 0 stamps the time it leaves every grid barrier with
// the phase that barrier ends; a phase's time is the gap to the previous
// stamp (the first phase counts from the kernel's start event).
static iccg_status profile_persistent(iccg_ctx *ctx, const double *b, double *x, double tol, int32_t maxit,
                                      int32_t *iters, double *ms, int64_t *launches) {
  const int64_t cap64 = (int64_t(maxit) + 3) * (2 * int64_t(ctx->H.n_c) + 4) + 16;
  if (cap64 > (int64_t(1) << 28)) return ICCG_ERR_ARG;
  const int32_t cap = int32_t(cap64);
  unsigned long long *tr = nullptr;
  int32_t *tlen = nullptr;
  CK(cudaMalloc(&tr, sizeof(unsigned long long) * size_t(cap)), "alloc trace");
  if (cudaMalloc(&tlen, sizeof(int32_t)) != cudaSuccess) {
    cudaFree(tr);
    return cuda_fail(ctx, cudaGetLastError(), "alloc trace");
  }
  struct Free {
    void *a, *b;
    ~Free() { cudaFree(a); cudaFree(b); }
  } fr{tr, tlen};
  cudaEvent_t a0, a1;
  CK(cudaEventCreate(&a0), "event");
  CK(cudaEventCreate(&a1), "event");
  struct FreeEv {
    cudaEvent_t a, b;
    ~FreeEv() { cudaEventDestroy(a); cudaEventDestroy(b); }
  } fe{a0, a1};
  ctx->P.trace = tr;
  ctx->P.trace_len = tlen;
  ctx->P.trace_cap = cap;
  CK(cudaEventRecord(a0, ctx->stream), "event");
  iccg_status st = solve_impl(ctx, b, x, tol, maxit, iters, nullptr, nullptr);
  cudaEventRecord(a1, ctx->stream);
  ctx->P.trace = nullptr;
  ctx->P.trace_len = nullptr;
  ctx->P.trace_cap = 0;
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  int32_t len = 0;
  CK(cudaMemcpy(&len, tlen, sizeof(len), cudaMemcpyDeviceToHost), "trace");
  len = std::max(0, std::min(len, cap));
  std::vector<unsigned long long> h(size_t(len) + 1);
  if (len) CK(cudaMemcpy(h.data(), tr, sizeof(unsigned long long) * size_t(len), cudaMemcpyDeviceToHost), "trace");
  float tall = 0.f;
  cudaEventElapsedTime(&tall, a0, a1);
  double pms[PH_COUNT] = {0};
  int64_t pn[PH_COUNT] = {0};
  for (int32_t k = 1; k < len; ++k) {
    const int tag = int(h[size_t(k)] & 15u);
    const double dt = double((h[size_t(k)] >> 4) - (h[size_t(k) - 1] >> 4)) * 1e-6;
    const int ph = tag == PH_ALL ? PH_BWD : tag;   // the tail after the last barrier
    if (ph >= 0 && ph < PH_ALL) { pms[ph] += dt; pn[ph] += tag == PH_ALL ? 0 : 1; }
  }
  pms[PH_ALL] = tall;
  for (int k = 0; k < PH_ALL; ++k) pn[PH_ALL] += pn[k];
  for (int k = 0; k < PH_COUNT; ++k) {
    if (ms) ms[k] = pms[k];
    if (launches) launches[k] = pn[k];
  }
  return st;
}

iccg_status iccg_profile_solve(iccg_ctx *ctx, const double *b, double *x, double tol, int32_t maxit,
                               int32_t *iters, double *ms, int64_t *launches) {
  if (!ctx) return ICCG_ERR_ARG;
  DeviceGuard guard(ctx->device);
  if (ctx->persistent && ctx->H.n > 0) return profile_persistent(ctx, b, x, tol, maxit, iters, ms, launches);
  ProfileState ps;
  ps.s = ctx->stream;
  ps.ev.resize(4096);
  ps.phase.resize(4096);
  for (auto &e : ps.ev) CK(cudaEventCreate(&e), "event");
  // the ALL phase is bracketed by its own pair of events
  cudaEvent_t a0, a1;
  CK(cudaEventCreate(&a0), "event");
  CK(cudaEventCreate(&a1), "event");
  CK(cudaEventRecord(a0, ctx->stream), "event");
  iccg_status st = solve_impl(ctx, b, x, tol, maxit, iters, nullptr, &ps);
  cudaEventRecord(a1, ctx->stream);
  cudaStreamSynchronize(ctx->stream);
  ps.flush();
  float tall = 0.f;
  cudaEventElapsedTime(&tall, a0, a1);
  ps.ms[PH_ALL] = tall;
  ps.launches[PH_ALL] = 0;
  for (int k = 0; k < PH_ALL; ++k) ps.launches[PH_ALL] += ps.launches[k];
  for (auto &e : ps.ev) cudaEventDestroy(e);
  cudaEventDestroy(a0);
  cudaEventDestroy(a1);
  for (int k = 0; k < PH_COUNT; ++k) {
    if (ms) ms[k] = ps.ms[k];
    if (launches) launches[k] = ps.launches[k];
  }
  return st;
}

iccg_status iccg_time_spmv_phase(iccg_ctx *ctx, int32_t reps, double *ms) {
  if (!ctx || reps < 1 || !ms) return ICCG_ERR_ARG;
  DeviceGuard guard(ctx->device);
  if (!ctx->factored) return ICCG_ERR_STATE;
  *ms = 0.0;
  if (ctx->H.n == 0) return ICCG_OK;
  cudaStream_t s = ctx->stream;
  // beta = 0: every repetition computes p = z (no growth of p across them)
  static const double zero = 0.0;
  CK(cudaMemcpyAsync(&ctx->P.sc->beta, &zero, sizeof(double), cudaMemcpyHostToDevice, s), "scalars");
  CK(cudaStreamSynchronize(s), "sync");
  cudaEvent_t a0, a1;
  CK(cudaEventCreate(&a0), "event");
  if (cudaEventCreate(&a1) != cudaSuccess) {
    cudaEventDestroy(a0);
    return cuda_fail(ctx, cudaGetLastError(), "event");
  }
  struct FreeEv {
    cudaEvent_t a, b;
    ~FreeEv() { cudaEventDestroy(a); cudaEventDestroy(b); }
  } fe{a0, a1};
  CK(launch_spmv_phase(ctx->P, ctx->plan, ctx->fp32), "spmv phase");   // warm-up
  CK(cudaEventRecord(a0, s), "event");
  for (int32_t k = 0; k < reps; ++k) CK(launch_spmv_phase(ctx->P, ctx->plan, ctx->fp32), "spmv phase");
  CK(cudaEventRecord(a1, s), "event");
  CK(cudaStreamSynchronize(s), "sync");
  float t = 0.f;
  CK(cudaEventElapsedTime(&t, a0, a1), "event");
  *ms = double(t) / double(reps);
  return ICCG_OK;
}

iccg_status iccg_precond(iccg_ctx *ctx, const double *r, double *z) {
  if (!ctx) return ICCG_ERR_ARG;
  DeviceGuard guard(ctx->device);
  const int32_t n = ctx->H.n;
  if (n == 0) return ICCG_OK;
  if (!r || !z) return ICCG_ERR_ARG;
  if (!ctx->factored) return ICCG_ERR_STATE;
  cudaStream_t s = ctx->stream;
  const Plan &L = ctx->plan;
  CK(copy_in(ctx, ctx->bin, r, size_t(n)), "copy r");
  CK(launch_permute(ctx->bin, ctx->P.r, ctx->P.perm, n, true, L.grid_v, s), "permute");
  CK(launch_precond(ctx->P, L, ctx->fp32), "precond");
  const double *zsrc = static_cast<const double *>(ctx->P.z);
  if (ctx->fp32) {
    CK(launch_widen(static_cast<const float *>(ctx->P.z), ctx->P.q, n, L.grid_v, s), "widen");
    zsrc = ctx->P.q;
  }
  CK(launch_permute(zsrc, ctx->xout, ctx->P.perm, n, false, L.grid_v, s), "permute");
  CK(copy_out(ctx, z, ctx->xout, size_t(n)), "copy z");
  CK(cudaStreamSynchronize(s), "sync");
  return ICCG_OK;
}

iccg_status iccg_spmv(iccg_ctx *ctx, const double *p, double *q) {
  if (!ctx) return ICCG_ERR_ARG;
  DeviceGuard guard(ctx->device);
  const int32_t n = ctx->H.n;
  if (n == 0) return ICCG_OK;
  if (!p || !q) return ICCG_ERR_ARG;
  cudaStream_t s = ctx->stream;
  const Plan &L = ctx->plan;
  CK(copy_in(ctx, ctx->bin, p, size_t(n)), "copy p");
  CK(launch_permute(ctx->bin, ctx->P.xh, ctx->P.perm, n, true, L.grid_v, s), "permute");
  CK(launch_spmv_plain(ctx->P, L), "spmv");
  CK(launch_permute(ctx->P.q, ctx->xout, ctx->P.perm, n, false, L.grid_v, s), "permute");
  CK(copy_out(ctx, q, ctx->xout, size_t(n)), "copy q");
  CK(cudaStreamSynchronize(s), "sync");
  return ICCG_OK;
}

iccg_status iccg_get_factor(iccg_ctx *ctx, double *lval, int64_t *nnz_lower) {
  if (!ctx || !nnz_lower) return ICCG_ERR_ARG;
  DeviceGuard guard(ctx->device);
  const HostLayout &H = ctx->H;
  *nnz_lower = H.nL + H.n;
  if (!lval) return ICCG_OK;
  if (!ctx->factored) return ICCG_ERR_STATE;
  std::vector<double> lv(size_t(H.nL)), dg(size_t(H.n));
  if (H.nL) CK(cudaMemcpyAsync(lv.data(), ctx->P.lval, sizeof(double) * lv.size(), cudaMemcpyDeviceToHost, ctx->stream), "copy L");
  if (H.n) CK(cudaMemcpyAsync(dg.data(), ctx->P.ldiag, sizeof(double) * dg.size(), cudaMemcpyDeviceToHost, ctx->stream), "copy D");
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  // rows and columns back in the caller's block-multicolor order (lane tiles
  // store a color's rows step-major)
  std::vector<int32_t> iord(size_t(H.n));
  for (int32_t i = 0; i < H.n; ++i) iord[size_t(H.ord[size_t(i)])] = i;
  std::vector<std::pair<int32_t, double>> row;
  int64_t k = 0;
  for (int32_t u = 0; u < H.n; ++u) {
    const int32_t i = iord[size_t(u)];
    row.clear();
    for (int32_t p = H.lrp[i]; p < H.lrp[i + 1]; ++p) row.emplace_back(H.ord[size_t(H.lcol[p])], lv[size_t(p)]);
    std::sort(row.begin(), row.end(),
              [](const std::pair<int32_t, double> &a, const std::pair<int32_t, double> &b) { return a.first < b.first; });
    for (const auto &pr : row) lval[k++] = pr.second;
    lval[k++] = dg[size_t(i)];
  }
  return ICCG_OK;
}

iccg_status iccg_info(const iccg_ctx *ctx, int64_t out[18]) {
  if (!ctx || !out) return ICCG_ERR_ARG;
  const HostLayout &H = ctx->H;
  out[0] = H.n;
  out[1] = H.nnz;
  out[2] = H.n_b;
  out[3] = H.n_c;
  out[4] = int64_t(H.groups.size());
  out[5] = 0;
  for (const GroupDesc &d : H.groups) out[5] += d.fit ? 0 : 1;
  out[6] = H.nL;
  out[7] = H.max_levels;
  out[8] = H.max_group_rows;
  out[9] = int64_t(H.tiles.size());
  out[10] = H.tile_colors;
  out[11] = out[12] = 0;
  for (char w : ctx->plan.wtile) {
    out[11] += w == 1 ? 1 : 0;
    out[12] += w == 2 ? 1 : 0;
  }
  out[13] = H.unit_colors;
  out[14] = ctx->plan.coop ? 1 : (ctx->plan.tail_c > 0 ? 2 : 0);
  const Plan &L = ctx->plan;
  int64_t fac = 1;    // factor_finish
  for (int c = 0; c < L.n_c; ++c)
    fac += (L.tile1[c] > L.tile0[c] || L.unit1[c] > L.unit0[c]) ? L.fac_nlev[c] : 1;
  const int64_t sw = L.n_c == 0 ? 0 : (L.coop ? 1 : (L.tail_c > 0 ? 2 * int64_t(L.tail_c) + 1 : 2 * int64_t(L.n_c) - 1));
  out[15] = fac;
  out[16] = 2 + sw;
  out[17] = 3 + sw;
  return ICCG_OK;
}

iccg_status iccg_set_wait_limit(iccg_ctx *ctx, uint64_t wait_ns) {
  if (!ctx) return ICCG_ERR_ARG;
  DeviceGuard guard(ctx->device);
  ctx->P.wait_ns = wait_ns ? wait_ns : kDefaultWaitNs;
  destroy_graph(ctx);   // the captured launches hold the old limit
  return ICCG_OK;
}

iccg_status iccg_last_error(const iccg_ctx *ctx, int64_t *row_or_block, const char **msg) {
  if (!ctx) return ICCG_ERR_ARG;
  if (row_or_block) *row_or_block = ctx->err_index;
  if (msg) *msg = ctx->err_msg.c_str();
  return ICCG_OK;
}

void iccg_destroy(iccg_ctx *ctx) {
  if (!ctx) return;
  {
    DeviceGuard guard(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    destroy_graph(ctx);
    if (ctx->fexec) cudaGraphExecDestroy(ctx->fexec);
    ctx->fexec = nullptr;
    for (void *p : ctx->allocs) cudaFree(p);
    if (ctx->sc_host) cudaFreeHost(ctx->sc_host);
    if (ctx->hist_host) cudaFreeHost(ctx->hist_host);
  }
  delete ctx;
}

}  // extern "C"
