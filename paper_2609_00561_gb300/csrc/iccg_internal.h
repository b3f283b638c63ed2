// Internal declarations of libiccg (not part of the C ABI).
//
// Device data layout (all in the block-multicolor numbering, Sec. 3):
//   A_hat   CSR (arp/acol/aval), and its off-diagonal entries sliced-ELL in
//           32-row slices (sa_ptr/sa_col/sa_val) with the diagonal (adiag)
//           for the SpMV of Table 8's "SpMV" phase.
//   L       strictly lower part of the IC(0) factor in CSR (lrp/lcol/lval),
//           diagonal separately (ldiag, invd = 1/L_ii).
//   U = L^T strictly upper part in CSR (urp/ucol/uval); umap[k] is the L
//           entry that U entry k mirrors.
//   A color is processed in one of two layouts:
//   Lane tiles (colors whose blocks all have at most lane_max rows): 32
//           blocks of the color form a tile, one block per lane of a warp;
//           the lane walks its block's rows in order (step k = k-th row).  The
//           tile's rows are stored step-major (the rows of step k of all its
//           lanes are consecutive), so every step reads and writes 32
//           consecutive rows.  Blocks of one color share no edge, so this
//           renumbering keeps every row's order relative to all rows it is
//           connected to: the IC(0) factor and the substitutions are the same
//           as in the user's block-multicolor order.  L and U rows of a step
//           are stored sliced-ELL (entry j of lane l at off + j*cnt + l), with
//           a reference to an earlier (later) row of the same block coded as
//           -(step + 1): that value sits in the warp's shared memory.
//   Groups  (other colors): consecutive whole blocks of one color up to
//           group_rows rows, or one larger block; one CTA each, rows resolved
//           level by level of the in-group dependency DAG.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/iccg.h"

namespace iccg {

constexpr int kWarp = 32;
constexpr int kMaxWarpsPerCta = 16;
constexpr int kSpmvWarps = 8;    // warps per CTA of the SpMV (one warp per 32-row slice)

// A group: consecutive whole blocks of one color (or one big block), the
// work of one warp.  Its forward / backward schedules list the group's rows
// (as offsets from r0) level by level; they are stored at sched_f[r0 ..],
// sched_b[r0 ..], with level pointers at levp[lf ..] / levp[lb ..].
struct __align__(16) GroupDesc {
  int32_t r0, r1;      // rows [r0, r1)
  int32_t l0, l1;      // L entries [l0, l1)
  int32_t u0, u1;      // U entries [u0, u1)
  int32_t lf, lb;      // level-pointer offsets (forward, backward)
  int32_t nlf, nlb;    // level counts
  int32_t fit;         // 1: the group fits the per-warp shared-memory plan
  int32_t pad0, pad1, pad2, pad3, pad4;
};

constexpr int kGroup = 32;   // CTAs per first-level reduction group
constexpr unsigned long long kDefaultWaitNs = 4000000000ull;   // device-side wait limit (4 s)

// A lane tile: rows [row0, row0 + nrows), step descriptors steps[step0 ..
// step0 + nsteps); its sliced-ELL entries are the contiguous ranges
// [lo0, lo1) (L, other colors), [li0, li1) (L, in-block), [uo0, uo1),
// [ui0, ui1) (U); wl / wu: its widest in-block L / U step; lw0 / uw0: the
// widths of its first step's entries to other colors (a one-step tile is
// fully described without its step descriptor).
struct __align__(16) TileDesc {
  int32_t row0, nrows, nsteps, step0, lo0, lo1, li0, li1, uo0, uo1, ui0, ui1, wl, wu, lw0, uw0;
};
// One step of a tile: rows [row, row + cnt) (lanes 0 .. cnt-1; blocks are
// sorted by size, so the active lanes are a prefix).  Sliced-ELL entry j of
// lane l sits at off + j*cnt + l: L entries to other colors at (lo, lw),
// in-block L entries at (li, liw), U likewise (uo, uw), (ui, uiw).
struct __align__(16) StepDesc {
  int32_t row, cnt, lo, lw, li, liw, uo, uw, ui, uiw, pad0, pad1;
};
// A tile of at most two steps in one descriptor (blocks of one or two rows):
// step 0 = rows [row0, row0 + c0), step 1 = rows [row0 + c0, row0 + c0 + c1);
// other-color entries of step 0 at lo, of step 1 at lo + lw0 * c0 (U: uo,
// uo + uw0 * c0); the in-block L entries are step 1's (at li, width liw1,
// each referring to step 0), the in-block U entries step 0's (at ui, width
// uiw0, each referring to step 1).
struct __align__(16) PairDesc {
  int32_t row0, c0, c1, lo, lw0, lw1, li, liw1, uo, uw0, uw1, ui, uiw0, pad0, pad1, pad2;
};
// A warp unit (a color whose blocks have at most 32 rows): 32 / S consecutive
// blocks of one color, each at most S rows (S a power of two), one warp;
// lane l holds row l % S of block blk0 + l / S (rows of a block are
// consecutive in the caller's order, which these colors keep).  Its entries
// to other colors are sliced-ELL over the 32 lanes (entry j of lane l at
// off + 32 j + l; L at (lo, lw), U at (uo, uw)).  Its in-block recurrence runs
// as lm (forward) / um (backward) chain steps: at step m a lane subtracts at
// most one in-block term, coefficient x the final value of the source lane;
// coefficient m of lane l at li + 32 m + l (ui for U), the source lanes as
// bytes, four steps per word, word w of lane l at ls + 32 w + l (us for U),
// and bit m of the lane's mask (wl_mask / wu_mask) marks a step with a term.
struct __align__(16) WarpUnit {
  int32_t blk0, nblk, lo, lw, uo, uw, li, lm, ui, um, row0, nrows, ls, us, pad0, pad1;
};
constexpr int32_t kPadCol = 0x7fffffff;   // padding entry of a sliced-ELL step
constexpr int kTileSmemBudget = 96 * 1024;      // lane-tile CTA with two buffers, bytes
constexpr int kTileSmemBudget1 = 200 * 1024;    // lane-tile CTA with one buffer, bytes

// Shared memory of a lane tile's CTA (offsets in bytes, 16-byte aligned).
// Two buffers, each: the step descriptors, 1/L_ii of the tile's rows and
// the in-block sliced-ELL entries (steps, values) of L and/or U, copied as the
// 16-byte-aligned cover of the tile's range (capacity cap_i entries + 16 bytes
// on either side; a tile with more in-block entries reads them from global
// memory); the CTA computes one tile from one buffer while the next tile is
// copied into the other.  Then the row values w[step][lane].
struct TilePlan {
  int cap_s, cap_r, cap_i;          // steps, rows, in-block entries per tile
  int cap_o;                        // other-color entries per tile staged (0: read from global memory)
  int o_steps, o_dv, o_ic, o_iv;    // within a buffer
  int o_oc, o_ov, o_vec;            // other-color entries (columns, values), four row vectors
  int o_ic2, o_iv2;                 // second entry set (U of a fused launch)
  int buf1, buf2;                   // buffer bytes with one / two entry sets
  int w_bytes;
  int nbuf;                         // 2: the next tile is copied while one is computed; 1: in turn
  int cap_i2;                       // second-set capacity of a fused launch (0: read from global memory)
};

__host__ __device__ inline int r16b(int bytes) { return (bytes + 15) & ~15; }

// With cap_o > 0 a buffer also holds the tile's entries to other colors (L
// forward, U backward) and four vectors over its rows (r, q, x, p forward;
// y, r backward), so that a tile's loads are issued while the previous tile
// is computed.
__host__ __device__ inline TilePlan tile_plan(int cap_s, int cap_r, int cap_i, int elem, int cap_o = 0) {
  TilePlan p;
  p.cap_s = cap_s; p.cap_r = cap_r; p.cap_i = cap_i; p.cap_o = cap_o;
  int o = 0;
  p.o_steps = o; o += r16b(cap_s * 48);
  p.o_dv = o; o += r16b((cap_r + 8) * elem);
  p.o_oc = p.o_ov = p.o_vec = o;
  if (cap_o > 0) {
    p.o_oc = o; o += r16b((cap_o + 8) * 4);
    p.o_ov = o; o += r16b((cap_o + 8) * elem);
    p.o_vec = o; o += 4 * r16b((cap_r + 8) * 8);
  }
  p.o_ic = o; o += r16b((cap_i + 8) * 4);
  p.o_iv = o; o += r16b((cap_i + 8) * elem);
  p.buf1 = o;
  p.o_ic2 = o; o += r16b((cap_i + 8) * 4);
  p.o_iv2 = o; o += r16b((cap_i + 8) * elem);
  p.buf2 = o;
  p.w_bytes = r16b(cap_s * kWarp * elem);
  p.nbuf = 2;
  p.cap_i2 = cap_i;
  return p;
}

// bytes of a lane-tile launch: nbuf buffers and w
__host__ __device__ inline int tile_launch_bytes(const TilePlan &p, bool two_sets) {
  return p.nbuf * (two_sets && p.cap_i2 > 0 ? p.buf2 : p.buf1) + p.w_bytes;
}

// Grid barrier of the persistent solve kernel: arrival count, generation
// (bumped by the last arrival) and a sticky error word set by a CTA whose
// bounded wait gave up.  count and err start at zero for every launch.
struct GridBar {
  uint32_t count, gen, err, pad;
};

// Device-resident scalars of one solve.
struct Scalars {
  double bb, bnorm, rr, rz, pq, alpha, beta, tol;
  int32_t iter, maxit, done, status;
  uint32_t ticket;       // arrival counter for "last CTA reduces" epilogues
  int32_t use_cond;      // 1 when a graph conditional handle is live
  unsigned long long cond_handle;
};

// Everything a kernel needs; passed by value.
struct Params {
  int32_t n, R, W, n_c;
  // A_hat
  const int32_t *arp, *acol;
  const double *aval;
  // L / U
  const int32_t *lrp, *lcol, *urp, *ucol, *umap;
  double *lval, *uval, *ldiag, *invd;
  float *lval32, *uval32, *invd32;
  const double *ainit, *adiag;
  // A_hat's off-diagonal entries sliced-ELL (slice s = rows [32s, 32s+32):
  // entry j of lane l at sa_ptr[s] + 32 j + l; padding (row, 0.0))
  const int32_t *sa_ptr, *sa_col;
  const double *sa_val;
  // groups and their level schedules
  const GroupDesc *groups;
  const int32_t *sched_f, *sched_b, *levp;
  // per-warp shared-memory plan: entries of the staged L / U segment, rows
  // and levels of a fitting group
  int32_t cap_l, cap_u, cap_a, cap_rows, cap_lev;
  // vectors (permuted numbering)
  double *xh, *r, *q, *p0, *p1, *bh;
  void *y, *z;                  // double or float, by precision
  const double *bin, *xin;      // original-order inputs
  double *xout;                 // original-order output
  const int32_t *perm;
  // reductions.  Every color launch stores one <r,r> and/or <r,z> partial
  // per CTA into slot_rr / slot_rz (its own region, plain stores); the last
  // launch of an iteration sums all slots: each of its CTAs sums a fixed chunk
  // of the earlier launches' slots plus its own partial into part0 / part1,
  // the last CTA of each group of kGroup CTAs sums its group into gsum0 /
  // gsum1, and the last group runs the epilogue.  The SpMV stores one <p,q>
  // partial per CTA in part_a; its last CTA sums them.  init_bb / part_a hold
  // <b,b> and <r0,r0> partials at the solve start.
  double *slot_rr, *slot_rz;    // [nslot]
  double *part0, *part1;        // [npart]
  double *gsum0, *gsum1;        // [ngroup]
  double *part_a, *init_bb;     // [npart_a], [nbb]
  uint32_t *gticket;            // [ngroup] group arrival counters
  int32_t nslot, npart, ngroup, npart_a, nbb;
  Scalars *sc;
  // lane tiles: sliced-ELL entries to other colors (sl_ / su_: column, or
  // kPadCol for padding) and in-block entries (si_ / ui_: the step of the
  // same block's row); values are filled from the factor through the maps
  // (the L entry an entry takes, -1: padding)
  const TileDesc *tiles;
  const PairDesc *pairs;        // [tiles]: the tile as a PairDesc (tiles of <= 2 steps)
  const StepDesc *steps;
  const int32_t *sl_col, *su_col, *sl_map, *su_map;
  const int32_t *si_col, *ui_col, *si_map, *ui_map;
  double *sl_val, *su_val, *si_val, *ui_val;
  float *sl_val32, *su_val32, *si_val32, *ui_val32;
  int32_t nsl, nsu, nsi, nui;
  int32_t lane_max, wi_max;     // largest tile block (steps) and in-block width
  int32_t tcap_r, tcap_i;       // largest tile rows; in-block entries staged per tile (L or U)
  int32_t tcap_o;               // other-color entries staged per tile (0: global memory)
  int32_t tnbuf;                // lane-tile staging buffers per CTA (1 or 2)
  int32_t tcap_i2;              // fused launch: second-set staging capacity (0: global)
  // persistent solve: first group of each color [n_c + 1], grid barrier
  const int32_t *color_group;
  GridBar *bar;
  unsigned long long wait_ns;   // bounded grid-barrier wait (ns)
  // optional phase trace of the persistent solve: (ns << 4 | phase) per
  // barrier, written by CTA 0 (null: off); trace_len receives the count
  unsigned long long *trace;
  int32_t *trace_len;
  int32_t trace_cap;
  double *hist;
  unsigned long long *err_row;  // IC(0) breakdown row (new numbering), ~0 = none
  const int32_t *fac_rows;      // IC(0) rows of the lane-tile colors, level by level
  const int4 *fac_rec;          // per fac_rows entry: row, first L entry, first pair, entries | pairs << 8
  const int32_t *fp_ptr, *fp_b;  // IC(0) update pairs (null: not built)
  const uint8_t *fp_pos;
  // warp units: descriptors, per-lane in-block masks, in-block coefficients
  // (forward: L_lk / L_kk; backward: L_kl / L_kk, k the source step's row),
  // filled from the factor through (entry map, scaling row); block pointers
  const WarpUnit *units;
  const uint32_t *wl_mask, *wu_mask;
  const uint32_t *wl_src, *wu_src;    // chain-step source lanes, four bytes a word
  const int32_t *wl_map, *wl_srow, *wu_map, *wu_srow;
  double *wl_val, *wu_val;
  float *wl_val32, *wu_val32;
  int32_t nwl, nwu;
  const int32_t *bptr;
  const int32_t *ctile;         // first lane tile of each color [n_c + 1] (cooperative sweep)
};

// ---- host-side layout built by iccg_setup --------------------------------
struct HostLayout {
  int32_t n = 0, n_b = 0, n_c = 0;
  int64_t nnz = 0, nL = 0;
  std::vector<int32_t> perm, iperm;
  std::vector<int32_t> arp, acol;
  std::vector<double> aval;
  std::vector<int32_t> lrp, lcol, urp, ucol, umap;
  std::vector<double> ainit, adiag;
  std::vector<int32_t> sa_ptr, sa_col;          // A_hat off-diagonal, sliced-ELL (32-row slices)
  std::vector<double> sa_val;
  std::vector<GroupDesc> groups;
  std::vector<int32_t> sched_f, sched_b, levp;
  std::vector<int32_t> color_group;   // n_c + 1 (no groups for a tile color)
  std::vector<int32_t> color_tile;    // n_c + 1 (no tiles for a group color)
  std::vector<TileDesc> tiles;
  std::vector<PairDesc> pairs;
  std::vector<StepDesc> steps;
  std::vector<int32_t> sl_col, su_col, sl_map, su_map;
  std::vector<int32_t> si_col, ui_col, si_map, ui_map;
  int32_t wi_max = 0;                 // widest in-block step of any tile
  int32_t tcap_r = 0, tcap_i = 0;     // largest tile: rows, in-block entries
  int32_t tcap_o = 0;                 // largest tile: entries to other colors (L or U)
  std::vector<int32_t> ord;           // internal row -> row of the caller's block-multicolor order
  // IC(0) schedule of the lane-tile colors: the color's rows by in-block
  // dependency level (level 0: no earlier row of the same block in the
  // pattern); rows of level v of color c are fac_rows[fac_ptr[fac_lev0[c] + v]
  // .. fac_ptr[fac_lev0[c] + v + 1]), fac_nlev[c] levels (0 for a group color)
  std::vector<int32_t> fac_rows, fac_ptr, fac_lev0, fac_nlev;
  std::vector<int32_t> fac_wide;      // per level: the widest row's lower entries
  // IC(0) update pairs (symbolic factorisation, when small enough): for L
  // entry e = (i, j), the terms L_ik L_jk with k < j in both patterns, k
  // ascending, as pairs fp_pos[q] (position of k in row i) and fp_b[q] (the L
  // entry (j, k)), q in [fp_ptr[e], fp_ptr[e + 1]); empty when not built
  std::vector<int32_t> fp_ptr, fp_b;
  std::vector<uint8_t> fp_pos;
  // warp units (colors of blocks of at most 32 rows when enabled): color c's units
  // [color_unit[c], color_unit[c + 1]), unit_S[c] rows per segment
  std::vector<WarpUnit> units;
  std::vector<int32_t> color_unit, unit_S;
  std::vector<uint32_t> wl_mask, wu_mask, wl_src, wu_src;
  std::vector<int32_t> wl_map, wl_srow, wu_map, wu_srow;
  int32_t unit_colors = 0;
  int32_t lane_max = 0;               // largest block of a tile color
  int32_t tile_colors = 0;
  std::vector<int32_t> block_ptr, color_ptr;
  int32_t max_group_rows = 0, max_levels = 0;   // over all groups
  int32_t fit_rows = 0, fit_levels = 0;         // over groups of at most 32R rows
  int32_t seg_l = 0, seg_u = 0, seg_a = 0;      // largest segments (entries)
};

// Validates inputs and builds the layout (groups of at most group_rows rows);
// returns ICCG_OK or an error with (bad_index, message) filled in.
// Colors whose blocks all have at most lane_max rows (<= 32; 0 = none) use
// lane tiles.
// Colors whose largest block has unit_min..32 rows use warp units instead
// of lane tiles (unit_min = 0: no warp units).
iccg_status build_layout(int32_t n, int64_t nnz, const int64_t *rowptr, const int32_t *colind,
                         const double *val, const int32_t *perm, const int32_t *block_ptr,
                         const int32_t *color_ptr, int32_t n_b, int32_t n_c, int32_t group_rows,
                         int32_t lane_max, int32_t unit_min, HostLayout &out, int64_t &bad_index,
                         std::string &msg);

// ---- launch plan (host side) ---------------------------------------------
struct Plan {
  cudaStream_t stream = nullptr;
  bool pdl = true;                      // programmatic dependent launch
  int32_t W = 8, R = 1, n_c = 0, n = 0;
  int32_t Wa = 4;                       // warps per CTA of the SpMV
  std::vector<int32_t> task0, task1;    // group range of each color
  std::vector<int32_t> grid_c;          // CTAs of the color-c kernels
  std::vector<int32_t> tile0, tile1;    // tile range of each color (empty: groups)
  int32_t Wt = 8;                       // warps per CTA of the lane-tile kernels (one tile at a time)
  int32_t smem_tile = 0, smem_tile2 = 0;  // bytes per CTA of the lane-tile kernels (one / two entry sets)
  int32_t smem_tile_x = 0;              // bytes per CTA with the entries to other colors staged as well
  int32_t cap_ti = 0;                   // in-block entries of a tile staged in shared memory
  int32_t nbuf_t = 2;                   // lane-tile staging buffers per CTA
  int32_t cap_ti2 = 0;                  // second-set (fused launch) staging capacity
  int32_t cap_to = 0;                   // other-color entries staged per tile (0: global)
  std::vector<char> stage_ext;          // color c's lane-tile launches stage those entries (tiles of <= 2 steps)
  std::vector<char> wtile;              // color c: 0 CTA per tile, 1 warp-tile kernels, 2 pair kernels, 3 warp units
  std::vector<int32_t> unit0, unit1, unit_S;   // warp-unit range and segment size of each color
  int32_t Wu = 8;                       // warps per CTA of the warp-unit kernels
  bool coop = false;                    // every sweep as one cooperative launch (pair-tile layouts)
  int32_t grid_coop = 0;                // CTAs of that launch (all resident)
  int32_t tail_c = 0;                   // > 0: colors tail_c.. of every sweep in one cooperative launch
  int32_t grid_tail = 0;                // CTAs of that launch (one per SM)
  int32_t Ww = 8;                       // warps per CTA of the warp-tile kernels
  int32_t Wp = 4;                       // warps per CTA of the pair kernels
  std::vector<char> pstage_f, pstage_b; // pair color c's forward / backward launches stage their entries
  int32_t smem_wt = 0;                  // bytes per CTA of the warp-tile kernels
  int32_t cap_ws = 0;                   // steps per tile held in a warp's buffer
  std::vector<int32_t> off_rr, off_rz;  // slot regions of the color-c forward / backward launches
  std::vector<int32_t> fac_ptr, fac_lev0, fac_nlev, fac_wide;   // IC(0) level schedule (host copy)
  int32_t last_rr = 0, last_rz = 0;     // slots written before the final launch of an iteration
  int32_t grid_a = 0;                   // CTAs of the SpMV-shaped kernels
  int32_t grid_v = 0;                   // CTAs of the vector kernels
  int32_t smem_fwd = 0, smem_bwd = 0, smem_fused = 0, smem_a = 0;  // bytes per CTA
  int32_t grid_p = 0, smem_p = 0;       // persistent kernel: CTAs (all co-resident), bytes per CTA
  int32_t cap_p = 0;                    // persistent kernel: staged SpMV entries per warp
};

// phase ids for the profiling hook
enum Phase { PH_INIT = 0, PH_SPMV = 1, PH_FWD = 2, PH_FUSED = 3, PH_BWD = 4, PH_ALL = 5, PH_COUNT = 6 };
typedef void (*PhaseHook)(void *user, int phase, int begin);

// ---- kernel launchers (kernels.cu) ----------------------------------------
cudaError_t configure_kernels();
int group_smem_bytes(int cap, int rows, int levs, int elem);  // per-warp plan of the color kernels
int spmv_smem_bytes(int cap);                                // per-warp staging of the SpMV
int spmv_resident_ctas(int Wa, int smem);                    // CTAs per SM of the SpMV
int tile_resident_ctas(bool fp32, int threads, int smem);    // CTAs per SM of the lane-tile kernels
int wtile_resident_ctas(bool fp32, int threads, int smem);   // CTAs per SM of the warp-tile kernels
int pair_resident_ctas(bool fp32, int threads);              // CTAs per SM of the pair kernels
int unit_resident_ctas(bool fp32, int S, int threads);       // CTAs per SM of the warp-unit kernels
int coop_sweep_resident_ctas(bool fp32);                     // CTAs per SM of the cooperative sweep (0: none)
cudaError_t launch_factor(const Params &P, const Plan &L, int nL);
cudaError_t launch_solve_init(const Params &P, const Plan &L, bool fp32, PhaseHook h, void *u);
cudaError_t launch_solve_body(const Params &P, const Plan &L, bool fp32, PhaseHook h, void *u);
// the SpMV phase of a PCG iteration: p = z + beta p, then q = A p and <p,q>
cudaError_t launch_spmv_phase(const Params &P, const Plan &L, bool fp32);
cudaError_t launch_solve_final(const Params &P, const Plan &L);
// bytes per CTA of the persistent kernel within max(group plan, budget);
// *cap_spmv = staged SpMV entries per warp
int persistent_smem_bytes(const Params &P, bool fp32, int W, int budget, int *cap_spmv);
int persistent_resident_ctas(bool fp32, int W, int smem);        // CTAs per SM
cudaError_t launch_solve_persistent(const Params &P, const Plan &L, bool fp32);  // whole solve, one launch
cudaError_t launch_precond(const Params &P, const Plan &L, bool fp32);  // z(perm) from r(perm)
cudaError_t launch_spmv_plain(const Params &P, const Plan &L);          // q = A_hat xh
cudaError_t launch_permute(const double *src, double *dst, const int32_t *perm, int32_t n,
                           bool gather, int32_t grid, cudaStream_t s);
cudaError_t launch_widen(const float *src, double *dst, int32_t n, int32_t grid, cudaStream_t s);

}  // namespace iccg

// A context (C ABI handle): the layout, the launch plan, device arrays and
// solve state of one system.
struct iccg_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  iccg_opts opts{};
  bool fp32 = false;
  bool persistent = false;         // the whole solve as one cooperative launch
  iccg::HostLayout H;
  iccg::Plan plan;
  iccg::Params P{};
  bool factored = false;
  std::vector<void *> allocs;
  // solve state
  double *hist = nullptr;
  int32_t hist_cap = 0;
  double *bin = nullptr, *xin = nullptr, *xout = nullptr;
  iccg::Scalars *sc_host = nullptr;      // pinned
  double *hist_host = nullptr;     // pinned
  int32_t hist_host_cap = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaGraphExec_t fexec = nullptr;      // IC(0): its launch sequence as one graph
  bool fgraph_failed = false;
  unsigned long long cond_handle = 0;
  // error record
  int64_t err_index = -1;
  std::string err_msg;
};
