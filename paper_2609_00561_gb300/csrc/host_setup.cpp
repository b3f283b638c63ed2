// Host-side setup of the block-multicolor layout (the one-time step before
// the solve; the paper excludes blocking and setup from the ICCG time,
// Sec. 6.6).  Validates the CSR matrix, the permutation, the block and color
// pointers and the coloring invariant of Sec. 3 (blocks of one color share no
// edge), then builds the permuted matrix, the strictly lower / upper parts of
// the IC(0) pattern and the per-color warp tiles.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "iccg_internal.h"

namespace iccg {

namespace {

iccg_status fail(iccg_status st, int64_t idx, const char *what, int64_t &bad, std::string &msg) {
  bad = idx;
  msg = what;
  return st;
}

}  // namespace

iccg_status build_layout(int32_t n, int64_t nnz, const int64_t *rowptr, const int32_t *colind,
                         const double *val, const int32_t *perm, const int32_t *block_ptr,
                         const int32_t *color_ptr, int32_t n_b, int32_t n_c, int32_t R,
                         HostLayout &H, int64_t &bad, std::string &msg) {
  bad = -1;
  if (n < 0 || nnz < 0 || nnz >= (int64_t(1) << 31)) return fail(ICCG_ERR_ARG, -1, "n or nnz out of range", bad, msg);
  if (n > 0 && (n_b < 1 || n_c < 1 || n_b > n || n_c > n_b)) return fail(ICCG_ERR_ARG, -1, "n_b / n_c out of range", bad, msg);
  if (n == 0 && (n_b != 0 || n_c != 0)) return fail(ICCG_ERR_ARG, -1, "empty matrix needs n_b = n_c = 0", bad, msg);
  if (rowptr[0] != 0 || rowptr[n] != nnz) return fail(ICCG_ERR_ARG, -1, "rowptr[0] must be 0 and rowptr[n] = nnz", bad, msg);
  for (int32_t i = 0; i < n; ++i)
    if (rowptr[i + 1] < rowptr[i]) return fail(ICCG_ERR_ARG, i, "rowptr not monotone", bad, msg);
  for (int64_t e = 0; e < nnz; ++e) {
    if (colind[e] < 0 || colind[e] >= n) return fail(ICCG_ERR_ARG, e, "column index out of range", bad, msg);
    if (!std::isfinite(val[e])) return fail(ICCG_ERR_ARG, e, "non-finite matrix value", bad, msg);
  }
  // permutation: a bijection on [0, n)
  H.n = n; H.nnz = nnz; H.n_b = n_b; H.n_c = n_c;
  H.perm.assign(perm, perm + n);
  H.iperm.assign(n, -1);
  for (int32_t i = 0; i < n; ++i) {
    int32_t o = perm[i];
    if (o < 0 || o >= n || H.iperm[o] >= 0) return fail(ICCG_ERR_ARG, i, "perm is not a permutation", bad, msg);
    H.iperm[o] = i;
  }
  if (n > 0) {
    if (block_ptr[0] != 0 || block_ptr[n_b] != n) return fail(ICCG_ERR_ARG, -1, "block_ptr must run from 0 to n", bad, msg);
    for (int32_t j = 0; j < n_b; ++j)
      if (block_ptr[j + 1] <= block_ptr[j]) return fail(ICCG_ERR_ARG, j, "block_ptr not strictly increasing", bad, msg);
    if (color_ptr[0] != 0 || color_ptr[n_c] != n_b) return fail(ICCG_ERR_ARG, -1, "color_ptr must run from 0 to n_b", bad, msg);
    for (int32_t c = 0; c < n_c; ++c)
      if (color_ptr[c + 1] <= color_ptr[c]) return fail(ICCG_ERR_ARG, c, "color_ptr not strictly increasing", bad, msg);
  }
  H.block_ptr.assign(block_ptr, block_ptr + (n > 0 ? n_b + 1 : 1));
  H.color_ptr.assign(color_ptr, color_ptr + (n > 0 ? n_c + 1 : 1));
  if (n == 0) H.block_ptr.assign(1, 0), H.color_ptr.assign(1, 0);

  // block and color of every new row
  std::vector<int32_t> blk(n), colr(n_b > 0 ? n_b : 1);
  for (int32_t j = 0; j < n_b; ++j)
    for (int32_t i = block_ptr[j]; i < block_ptr[j + 1]; ++i) blk[i] = j;
  for (int32_t c = 0; c < n_c; ++c)
    for (int32_t j = color_ptr[c]; j < color_ptr[c + 1]; ++j) colr[j] = c;

  // permuted matrix A_hat[i][j] = A[perm[i]][perm[j]], columns ascending
  H.arp.assign(n + 1, 0);
  for (int32_t i = 0; i < n; ++i) H.arp[i + 1] = H.arp[i] + int32_t(rowptr[perm[i] + 1] - rowptr[perm[i]]);
  H.acol.resize(nnz);
  H.aval.resize(nnz);
  int64_t err_row = -1;
  int err_kind = 0;
#pragma omp parallel
  {
    std::vector<std::pair<int32_t, double>> tmp;
#pragma omp for schedule(dynamic, 1024)
    for (int32_t i = 0; i < n; ++i) {
      int32_t o = perm[i];
      tmp.clear();
      for (int64_t e = rowptr[o]; e < rowptr[o + 1]; ++e) tmp.emplace_back(H.iperm[colind[e]], val[e]);
      std::sort(tmp.begin(), tmp.end(), [](const std::pair<int32_t, double> &a, const std::pair<int32_t, double> &b) { return a.first < b.first; });
      bool diag = false, dup = false;
      for (size_t k = 0; k < tmp.size(); ++k) {
        if (k && tmp[k].first == tmp[k - 1].first) dup = true;
        if (tmp[k].first == i) diag = true;
        H.acol[H.arp[i] + k] = tmp[k].first;
        H.aval[H.arp[i] + k] = tmp[k].second;
      }
      if (!diag || dup) {
#pragma omp critical
        {
          if (err_row < 0 || o < err_row) { err_row = o; err_kind = dup ? 2 : 1; }
        }
      }
    }
  }
  if (err_row >= 0)
    return fail(ICCG_ERR_ARG, err_row, err_kind == 2 ? "duplicate column in a row" : "missing diagonal entry", bad, msg);

  // structural symmetry and the coloring invariant
  int64_t sym_bad = -1, col_bad = -1;
#pragma omp parallel for schedule(dynamic, 1024)
  for (int32_t i = 0; i < n; ++i) {
    for (int32_t e = H.arp[i]; e < H.arp[i + 1]; ++e) {
      int32_t j = H.acol[e];
      if (j == i) continue;
      const int32_t *b0 = H.acol.data() + H.arp[j], *b1 = H.acol.data() + H.arp[j + 1];
      if (!std::binary_search(b0, b1, i)) {
#pragma omp critical
        { if (sym_bad < 0 || perm[i] < sym_bad) sym_bad = perm[i]; }
      }
      if (blk[i] != blk[j] && colr[blk[i]] == colr[blk[j]]) {
#pragma omp critical
        { if (col_bad < 0 || blk[i] < col_bad) col_bad = blk[i]; }
      }
    }
  }
  if (sym_bad >= 0) return fail(ICCG_ERR_ARG, sym_bad, "pattern of A is not symmetric", bad, msg);
  if (col_bad >= 0) return fail(ICCG_ERR_COLORING, col_bad, "two blocks of one color share an edge", bad, msg);

  // strictly lower (L) and strictly upper (U = L^T) parts
  H.lrp.assign(n + 1, 0);
  H.urp.assign(n + 1, 0);
  for (int32_t i = 0; i < n; ++i) {
    int32_t lo = 0, up = 0;
    for (int32_t e = H.arp[i]; e < H.arp[i + 1]; ++e) {
      if (H.acol[e] < i) lo++;
      else if (H.acol[e] > i) up++;
    }
    H.lrp[i + 1] = H.lrp[i] + lo;
    H.urp[i + 1] = H.urp[i] + up;
  }
  H.nL = H.lrp[n];
  H.lcol.resize(H.nL);
  H.ainit.resize(H.nL);
  H.ucol.resize(H.urp[n]);
  H.umap.resize(H.urp[n]);
  H.adiag.resize(n);
#pragma omp parallel for schedule(static)
  for (int32_t i = 0; i < n; ++i) {
    int32_t l = H.lrp[i], u = H.urp[i];
    for (int32_t e = H.arp[i]; e < H.arp[i + 1]; ++e) {
      int32_t j = H.acol[e];
      if (j < i) { H.lcol[l] = j; H.ainit[l] = H.aval[e]; ++l; }
      else if (j > i) { H.ucol[u] = j; ++u; }
      else H.adiag[i] = H.aval[e];
    }
  }
  // U entry (i, j), j > i, mirrors L entry (j, i)
#pragma omp parallel for schedule(static)
  for (int32_t i = 0; i < n; ++i) {
    for (int32_t u = H.urp[i]; u < H.urp[i + 1]; ++u) {
      int32_t j = H.ucol[u];
      const int32_t *b0 = H.lcol.data() + H.lrp[j], *b1 = H.lcol.data() + H.lrp[j + 1];
      H.umap[u] = int32_t(std::lower_bound(b0, b1, i) - H.lcol.data());
    }
  }

  // tiles and tasks per color
  const int32_t T = kWarp * R;
  std::vector<int32_t> tile_row(1, 0), task_tile(1, 0);
  H.color_task.assign(n_c + 1, 0);
  H.max_task_rows = 0;
  for (int32_t c = 0; c < n_c; ++c) {
    H.color_task[c] = int32_t(task_tile.size()) - 1;
    int32_t j = color_ptr[c];
    while (j < color_ptr[c + 1]) {
      int32_t size = block_ptr[j + 1] - block_ptr[j];
      if (size > T) {
        for (int32_t r0 = block_ptr[j] + T; r0 < block_ptr[j + 1]; r0 += T) tile_row.push_back(r0);
        tile_row.push_back(block_ptr[j + 1]);
        H.max_task_rows = std::max(H.max_task_rows, size);
        ++j;
      } else {
        int32_t end = j + 1;
        while (end < color_ptr[c + 1] && block_ptr[end + 1] - block_ptr[j] <= T) ++end;
        tile_row.push_back(block_ptr[end]);
        H.max_task_rows = std::max(H.max_task_rows, block_ptr[end] - block_ptr[j]);
        j = end;
      }
      task_tile.push_back(int32_t(tile_row.size()) - 1);
    }
  }
  H.color_task[n_c] = int32_t(task_tile.size()) - 1;
  const int32_t ntiles = int32_t(tile_row.size()) - 1;
  const int32_t ntasks = int32_t(task_tile.size()) - 1;

  // in-tile dependency depth: forward over L (rows ascending), backward over U
  H.lev.assign(n, 0);
  H.tiles.assign(ntiles, TileDesc{});
  std::vector<uint8_t> ulev(n, 0);
  int32_t maxr = 0, seg_l = 0, seg_u = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(max : maxr, seg_l, seg_u)
  for (int32_t t = 0; t < ntiles; ++t) {
    const int32_t t0 = tile_row[t], t1 = tile_row[t + 1];
    int32_t df = 0, db = 0;
    for (int32_t i = t0; i < t1; ++i) {
      int32_t lv = 0;
      for (int32_t e = H.lrp[i]; e < H.lrp[i + 1]; ++e)
        if (H.lcol[e] >= t0) lv = std::max(lv, H.lev[H.lcol[e]] + 1);
      H.lev[i] = uint8_t(lv);
      df = std::max(df, lv);
    }
    for (int32_t i = t1 - 1; i >= t0; --i) {
      int32_t lv = 0;
      for (int32_t e = H.urp[i]; e < H.urp[i + 1]; ++e)
        if (H.ucol[e] < t1) lv = std::max(lv, ulev[H.ucol[e]] + 1);
      ulev[i] = uint8_t(lv);
      db = std::max(db, lv);
    }
    TileDesc &d = H.tiles[t];
    d.r0 = t0; d.r1 = t1;
    d.rounds = (df + 1) | ((db + 1) << 16);
    d.pad = 0;
    d.l0 = H.lrp[t0]; d.l1 = H.lrp[t1];
    d.u0 = H.urp[t0]; d.u1 = H.urp[t1];
    maxr = std::max(maxr, std::max(df, db) + 1);
    seg_l = std::max(seg_l, d.l1 - d.l0);
    seg_u = std::max(seg_u, d.u1 - d.u0);
  }
  H.max_rounds = maxr;
  H.seg_l = seg_l;
  H.seg_u = seg_u;
  H.tasks.assign(ntasks, TaskDesc{});
  for (int32_t k = 0; k < ntasks; ++k) {
    TaskDesc &td = H.tasks[k];
    td.tile0 = task_tile[k];
    td.ntiles = task_tile[k + 1] - task_tile[k];
    td.first = H.tiles[td.tile0];
    td.pad0 = td.pad1 = 0;
  }
  int32_t seg_a = 0;
  for (int32_t r0 = 0; r0 < n; r0 += T) seg_a = std::max(seg_a, H.arp[std::min(n, r0 + T)] - H.arp[r0]);
  H.seg_a = seg_a;
  return ICCG_OK;
}

}  // namespace iccg
