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
                         const int32_t *color_ptr, int32_t n_b, int32_t n_c, int32_t group_rows,
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

  // groups: consecutive whole blocks of one color, at most G rows (a larger
  // block is a group of its own); one CTA per group
  const int32_t G = std::max(group_rows, 1);
  std::vector<int32_t> grow(1, 0);
  H.color_group.assign(n_c + 1, 0);
  for (int32_t c = 0; c < n_c; ++c) {
    H.color_group[c] = int32_t(grow.size()) - 1;
    int32_t j = color_ptr[c];
    while (j < color_ptr[c + 1]) {
      int32_t end = j + 1;
      while (end < color_ptr[c + 1] && block_ptr[end + 1] - block_ptr[j] <= G) ++end;
      grow.push_back(block_ptr[end]);
      j = end;
    }
  }
  H.color_group[n_c] = int32_t(grow.size()) - 1;
  const int32_t ngroups = int32_t(grow.size()) - 1;

  // in-group levels: forward over L (rows ascending), backward over U (rows
  // descending); the schedule of a group lists its rows level by level
  // (ascending row inside a level) and is stored at the group's row offset
  std::vector<int32_t> levf(n, 0), levb(n, 0), nlf(ngroups), nlb(ngroups);
#pragma omp parallel for schedule(dynamic, 64)
  for (int32_t g = 0; g < ngroups; ++g) {
    const int32_t r0 = grow[g], r1 = grow[g + 1];
    int32_t df = 0, db = 0;
    for (int32_t i = r0; i < r1; ++i) {
      int32_t lv = 0;
      for (int32_t e = H.lrp[i]; e < H.lrp[i + 1]; ++e)
        if (H.lcol[e] >= r0) lv = std::max(lv, levf[H.lcol[e]] + 1);
      levf[i] = lv;
      df = std::max(df, lv);
    }
    for (int32_t i = r1 - 1; i >= r0; --i) {
      int32_t lv = 0;
      for (int32_t e = H.urp[i]; e < H.urp[i + 1]; ++e)
        if (H.ucol[e] < r1) lv = std::max(lv, levb[H.ucol[e]] + 1);
      levb[i] = lv;
      db = std::max(db, lv);
    }
    nlf[g] = df + 1;
    nlb[g] = db + 1;
  }
  H.groups.assign(ngroups, GroupDesc{});
  int32_t off = 0;
  for (int32_t g = 0; g < ngroups; ++g) {
    GroupDesc &d = H.groups[g];
    d.r0 = grow[g]; d.r1 = grow[g + 1];
    d.l0 = H.lrp[d.r0]; d.l1 = H.lrp[d.r1];
    d.u0 = H.urp[d.r0]; d.u1 = H.urp[d.r1];
    d.nlf = nlf[g]; d.nlb = nlb[g];
    d.lf = off; off += d.nlf + 1;
    d.lb = off; off += d.nlb + 1;
    d.fit = 0; d.pad0 = d.pad1 = d.pad2 = 0;
  }
  H.sched_f.assign(n, 0);
  H.sched_b.assign(n, 0);
  H.levp.assign(off, 0);
#pragma omp parallel for schedule(dynamic, 64)
  for (int32_t g = 0; g < ngroups; ++g) {
    const GroupDesc &d = H.groups[g];
    for (int pass = 0; pass < 2; ++pass) {
      const std::vector<int32_t> &lev = pass == 0 ? levf : levb;
      const int32_t nl = pass == 0 ? d.nlf : d.nlb;
      int32_t *lp = H.levp.data() + (pass == 0 ? d.lf : d.lb);
      int32_t *sc = (pass == 0 ? H.sched_f.data() : H.sched_b.data()) + d.r0;
      for (int32_t l = 0; l <= nl; ++l) lp[l] = 0;
      for (int32_t i = d.r0; i < d.r1; ++i) lp[lev[i] + 1]++;
      for (int32_t l = 0; l < nl; ++l) lp[l + 1] += lp[l];
      std::vector<int32_t> fill(lp, lp + nl);
      for (int32_t i = d.r0; i < d.r1; ++i) sc[fill[lev[i]]++] = i - d.r0;
    }
  }
  // the shared-memory plan covers groups of at most G rows; a larger group
  // (one big block) reads its data from global memory
  int32_t seg_l = 0, seg_u = 0, maxlev = 1, maxrows = 1;
  H.max_group_rows = 0;
  H.max_levels = 0;
  for (int32_t g = 0; g < ngroups; ++g) {
    const GroupDesc &d = H.groups[g];
    H.max_group_rows = std::max(H.max_group_rows, d.r1 - d.r0);
    H.max_levels = std::max(H.max_levels, std::max(d.nlf, d.nlb));
    if (d.r1 - d.r0 > G) continue;
    seg_l = std::max(seg_l, d.l1 - d.l0);
    seg_u = std::max(seg_u, d.u1 - d.u0);
    maxlev = std::max(maxlev, std::max(d.nlf, d.nlb));
    maxrows = std::max(maxrows, d.r1 - d.r0);
  }
  H.seg_l = seg_l;
  H.seg_u = seg_u;
  H.fit_levels = maxlev;
  H.fit_rows = maxrows;
  int32_t seg_a = 0;
  for (int32_t r0 = 0; r0 < n; r0 += kWarp) seg_a = std::max(seg_a, H.arp[std::min(n, r0 + kWarp)] - H.arp[r0]);
  H.seg_a = seg_a;
  return ICCG_OK;
}

}  // namespace iccg
