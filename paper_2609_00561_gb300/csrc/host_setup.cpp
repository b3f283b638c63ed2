// Host-side setup of the block-multicolor layout (the one-time step before
// the solve; the paper excludes blocking and setup from the ICCG time,
// Sec. 6.6).  Validates the CSR matrix, the permutation, the block and color
// pointers and the coloring invariant of Sec. 3 (blocks of one color share no
// edge), then builds the permuted matrix, the strictly lower / upper parts of
// the IC(0) pattern, the lane tiles of small-block colors and the groups of
// the other colors.
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
                         int32_t lane_max, int32_t unit_min, HostLayout &H, int64_t &bad, std::string &msg) {
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

  // lane tiles: a color whose blocks all have at most lane_max rows is cut
  // into tiles of 32 blocks (sorted by size, largest first, so the lanes still
  // active at a step are a prefix), its rows stored step-major per tile
  lane_max = std::max(0, std::min(lane_max, 32));
  std::vector<char> tcol(n_c > 0 ? n_c : 1, 0);
  // warp units: colors whose largest block has unit_min..32 rows (when
  // enabled, unit_min >= 1); they keep the caller's row order
  std::vector<char> wcol(n_c > 0 ? n_c : 1, 0);
  H.unit_colors = 0;
  for (int32_t c = 0; c < n_c && unit_min > 0; ++c) {
    int32_t mb = 0;
    for (int32_t j = color_ptr[c]; j < color_ptr[c + 1]; ++j) mb = std::max(mb, block_ptr[j + 1] - block_ptr[j]);
    if (mb >= unit_min && mb <= kWarp) {
      wcol[c] = 1;
      H.unit_colors++;
    }
  }
  H.ord.resize(n);
  for (int32_t i = 0; i < n; ++i) H.ord[i] = i;
  H.lane_max = 0;
  H.tile_colors = 0;
  struct TileRows { int32_t row0, nsteps, nlanes; std::vector<int32_t> cnt; };
  std::vector<std::vector<TileRows>> ctiles(n_c > 0 ? n_c : 1);
  for (int32_t c = 0; c < n_c && lane_max > 0; ++c) {
    if (wcol[c]) continue;
    int32_t mb = 0;
    for (int32_t j = color_ptr[c]; j < color_ptr[c + 1]; ++j) mb = std::max(mb, block_ptr[j + 1] - block_ptr[j]);
    if (mb > lane_max) continue;
    // a tile's step descriptors, 1/L_ii and row values must fit the CTA's
    // shared memory (its in-block entries are staged only when they fit too)
    if (tile_launch_bytes(tile_plan(mb, kWarp * mb, 0, 8), true) > kTileSmemBudget) continue;
    tcol[c] = 1;
    H.tile_colors++;
    H.lane_max = std::max(H.lane_max, mb);
    std::vector<int32_t> bl;
    for (int32_t j = color_ptr[c]; j < color_ptr[c + 1]; ++j) bl.push_back(j);
    std::stable_sort(bl.begin(), bl.end(), [&](int32_t a, int32_t b) {
      return block_ptr[a + 1] - block_ptr[a] > block_ptr[b + 1] - block_ptr[b];
    });
    int32_t row = block_ptr[color_ptr[c]];
    for (size_t t0 = 0; t0 < bl.size(); t0 += kWarp) {
      const int32_t nl = int32_t(std::min<size_t>(kWarp, bl.size() - t0));
      TileRows tr;
      tr.row0 = row;
      tr.nlanes = nl;
      tr.nsteps = block_ptr[bl[t0] + 1] - block_ptr[bl[t0]];
      for (int32_t k = 0; k < tr.nsteps; ++k) {
        int32_t cnt = 0;
        while (cnt < nl && block_ptr[bl[t0 + cnt] + 1] - block_ptr[bl[t0 + cnt]] > k) ++cnt;
        for (int32_t l = 0; l < cnt; ++l) H.ord[row++] = block_ptr[bl[t0 + l]] + k;
        tr.cnt.push_back(cnt);
      }
      ctiles[c].push_back(std::move(tr));
    }
  }
  if (H.tile_colors > 0) {
    // renumber: internal row i is row ord[i] of the caller's order
    std::vector<int32_t> iord(n);
    for (int32_t i = 0; i < n; ++i) iord[H.ord[i]] = i;
    std::vector<int32_t> arp(n + 1, 0), acol(nnz);
    std::vector<double> aval(nnz);
    for (int32_t i = 0; i < n; ++i) arp[i + 1] = arp[i] + (H.arp[H.ord[i] + 1] - H.arp[H.ord[i]]);
#pragma omp parallel
    {
      std::vector<std::pair<int32_t, double>> tmp;
#pragma omp for schedule(dynamic, 1024)
      for (int32_t i = 0; i < n; ++i) {
        const int32_t u = H.ord[i];
        tmp.clear();
        for (int32_t e = H.arp[u]; e < H.arp[u + 1]; ++e) tmp.emplace_back(iord[H.acol[e]], H.aval[e]);
        std::sort(tmp.begin(), tmp.end(),
                  [](const std::pair<int32_t, double> &a, const std::pair<int32_t, double> &b) { return a.first < b.first; });
        for (size_t k = 0; k < tmp.size(); ++k) {
          acol[arp[i] + k] = tmp[k].first;
          aval[arp[i] + k] = tmp[k].second;
        }
      }
    }
    H.arp.swap(arp);
    H.acol.swap(acol);
    H.aval.swap(aval);
    for (int32_t i = 0; i < n; ++i) {
      H.perm[i] = perm[H.ord[i]];
      H.iperm[H.perm[i]] = i;
    }
  }
  // block of every internal row and the row's position (step) in its block
  std::vector<int32_t> iblk(n), istep(n);
  for (int32_t i = 0; i < n; ++i) {
    iblk[i] = blk[H.ord[i]];
    istep[i] = H.ord[i] - block_ptr[iblk[i]];
  }

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

  // IC(0) update pairs of every L entry (the symbolic part of the factor),
  // built when every row has at most 32 lower entries and the pairs stay
  // within a budget; otherwise the numeric factor finds them itself
  H.fp_ptr.clear(); H.fp_b.clear(); H.fp_pos.clear();
  {
    constexpr int64_t kPairBudget = int64_t(64) << 20;
    bool ok = true;
    for (int32_t i = 0; i < n && ok; ++i) ok = H.lrp[i + 1] - H.lrp[i] <= 32;
    std::vector<int32_t> cnt;
    if (ok) {
      cnt.assign(size_t(H.nL), 0);
#pragma omp parallel for schedule(dynamic, 1024)
      for (int32_t i = 0; i < n; ++i) {
        for (int32_t e = H.lrp[i]; e < H.lrp[i + 1]; ++e) {
          const int32_t j = H.lcol[e];
          int32_t a = H.lrp[i], b = H.lrp[j], c = 0;
          while (a < e && b < H.lrp[j + 1]) {
            if (H.lcol[a] == H.lcol[b]) { ++c; ++a; ++b; }
            else if (H.lcol[a] < H.lcol[b]) ++a;
            else ++b;
          }
          cnt[size_t(e)] = c;
        }
      }
      int64_t tot = 0;
      for (int32_t c : cnt) tot += c;
      ok = tot <= kPairBudget;
    }
    if (ok && H.nL > 0) {
      H.fp_ptr.assign(size_t(H.nL) + 1, 0);
      for (int64_t e = 0; e < H.nL; ++e) H.fp_ptr[size_t(e) + 1] = H.fp_ptr[size_t(e)] + cnt[size_t(e)];
      H.fp_b.resize(size_t(H.fp_ptr[size_t(H.nL)]));
      H.fp_pos.resize(H.fp_b.size());
#pragma omp parallel for schedule(dynamic, 1024)
      for (int32_t i = 0; i < n; ++i) {
        for (int32_t e = H.lrp[i]; e < H.lrp[i + 1]; ++e) {
          const int32_t j = H.lcol[e];
          int32_t a = H.lrp[i], b = H.lrp[j], q = H.fp_ptr[size_t(e)];
          while (a < e && b < H.lrp[j + 1]) {
            if (H.lcol[a] == H.lcol[b]) {
              H.fp_pos[size_t(q)] = uint8_t(a - H.lrp[i]);
              H.fp_b[size_t(q)] = b;
              ++q; ++a; ++b;
            } else if (H.lcol[a] < H.lcol[b]) ++a;
            else ++b;
          }
        }
      }
    }
  }

  // lane tiles: descriptors and the sliced-ELL L / U entries of every step,
  // split into entries to other colors and in-block entries
  H.color_tile.assign(n_c + 1, 0);
  H.tiles.clear();
  H.steps.clear();
  H.sl_col.clear(); H.su_col.clear(); H.sl_map.clear(); H.su_map.clear();
  H.si_col.clear(); H.ui_col.clear(); H.si_map.clear(); H.ui_map.clear();
  H.wi_max = 0;
  H.tcap_r = H.tcap_i = H.tcap_o = 0;
  // appends, sliced-ELL, the entries of rows row .. row+cnt-1 that are
  // in-block (inb) or not; emap maps a CSR entry to its L entry (null:
  // itself); returns the width
  std::vector<std::vector<int32_t>> sel;
  auto sell = [&](int32_t row, int32_t cnt, const std::vector<int32_t> &rp, const std::vector<int32_t> &cols,
                  const int32_t *emap, bool inb, std::vector<int32_t> &ocol, std::vector<int32_t> &omap) {
    int32_t width = 0;
    sel.assign(size_t(cnt), std::vector<int32_t>());
    for (int32_t l = 0; l < cnt; ++l) {
      const int32_t i = row + l;
      for (int32_t e = rp[i]; e < rp[i + 1]; ++e)
        if ((iblk[cols[e]] == iblk[i]) == inb) sel[size_t(l)].push_back(e);
      width = std::max(width, int32_t(sel[size_t(l)].size()));
    }
    for (int32_t j = 0; j < width; ++j)
      for (int32_t l = 0; l < cnt; ++l) {
        if (j < int32_t(sel[size_t(l)].size())) {
          const int32_t e = sel[size_t(l)][size_t(j)];
          ocol.push_back(inb ? istep[cols[e]] : cols[e]);
          omap.push_back(emap ? emap[e] : e);
        } else {
          ocol.push_back(inb ? 0 : kPadCol);
          omap.push_back(-1);
        }
      }
    return width;
  };
  for (int32_t c = 0; c < n_c; ++c) {
    H.color_tile[c] = int32_t(H.tiles.size());
    for (const TileRows &tr : ctiles[c]) {
      TileDesc td{};
      td.row0 = tr.row0;
      td.nsteps = tr.nsteps;
      td.step0 = int32_t(H.steps.size());
      td.lo0 = int32_t(H.sl_col.size());
      td.li0 = int32_t(H.si_col.size());
      td.uo0 = int32_t(H.su_col.size());
      td.ui0 = int32_t(H.ui_col.size());
      int32_t row = tr.row0;
      for (int32_t k = 0; k < tr.nsteps; ++k) {
        const int32_t cnt = tr.cnt[k];
        StepDesc sd{};
        sd.row = row;
        sd.cnt = cnt;
        sd.lo = int32_t(H.sl_col.size());
        sd.lw = sell(row, cnt, H.lrp, H.lcol, nullptr, false, H.sl_col, H.sl_map);
        sd.li = int32_t(H.si_col.size());
        sd.liw = sell(row, cnt, H.lrp, H.lcol, nullptr, true, H.si_col, H.si_map);
        sd.uo = int32_t(H.su_col.size());
        sd.uw = sell(row, cnt, H.urp, H.ucol, H.umap.data(), false, H.su_col, H.su_map);
        sd.ui = int32_t(H.ui_col.size());
        sd.uiw = sell(row, cnt, H.urp, H.ucol, H.umap.data(), true, H.ui_col, H.ui_map);
        td.wl = std::max(td.wl, sd.liw);
        td.wu = std::max(td.wu, sd.uiw);
        if (k == 0) { td.lw0 = sd.lw; td.uw0 = sd.uw; }
        H.steps.push_back(sd);
        row += cnt;
      }
      td.nrows = row - tr.row0;
      td.lo1 = int32_t(H.sl_col.size());
      td.li1 = int32_t(H.si_col.size());
      td.uo1 = int32_t(H.su_col.size());
      td.ui1 = int32_t(H.ui_col.size());
      H.wi_max = std::max(H.wi_max, std::max(td.wl, td.wu));
      H.tcap_r = std::max(H.tcap_r, td.nrows);
      H.tcap_i = std::max(H.tcap_i, std::max(td.li1 - td.li0, td.ui1 - td.ui0));
      H.tcap_o = std::max(H.tcap_o, std::max(td.lo1 - td.lo0, td.uo1 - td.uo0));
      H.tiles.push_back(td);
    }
  }
  H.color_tile[n_c] = int32_t(H.tiles.size());
  // IC(0) schedule of the lane-tile and warp-unit colors: a row's in-block level is one
  // more than the deepest earlier row of its block it refers to (internal
  // numbering: earlier steps of a block have smaller indices); the rows of a
  // level depend only on earlier levels and earlier colors
  H.fac_rows.clear();
  H.fac_wide.clear();
  H.fac_ptr.assign(1, 0);
  H.fac_lev0.assign(n_c + 1, 0);
  H.fac_nlev.assign(n_c + 1, 0);
  {
    std::vector<int32_t> lev(n, 0), cnt;
    for (int32_t c = 0; c < n_c; ++c) {
      H.fac_lev0[c] = int32_t(H.fac_ptr.size()) - 1;
      if (!tcol[c] && !wcol[c]) continue;
      const int32_t r0 = block_ptr[color_ptr[c]], r1 = block_ptr[color_ptr[c + 1]];
      int32_t depth = 0;
      for (int32_t i = r0; i < r1; ++i) {
        int32_t lv = 0;
        for (int32_t e = H.lrp[i]; e < H.lrp[i + 1]; ++e)
          if (H.lcol[e] >= r0 && iblk[H.lcol[e]] == iblk[i]) lv = std::max(lv, lev[H.lcol[e]] + 1);
        lev[i] = lv;
        depth = std::max(depth, lv + 1);
      }
      cnt.assign(size_t(depth) + 1, 0);
      for (int32_t i = r0; i < r1; ++i) cnt[size_t(lev[i]) + 1]++;
      for (int32_t v = 0; v < depth; ++v) cnt[size_t(v) + 1] += cnt[size_t(v)];
      const int32_t base = int32_t(H.fac_rows.size());
      H.fac_rows.resize(size_t(base) + size_t(r1 - r0));
      std::vector<int32_t> fill(cnt.begin(), cnt.end() - 1);
      for (int32_t i = r0; i < r1; ++i) H.fac_rows[size_t(base + fill[size_t(lev[i])]++)] = i;
      for (int32_t v = 1; v <= depth; ++v) H.fac_ptr.push_back(base + cnt[size_t(v)]);
      H.fac_nlev[c] = depth;
      std::vector<int32_t> wide(size_t(depth), 0);
      for (int32_t i = r0; i < r1; ++i) wide[size_t(lev[i])] = std::max(wide[size_t(lev[i])], H.lrp[i + 1] - H.lrp[i]);
      H.fac_wide.insert(H.fac_wide.end(), wide.begin(), wide.end());
    }
    H.fac_lev0[n_c] = int32_t(H.fac_ptr.size()) - 1;
  }
  // tiles of at most two steps, each in one descriptor
  H.pairs.assign(H.tiles.size(), PairDesc{});
  for (size_t t = 0; t < H.tiles.size(); ++t) {
    const TileDesc &td = H.tiles[t];
    if (td.nsteps > 2) continue;
    const StepDesc &s0 = H.steps[size_t(td.step0)];
    PairDesc &pd = H.pairs[t];
    pd.row0 = td.row0; pd.c0 = s0.cnt; pd.lo = s0.lo; pd.lw0 = s0.lw; pd.uo = s0.uo; pd.uw0 = s0.uw;
    pd.ui = s0.ui; pd.uiw0 = s0.uiw;
    pd.li = td.li0;
    if (td.nsteps == 2) {
      const StepDesc &s1 = H.steps[size_t(td.step0) + 1];
      pd.c1 = s1.cnt; pd.lw1 = s1.lw; pd.liw1 = s1.liw; pd.uw1 = s1.uw; pd.li = s1.li;
    }
  }
  // warp units: 32 / S blocks per warp, lane l = row l % S of block l / S
  H.color_unit.assign(n_c + 1, 0);
  H.unit_S.assign(n_c + 1, 0);
  H.units.clear();
  H.wl_mask.clear(); H.wu_mask.clear(); H.wl_src.clear(); H.wu_src.clear();
  H.wl_map.clear(); H.wl_srow.clear(); H.wu_map.clear(); H.wu_srow.clear();
  {
    std::vector<std::vector<int32_t>> se(kWarp), sw(kWarp);
    // appends the per-lane lists sliced-ELL over 32 lanes, padding (pad, -1)
    auto slab = [&](std::vector<std::vector<int32_t>> &a, std::vector<std::vector<int32_t>> &b,
                    std::vector<int32_t> &oa, std::vector<int32_t> &ob, int32_t pad) {
      int32_t w = 0;
      for (int l = 0; l < kWarp; ++l) w = std::max(w, int32_t(a[size_t(l)].size()));
      for (int32_t j = 0; j < w; ++j)
        for (int l = 0; l < kWarp; ++l) {
          const bool ok = j < int32_t(a[size_t(l)].size());
          oa.push_back(ok ? a[size_t(l)][size_t(j)] : pad);
          ob.push_back(ok ? b[size_t(l)][size_t(j)] : -1);
        }
      return w;
    };
    for (int32_t c = 0; c < n_c; ++c) {
      H.color_unit[c] = int32_t(H.units.size());
      if (!wcol[c]) continue;
      int32_t mb = 0;
      for (int32_t j = color_ptr[c]; j < color_ptr[c + 1]; ++j) mb = std::max(mb, block_ptr[j + 1] - block_ptr[j]);
      int32_t S = 1;
      while (S < mb) S <<= 1;
      H.unit_S[c] = S;
      const int32_t per = kWarp / S;
      for (int32_t j = color_ptr[c]; j < color_ptr[c + 1]; j += per) {
        WarpUnit u{};
        u.blk0 = j;
        u.nblk = std::min(per, color_ptr[c + 1] - j);
        u.row0 = block_ptr[j];
        u.nrows = block_ptr[j + u.nblk] - u.row0;
        std::vector<int32_t> lrow(kWarp, -1);
        for (int l = 0; l < kWarp; ++l) {
          const int32_t b = j + l / S;
          if (l / S < u.nblk && block_ptr[b] + l % S < block_ptr[b + 1]) lrow[size_t(l)] = block_ptr[b] + l % S;
        }
        for (int pass = 0; pass < 2; ++pass) {
          const std::vector<int32_t> &rp = pass ? H.urp : H.lrp, &cols = pass ? H.ucol : H.lcol;
          // entries to other colors
          for (int l = 0; l < kWarp; ++l) {
            se[size_t(l)].clear();
            sw[size_t(l)].clear();
            const int32_t i = lrow[size_t(l)];
            if (i < 0) continue;
            for (int32_t e = rp[size_t(i)]; e < rp[size_t(i) + 1]; ++e)
              if (iblk[cols[size_t(e)]] != iblk[i]) {
                se[size_t(l)].push_back(cols[size_t(e)]);
                sw[size_t(l)].push_back(pass ? H.umap[size_t(e)] : e);
              }
          }
          if (pass == 0) { u.lo = int32_t(H.sl_col.size()); u.lw = slab(se, sw, H.sl_col, H.sl_map, kPadCol); }
          else { u.uo = int32_t(H.su_col.size()); u.uw = slab(se, sw, H.su_col, H.su_map, kPadCol); }
          // in-block terms as a chain schedule: lane l's terms (source row
          // k, coefficient) in the order their sources become final, one per
          // step (a source is final the step after its own last term; rows
          // are visited in dependency order: ascending forward, descending
          // backward), each at the earliest step both it and the lane allow
          std::vector<int32_t> ready(size_t(kWarp), 0);
          std::vector<std::vector<std::pair<int32_t, int32_t>>> sched(kWarp);   // (step, term index)
          std::vector<std::vector<int32_t>> tsrc(kWarp), tmap(kWarp), trow(kWarp);
          for (int l = 0; l < kWarp; ++l) {
            const int32_t i = lrow[size_t(l)];
            if (i < 0) continue;
            for (int32_t e = rp[size_t(i)]; e < rp[size_t(i) + 1]; ++e) {
              const int32_t k = cols[size_t(e)];
              if (iblk[k] != iblk[i]) continue;
              tsrc[size_t(l)].push_back((l / S) * S + (k - block_ptr[iblk[i]]));
              tmap[size_t(l)].push_back(pass ? H.umap[size_t(e)] : e);
              trow[size_t(l)].push_back(k);
            }
          }
          int32_t M = 0;
          for (int q = 0; q < kWarp; ++q) {
            const int l = pass ? kWarp - 1 - q : q;   // sources before their targets within a block
            const size_t nt = tsrc[size_t(l)].size();
            std::vector<int32_t> ord(nt);
            for (size_t x = 0; x < nt; ++x) ord[x] = int32_t(x);
            std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) {
              return ready[size_t(tsrc[size_t(l)][size_t(a)])] < ready[size_t(tsrc[size_t(l)][size_t(b)])];
            });
            int32_t t = 0;
            for (int32_t x : ord) {
              const int32_t st = std::max(t, ready[size_t(tsrc[size_t(l)][size_t(x)])]);
              sched[size_t(l)].push_back({st, x});
              t = st + 1;
            }
            ready[size_t(l)] = t;
            M = std::max(M, t);
          }
          if (M > kWarp) return fail(ICCG_ERR_ARG, u.blk0, "warp-unit chain longer than 32 steps", bad, msg);
          const int32_t co = int32_t((pass ? H.wu_map : H.wl_map).size());
          const int32_t so = int32_t((pass ? H.wu_src : H.wl_src).size());
          std::vector<int32_t> &mp = pass ? H.wu_map : H.wl_map, &sr = pass ? H.wu_srow : H.wl_srow;
          std::vector<uint32_t> &swd = pass ? H.wu_src : H.wl_src, &mk = pass ? H.wu_mask : H.wl_mask;
          // coefficients term-major: lane l's j-th term (in step order) at
          // co + j * 32 + l, the block as deep as the lane with most terms
          size_t T = 0;
          for (int l = 0; l < kWarp; ++l) T = std::max(T, sched[size_t(l)].size());
          mp.resize(size_t(co) + T * kWarp, -1);
          sr.resize(size_t(co) + T * kWarp, -1);
          const int32_t nw = (M + 3) / 4;
          swd.resize(size_t(so) + size_t(nw) * kWarp, 0u);
          for (int l = 0; l < kWarp; ++l) {
            uint32_t mask = 0;
            for (int m = 0; m < nw * 4; ++m) {   // idle steps read the lane itself
              const size_t w = size_t(so) + size_t(m / 4) * kWarp + size_t(l);
              swd[w] |= uint32_t(l) << (8 * (m % 4));
            }
            size_t j = 0;
            for (const auto &pr : sched[size_t(l)]) {
              const int32_t m = pr.first, x = pr.second;
              mask |= 1u << m;
              mp[size_t(co) + j * kWarp + size_t(l)] = tmap[size_t(l)][size_t(x)];
              sr[size_t(co) + j * kWarp + size_t(l)] = trow[size_t(l)][size_t(x)];
              ++j;
              const size_t w = size_t(so) + size_t(m / 4) * kWarp + size_t(l);
              swd[w] = (swd[w] & ~(0xffu << (8 * (m % 4)))) | (uint32_t(tsrc[size_t(l)][size_t(x)]) << (8 * (m % 4)));
            }
            mk.push_back(mask);
          }
          if (pass == 0) { u.li = co; u.lm = M; u.ls = so; }
          else { u.ui = co; u.um = M; u.us = so; }
        }
        H.units.push_back(u);
      }
    }
    H.color_unit[n_c] = int32_t(H.units.size());
  }
  const size_t lim = size_t(1) << 31;
  if (H.wl_map.size() >= lim || H.wu_map.size() >= lim) return fail(ICCG_ERR_ARG, -1, "warp-unit layout exceeds 2^31 entries", bad, msg);
  if (H.sl_col.size() >= lim || H.su_col.size() >= lim || H.si_col.size() >= lim || H.ui_col.size() >= lim)
    return fail(ICCG_ERR_ARG, -1, "lane-tile layout exceeds 2^31 entries", bad, msg);

  // groups (the other colors): consecutive whole blocks of one color, at most
  // G rows (a larger block is a group of its own); one CTA per group
  const int32_t G = std::max(group_rows, 1);
  std::vector<int32_t> gr0, gr1;   // rows [gr0[g], gr1[g]) of group g
  H.color_group.assign(n_c + 1, 0);
  for (int32_t c = 0; c < n_c; ++c) {
    H.color_group[c] = int32_t(gr0.size());
    if (tcol[c] || wcol[c]) continue;
    int32_t j = color_ptr[c];
    while (j < color_ptr[c + 1]) {
      int32_t end = j + 1;
      while (end < color_ptr[c + 1] && block_ptr[end + 1] - block_ptr[j] <= G) ++end;
      gr0.push_back(block_ptr[j]);
      gr1.push_back(block_ptr[end]);
      j = end;
    }
  }
  H.color_group[n_c] = int32_t(gr0.size());
  const int32_t ngroups = int32_t(gr0.size());

  // in-group levels: forward over L (rows ascending), backward over U (rows
  // descending); the schedule of a group lists its rows level by level
  // (ascending row inside a level) and is stored at the group's row offset
  std::vector<int32_t> levf(n, 0), levb(n, 0), nlf(ngroups), nlb(ngroups);
  // (group colors keep the caller's order: internal row = caller's row)
#pragma omp parallel for schedule(dynamic, 64)
  for (int32_t g = 0; g < ngroups; ++g) {
    const int32_t r0 = gr0[g], r1 = gr1[g];
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
    d.r0 = gr0[g]; d.r1 = gr1[g];
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

  // A_hat's off-diagonal entries sliced-ELL for the SpMV: slice s holds rows
  // [32s, 32s + 32), width w_s = its longest row; entry j of lane l at
  // sa_ptr[s] + 32 j + l; padding (the row itself, 0.0)
  const int32_t nsl = (n + kWarp - 1) / kWarp;
  H.sa_ptr.assign(nsl + 1, 0);
  int64_t tot = 0;
  for (int32_t s = 0; s < nsl; ++s) {
    int32_t w = 0;
    for (int32_t i = s * kWarp; i < std::min(n, (s + 1) * kWarp); ++i) w = std::max(w, H.arp[i + 1] - H.arp[i] - 1);
    tot += int64_t(w) * kWarp;
    if (tot > INT32_MAX) return fail(ICCG_ERR_ARG, -1, "matrix too large for 32-bit sliced-ELL offsets", bad, msg);
    H.sa_ptr[s + 1] = int32_t(tot);
  }
  H.sa_col.assign(size_t(tot), 0);
  H.sa_val.assign(size_t(tot), 0.0);
#pragma omp parallel for schedule(static)
  for (int32_t s = 0; s < nsl; ++s) {
    const int32_t w = (H.sa_ptr[s + 1] - H.sa_ptr[s]) / kWarp;
    for (int32_t l = 0; l < kWarp; ++l) {
      const int32_t i = s * kWarp + l;
      int32_t j = 0;
      if (i < n)
        for (int32_t e = H.arp[i]; e < H.arp[i + 1]; ++e) {
          if (H.acol[e] == i) continue;
          H.sa_col[H.sa_ptr[s] + j * kWarp + l] = H.acol[e];
          H.sa_val[H.sa_ptr[s] + j * kWarp + l] = H.aval[e];
          ++j;
        }
      for (; j < w; ++j) H.sa_col[H.sa_ptr[s] + j * kWarp + l] = i < n ? i : 0;
    }
  }
  return ICCG_OK;
}

}  // namespace iccg

// ---------------------------------------------------------------------------
// Diagnostics: build the layout as iccg_setup does (host only) and check the
// index ranges the kernels rely on.
// ---------------------------------------------------------------------------
namespace {

struct Checker {
  int64_t failed = 0, first = -1;
  const char *what = nullptr;
  void operator()(bool ok, int64_t where, const char *msg) {
    if (ok) return;
    if (failed++ == 0) {
      first = where;
      what = msg;
    }
  }
};

}  // namespace

extern "C" iccg_status iccg_check_layout(int32_t n, int64_t nnz, const int64_t *rowptr, const int32_t *colind,
                                         const double *val, const int32_t *perm, const int32_t *block_ptr,
                                         const int32_t *color_ptr, int32_t n_b, int32_t n_c, int32_t group_rows,
                                         int32_t lane_max, int32_t use_units, int64_t report[4],
                                         const char **what) {
  using namespace iccg;
  if (!report || !rowptr) return ICCG_ERR_ARG;
  HostLayout H;
  int64_t bad = -1;
  std::string msg;
  const iccg_status st = build_layout(n, nnz, rowptr, colind, val, perm, block_ptr, color_ptr, n_b, n_c,
                                      std::max(group_rows, 1), lane_max, use_units ? 1 : 0, H, bad, msg);
  report[0] = report[1] = report[2] = report[3] = 0;
  if (st != ICCG_OK) {
    report[3] = bad;
    return st;
  }
  Checker ck;
  // A_hat sliced-ELL: slice widths, padding on the row itself, every
  // off-diagonal CSR entry once
  {
    const int32_t nsl = (n + kWarp - 1) / kWarp;
    ck(int32_t(H.sa_ptr.size()) == nsl + 1 && H.sa_ptr[0] == 0, -1, "A slices");
    for (int32_t sl = 0; sl < nsl; ++sl) {
      const int32_t e0 = H.sa_ptr[size_t(sl)], e1 = H.sa_ptr[size_t(sl) + 1];
      ck(e1 >= e0 && (e1 - e0) % kWarp == 0, sl, "A slice width");
      const int32_t w = (e1 - e0) / kWarp;
      for (int32_t l = 0; l < kWarp; ++l) {
        const int32_t i = sl * kWarp + l;
        int32_t j = 0;
        if (i < n)
          for (int32_t e = H.arp[size_t(i)]; e < H.arp[size_t(i) + 1]; ++e) {
            if (H.acol[size_t(e)] == i) continue;
            const int32_t k = e0 + j * kWarp + l;
            ck(j < w && H.sa_col[size_t(k)] == H.acol[size_t(e)] && H.sa_val[size_t(k)] == H.aval[size_t(e)], sl,
               "A slice entry");
            ++j;
          }
        for (; j < w; ++j) {
          const int32_t k = e0 + j * kWarp + l;
          ck(H.sa_val[size_t(k)] == 0.0 && H.sa_col[size_t(k)] == (i < n ? i : 0), sl, "A slice padding");
        }
      }
    }
  }
  // tiles: step rows consecutive, active lanes a prefix, entries inside their
  // step's range, in-block references to existing earlier (L) or later (U)
  // steps of the same lane, other-color columns in range
  for (size_t t = 0; t < H.tiles.size(); ++t) {
    const TileDesc &td = H.tiles[t];
    ck(td.nsteps >= 1 && td.nsteps <= H.lane_max, int64_t(t), "tile steps");
    ck(td.nrows <= H.tcap_r, int64_t(t), "tile rows");
    int32_t row = td.row0;
    for (int s = 0; s < td.nsteps; ++s) {
      const StepDesc &sd = H.steps[size_t(td.step0 + s)];
      ck(sd.row == row, int64_t(t), "step rows");
      ck(sd.cnt >= 1 && sd.cnt <= kWarp, int64_t(t), "step lanes");
      if (s == 0) ck(sd.lo == td.lo0 && sd.lw == td.lw0 && sd.li == td.li0 && sd.uo == td.uo0 && sd.uw == td.uw0 &&
                     sd.ui == td.ui0, int64_t(t), "first step in the tile descriptor");
      if (td.nsteps == 1) ck(sd.cnt == td.nrows && sd.liw == td.wl && sd.uiw == td.wu, int64_t(t), "one-step tile");
      if (td.nsteps <= 2) {
        const PairDesc &pd = H.pairs[t];
        if (s == 0)
          ck(pd.row0 == sd.row && pd.c0 == sd.cnt && pd.lo == sd.lo && pd.lw0 == sd.lw && sd.liw == 0 &&
                 pd.uo == sd.uo && pd.uw0 == sd.uw && pd.ui == sd.ui && pd.uiw0 == sd.uiw &&
                 (td.nsteps == 2 || (pd.c1 == 0 && pd.liw1 == 0 && sd.uiw == 0)),
             int64_t(t), "pair descriptor, step 0");
        else
          ck(pd.c1 == sd.cnt && sd.row == pd.row0 + pd.c0 && sd.lo == pd.lo + pd.lw0 * pd.c0 && pd.lw1 == sd.lw &&
                 pd.li == sd.li && pd.liw1 == sd.liw && sd.uo == pd.uo + pd.uw0 * pd.c0 && pd.uw1 == sd.uw &&
                 sd.uiw == 0,
             int64_t(t), "pair descriptor, step 1");
      }
      if (s) ck(sd.cnt <= H.steps[size_t(td.step0 + s - 1)].cnt, int64_t(t), "active lanes a prefix");
      ck(sd.lo >= td.lo0 && sd.lo + sd.lw * sd.cnt <= td.lo1, int64_t(t), "L other-color range");
      ck(sd.li >= td.li0 && sd.li + sd.liw * sd.cnt <= td.li1, int64_t(t), "L in-block range");
      ck(sd.uo >= td.uo0 && sd.uo + sd.uw * sd.cnt <= td.uo1, int64_t(t), "U other-color range");
      ck(sd.ui >= td.ui0 && sd.ui + sd.uiw * sd.cnt <= td.ui1, int64_t(t), "U in-block range");
      for (int j = 0; j < sd.liw; ++j)
        for (int l = 0; l < sd.cnt; ++l) {
          const size_t e = size_t(sd.li + j * sd.cnt + l);
          const int c = H.si_col[e];
          ck(c >= 0 && c < td.nsteps, int64_t(t), "in-block L step");
          if (H.si_map[e] >= 0) ck(c < s && l < H.steps[size_t(td.step0 + c)].cnt, int64_t(t), "in-block L order");
        }
      for (int j = 0; j < sd.uiw; ++j)
        for (int l = 0; l < sd.cnt; ++l) {
          const size_t e = size_t(sd.ui + j * sd.cnt + l);
          const int c = H.ui_col[e];
          ck(c >= 0 && c < td.nsteps, int64_t(t), "in-block U step");
          if (H.ui_map[e] >= 0) ck(c > s && l < H.steps[size_t(td.step0 + c)].cnt, int64_t(t), "in-block U order");
        }
      for (int j = 0; j < sd.lw; ++j)
        for (int l = 0; l < sd.cnt; ++l) {
          const int c = H.sl_col[size_t(sd.lo + j * sd.cnt + l)];
          ck(c == kPadCol || (c >= 0 && c < n), int64_t(t), "L other-color column");
        }
      for (int j = 0; j < sd.uw; ++j)
        for (int l = 0; l < sd.cnt; ++l) {
          const int c = H.su_col[size_t(sd.uo + j * sd.cnt + l)];
          ck(c == kPadCol || (c >= 0 && c < n), int64_t(t), "U other-color column");
        }
      row += sd.cnt;
    }
    ck(row == td.row0 + td.nrows, int64_t(t), "tile row count");
  }
  // groups: level pointers monotone and complete, schedules a permutation
  for (size_t g = 0; g < H.groups.size(); ++g) {
    const GroupDesc &gd = H.groups[g];
    const int rows = gd.r1 - gd.r0;
    ck(rows >= 1, int64_t(g), "group rows");
    for (int pass = 0; pass < 2; ++pass) {
      const int lp0 = pass ? gd.lb : gd.lf, nl = pass ? gd.nlb : gd.nlf;
      ck(H.levp[size_t(lp0)] == 0 && H.levp[size_t(lp0 + nl)] == rows, int64_t(g), "level pointers");
      for (int lv = 0; lv < nl; ++lv) ck(H.levp[size_t(lp0 + lv)] <= H.levp[size_t(lp0 + lv + 1)], int64_t(g), "levels");
      std::vector<char> seen(size_t(rows), 0);
      const std::vector<int32_t> &sch = pass ? H.sched_b : H.sched_f;
      for (int i = gd.r0; i < gd.r1; ++i) {
        const int l = sch[size_t(i)];
        ck(l >= 0 && l < rows && !seen[size_t(std::max(0, std::min(l, rows - 1)))], int64_t(g), "schedule");
        if (l >= 0 && l < rows) seen[size_t(l)] = 1;
      }
    }
  }
  // IC(0) schedule of the lane-tile colors: every row of the color once, and
  // every in-block reference of a row at an earlier level
  {
    std::vector<int32_t> level(size_t(n), -1);
    for (int c = 0; c < n_c; ++c) {
      const bool tile = H.color_tile[size_t(c) + 1] > H.color_tile[size_t(c)] ||
                        H.color_unit[size_t(c) + 1] > H.color_unit[size_t(c)];
      if (!tile) { ck(H.fac_nlev[size_t(c)] == 0, c, "factor schedule of a group color"); continue; }
      const int32_t r0 = H.block_ptr[size_t(H.color_ptr[size_t(c)])], r1 = H.block_ptr[size_t(H.color_ptr[size_t(c) + 1])];
      int64_t seen = 0;
      for (int v = 0; v < H.fac_nlev[size_t(c)]; ++v) {
        const int32_t k0 = H.fac_ptr[size_t(H.fac_lev0[size_t(c)] + v)], k1 = H.fac_ptr[size_t(H.fac_lev0[size_t(c)] + v + 1)];
        ck(k0 <= k1, c, "factor level pointers");
        for (int32_t k = k0; k < k1; ++k) {
          const int32_t i = H.fac_rows[size_t(k)];
          const bool in = i >= r0 && i < r1;
          ck(in && level[size_t(std::max(0, std::min(i, n - 1)))] < 0, c, "factor schedule rows");
          if (in) level[size_t(i)] = v;
          ++seen;
        }
      }
      ck(seen == r1 - r0, c, "factor schedule covers the color");
      for (int32_t i = r0; i < r1; ++i)
        for (int32_t e = H.lrp[size_t(i)]; e < H.lrp[size_t(i) + 1]; ++e) {
          const int32_t j = H.lcol[size_t(e)];
          if (j >= r0) ck(level[size_t(j)] >= 0 && level[size_t(j)] < level[size_t(i)], c, "factor schedule order");
        }
    }
  }
  // warp units: lanes on the rows of their blocks; each chain holds every
  // in-block term of a row once, from a lane of the same block whose own last
  // term comes at an earlier step; entries to other colors outside the block
  for (int c = 0; c < n_c; ++c) {
    const int S = H.unit_S[size_t(c)];
    for (int32_t t = H.color_unit[size_t(c)]; t < H.color_unit[size_t(c) + 1]; ++t) {
      const WarpUnit &u = H.units[size_t(t)];
      ck(S >= 1 && S <= kWarp && (S & (S - 1)) == 0 && u.nblk >= 1 && u.nblk <= kWarp / S, t, "unit shape");
      ck(u.blk0 >= H.color_ptr[size_t(c)] && u.blk0 + u.nblk <= H.color_ptr[size_t(c) + 1], t, "unit blocks");
      ck(u.row0 == H.block_ptr[size_t(u.blk0)] && u.row0 + u.nrows == H.block_ptr[size_t(u.blk0 + u.nblk)], t, "unit rows");
      for (int l = 0; l < kWarp; ++l) {
        const int32_t b = u.blk0 + l / S;
        const bool on = l / S < u.nblk && H.block_ptr[size_t(b)] + l % S < H.block_ptr[size_t(b) + 1];
        const int32_t i = on ? H.block_ptr[size_t(b)] + l % S : -1;
        for (int pass = 0; pass < 2; ++pass) {
          const uint32_t m = (pass ? H.wu_mask : H.wl_mask)[size_t(t) * kWarp + l];
          const int32_t off = pass ? u.ui : u.li, M = pass ? u.um : u.lm, so = pass ? u.us : u.ls;
          const std::vector<int32_t> &mp = pass ? H.wu_map : H.wl_map, &sr = pass ? H.wu_srow : H.wl_srow;
          const std::vector<uint32_t> &swd = pass ? H.wu_src : H.wl_src;
          ck(M >= 0 && M <= kWarp && (M == kWarp || (m >> M) == 0u), t, "chain steps");
          if (!on) { ck(m == 0u, t, "idle lane mask"); continue; }
          // every in-block entry of the row exactly once, from its own block,
          // after the source lane's last term
          std::vector<int32_t> want;
          const std::vector<int32_t> &rp = pass ? H.urp : H.lrp, &cols = pass ? H.ucol : H.lcol;
          for (int32_t e = rp[size_t(i)]; e < rp[size_t(i) + 1]; ++e)
            if (cols[size_t(e)] >= H.block_ptr[size_t(b)] && cols[size_t(e)] < H.block_ptr[size_t(b) + 1])
              want.push_back(pass ? H.umap[size_t(e)] : e);
          std::vector<int32_t> got;
          int32_t j = 0;
          for (int k = 0; k < M; ++k) {
            const uint32_t src = (swd[size_t(so) + size_t(k / 4) * kWarp + size_t(l)] >> (8 * (k % 4))) & 0xffu;
            if (!((m >> k) & 1u)) continue;
            // the lane's terms are stored term-major: its j-th term at off + j * 32 + l
            const size_t e = size_t(off) + size_t(j++) * kWarp + size_t(l);
            ck(e < mp.size(), t, "chain term slot");
            if (e >= mp.size()) break;
            got.push_back(mp[e]);
            const int32_t srow = H.block_ptr[size_t(b)] + int32_t(src) % S;
            ck(int32_t(src) / S == l / S && sr[e] == srow && (pass ? srow > i : srow < i), t, "chain source");
            // the source lane has no term at this step or later
            const uint32_t ms = (pass ? H.wu_mask : H.wl_mask)[size_t(t) * kWarp + src];
            ck((ms >> k) == 0u, t, "chain order");
          }
          std::sort(want.begin(), want.end());
          std::sort(got.begin(), got.end());
          ck(want == got, t, "chain terms");
          const int32_t eo = pass ? u.uo : u.lo, ew = pass ? u.uw : u.lw;
          const std::vector<int32_t> &ec = pass ? H.su_col : H.sl_col;
          for (int32_t q = 0; q < ew; ++q) {
            const int32_t col = ec[size_t(eo) + size_t(q) * kWarp + size_t(l)];
            ck(col == kPadCol || (col >= 0 && col < n && (pass ? col > i : col < i) &&
                                  (col < H.block_ptr[size_t(b)] || col >= H.block_ptr[size_t(b) + 1])),
               t, "unit entry to another color");
          }
        }
      }
    }
  }
  // every color tiles, groups or units, covering its rows
  for (int c = 0; c < n_c; ++c) {
    const bool tile = H.color_tile[size_t(c) + 1] > H.color_tile[size_t(c)];
    const bool grp = H.color_group[size_t(c) + 1] > H.color_group[size_t(c)];
    const bool unit = H.color_unit[size_t(c) + 1] > H.color_unit[size_t(c)];
    ck(int(tile) + int(grp) + int(unit) == 1, c, "color layout");
  }
  report[0] = int64_t(H.tiles.size() + H.units.size());
  report[1] = int64_t(H.groups.size());
  report[2] = ck.failed;
  report[3] = ck.first;
  if (what) *what = ck.what;
  return ck.failed ? ICCG_ERR_STATE : ICCG_OK;
}
