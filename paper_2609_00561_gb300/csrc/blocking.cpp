// Production host-side blocking: adjacency graph, ABMC, greedy block
// coloring with the block-multicolor ordering, and Leiden (modularity / CPM).
//
// The results are integer labellings and must be reproducible bit for bit,
// so every order-dependent choice is fixed:
//   * ABMC (Sec. 3): FIFO candidate set, neighbours in ascending index, a new
//     seed / an empty candidate set takes the smallest unassigned node.
//   * greedy coloring (Sec. 3, Sec. 5.1): blocks in index order, smallest
//     color unused by already-colored neighbour blocks.
//   * ordering: colors ascending, blocks ascending, rows ascending.
//   * Leiden (Sec. 4; Traag, Waltman & van Eck 2019), with the quality
//     H = sum_c (e_c - gp W_c^2 / 2) (H/m is Eq. 1 with gp = gamma/2m and
//     node weight = degree, or Eq. 2 with gp = gamma and weight 1):
//       - local moving: random visiting queue, best gain, strictly better
//         than staying, ties to the lowest community id, the smallest empty
//         community as the "new community" candidate;
//       - refinement: well-connected nodes of each community in random order,
//         merged into a well-connected sub-community drawn with probability
//         proportional to exp(gain / beta) (one uniform draw per visit);
//       - aggregation on the refined partition (on the unrefined one when the
//         refinement merged nothing), communities renumbered by first
//         appearance; n_iter full passes.
//     Random numbers: Philox4x64-10 (Salmon et al. 2011), key (seed, 0),
//     counter incremented before each block, uniform integers by rejection
//     of draws below 2^64 mod k, unit doubles from the top 53 bits.
// Compiled with -ffp-contract=off: every gain is the plain IEEE evaluation of
// k - gp * w * W, left to right.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <set>
#include <vector>

#include "../../include/iccg.h"

namespace {

// ---------------------------------------------------------------------------
class Philox {
 public:
  explicit Philox(uint64_t seed) : key_{seed, 0}, ctr_{0, 0, 0, 0} {}
  uint64_t next() {
    if (pos_ == 4) refill();
    return out_[pos_++];
  }
  double unit() { return double(next() >> 11) * (1.0 / 9007199254740992.0); }
  uint64_t below(uint64_t k) {
    const uint64_t reject = (0 - k) % k;
    for (;;) {
      const uint64_t x = next();
      if (x >= reject) return x % k;
    }
  }
  template <typename T>
  void shuffle(std::vector<T> &a) {
    for (size_t i = a.size(); i-- > 1;) std::swap(a[i], a[below(uint64_t(i + 1))]);
  }

 private:
  void refill() {
    for (auto &c : ctr_)
      if (++c != 0) break;
    uint64_t x0 = ctr_[0], x1 = ctr_[1], x2 = ctr_[2], x3 = ctr_[3];
    uint64_t k0 = key_[0], k1 = key_[1];
    for (int rnd = 0; rnd < 10; ++rnd) {
      const unsigned __int128 m0 = (unsigned __int128)0xD2E7470EE14C6C93ULL * x0;
      const unsigned __int128 m1 = (unsigned __int128)0xCA5A826395121157ULL * x2;
      const uint64_t y0 = uint64_t(m1 >> 64) ^ x1 ^ k0;
      const uint64_t y2 = uint64_t(m0 >> 64) ^ x3 ^ k1;
      x1 = uint64_t(m1);
      x3 = uint64_t(m0);
      x0 = y0;
      x2 = y2;
      k0 += 0x9E3779B97F4A7C15ULL;
      k1 += 0xBB67AE8584CAA73BULL;
    }
    out_[0] = x0; out_[1] = x1; out_[2] = x2; out_[3] = x3;
    pos_ = 0;
  }
  uint64_t key_[2];
  uint64_t ctr_[4];
  uint64_t out_[4] = {0, 0, 0, 0};
  int pos_ = 4;
};

// Relabel by first appearance; returns the number of labels.
int32_t first_appearance(std::vector<int32_t> &lab) {
  int32_t hi = 0;
  for (int32_t v : lab) hi = std::max(hi, v + 1);
  std::vector<int32_t> map(static_cast<size_t>(hi), -1);
  int32_t k = 0;
  for (int32_t &v : lab) {
    if (map[v] < 0) map[v] = k++;
    v = map[v];
  }
  return k;
}

// Weighted undirected graph without self-loops (CSR, neighbours ascending).
struct Graph {
  int32_t n = 0;
  std::vector<int64_t> off;
  std::vector<int32_t> nbr;
  std::vector<double> ew;   // edge weights
  std::vector<double> vw;   // node weights
};

// ---------------------------------------------------------------------------
class Leiden {
 public:
  Leiden(double gp, double beta, Philox &rng) : gp_(gp), beta_(beta), rng_(rng) {}

  // one full multilevel pass starting from `memb` (labels on g0's nodes)
  void pass(const Graph &g0, std::vector<int32_t> &memb) {
    const int32_t n0 = g0.n;
    std::vector<int32_t> where(n0);
    std::iota(where.begin(), where.end(), 0);
    Graph level;               // aggregate graphs (level 0 uses g0 directly)
    const Graph *g = &g0;
    std::vector<int32_t> part = memb;
    first_appearance(part);
    for (;;) {
      move_nodes(*g, part);
      std::vector<int32_t> probe = part;
      if (first_appearance(probe) == g->n) break;
      std::vector<int32_t> sub = refine(*g, part);
      int32_t m = first_appearance(sub);
      std::vector<int32_t> next_part;
      if (m == g->n) {
        sub = part;
        m = first_appearance(sub);
        next_part.resize(size_t(m));
        std::iota(next_part.begin(), next_part.end(), 0);
      } else {
        next_part.assign(size_t(m), 0);
        for (int32_t v = 0; v < g->n; ++v) next_part[sub[v]] = part[v];
        first_appearance(next_part);
      }
      Graph agg = aggregate(*g, sub, m);
      for (int32_t &w : where) w = sub[w];
      level = std::move(agg);
      g = &level;
      part = std::move(next_part);
    }
    for (int32_t v = 0; v < n0; ++v) memb[v] = part[where[v]];
    first_appearance(memb);
  }

 private:
  double gain(double k, double w, double W) const { return k - gp_ * w * W; }

  void move_nodes(const Graph &g, std::vector<int32_t> &part) {
    const int32_t n = g.n;
    std::vector<double> W(n, 0.0);
    std::vector<int64_t> members(n, 0);
    for (int32_t v = 0; v < n; ++v) {
      W[part[v]] += g.vw[v];
      members[part[v]]++;
    }
    std::set<int32_t> empties;
    for (int32_t c = 0; c < n; ++c)
      if (members[c] == 0) empties.insert(c);
    std::vector<int32_t> order(n);
    std::iota(order.begin(), order.end(), 0);
    rng_.shuffle(order);
    std::vector<int32_t> ring(order);   // circular FIFO, capacity n
    std::vector<char> queued(n, 1);
    size_t head = 0, count = size_t(n);
    std::vector<double> link(n, 0.0);
    std::vector<char> seen(n, 0);
    std::vector<int32_t> touched, cand;
    while (count > 0) {
      const int32_t v = ring[head];
      head = (head + 1) % size_t(n);
      --count;
      queued[v] = 0;
      const int32_t cur = part[v];
      const double wv = g.vw[v];
      touched.clear();
      for (int64_t e = g.off[v]; e < g.off[v + 1]; ++e) {
        const int32_t c = part[g.nbr[e]];
        if (!seen[c]) { seen[c] = 1; touched.push_back(c); }
        link[c] += g.ew[e];
      }
      double best_gain = gain(link[cur], wv, W[cur] - wv);
      int32_t best = cur;
      cand.clear();
      for (int32_t c : touched)
        if (c != cur) cand.push_back(c);
      int32_t fresh = -1;
      if (members[cur] > 1 && !empties.empty()) {
        fresh = *empties.begin();
        cand.push_back(fresh);
      }
      std::sort(cand.begin(), cand.end());
      for (int32_t c : cand) {
        const double gc = (c == fresh) ? 0.0 : gain(link[c], wv, W[c]);
        if (gc > best_gain) { best_gain = gc; best = c; }
      }
      for (int32_t c : touched) { link[c] = 0.0; seen[c] = 0; }
      if (best == cur) continue;
      W[cur] -= wv;
      members[cur]--;
      if (best == fresh) empties.erase(fresh);
      if (members[cur] == 0) empties.insert(cur);
      W[best] += wv;
      members[best]++;
      part[v] = best;
      for (int64_t e = g.off[v]; e < g.off[v + 1]; ++e) {
        const int32_t u = g.nbr[e];
        if (part[u] != best && !queued[u]) {
          queued[u] = 1;
          ring[(head + count) % size_t(n)] = u;
          ++count;
        }
      }
    }
  }

  std::vector<int32_t> refine(const Graph &g, const std::vector<int32_t> &part) {
    const int32_t n = g.n;
    std::vector<int32_t> sub(n);
    std::iota(sub.begin(), sub.end(), 0);
    std::vector<double> subW(g.vw), subE(n, 0.0);
    std::vector<int64_t> subN(n, 1);
    // members of every community, ascending
    std::vector<std::vector<int32_t>> comm(n);
    for (int32_t v = 0; v < n; ++v) comm[part[v]].push_back(v);
    std::vector<double> link(n, 0.0);
    std::vector<char> seen(n, 0);
    std::vector<int32_t> touched, cand;
    std::vector<double> wts;
    for (int32_t c = 0; c < n; ++c) {
      const std::vector<int32_t> &S = comm[c];
      if (S.empty()) continue;
      double WS = 0.0;
      for (int32_t v : S) WS += g.vw[v];
      std::vector<int32_t> pool;
      for (int32_t v : S) {
        double inside = 0.0;
        for (int64_t e = g.off[v]; e < g.off[v + 1]; ++e)
          if (part[g.nbr[e]] == c) inside += g.ew[e];
        subE[v] = inside;
        if (inside >= gp_ * g.vw[v] * (WS - g.vw[v])) pool.push_back(v);
      }
      rng_.shuffle(pool);
      for (int32_t v : pool) {
        if (subN[sub[v]] != 1) continue;
        const double u01 = rng_.unit();
        const int32_t own = sub[v];
        const double wv = g.vw[v];
        touched.clear();
        for (int64_t e = g.off[v]; e < g.off[v + 1]; ++e) {
          const int32_t u = g.nbr[e];
          if (part[u] != c) continue;
          const int32_t t = sub[u];
          if (!seen[t]) { seen[t] = 1; touched.push_back(t); }
          link[t] += g.ew[e];
        }
        cand.clear();
        for (int32_t t : touched) {
          if (t == own) continue;
          if (!(subE[t] >= gp_ * subW[t] * (WS - subW[t]))) continue;
          if (gain(link[t], wv, subW[t]) >= 0.0) cand.push_back(t);
        }
        cand.push_back(own);
        std::sort(cand.begin(), cand.end());
        wts.assign(cand.size(), 0.0);
        double top = 0.0;
        for (size_t j = 0; j < cand.size(); ++j) {
          wts[j] = (cand[j] == own) ? 0.0 : gain(link[cand[j]], wv, subW[cand[j]]);
          top = std::max(top, wts[j]);
        }
        double total = 0.0;
        for (double &x : wts) {
          x = std::exp((x - top) / beta_);
          total += x;
        }
        const double target = u01 * total;
        double run = 0.0;
        int32_t pick = cand.back();
        for (size_t j = 0; j < cand.size(); ++j) {
          run += wts[j];
          if (target < run) { pick = cand[j]; break; }
        }
        const double kpick = (pick == own) ? 0.0 : link[pick];
        for (int32_t t : touched) { link[t] = 0.0; seen[t] = 0; }
        if (pick == own) continue;
        subE[pick] = subE[pick] + subE[own] - 2.0 * kpick;
        subW[pick] += wv;
        subN[pick] += 1;
        subN[own] = 0;
        sub[v] = pick;
      }
    }
    return sub;
  }

  static Graph aggregate(const Graph &g, const std::vector<int32_t> &grp, int32_t m) {
    Graph a;
    a.n = m;
    a.vw.assign(size_t(m), 0.0);
    a.off.assign(size_t(m) + 1, 0);
    std::vector<std::vector<int32_t>> mem(static_cast<size_t>(m));
    for (int32_t v = 0; v < g.n; ++v) mem[grp[v]].push_back(v);
    std::vector<double> acc(static_cast<size_t>(m), 0.0);
    std::vector<char> seen(static_cast<size_t>(m), 0);
    std::vector<int32_t> lst;
    for (int32_t x = 0; x < m; ++x) {
      lst.clear();
      for (int32_t v : mem[x]) {
        a.vw[x] += g.vw[v];
        for (int64_t e = g.off[v]; e < g.off[v + 1]; ++e) {
          const int32_t y = grp[g.nbr[e]];
          if (y == x) continue;
          if (!seen[y]) { seen[y] = 1; lst.push_back(y); }
          acc[y] += g.ew[e];
        }
      }
      std::sort(lst.begin(), lst.end());
      for (int32_t y : lst) {
        a.nbr.push_back(y);
        a.ew.push_back(acc[y]);
        acc[y] = 0.0;
        seen[y] = 0;
      }
      a.off[x + 1] = int64_t(a.nbr.size());
    }
    return a;
  }

  double gp_, beta_;
  Philox &rng_;
};

}  // namespace

extern "C" {

iccg_status iccg_graph(int32_t n, const int64_t *rowptr, const int32_t *colind, int64_t *gptr, int32_t *gadj,
                       int64_t *m) {
  if (n < 0 || !rowptr || !gptr || (n > 0 && !colind)) return ICCG_ERR_ARG;
  std::vector<std::vector<int32_t>> adj(static_cast<size_t>(n));
  for (int32_t i = 0; i < n; ++i)
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      const int32_t j = colind[e];
      if (j < 0 || j >= n) return ICCG_ERR_ARG;
      if (j == i) continue;
      adj[i].push_back(j);
      adj[j].push_back(i);
    }
  gptr[0] = 0;
  int64_t k = 0;
  for (int32_t i = 0; i < n; ++i) {
    std::vector<int32_t> &a = adj[i];
    std::sort(a.begin(), a.end());
    a.erase(std::unique(a.begin(), a.end()), a.end());
    if (gadj) std::copy(a.begin(), a.end(), gadj + k);
    k += int64_t(a.size());
    gptr[i + 1] = k;
  }
  if (m) *m = k;
  return ICCG_OK;
}

iccg_status iccg_block_abmc(int32_t n, const int64_t *gptr, const int32_t *gadj, int32_t s, int32_t *block_of,
                            int32_t *n_b) {
  if (n < 0 || s < 1 || !gptr || !block_of || !n_b) return ICCG_ERR_ARG;
  std::fill(block_of, block_of + n, -1);
  std::vector<int32_t> stamp(static_cast<size_t>(n), -1), fifo;
  fifo.reserve(size_t(n));
  int32_t blocks = 0, lowest = 0, done = 0;
  while (done < n) {
    fifo.clear();
    size_t head = 0;
    for (int32_t filled = 0; filled < s && done < n; ++filled) {
      int32_t v = -1;
      while (head < fifo.size() && v < 0) {
        const int32_t c = fifo[head++];
        if (block_of[c] < 0) v = c;
      }
      if (v < 0) {
        while (block_of[lowest] >= 0) ++lowest;
        v = lowest;
      }
      block_of[v] = blocks;
      ++done;
      for (int64_t e = gptr[v]; e < gptr[v + 1]; ++e) {
        const int32_t u = gadj[e];
        if (block_of[u] < 0 && stamp[u] != blocks) {
          stamp[u] = blocks;
          fifo.push_back(u);
        }
      }
    }
    ++blocks;
  }
  *n_b = blocks;
  return ICCG_OK;
}

iccg_status iccg_block_leiden(int32_t n, const int64_t *gptr, const int32_t *gadj, int32_t quality, double gamma,
                              int32_t n_iter, double beta, uint64_t seed, int32_t *block_of, int32_t *n_b) {
  if (n < 0 || !gptr || !block_of || !n_b || (quality != 0 && quality != 1) || n_iter < 0 || !(beta > 0.0))
    return ICCG_ERR_ARG;
  if (n == 0) { *n_b = 0; return ICCG_OK; }
  Graph g;
  g.n = n;
  g.off.assign(gptr, gptr + n + 1);
  g.nbr.assign(gadj, gadj + gptr[n]);
  g.ew.assign(size_t(gptr[n]), 1.0);
  g.vw.resize(size_t(n));
  double gp;
  if (quality == 0) {
    for (int32_t v = 0; v < n; ++v) g.vw[v] = double(gptr[v + 1] - gptr[v]);
    gp = gptr[n] > 0 ? gamma / double(gptr[n]) : 0.0;
  } else {
    std::fill(g.vw.begin(), g.vw.end(), 1.0);
    gp = gamma;
  }
  Philox rng(seed);
  Leiden alg(gp, beta, rng);
  std::vector<int32_t> memb(static_cast<size_t>(n));
  std::iota(memb.begin(), memb.end(), 0);
  for (int32_t it = 0; it < n_iter; ++it) alg.pass(g, memb);
  *n_b = first_appearance(memb);
  std::copy(memb.begin(), memb.end(), block_of);
  return ICCG_OK;
}

iccg_status iccg_sort_blocks_desc(int32_t n, int32_t n_b, int32_t *block_of) {
  if (n < 0 || n_b < 0 || !block_of) return ICCG_ERR_ARG;
  std::vector<int32_t> size(static_cast<size_t>(n_b), 0), first(static_cast<size_t>(n_b), n);
  for (int32_t i = 0; i < n; ++i) {
    const int32_t b = block_of[i];
    if (b < 0 || b >= n_b) return ICCG_ERR_ARG;
    size[b]++;
    first[b] = std::min(first[b], i);
  }
  std::vector<int32_t> order(static_cast<size_t>(n_b));
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
    if (size[a] != size[b]) return size[a] > size[b];
    return first[a] < first[b];
  });
  std::vector<int32_t> rank(static_cast<size_t>(n_b));
  for (int32_t k = 0; k < n_b; ++k) rank[order[k]] = k;
  for (int32_t i = 0; i < n; ++i) block_of[i] = rank[block_of[i]];
  return ICCG_OK;
}

iccg_status iccg_color_order(int32_t n, const int64_t *gptr, const int32_t *gadj, int32_t n_b,
                             const int32_t *block_of, int32_t *color_of, int32_t *n_c, int32_t *perm,
                             int32_t *block_ptr, int32_t *color_ptr) {
  if (n < 0 || n_b < 0 || !gptr || !block_of || !color_of || !n_c || !perm || !block_ptr || !color_ptr)
    return ICCG_ERR_ARG;
  // rows of every block, ascending
  std::vector<std::vector<int32_t>> rows(static_cast<size_t>(n_b));
  for (int32_t i = 0; i < n; ++i) {
    if (block_of[i] < 0 || block_of[i] >= n_b) return ICCG_ERR_ARG;
    rows[block_of[i]].push_back(i);
  }
  std::vector<int32_t> used(size_t(n_b) + 1, -1);
  int32_t ncol = 0;
  for (int32_t b = 0; b < n_b; ++b) color_of[b] = -1;
  for (int32_t b = 0; b < n_b; ++b) {
    for (int32_t v : rows[b])
      for (int64_t e = gptr[v]; e < gptr[v + 1]; ++e) {
        const int32_t nb = block_of[gadj[e]];
        if (nb != b && color_of[nb] >= 0) used[color_of[nb]] = b;
      }
    int32_t c = 0;
    while (used[c] == b) ++c;
    color_of[b] = c;
    ncol = std::max(ncol, c + 1);
  }
  *n_c = ncol;
  // colors ascending, blocks ascending, rows ascending
  std::vector<std::vector<int32_t>> by_color(static_cast<size_t>(ncol));
  for (int32_t b = 0; b < n_b; ++b) by_color[color_of[b]].push_back(b);
  int32_t nb_new = 0, row = 0;
  for (int32_t c = 0; c < ncol; ++c) {
    color_ptr[c] = nb_new;
    for (int32_t b : by_color[c]) {
      block_ptr[nb_new++] = row;
      for (int32_t v : rows[b]) perm[row++] = v;
    }
  }
  color_ptr[ncol] = nb_new;
  block_ptr[nb_new] = row;
  return ICCG_OK;
}

// Level-set ordering (the level scheduling of Sec. 2): the level of row i is
// 0 when no neighbour precedes it in the natural order, else one more than
// the deepest preceding neighbour.  Rows of one level are never adjacent, so
// the levels are colors of one-row blocks; ordering rows by level (ascending
// index within a level) keeps the relative order of every adjacent pair, so
// IC(0) and its substitutions are those of the natural order.
iccg_status iccg_level_order(int32_t n, const int64_t *gptr, const int32_t *gadj, int32_t *level_of, int32_t *n_lev,
                             int32_t *perm, int32_t *block_ptr, int32_t *color_ptr) {
  if (n < 0 || !gptr || !level_of || !n_lev || !perm || !block_ptr || !color_ptr) return ICCG_ERR_ARG;
  int32_t nl = 0;
  for (int32_t i = 0; i < n; ++i) {
    int32_t lv = 0;
    for (int64_t e = gptr[i]; e < gptr[i + 1]; ++e) {
      const int32_t j = gadj[e];
      if (j < 0 || j >= n) return ICCG_ERR_ARG;
      if (j < i) lv = std::max(lv, level_of[j] + 1);
    }
    level_of[i] = lv;
    nl = std::max(nl, lv + 1);
  }
  *n_lev = nl;
  std::vector<int32_t> cnt(size_t(nl) + 1, 0);
  for (int32_t i = 0; i < n; ++i) cnt[size_t(level_of[i]) + 1]++;
  for (int32_t v = 0; v < nl; ++v) cnt[size_t(v) + 1] += cnt[size_t(v)];
  for (int32_t v = 0; v <= nl; ++v) color_ptr[v] = cnt[size_t(v)];
  for (int32_t i = 0; i < n; ++i) perm[cnt[size_t(level_of[i])]++] = i;
  for (int32_t k = 0; k <= n; ++k) block_ptr[k] = k;
  return ICCG_OK;
}

// Intra-block level sets for oversized blocks: every block of more than
// max_rows rows is split into its in-block dependency levels (level 0: rows
// with no earlier row of the block in the pattern; a row one deeper than its
// deepest earlier in-block neighbour), each level of each color becoming a
// color of one-row blocks.  Rows of one level of one color are never
// adjacent (blocks of a color share no edge; in a block, adjacent rows sit at
// different levels), and ordering a block's rows by level keeps the relative
// order of every adjacent pair, so IC(0) and the substitutions are those of
// the input ordering.  Blocks of at most max_rows rows are kept; every color
// of the input keeps its position.  Outputs sized n, n+1, n+1.
iccg_status iccg_split_levels(int32_t n, const int64_t *rowptr, const int32_t *colind, const int32_t *perm,
                              const int32_t *block_ptr, const int32_t *color_ptr, int32_t n_b, int32_t n_c,
                              int32_t max_rows, int32_t *perm_out, int32_t *block_ptr_out,
                              int32_t *color_ptr_out, int32_t *n_b_out, int32_t *n_c_out) {
  if (n < 0 || n_b < 0 || n_c < 0 || max_rows < 1 || !rowptr || !perm || !block_ptr || !color_ptr || !perm_out ||
      !block_ptr_out || !color_ptr_out || !n_b_out || !n_c_out)
    return ICCG_ERR_ARG;
  std::vector<int32_t> iperm(size_t(n), -1), blk(size_t(n), 0);
  for (int32_t i = 0; i < n; ++i) {
    if (perm[i] < 0 || perm[i] >= n || iperm[size_t(perm[i])] >= 0) return ICCG_ERR_ARG;
    iperm[size_t(perm[i])] = i;
  }
  for (int32_t b = 0; b < n_b; ++b)
    for (int32_t i = block_ptr[b]; i < block_ptr[b + 1]; ++i) blk[size_t(i)] = b;
  // in-block level of every (new) row of an oversized block
  std::vector<int32_t> lev(size_t(n), 0);
  for (int32_t b = 0; b < n_b; ++b) {
    if (block_ptr[b + 1] - block_ptr[b] <= max_rows) continue;
    for (int32_t i = block_ptr[b]; i < block_ptr[b + 1]; ++i) {
      const int32_t o = perm[i];
      int32_t lv = 0;
      for (int64_t e = rowptr[o]; e < rowptr[o + 1]; ++e) {
        const int32_t c = colind[e];
        if (c < 0 || c >= n) return ICCG_ERR_ARG;
        const int32_t j = iperm[size_t(c)];
        if (j < i && blk[size_t(j)] == b) lv = std::max(lv, lev[size_t(j)] + 1);
      }
      lev[size_t(i)] = lv;
    }
  }
  int32_t nb = 0, nc = 0, row = 0;
  for (int32_t c = 0; c < n_c; ++c) {
    // the color's small blocks stay one color; its oversized blocks give one
    // color per level
    color_ptr_out[nc++] = nb;
    int32_t depth = 0;
    bool small = false;
    for (int32_t b = color_ptr[c]; b < color_ptr[c + 1]; ++b) {
      if (block_ptr[b + 1] - block_ptr[b] <= max_rows) {
        small = true;
        block_ptr_out[nb++] = row;
        for (int32_t i = block_ptr[b]; i < block_ptr[b + 1]; ++i) perm_out[row++] = perm[i];
      } else {
        for (int32_t i = block_ptr[b]; i < block_ptr[b + 1]; ++i) depth = std::max(depth, lev[size_t(i)] + 1);
      }
    }
    if (!small) --nc;
    for (int32_t v = 0; v < depth; ++v) {
      color_ptr_out[nc++] = nb;
      for (int32_t b = color_ptr[c]; b < color_ptr[c + 1]; ++b) {
        if (block_ptr[b + 1] - block_ptr[b] <= max_rows) continue;
        for (int32_t i = block_ptr[b]; i < block_ptr[b + 1]; ++i)
          if (lev[size_t(i)] == v) {
            block_ptr_out[nb++] = row;
            perm_out[row++] = perm[i];
          }
      }
    }
  }
  color_ptr_out[nc] = nb;
  block_ptr_out[nb] = row;
  *n_b_out = nb;
  *n_c_out = nc;
  return ICCG_OK;
}

}  // extern "C"
