/*
 * Parallel Leiden, restated sequentially -- TEST INFRASTRUCTURE ONLY.
 *
 * The GPU library runs Leiden (Sec. 4; Traag, Waltman & van Eck 2019) in a
 * parallel form whose every decision is taken from the state at the start of
 * a synchronous sub-round.  This file states the same procedure as plain
 * sequential loops over the nodes, so the two must give the same partition
 * integer for integer:
 *
 *   quality H = sum_c (e_c - gp W_c^2 / 2); the gain of placing node v
 *   (weight w) in community c is k_vc - gp w W_c (W_c without v); CPM: node
 *   weight 1, gp = gamma; modularity: node weight = degree, gp = gamma / m
 *   (m = adjacency entries, twice the edges);
 *
 *   local moving, sub-round r (at most 128; until two sub-rounds move
 *   nothing): every node v of community C takes the neighbouring community
 *   of largest gain, strictly better than staying, ties to the smallest
 *   label, only labels below C in even sub-rounds and above C in odd ones;
 *   a node of a community with other members may instead open its own label
 *   v when no node holds it and staying has a negative gain.  A move to an
 *   existing community is a proposal; a community accepts the proposal of
 *   largest key (gain over staying as a float in the high 32 bits, 2^32 - 1 -
 *   v in the low ones) and a node moves only when its proposal is the
 *   accepted one and no proposal targets its own community;
 *
 *   refinement, inside each community: singleton sub-communities of
 *   well-connected nodes (edges into the rest of the community >= gp w (W_C
 *   - w)) join the well-connected sub-community T (E(T, C - T) >= gp W_T
 *   (W_C - W_T)) of largest gain >= 0, ties to the smallest label, with the
 *   same direction rule and one accepted proposal per sub-community (key:
 *   gain + 1), no move out of a sub-community that receives one;
 *
 *   aggregation on the refined partition (the unrefined one when nothing was
 *   merged), the aggregate starting from the unrefined communities; labels
 *   are renumbered by ascending old label after every stage; until local
 *   moving leaves every node alone; n_iter passes, the second from the
 *   first's result; then every community is split into its connected
 *   components, numbered by their smallest node.
 *
 * Every floating-point expression is evaluated as written, one rounding per
 * operation (the file is compiled with -ffp-contract=off).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int32_t n;
  int64_t m;
  int64_t *ptr;
  int32_t *adj;
  int64_t *ew;
  int64_t *vw;
} PGraph;

#define PL_SUBROUNDS 128
#define PL_LEVELS 64

static double pl_penalty(double gp, int64_t w, int64_t W) {
  const double a = gp * (double)w;
  return a * (double)W;
}

static double pl_gain(int64_t k, int64_t w, int64_t W, double gp) { return (double)k - pl_penalty(gp, w, W); }

static uint64_t pl_key(double delta, int32_t v) {
  float f = (float)delta;
  f = fmaxf(f, 1e-30f);
  uint32_t bits;
  memcpy(&bits, &f, sizeof(bits));
  return ((uint64_t)bits << 32) | (uint64_t)(0xffffffffu - (uint32_t)v);
}

static void pl_weights(const PGraph *g, const int32_t *comm, int64_t *W, int32_t *cnt) {
  memset(W, 0, sizeof(int64_t) * (size_t)g->n);
  memset(cnt, 0, sizeof(int32_t) * (size_t)g->n);
  for (int32_t v = 0; v < g->n; ++v) {
    W[comm[v]] += g->vw[v];
    cnt[comm[v]] += 1;
  }
}

/* labels with cnt > 0 renumbered 0.. in ascending order; returns how many */
static int32_t pl_compact(int32_t n, int32_t *a, const int32_t *cnt) {
  int32_t *id = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int32_t k = 0;
  for (int32_t c = 0; c < n; ++c) id[c] = cnt[c] > 0 ? k++ : -1;
  for (int32_t i = 0; i < n; ++i) a[i] = id[a[i]];
  free(id);
  return k;
}

static void pl_move_nodes(const PGraph *g, int32_t *comm, int64_t *W, int32_t *cnt, double gp) {
  const int32_t n = g->n;
  int32_t *newc = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int32_t *out = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  uint64_t *join = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
  int idle = 0;
  for (int r = 0; r < PL_SUBROUNDS && idle < 2; ++r) {
    const int dir = r & 1;
    pl_weights(g, comm, W, cnt);
    memset(join, 0, sizeof(uint64_t) * (size_t)n);
    for (int32_t v = 0; v < n; ++v) {
      const int32_t C = comm[v];
      const int64_t wv = g->vw[v], e0 = g->ptr[v], e1 = g->ptr[v + 1];
      int64_t kC = 0;
      for (int64_t e = e0; e < e1; ++e)
        if (comm[g->adj[e]] == C) kC += g->ew[e];
      int32_t best = C;
      double bestg = pl_gain(kC, wv, W[C] - wv, gp);
      for (int64_t e = e0; e < e1; ++e) {
        const int32_t c = comm[g->adj[e]];
        if (c == C || (dir == 0 ? c > C : c < C)) continue;
        int dup = 0;
        for (int64_t f = e0; f < e && !dup; ++f) dup = comm[g->adj[f]] == c;
        if (dup) continue;
        int64_t kc = 0;
        for (int64_t f = e; f < e1; ++f)
          if (comm[g->adj[f]] == c) kc += g->ew[f];
        const double gc = pl_gain(kc, wv, W[c], gp);
        if (gc > bestg || (gc == bestg && best != C && c < best)) {
          best = c;
          bestg = gc;
        }
      }
      const double stay = pl_gain(kC, wv, W[C] - wv, gp);
      if (cnt[C] > 1 && cnt[v] == 0 && 0.0 > bestg) {
        best = v;
        bestg = 0.0;
      }
      newc[v] = best;
      if (best != C && best != v) {
        const uint64_t key = pl_key(bestg - stay, v);
        if (key > join[best]) join[best] = key;
      }
    }
    int32_t moved = 0;
    for (int32_t v = 0; v < n; ++v) {
      const int32_t C = comm[v], D = newc[v];
      int32_t r2 = C;
      if (D != C) {
        if (D == v && cnt[v] == 0) r2 = D;
        else if (join[C] == 0 && (join[D] & 0xffffffffull) == 0xffffffffull - (uint32_t)v) r2 = D;
      }
      out[v] = r2;
      if (r2 != C) ++moved;
    }
    memcpy(comm, out, sizeof(int32_t) * (size_t)n);
    idle = moved == 0 ? idle + 1 : 0;
  }
  pl_weights(g, comm, W, cnt);
  free(newc);
  free(out);
  free(join);
}

static void pl_refine(const PGraph *g, const int32_t *comm, const int64_t *W, int32_t *sub, double gp) {
  const int32_t n = g->n;
  int64_t *SW = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  int32_t *subN = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int64_t *subE = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  int32_t *newsub = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int32_t *out = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  uint64_t *join = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
  for (int32_t v = 0; v < n; ++v) sub[v] = v;
  int idle = 0;
  for (int r = 0; r < PL_SUBROUNDS && idle < 2; ++r) {
    const int dir = r & 1;
    pl_weights(g, sub, SW, subN);
    memset(subE, 0, sizeof(int64_t) * (size_t)n);
    for (int32_t v = 0; v < n; ++v)
      for (int64_t e = g->ptr[v]; e < g->ptr[v + 1]; ++e) {
        const int32_t u = g->adj[e];
        if (comm[u] == comm[v] && sub[u] != sub[v]) subE[sub[v]] += g->ew[e];
      }
    memset(join, 0, sizeof(uint64_t) * (size_t)n);
    for (int32_t v = 0; v < n; ++v) {
      const int32_t C = comm[v];
      newsub[v] = sub[v];
      if (sub[v] != v || subN[v] != 1) continue;
      const int64_t wv = g->vw[v], e0 = g->ptr[v], e1 = g->ptr[v + 1], WC = W[C];
      int64_t inside = 0;
      for (int64_t e = e0; e < e1; ++e)
        if (comm[g->adj[e]] == C) inside += g->ew[e];
      if (!((double)inside >= pl_penalty(gp, wv, WC - wv))) continue;
      int32_t best = v;
      double bestg = 0.0;
      int found = 0;
      for (int64_t e = e0; e < e1; ++e) {
        const int32_t u = g->adj[e];
        if (comm[u] != C) continue;
        const int32_t t = sub[u];
        if (t == v || (dir == 0 ? t > v : t < v)) continue;
        int dup = 0;
        for (int64_t f = e0; f < e && !dup; ++f) dup = comm[g->adj[f]] == C && sub[g->adj[f]] == t;
        if (dup) continue;
        if (!((double)subE[t] >= pl_penalty(gp, SW[t], WC - SW[t]))) continue;
        int64_t kt = 0;
        for (int64_t f = e; f < e1; ++f)
          if (comm[g->adj[f]] == C && sub[g->adj[f]] == t) kt += g->ew[f];
        const double gt = pl_gain(kt, wv, SW[t], gp);
        if (gt >= 0.0 && (!found || gt > bestg || (gt == bestg && t < best))) {
          best = t;
          bestg = gt;
          found = 1;
        }
      }
      if (found) {
        newsub[v] = best;
        const uint64_t key = pl_key(bestg + 1.0, v);
        if (key > join[best]) join[best] = key;
      }
    }
    int32_t moved = 0;
    for (int32_t v = 0; v < n; ++v) {
      const int32_t s0 = sub[v], t = newsub[v];
      int32_t r2 = s0;
      if (t != s0 && join[v] == 0 && (join[t] & 0xffffffffull) == 0xffffffffull - (uint32_t)v) r2 = t;
      out[v] = r2;
      if (r2 != s0) ++moved;
    }
    memcpy(sub, out, sizeof(int32_t) * (size_t)n);
    idle = moved == 0 ? idle + 1 : 0;
  }
  free(SW);
  free(subN);
  free(subE);
  free(newsub);
  free(out);
  free(join);
}

/* the aggregate of g by grp (labels 0..K-1): node weights summed, edges
 * between different groups summed (ascending neighbour), the aggregate's
 * starting communities comm2[grp[v]] = comm[v] */
static PGraph pl_aggregate(const PGraph *g, const int32_t *grp, int32_t K, const int32_t *comm, int32_t *comm2) {
  PGraph a;
  a.n = K;
  a.vw = (int64_t *)calloc((size_t)(K > 0 ? K : 1), sizeof(int64_t));
  a.ptr = (int64_t *)calloc((size_t)K + 1, sizeof(int64_t));
  for (int32_t v = 0; v < g->n; ++v) {
    a.vw[grp[v]] += g->vw[v];
    comm2[grp[v]] = comm[v];
  }
  /* members of every group */
  int64_t *mp = (int64_t *)calloc((size_t)K + 1, sizeof(int64_t));
  int32_t *mem = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->n > 0 ? g->n : 1));
  for (int32_t v = 0; v < g->n; ++v) mp[grp[v] + 1]++;
  for (int32_t x = 0; x < K; ++x) mp[x + 1] += mp[x];
  int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(K > 0 ? K : 1));
  for (int32_t x = 0; x < K; ++x) fill[x] = mp[x];
  for (int32_t v = 0; v < g->n; ++v) mem[fill[grp[v]]++] = v;
  int64_t *acc = (int64_t *)calloc((size_t)(K > 0 ? K : 1), sizeof(int64_t));
  char *seen = (char *)calloc((size_t)(K > 0 ? K : 1), 1);
  int32_t *lst = (int32_t *)malloc(sizeof(int32_t) * (size_t)(K > 0 ? K : 1));
  int64_t cap = g->m > 0 ? g->m : 1, na = 0;
  a.adj = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
  a.ew = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
  for (int32_t x = 0; x < K; ++x) {
    int32_t nl = 0;
    for (int64_t q = mp[x]; q < mp[x + 1]; ++q) {
      const int32_t v = mem[q];
      for (int64_t e = g->ptr[v]; e < g->ptr[v + 1]; ++e) {
        const int32_t y = grp[g->adj[e]];
        if (y == x) continue;
        if (!seen[y]) {
          seen[y] = 1;
          lst[nl++] = y;
        }
        acc[y] += g->ew[e];
      }
    }
    /* ascending neighbour (insertion sort: the lists are short) */
    for (int32_t i = 1; i < nl; ++i) {
      const int32_t t = lst[i];
      int32_t j = i - 1;
      while (j >= 0 && lst[j] > t) {
        lst[j + 1] = lst[j];
        --j;
      }
      lst[j + 1] = t;
    }
    for (int32_t i = 0; i < nl; ++i) {
      a.adj[na] = lst[i];
      a.ew[na] = acc[lst[i]];
      ++na;
      acc[lst[i]] = 0;
      seen[lst[i]] = 0;
    }
    a.ptr[x + 1] = na;
  }
  a.m = na;
  free(mp);
  free(mem);
  free(fill);
  free(acc);
  free(seen);
  free(lst);
  return a;
}

static void pl_free(PGraph *g) {
  free(g->ptr);
  free(g->adj);
  free(g->ew);
  free(g->vw);
}

static void pl_pass(const PGraph *g0, int32_t *memb, double gp) {
  const int32_t n0 = g0->n;
  int32_t *where = (int32_t *)malloc(sizeof(int32_t) * (size_t)n0);
  for (int32_t i = 0; i < n0; ++i) where[i] = i;
  PGraph g = *g0;
  int owned = 0;
  int32_t *comm = (int32_t *)malloc(sizeof(int32_t) * (size_t)n0);
  memcpy(comm, memb, sizeof(int32_t) * (size_t)n0);
  for (int level = 0; level < PL_LEVELS; ++level) {
    const int32_t n = g.n;
    int64_t *W = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int32_t *cnt = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *sub = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int64_t *SW = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int32_t *subN = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    pl_move_nodes(&g, comm, W, cnt, gp);
    memcpy(tmp, comm, sizeof(int32_t) * (size_t)n);
    const int32_t ncomm = pl_compact(n, tmp, cnt);
    int stop = ncomm == n;
    int32_t *comm2 = NULL;
    if (!stop) {
      memcpy(comm, tmp, sizeof(int32_t) * (size_t)n);
      pl_weights(&g, comm, W, cnt);
      pl_refine(&g, comm, W, sub, gp);
      pl_weights(&g, sub, SW, subN);
      int32_t K = pl_compact(n, sub, subN);
      PGraph a;
      if (K == n) {
        /* the refinement merged nothing: aggregate on the communities */
        memcpy(sub, comm, sizeof(int32_t) * (size_t)n);
        K = ncomm;
        comm2 = (int32_t *)malloc(sizeof(int32_t) * (size_t)K);
        a = pl_aggregate(&g, sub, K, comm, comm2);
        for (int32_t x = 0; x < K; ++x) comm2[x] = x;
      } else {
        comm2 = (int32_t *)malloc(sizeof(int32_t) * (size_t)K);
        a = pl_aggregate(&g, sub, K, comm, comm2);
      }
      for (int32_t i = 0; i < n0; ++i) where[i] = sub[where[i]];
      if (owned) pl_free(&g);
      g = a;
      owned = 1;
    }
    free(W);
    free(cnt);
    free(tmp);
    free(sub);
    free(SW);
    free(subN);
    if (stop) break;
    free(comm);
    comm = comm2;
  }
  for (int32_t i = 0; i < n0; ++i) memb[i] = comm[where[i]];
  int32_t *cnt0 = (int32_t *)calloc((size_t)n0, sizeof(int32_t));
  for (int32_t i = 0; i < n0; ++i) cnt0[memb[i]]++;
  pl_compact(n0, memb, cnt0);
  free(cnt0);
  free(comm);
  free(where);
  if (owned) pl_free(&g);
}

/* block_of[n]: the communities split into connected components, numbered by
 * ascending smallest node; returns their number */
int32_t orc_par_leiden(int32_t n, const int64_t *gptr, const int32_t *gadj, int32_t quality, double gamma,
                       int32_t n_iter, int32_t *block_of) {
  if (n <= 0) return 0;
  PGraph g;
  g.n = n;
  g.m = gptr[n];
  g.ptr = (int64_t *)gptr;
  g.adj = (int32_t *)gadj;
  g.ew = (int64_t *)malloc(sizeof(int64_t) * (size_t)(g.m > 0 ? g.m : 1));
  g.vw = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  for (int64_t e = 0; e < g.m; ++e) g.ew[e] = 1;
  for (int32_t v = 0; v < n; ++v) g.vw[v] = quality == 1 ? 1 : gptr[v + 1] - gptr[v];
  const double gp = quality == 1 ? gamma : (g.m > 0 ? gamma / (double)g.m : 0.0);
  int32_t *memb = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  for (int32_t v = 0; v < n; ++v) memb[v] = v;
  for (int32_t it = 0; it < n_iter; ++it) pl_pass(&g, memb, gp);
  /* connected components inside the communities: the smallest node of each
   * (breadth-first from nodes in ascending order) */
  int32_t *lab = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  for (int32_t v = 0; v < n; ++v) lab[v] = -1;
  for (int32_t s = 0; s < n; ++s) {
    if (lab[s] >= 0) continue;
    int32_t head = 0, tail = 0;
    lab[s] = s;
    queue[tail++] = s;
    while (head < tail) {
      const int32_t v = queue[head++];
      for (int64_t e = gptr[v]; e < gptr[v + 1]; ++e) {
        const int32_t u = gadj[e];
        if (lab[u] < 0 && memb[u] == memb[v]) {
          lab[u] = s;
          queue[tail++] = u;
        }
      }
    }
  }
  int32_t *cnt = (int32_t *)calloc((size_t)n, sizeof(int32_t));
  for (int32_t v = 0; v < n; ++v) cnt[lab[v]]++;
  const int32_t nb = pl_compact(n, lab, cnt);
  memcpy(block_of, lab, sizeof(int32_t) * (size_t)n);
  free(cnt);
  free(lab);
  free(queue);
  free(memb);
  free(g.ew);
  free(g.vw);
  return nb;
}
