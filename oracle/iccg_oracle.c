/*
 * CPU oracle for block-multicolor ICCG -- TEST INFRASTRUCTURE ONLY.
 *
 * This file is the plain, slow, single-threaded FP64 statement of what the
 * GPU path computes.  Only tests/, the smoke check and the CPU-baseline leg
 * of the benchmark may load it.  It shares no code with the CUDA library.
 *
 * Source of each step (Suzuki, "Comparison of Algebraic Block Multi-Coloring
 * and Leiden Methods for Parallel Preconditioning in the ICCG Method"):
 *   - adjacency graph of A ............................ Sec. 3 (first par.)
 *   - ABMC blocking (seed + candidate set) ............ Sec. 3; Sec. 5.1 (s = ceil(n/n_b))
 *   - greedy block coloring ........................... Sec. 3; Sec. 5.1 (Saad's greedy)
 *   - Leiden with modularity (Eq. 1) / CPM (Eq. 2) .... Sec. 4; Sec. 6.1 (2 iterations, beta 0.01)
 *   - block ordering (Leiden: size descending) ........ Sec. 6.1
 *   - level-set ordering (level scheduling baseline) .. Sec. 2
 *   - IC(0) factor, L L^T form ........................ Sec. 3 (Alg. 1 divides by L_ii)
 *   - forward / backward substitution ................. Sec. 3, Alg. 1 and the text after it
 *   - PCG, stop at ||r||_2/||b||_2 <= tol .............. Sec. 1; Sec. 4 (tol 1e-8)
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   - graph: unweighted, edge {i,j} iff i != j and a_ij or a_ji is stored;
 *   - ABMC: FIFO candidate queue; neighbours pushed in ascending index;
 *     an empty queue is refilled with the smallest unassigned node;
 *   - Leiden: the published algorithm of Traag, Waltman & van Eck (2019)
 *     with the unnormalised quality H = sum_c (e_c - gamma' W_c^2 / 2);
 *     modularity uses gamma' = gamma/(2m) and node weight = degree, CPM uses
 *     gamma' = gamma and node weight = 1.  Random numbers come from
 *     Philox4x64-10 (Salmon et al. 2011), keyed by the seed.
 *   - the block-multicolor substitution equals the sequential substitution
 *     on the permuted matrix (same-color blocks share no edge and IC(0) adds
 *     no fill), so the oracle solves sequentially over the new numbering.
 *
 * Build: gcc -O2 -ffp-contract=off -shared -fPIC (no fused multiply-add, so
 * the arithmetic is the plain IEEE expression order written here).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11).  A counter-based        */
/* generator: output block k is the 10-round bijection of counter k under    */
/* the key.  The counter is incremented before each block is produced.       */
/* ------------------------------------------------------------------------- */
typedef struct {
  uint64_t key[2];
  uint64_t ctr[4];
  uint64_t out[4];
  int pos;
} orc_rng;

static void mul128(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo) {
  __uint128_t p = (__uint128_t)a * (__uint128_t)b;
  *hi = (uint64_t)(p >> 64);
  *lo = (uint64_t)p;
}

static void philox_block(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4]) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
  uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint64_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += W0; k1 += W1; }
    uint64_t hi0, lo0, hi1, lo1;
    mul128(M0, c0, &hi0, &lo0);
    mul128(M1, c2, &hi1, &lo1);
    uint64_t n0 = hi1 ^ c1 ^ k0;
    uint64_t n1 = lo1;
    uint64_t n2 = hi0 ^ c3 ^ k1;
    uint64_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void rng_init(orc_rng *r, uint64_t seed) {
  r->key[0] = seed; r->key[1] = 0;
  r->ctr[0] = r->ctr[1] = r->ctr[2] = r->ctr[3] = 0;
  r->pos = 4;
}

static uint64_t rng_u64(orc_rng *r) {
  if (r->pos == 4) {
    /* 256-bit counter increment */
    if (++r->ctr[0] == 0) if (++r->ctr[1] == 0) if (++r->ctr[2] == 0) ++r->ctr[3];
    philox_block(r->ctr, r->key, r->out);
    r->pos = 0;
  }
  return r->out[r->pos++];
}

/* uniform double in [0, 1): top 53 bits times 2^-53 */
static double rng_unit(orc_rng *r) { return (double)(rng_u64(r) >> 11) * 0x1.0p-53; }

/* uniform integer in [0, k): reject draws below (2^64 mod k), then take mod k */
static uint64_t rng_below(orc_rng *r, uint64_t k) {
  uint64_t t = (0 - k) % k;
  for (;;) {
    uint64_t x = rng_u64(r);
    if (x >= t) return x % k;
  }
}

/* Fisher-Yates: for i = len-1 down to 1, swap a[i] with a[uniform(i+1)] */
static void shuffle(orc_rng *r, int32_t *a, int64_t len) {
  for (int64_t i = len - 1; i >= 1; --i) {
    int64_t j = (int64_t)rng_below(r, (uint64_t)(i + 1));
    int32_t t = a[i]; a[i] = a[j]; a[j] = t;
  }
}

/* exported for the pin against an independent Philox implementation */
void orc_philox_stream(uint64_t seed, int64_t count, uint64_t *out) {
  orc_rng r; rng_init(&r, seed);
  for (int64_t i = 0; i < count; ++i) out[i] = rng_u64(&r);
}

void orc_shuffle_stream(uint64_t seed, int64_t len, int32_t *a) {
  orc_rng r; rng_init(&r, seed);
  for (int64_t i = 0; i < len; ++i) a[i] = (int32_t)i;
  shuffle(&r, a, len);
}

/* ------------------------------------------------------------------------- */
/* Adjacency graph of A (Sec. 3): symmetric pattern without the diagonal.    */
/* ------------------------------------------------------------------------- */
static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

/* Returns the number of adjacency entries; fills gptr[n+1] and, if gadj is not
 * NULL, gadj[...] (neighbours sorted ascending, no duplicates, no self). */
int64_t orc_graph(int32_t n, const int64_t *rowptr, const int32_t *colind,
                  int64_t *gptr, int32_t *gadj) {
  int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  for (int32_t i = 0; i < n; ++i)
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      int32_t j = colind[e];
      if (j == i) continue;
      cnt[i]++; cnt[j]++;
    }
  int64_t *tp = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
  tp[0] = 0;
  for (int32_t i = 0; i < n; ++i) tp[i + 1] = tp[i] + cnt[i];
  int32_t *tmp = (int32_t *)malloc((size_t)(tp[n] ? tp[n] : 1) * sizeof(int32_t));
  int64_t *fill = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
  memcpy(fill, tp, ((size_t)n + 1) * sizeof(int64_t));
  for (int32_t i = 0; i < n; ++i)
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      int32_t j = colind[e];
      if (j == i) continue;
      tmp[fill[i]++] = j;
      tmp[fill[j]++] = i;
    }
  int64_t total = 0;
  gptr[0] = 0;
  for (int32_t i = 0; i < n; ++i) {
    int32_t *row = tmp + tp[i];
    int64_t len = tp[i + 1] - tp[i];
    qsort(row, (size_t)len, sizeof(int32_t), cmp_i32);
    for (int64_t k = 0; k < len; ++k) {
      if (k > 0 && row[k] == row[k - 1]) continue;
      if (gadj) gadj[total] = row[k];
      total++;
    }
    gptr[i + 1] = total;
  }
  free(cnt); free(tp); free(tmp); free(fill);
  return total;
}

/* ------------------------------------------------------------------------- */
/* ABMC blocking (Sec. 3): pick a seed among the unassigned nodes and add    */
/* its neighbours from a candidate set until the block has s nodes.          */
/* Reading: FIFO candidate queue, neighbours pushed in ascending index, the  */
/* seed (and any refill of an empty queue) is the smallest unassigned node.  */
/* Returns the number of blocks.                                             */
/* ------------------------------------------------------------------------- */
int32_t orc_abmc(int32_t n, const int64_t *gptr, const int32_t *gadj, int32_t s,
                 int32_t *block_of) {
  if (n == 0) return 0;
  int32_t *queue = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  int32_t *queued_in = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  for (int32_t i = 0; i < n; ++i) { block_of[i] = -1; queued_in[i] = -1; }
  int32_t nb = 0, next_seed = 0, assigned = 0;
  while (assigned < n) {
    int64_t qh = 0, qt = 0;
    int32_t size = 0;
    while (size < s && assigned < n) {
      int32_t v = -1;
      while (qh < qt) {
        int32_t c = queue[qh++];
        if (block_of[c] < 0) { v = c; break; }
      }
      if (v < 0) {
        while (block_of[next_seed] >= 0) next_seed++;
        v = next_seed;
      }
      block_of[v] = nb;
      size++; assigned++;
      for (int64_t e = gptr[v]; e < gptr[v + 1]; ++e) {
        int32_t u = gadj[e];
        if (block_of[u] < 0 && queued_in[u] != nb) {
          queued_in[u] = nb;
          queue[qt++] = u;
        }
      }
    }
    nb++;
  }
  free(queue); free(queued_in);
  return nb;
}

/* ------------------------------------------------------------------------- */
/* Greedy block coloring (Sec. 3, Sec. 5.1): visit blocks in index order and */
/* give each the smallest color not used by an adjacent, already colored    */
/* block.  Blocks are adjacent iff some edge joins them.  Returns n_c.       */
/* ------------------------------------------------------------------------- */
int32_t orc_color_blocks(int32_t n, const int64_t *gptr, const int32_t *gadj,
                         int32_t n_b, const int32_t *block_of, int32_t *color_of) {
  /* rows of each block */
  int64_t *bptr = (int64_t *)calloc((size_t)n_b + 1, sizeof(int64_t));
  for (int32_t i = 0; i < n; ++i) bptr[block_of[i] + 1]++;
  for (int32_t b = 0; b < n_b; ++b) bptr[b + 1] += bptr[b];
  int32_t *rows = (int32_t *)malloc((size_t)(n ? n : 1) * sizeof(int32_t));
  int64_t *fill = (int64_t *)malloc(((size_t)n_b + 1) * sizeof(int64_t));
  memcpy(fill, bptr, ((size_t)n_b + 1) * sizeof(int64_t));
  for (int32_t i = 0; i < n; ++i) rows[fill[block_of[i]]++] = i;
  int32_t *mark = (int32_t *)malloc(((size_t)n_b + 1) * sizeof(int32_t));
  for (int32_t c = 0; c <= n_b; ++c) mark[c] = -1;
  for (int32_t b = 0; b < n_b; ++b) color_of[b] = -1;
  int32_t nc = 0;
  for (int32_t b = 0; b < n_b; ++b) {
    for (int64_t k = bptr[b]; k < bptr[b + 1]; ++k) {
      int32_t v = rows[k];
      for (int64_t e = gptr[v]; e < gptr[v + 1]; ++e) {
        int32_t ob = block_of[gadj[e]];
        if (ob != b && color_of[ob] >= 0) mark[color_of[ob]] = b;
      }
    }
    int32_t c = 0;
    while (mark[c] == b) c++;
    color_of[b] = c;
    if (c + 1 > nc) nc = c + 1;
  }
  free(bptr); free(rows); free(fill); free(mark);
  return nc;
}

/* ------------------------------------------------------------------------- */
/* Leiden (Sec. 4; Traag et al. 2019).  Weighted graph without self-loops.   */
/* ------------------------------------------------------------------------- */
typedef struct {
  int32_t n;
  int64_t *ptr;
  int32_t *adj;
  double *w;   /* edge weights */
  double *nw;  /* node weights */
} wgraph;

static void wgraph_free(wgraph *g) { free(g->ptr); free(g->adj); free(g->w); free(g->nw); }

/* Unnormalised gain of putting a node of weight w, joined to community D by
 * edge weight k_vD, into D of total weight W_D (v itself not counted):
 *     g = k_vD - gp * w * W_D.
 * With H = sum_c (e_c - gp W_c^2 / 2), moving v from C to D changes H by
 * g(D) - g(C without v); H / m is Eq. (1) (gp = gamma/2m, w = degree) or
 * Eq. (2) (gp = gamma, w = 1). */
static double gain_into(double k_vD, double w, double W_D, double gp) {
  return k_vD - gp * w * W_D;
}

/* binary min-heap of community ids (used to find the smallest empty community) */
typedef struct { int32_t *a; int64_t len; } minheap;
static void heap_push(minheap *h, int32_t x) {
  int64_t i = h->len++;
  h->a[i] = x;
  while (i > 0) {
    int64_t p = (i - 1) / 2;
    if (h->a[p] <= h->a[i]) break;
    int32_t t = h->a[p]; h->a[p] = h->a[i]; h->a[i] = t; i = p;
  }
}
static void heap_pop(minheap *h) {
  h->a[0] = h->a[--h->len];
  int64_t i = 0;
  for (;;) {
    int64_t l = 2 * i + 1, r = l + 1, m = i;
    if (l < h->len && h->a[l] < h->a[m]) m = l;
    if (r < h->len && h->a[r] < h->a[m]) m = r;
    if (m == i) break;
    int32_t t = h->a[m]; h->a[m] = h->a[i]; h->a[i] = t; i = m;
  }
}

/* Local moving (fast variant): queue of all nodes in random order; a node moves
 * to the neighbouring (or empty) community with the largest quality gain if
 * that gain is strictly positive; ties go to the lowest community id.  The
 * gain of putting v (weight w) into community D (weight W_D without v) is
 *     g(D) = k_{v,D} - gp * w * W_D
 * and v moves from C to D iff g(D) > g(C) with W_C taken without v. */
static void move_nodes_fast(const wgraph *g, int32_t *part, double gp, orc_rng *rng) {
  int32_t n = g->n;
  double *W = (double *)calloc((size_t)n, sizeof(double));
  int64_t *cnt = (int64_t *)calloc((size_t)n, sizeof(int64_t));
  for (int32_t v = 0; v < n; ++v) { W[part[v]] += g->nw[v]; cnt[part[v]]++; }
  minheap empty = {(int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t)), 0};
  for (int32_t c = 0; c < n; ++c) if (cnt[c] == 0) heap_push(&empty, c);
  int32_t *q = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  char *inq = (char *)malloc((size_t)n);
  for (int32_t v = 0; v < n; ++v) q[v] = v;
  shuffle(rng, q, n);
  memset(inq, 1, (size_t)n);
  int64_t head = 0, qlen = n;
  double *kvc = (double *)calloc((size_t)n, sizeof(double));
  char *touched_mark = (char *)calloc((size_t)n, 1);
  int32_t *cand = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
  while (qlen > 0) {
    int32_t v = q[head];
    head = (head + 1) % n; qlen--;
    inq[v] = 0;
    int32_t cur = part[v];
    double wv = g->nw[v];
    int64_t nc = 0;
    for (int64_t e = g->ptr[v]; e < g->ptr[v + 1]; ++e) {
      int32_t c = part[g->adj[e]];
      if (!touched_mark[c]) { touched_mark[c] = 1; cand[nc++] = c; }
      kvc[c] += g->w[e];
    }
    double best_gain = gain_into(kvc[cur], wv, W[cur] - wv, gp);
    int32_t best = cur;
    /* candidate communities: neighbours' communities and, unless v is alone,
     * the smallest empty community (gain 0) */
    int64_t ncand = 0;
    for (int64_t k = 0; k < nc; ++k) if (cand[k] != cur) cand[ncand++] = cand[k];
    int32_t empty_id = -1;
    if (cnt[cur] > 1 && empty.len > 0) { empty_id = empty.a[0]; cand[ncand++] = empty_id; }
    qsort(cand, (size_t)ncand, sizeof(int32_t), cmp_i32);
    for (int64_t k = 0; k < ncand; ++k) {
      int32_t c = cand[k];
      double gain = (c == empty_id) ? 0.0 : gain_into(kvc[c], wv, W[c], gp);
      if (gain > best_gain) { best_gain = gain; best = c; }
    }
    /* reset the scratch accumulators */
    for (int64_t e = g->ptr[v]; e < g->ptr[v + 1]; ++e) {
      int32_t c = part[g->adj[e]];
      kvc[c] = 0.0; touched_mark[c] = 0;
    }
    if (best != cur) {
      W[cur] -= wv; cnt[cur]--;
      if (best == empty_id) heap_pop(&empty);
      if (cnt[cur] == 0) heap_push(&empty, cur);
      W[best] += wv; cnt[best]++;
      part[v] = best;
      for (int64_t e = g->ptr[v]; e < g->ptr[v + 1]; ++e) {
        int32_t u = g->adj[e];
        if (part[u] != best && !inq[u]) {
          inq[u] = 1;
          q[(head + qlen) % n] = u;
          qlen++;
        }
      }
    }
  }
  free(W); free(cnt); free(empty.a); free(q); free(inq); free(kvc); free(touched_mark); free(cand);
}

/* Refinement: inside every community S of `part` (ascending community id),
 * start from singletons; visit the well-connected nodes of S,
 *     E(v, S - v) >= gp * w_v * (W_S - w_v),
 * in random order and, while v is still a singleton, merge it into a
 * well-connected refined community T of S,
 *     E(T, S - T) >= gp * W_T * (W_S - W_T),
 * chosen with probability proportional to exp(g(T) / beta) among those with
 * g(T) = k_{v,T} - gp * w_v * W_T >= 0 (v's own singleton has g = 0).
 * One uniform number is drawn for every visited singleton. */
static void refine(const wgraph *g, const int32_t *part, double gp, double beta,
                   orc_rng *rng, int32_t *ref) {
  int32_t n = g->n;
  double *Wr = (double *)malloc((size_t)n * sizeof(double));
  double *Er = (double *)malloc((size_t)n * sizeof(double));
  int64_t *sz = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  for (int32_t v = 0; v < n; ++v) { ref[v] = v; Wr[v] = g->nw[v]; Er[v] = 0.0; sz[v] = 1; }
  /* members of each community, ascending node id */
  int64_t *cptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  for (int32_t v = 0; v < n; ++v) cptr[part[v] + 1]++;
  for (int32_t c = 0; c < n; ++c) cptr[c + 1] += cptr[c];
  int32_t *mem = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  int64_t *fill = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
  memcpy(fill, cptr, ((size_t)n + 1) * sizeof(int64_t));
  for (int32_t v = 0; v < n; ++v) mem[fill[part[v]]++] = v;
  double *kvt = (double *)calloc((size_t)n, sizeof(double));
  char *tmark = (char *)calloc((size_t)n, 1);
  int32_t *cand = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
  double *gain = (double *)malloc(((size_t)n + 1) * sizeof(double));
  int32_t *R = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  for (int32_t c = 0; c < n; ++c) {
    int64_t s0 = cptr[c], s1 = cptr[c + 1];
    if (s1 == s0) continue;
    double WS = 0.0;
    for (int64_t k = s0; k < s1; ++k) WS += g->nw[mem[k]];
    int64_t nR = 0;
    for (int64_t k = s0; k < s1; ++k) {
      int32_t v = mem[k];
      double e_in = 0.0;
      for (int64_t e = g->ptr[v]; e < g->ptr[v + 1]; ++e)
        if (part[g->adj[e]] == c) e_in += g->w[e];
      Er[v] = e_in;
      if (e_in >= gp * g->nw[v] * (WS - g->nw[v])) R[nR++] = v;
    }
    shuffle(rng, R, nR);
    for (int64_t k = 0; k < nR; ++k) {
      int32_t v = R[k];
      if (sz[ref[v]] != 1) continue;   /* v is no longer a singleton */
      double u01 = rng_unit(rng);
      int32_t own = ref[v];
      double wv = g->nw[v];
      int64_t nc = 0;
      for (int64_t e = g->ptr[v]; e < g->ptr[v + 1]; ++e) {
        int32_t u = g->adj[e];
        if (part[u] != c) continue;
        int32_t t = ref[u];
        if (!tmark[t]) { tmark[t] = 1; cand[nc++] = t; }
        kvt[t] += g->w[e];
      }
      /* admissible candidates, own singleton included with gain 0 */
      int64_t na = 0;
      for (int64_t j = 0; j < nc; ++j) {
        int32_t t = cand[j];
        if (t == own) continue;
        if (!(Er[t] >= gp * Wr[t] * (WS - Wr[t]))) continue;
        double gt = gain_into(kvt[t], wv, Wr[t], gp);
        if (gt >= 0.0) cand[na++] = t;
      }
      cand[na++] = own;
      qsort(cand, (size_t)na, sizeof(int32_t), cmp_i32);
      double gmax = 0.0;
      for (int64_t j = 0; j < na; ++j) {
        int32_t t = cand[j];
        gain[j] = (t == own) ? 0.0 : gain_into(kvt[t], wv, Wr[t], gp);
        if (gain[j] > gmax) gmax = gain[j];
      }
      double total = 0.0;
      for (int64_t j = 0; j < na; ++j) { gain[j] = exp((gain[j] - gmax) / beta); total += gain[j]; }
      double target = u01 * total, cum = 0.0;
      int32_t pick = cand[na - 1];
      for (int64_t j = 0; j < na; ++j) {
        cum += gain[j];
        if (target < cum) { pick = cand[j]; break; }
      }
      double kpick = (pick == own) ? 0.0 : kvt[pick];
      for (int64_t e = g->ptr[v]; e < g->ptr[v + 1]; ++e) {
        int32_t u = g->adj[e];
        if (part[u] != c) continue;
        kvt[ref[u]] = 0.0; tmark[ref[u]] = 0;
      }
      if (pick != own) {
        Er[pick] = Er[pick] + Er[own] - 2.0 * kpick;
        Wr[pick] += wv;
        sz[pick] += 1;
        sz[own] = 0;
        ref[v] = pick;
      }
    }
  }
  free(Wr); free(Er); free(sz); free(cptr); free(mem); free(fill); free(kvt); free(tmark);
  free(cand); free(gain); free(R);
}

/* Renumber labels by first appearance over index order; returns the count. */
static int32_t renumber(int32_t n, int32_t *lab) {
  int32_t bound = 0;
  for (int32_t i = 0; i < n; ++i) if (lab[i] + 1 > bound) bound = lab[i] + 1;
  int32_t *map = (int32_t *)malloc((size_t)(bound ? bound : 1) * sizeof(int32_t));
  for (int32_t i = 0; i < bound; ++i) map[i] = -1;
  int32_t k = 0;
  for (int32_t i = 0; i < n; ++i) {
    if (map[lab[i]] < 0) map[lab[i]] = k++;
    lab[i] = map[lab[i]];
  }
  free(map);
  return k;
}

/* Aggregate graph: one node per group (labels 0..m-1), node weights summed,
 * edge weights between distinct groups summed, edges inside a group dropped
 * (they never enter a gain).  Neighbours sorted ascending. */
static void aggregate(const wgraph *g, const int32_t *grp, int32_t m, wgraph *out) {
  int32_t n = g->n;
  int64_t *gp_ = (int64_t *)calloc((size_t)m + 1, sizeof(int64_t));
  for (int32_t v = 0; v < n; ++v) gp_[grp[v] + 1]++;
  for (int32_t a = 0; a < m; ++a) gp_[a + 1] += gp_[a];
  int32_t *mem = (int32_t *)malloc((size_t)(n ? n : 1) * sizeof(int32_t));
  int64_t *fill = (int64_t *)malloc(((size_t)m + 1) * sizeof(int64_t));
  memcpy(fill, gp_, ((size_t)m + 1) * sizeof(int64_t));
  for (int32_t v = 0; v < n; ++v) mem[fill[grp[v]]++] = v;
  out->n = m;
  out->nw = (double *)calloc((size_t)(m ? m : 1), sizeof(double));
  out->ptr = (int64_t *)malloc(((size_t)m + 1) * sizeof(int64_t));
  int64_t cap = g->ptr[n] > 0 ? g->ptr[n] : 1;
  out->adj = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
  out->w = (double *)malloc((size_t)cap * sizeof(double));
  double *acc = (double *)calloc((size_t)(m ? m : 1), sizeof(double));
  char *mk = (char *)calloc((size_t)(m ? m : 1), 1);
  int32_t *lst = (int32_t *)malloc((size_t)(m ? m : 1) * sizeof(int32_t));
  int64_t tot = 0;
  out->ptr[0] = 0;
  for (int32_t a = 0; a < m; ++a) {
    int64_t nl = 0;
    for (int64_t k = gp_[a]; k < gp_[a + 1]; ++k) {
      int32_t v = mem[k];
      out->nw[a] += g->nw[v];
      for (int64_t e = g->ptr[v]; e < g->ptr[v + 1]; ++e) {
        int32_t b = grp[g->adj[e]];
        if (b == a) continue;
        if (!mk[b]) { mk[b] = 1; lst[nl++] = b; }
        acc[b] += g->w[e];
      }
    }
    qsort(lst, (size_t)nl, sizeof(int32_t), cmp_i32);
    for (int64_t k = 0; k < nl; ++k) {
      out->adj[tot] = lst[k]; out->w[tot] = acc[lst[k]]; tot++;
      acc[lst[k]] = 0.0; mk[lst[k]] = 0;
    }
    out->ptr[a + 1] = tot;
  }
  free(gp_); free(mem); free(fill); free(acc); free(mk); free(lst);
}

/* One multilevel Leiden run starting from the partition memb (on g0's nodes). */
static void leiden_run(const wgraph *g0, int32_t *memb, double gp, double beta, orc_rng *rng) {
  int32_t n0 = g0->n;
  int32_t *node_of = (int32_t *)malloc((size_t)(n0 ? n0 : 1) * sizeof(int32_t));
  for (int32_t v = 0; v < n0; ++v) node_of[v] = v;
  wgraph cur = *g0;      /* level 0 borrows g0's arrays */
  int owns = 0;
  int32_t *part = (int32_t *)malloc((size_t)(n0 ? n0 : 1) * sizeof(int32_t));
  memcpy(part, memb, (size_t)n0 * sizeof(int32_t));
  renumber(n0, part);
  for (;;) {
    int32_t n = cur.n;
    move_nodes_fast(&cur, part, gp, rng);
    int32_t ncomm;
    {
      int32_t *tmp = (int32_t *)malloc((size_t)n * sizeof(int32_t));
      memcpy(tmp, part, (size_t)n * sizeof(int32_t));
      ncomm = renumber(n, tmp);
      free(tmp);
    }
    if (ncomm == n) break;   /* every community is a single node: done */
    int32_t *ref = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    refine(&cur, part, gp, beta, rng, ref);
    int32_t m = renumber(n, ref);
    int32_t *newpart;
    wgraph next;
    if (m == n) {
      /* refinement merged nothing: aggregate on the unrefined partition */
      memcpy(ref, part, (size_t)n * sizeof(int32_t));
      m = renumber(n, ref);
      aggregate(&cur, ref, m, &next);
      newpart = (int32_t *)malloc((size_t)m * sizeof(int32_t));
      for (int32_t a = 0; a < m; ++a) newpart[a] = a;
    } else {
      aggregate(&cur, ref, m, &next);
      newpart = (int32_t *)malloc((size_t)m * sizeof(int32_t));
      for (int32_t v = 0; v < n; ++v) newpart[ref[v]] = part[v];
      renumber(m, newpart);
    }
    for (int32_t v = 0; v < n0; ++v) node_of[v] = ref[node_of[v]];
    free(ref);
    if (owns) wgraph_free(&cur);
    cur = next; owns = 1;
    free(part);
    part = newpart;
  }
  for (int32_t v = 0; v < n0; ++v) memb[v] = part[node_of[v]];
  renumber(n0, memb);
  if (owns) wgraph_free(&cur);
  free(part); free(node_of);
}

/* quality: 0 = modularity (Eq. 1), 1 = CPM (Eq. 2).  Returns the number of
 * communities; memb[n] receives community ids numbered by first appearance. */
int32_t orc_leiden(int32_t n, const int64_t *gptr, const int32_t *gadj, int32_t quality,
                   double gamma, int32_t n_iter, double beta, uint64_t seed, int32_t *memb) {
  if (n == 0) return 0;
  wgraph g;
  g.n = n;
  g.ptr = (int64_t *)gptr;
  g.adj = (int32_t *)gadj;
  int64_t m2 = gptr[n];
  g.w = (double *)malloc((size_t)(m2 ? m2 : 1) * sizeof(double));
  for (int64_t e = 0; e < m2; ++e) g.w[e] = 1.0;
  g.nw = (double *)malloc((size_t)n * sizeof(double));
  double gp;
  if (quality == 0) {
    for (int32_t v = 0; v < n; ++v) g.nw[v] = (double)(gptr[v + 1] - gptr[v]);
    gp = (m2 > 0) ? gamma / (double)m2 : 0.0;   /* gamma / (2m) */
  } else {
    for (int32_t v = 0; v < n; ++v) g.nw[v] = 1.0;
    gp = gamma;
  }
  orc_rng rng; rng_init(&rng, seed);
  for (int32_t v = 0; v < n; ++v) memb[v] = v;
  for (int32_t it = 0; it < n_iter; ++it) leiden_run(&g, memb, gp, beta, &rng);
  int32_t k = renumber(n, memb);
  free(g.w); free(g.nw);
  return k;
}

/* Change of Q (Eq. 1 for quality 0, Eq. 2 for quality 1) when node v moves
 * from its community to community `target` of partition memb, computed with
 * the same gain function the local moving uses: (g(D) - g(C - v)) / m. */
double orc_delta_quality(int32_t n, const int64_t *gptr, const int32_t *gadj, int32_t quality,
                         double gamma, const int32_t *memb, int32_t v, int32_t target) {
  int64_t m2 = gptr[n];
  double gp = quality == 0 ? gamma / (double)m2 : gamma;
  double wv = quality == 0 ? (double)(gptr[v + 1] - gptr[v]) : 1.0;
  int32_t cur = memb[v];
  double W_C = 0.0, W_D = 0.0, k_C = 0.0, k_D = 0.0;
  for (int32_t u = 0; u < n; ++u) {
    double wu = quality == 0 ? (double)(gptr[u + 1] - gptr[u]) : 1.0;
    if (memb[u] == cur) W_C += wu;
    if (memb[u] == target) W_D += wu;
  }
  for (int64_t e = gptr[v]; e < gptr[v + 1]; ++e) {
    int32_t u = gadj[e];
    if (memb[u] == cur) k_C += 1.0;
    if (memb[u] == target) k_D += 1.0;
  }
  if (target == cur) return 0.0;
  double dh = gain_into(k_D, wv, W_D, gp) - gain_into(k_C, wv, W_C - wv, gp);
  return dh / ((double)m2 / 2.0);
}

/* ------------------------------------------------------------------------- */
/* Block order and permutation.                                              */
/* ------------------------------------------------------------------------- */
static const int32_t *g_sort_size;
static const int32_t *g_sort_minrow;
static int cmp_block_desc(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  if (g_sort_size[x] != g_sort_size[y]) return g_sort_size[x] > g_sort_size[y] ? -1 : 1;
  return (g_sort_minrow[x] > g_sort_minrow[y]) - (g_sort_minrow[x] < g_sort_minrow[y]);
}

/* Leiden block order (Sec. 6.1): larger blocks get smaller indices.  Reading
 * for ties: ascending smallest original row.  Relabels block_of in place. */
void orc_sort_blocks_desc(int32_t n, int32_t n_b, int32_t *block_of) {
  int32_t *size = (int32_t *)calloc((size_t)n_b, sizeof(int32_t));
  int32_t *minrow = (int32_t *)malloc((size_t)n_b * sizeof(int32_t));
  for (int32_t b = 0; b < n_b; ++b) minrow[b] = n;
  for (int32_t i = 0; i < n; ++i) {
    size[block_of[i]]++;
    if (i < minrow[block_of[i]]) minrow[block_of[i]] = i;
  }
  int32_t *order = (int32_t *)malloc((size_t)n_b * sizeof(int32_t));
  for (int32_t b = 0; b < n_b; ++b) order[b] = b;
  g_sort_size = size; g_sort_minrow = minrow;
  qsort(order, (size_t)n_b, sizeof(int32_t), cmp_block_desc);
  int32_t *newid = (int32_t *)malloc((size_t)n_b * sizeof(int32_t));
  for (int32_t k = 0; k < n_b; ++k) newid[order[k]] = k;
  for (int32_t i = 0; i < n; ++i) block_of[i] = newid[block_of[i]];
  free(size); free(minrow); free(order); free(newid);
}

/* Block-multicolor ordering (Sec. 3, Alg. 1): colors ascending, then blocks
 * ascending, then rows of a block in ascending original index.
 * perm[new] = old; block_ptr[n_b+1] in new row numbering; color_ptr[n_c+1] in
 * new block numbering. */
void orc_order(int32_t n, int32_t n_b, int32_t n_c, const int32_t *block_of,
               const int32_t *color_of, int32_t *perm, int32_t *block_ptr, int32_t *color_ptr) {
  /* new block order: stable sort of block ids by color */
  int32_t *border = (int32_t *)malloc((size_t)(n_b ? n_b : 1) * sizeof(int32_t));
  int32_t k = 0;
  for (int32_t c = 0; c < n_c; ++c) {
    color_ptr[c] = k;
    for (int32_t b = 0; b < n_b; ++b) if (color_of[b] == c) border[k++] = b;
  }
  color_ptr[n_c] = k;
  int32_t *size = (int32_t *)calloc((size_t)n_b + 1, sizeof(int32_t));
  for (int32_t i = 0; i < n; ++i) size[block_of[i]]++;
  int32_t *start = (int32_t *)malloc(((size_t)n_b + 1) * sizeof(int32_t));
  int32_t pos = 0;
  for (int32_t j = 0; j < n_b; ++j) {
    block_ptr[j] = pos;
    start[border[j]] = pos;
    pos += size[border[j]];
  }
  block_ptr[n_b] = pos;
  for (int32_t i = 0; i < n; ++i) perm[start[block_of[i]]++] = i;
  free(border); free(size); free(start);
}

/* Level sets of the natural order (level scheduling, Sec. 2): a row's level
 * is the length of the longest chain of preceding neighbours ending at it,
 * i.e. 0 with no neighbour j < i, else 1 + the largest level of such j.  The
 * ordering lists levels ascending, rows ascending within a level; every row
 * is its own block and every level a color.  Returns the number of levels. */
int32_t orc_level_order(int32_t n, const int64_t *gptr, const int32_t *gadj, int32_t *level,
                        int32_t *perm, int32_t *block_ptr, int32_t *color_ptr) {
  int32_t nl = 0;
  for (int32_t i = 0; i < n; ++i) {
    int32_t lv = 0;
    for (int64_t e = gptr[i]; e < gptr[i + 1]; ++e) {
      const int32_t j = gadj[e];
      if (j < i && level[j] + 1 > lv) lv = level[j] + 1;
    }
    level[i] = lv;
    if (lv + 1 > nl) nl = lv + 1;
  }
  int32_t pos = 0;
  for (int32_t v = 0; v < nl; ++v) {
    color_ptr[v] = pos;
    for (int32_t i = 0; i < n; ++i)
      if (level[i] == v) perm[pos++] = i;
  }
  color_ptr[nl] = pos;
  for (int32_t k = 0; k <= n; ++k) block_ptr[k] = k;
  return nl;
}

/* ------------------------------------------------------------------------- */
/* IC(0) on the permuted matrix (Sec. 3): L has the pattern of tril(A_hat),  */
/* (L L^T)_ij = a_ij on that pattern, L_ii = sqrt(d_i).  Up-looking, row by  */
/* row.  Input: lower-triangular part of A_hat (CSR, columns ascending,      */
/* diagonal last in each row).  Output lval on the same pattern.             */
/* Returns -1 on success or the first row whose pivot is not positive.       */
/* ------------------------------------------------------------------------- */
int64_t orc_ic0(int32_t n, const int64_t *lptr, const int32_t *lcol, const double *aval,
                double *lval) {
  memcpy(lval, aval, (size_t)lptr[n] * sizeof(double));
  for (int32_t i = 0; i < n; ++i) {
    int64_t di = lptr[i + 1] - 1;
    if (di < lptr[i] || lcol[di] != i) return i;   /* no diagonal */
    for (int64_t p = lptr[i]; p < di; ++p) {
      int32_t j = lcol[p];
      /* s = a_ij - sum_{k<j, k in pat(i) and pat(j)} L_ik L_jk */
      double s = lval[p];
      int64_t a = lptr[i], b = lptr[j], bend = lptr[j + 1] - 1;
      while (a < p && b < bend) {
        if (lcol[a] == lcol[b]) { s -= lval[a] * lval[b]; a++; b++; }
        else if (lcol[a] < lcol[b]) a++;
        else b++;
      }
      lval[p] = s / lval[lptr[j + 1] - 1];
    }
    double d = lval[di];
    for (int64_t p = lptr[i]; p < di; ++p) d -= lval[p] * lval[p];
    if (!(d > 0.0) || !isfinite(d)) return i;
    lval[di] = sqrt(d);
  }
  return -1;
}

/* forward substitution L y = r (Alg. 1 in sequential order) */
void orc_forward(int32_t n, const int64_t *lptr, const int32_t *lcol, const double *lval,
                 const double *r, double *y) {
  for (int32_t i = 0; i < n; ++i) {
    double s = r[i];
    int64_t di = lptr[i + 1] - 1;
    for (int64_t p = lptr[i]; p < di; ++p) s -= lval[p] * y[lcol[p]];
    y[i] = s / lval[di];
  }
}

/* backward substitution L^T z = y: rows in reverse order; after z_i is known
 * its contribution L_ij z_i is removed from every earlier row j. */
void orc_backward(int32_t n, const int64_t *lptr, const int32_t *lcol, const double *lval,
                  const double *y, double *z) {
  double *w = (double *)malloc((size_t)(n ? n : 1) * sizeof(double));
  memcpy(w, y, (size_t)n * sizeof(double));
  for (int32_t i = n - 1; i >= 0; --i) {
    int64_t di = lptr[i + 1] - 1;
    z[i] = w[i] / lval[di];
    for (int64_t p = lptr[i]; p < di; ++p) w[lcol[p]] -= lval[p] * z[i];
  }
  free(w);
}

void orc_spmv(int32_t n, const int64_t *rowptr, const int32_t *colind, const double *val,
              const double *x, double *y) {
  for (int32_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) s += val[e] * x[colind[e]];
    y[i] = s;
  }
}

static double dot(int32_t n, const double *a, const double *b) {
  double s = 0.0;
  for (int32_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* Preconditioned CG with M = L L^T (Saad, Alg. 9.1):
 *   r0 = b - A x0, z0 = M^-1 r0, p0 = z0;
 *   for k = 0, 1, ...: q = A p; alpha = (r,z)/(p,q); x += alpha p;
 *     r -= alpha q; stop when ||r||/||b|| <= tol (iterations = k+1);
 *     z = M^-1 r; beta = (r,z)_new/(r,z)_old; p = z + beta p.
 * hist[k] = ||r_k||/||b|| for k = 0..iterations (hist may be NULL).
 * Returns 0 = converged, 1 = maxit reached, 2 = non-finite value.  b = 0
 * gives x = 0 and 0 iterations. */
int32_t orc_pcg(int32_t n, const int64_t *rowptr, const int32_t *colind, const double *val,
                const int64_t *lptr, const int32_t *lcol, const double *lval,
                const double *b, double *x, double tol, int32_t maxit,
                int32_t *iters, double *hist) {
  size_t sz = (size_t)(n ? n : 1) * sizeof(double);
  double *r = (double *)malloc(sz), *z = (double *)malloc(sz), *p = (double *)malloc(sz);
  double *q = (double *)malloc(sz), *y = (double *)malloc(sz);
  int32_t status = 1;
  double bnorm = sqrt(dot(n, b, b));
  *iters = 0;
  if (bnorm == 0.0) {
    for (int32_t i = 0; i < n; ++i) x[i] = 0.0;
    if (hist) hist[0] = 0.0;
    status = 0;
    goto done;
  }
  orc_spmv(n, rowptr, colind, val, x, q);
  for (int32_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
  double rn = sqrt(dot(n, r, r)) / bnorm;
  if (hist) hist[0] = rn;
  if (rn <= tol) { status = 0; goto done; }
  orc_forward(n, lptr, lcol, lval, r, y);
  orc_backward(n, lptr, lcol, lval, y, z);
  for (int32_t i = 0; i < n; ++i) p[i] = z[i];
  double rz = dot(n, r, z);
  for (int32_t k = 0; k < maxit; ++k) {
    orc_spmv(n, rowptr, colind, val, p, q);
    double alpha = rz / dot(n, p, q);
    for (int32_t i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
    rn = sqrt(dot(n, r, r)) / bnorm;
    *iters = k + 1;
    if (hist) hist[k + 1] = rn;
    if (!isfinite(rn)) { status = 2; goto done; }
    if (rn <= tol) { status = 0; goto done; }
    orc_forward(n, lptr, lcol, lval, r, y);
    orc_backward(n, lptr, lcol, lval, y, z);
    double rz_new = dot(n, r, z);
    double beta = rz_new / rz;
    rz = rz_new;
    for (int32_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
  }
done:
  free(r); free(z); free(p); free(q); free(y);
  return status;
}
