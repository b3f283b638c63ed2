// Device-side blocking: the graph of a sparse matrix, the greedy block
// coloring with the block-multicolor ordering, and the Leiden block order,
// computed on the GPU with the same results as the host helpers of
// blocking.cpp (the graph of Sec. 3: edge {i,j} iff a_ij or a_ji is stored,
// i != j; the greedy coloring of Sec. 3 / Sec. 5.1 with blocks visited in
// index order; colors ascending, blocks ascending, rows ascending; Leiden
// blocks by size descending, ties by smallest row, Sec. 6.1).
//
// Building blocks: an exclusive scan, a stable LSD radix sort of 64-bit keys
// (4-bit digits; each thread ranks 8 consecutive keys, so equal digits keep
// their order), and compaction by flags.  The greedy coloring is exact in
// parallel: block b's color depends only on the colors of its neighbours
// with a smaller index, so b is colored in the wave after the last of those
// (Jones-Plassmann with index priorities), and every wave gives exactly the
// colors of the sequential visit.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "iccg.h"

namespace iccg_dev {

constexpr int kT = 256;           // threads per CTA
constexpr int kItems = 8;         // keys per thread in scans and sorts
constexpr int kTile = kT * kItems;
constexpr int kDigitBits = 4;
constexpr int kDigits = 1 << kDigitBits;

// Stream-ordered scratch, freed (stream-ordered) when it goes out of scope.
struct Scratch {
  cudaStream_t s;
  std::vector<void *> ptrs;
  cudaError_t err = cudaSuccess;
  explicit Scratch(cudaStream_t st) : s(st) {}
  template <typename T>
  T *get(size_t n) {
    void *p = nullptr;
    if (err == cudaSuccess) err = cudaMallocAsync(&p, std::max<size_t>(n, 1) * sizeof(T), s);
    if (err != cudaSuccess) return nullptr;
    ptrs.push_back(p);
    return static_cast<T *>(p);
  }
  ~Scratch() {
    for (void *p : ptrs) cudaFreeAsync(p, s);
  }
};

inline int grid_for(int64_t n, int per = kT) {
  const int64_t g = (n + per - 1) / per;
  return int(std::max<int64_t>(1, std::min<int64_t>(g, 1 << 20)));
}

// ---------------------------------------------------------------------------
// exclusive scan (int64), any length, in place allowed
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t *total) {
  __shared__ int64_t ws[kT / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    int64_t s = lane < kT / 32 ? ws[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < kT / 32) ws[lane] = s;
  }
  __syncthreads();
  const int64_t before = (w > 0 ? ws[w - 1] : 0) + x - v;
  if (total) *total = ws[kT / 32 - 1];
  __syncthreads();
  return before;
}

__global__ void scan_tiles(const int64_t *in, int64_t *out, int64_t *sums, int64_t n) {
  const int64_t base = int64_t(blockIdx.x) * kTile + int64_t(threadIdx.x) * kItems;
  int64_t v[kItems], t = 0;
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    v[k] = base + k < n ? in[base + k] : 0;
    t += v[k];
  }
  int64_t tot;
  int64_t run = block_excl_scan(t, &tot);
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void scan_add(int64_t *out, const int64_t *offs, int64_t n) {
  const int64_t base = int64_t(blockIdx.x) * kTile;
  const int64_t o = offs[blockIdx.x];
  for (int k = threadIdx.x; k < kTile; k += kT)
    if (base + k < n) out[base + k] += o;
}

// out[k] = sum in[0..k); returns the total in *total (device) when given
cudaError_t scan(const int64_t *in, int64_t *out, int64_t n, Scratch &S, int64_t *total = nullptr) {
  if (n <= 0) {
    if (total) return cudaMemsetAsync(total, 0, sizeof(int64_t), S.s);
    return cudaSuccess;
  }
  const int64_t tiles = (n + kTile - 1) / kTile;
  int64_t *sums = S.get<int64_t>(size_t(tiles) + 1);
  if (S.err != cudaSuccess) return S.err;
  scan_tiles<<<unsigned(tiles), kT, 0, S.s>>>(in, out, sums, n);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (tiles == 1) {
    if (total) e = cudaMemcpyAsync(total, sums, sizeof(int64_t), cudaMemcpyDeviceToDevice, S.s);
    return e;
  }
  // scan of the tile sums (length tiles + 1: the last entry becomes the
  // total); tiles + 1 <= 2 (tiles - 1) + 1 keys fit in fewer tiles
  e = cudaMemsetAsync(sums + tiles, 0, sizeof(int64_t), S.s);
  if (e != cudaSuccess) return e;
  e = scan(sums, sums, tiles + 1, S);
  if (e != cudaSuccess) return e;
  scan_add<<<unsigned(tiles), kT, 0, S.s>>>(out, sums, n);
  e = cudaGetLastError();
  if (e == cudaSuccess && total) e = cudaMemcpyAsync(total, sums + tiles, sizeof(int64_t), cudaMemcpyDeviceToDevice, S.s);
  return e;
}

// ---------------------------------------------------------------------------
// stable LSD radix sort of (key, value) pairs on the low `bits` key bits
// ---------------------------------------------------------------------------
__global__ void radix_count(const uint64_t *key, int64_t n, int shift, int64_t *cnt, int64_t tiles) {
  __shared__ int c[kDigits];
  if (threadIdx.x < kDigits) c[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = int64_t(blockIdx.x) * kTile;
  for (int k = threadIdx.x; k < kTile; k += kT)
    if (base + k < n) atomicAdd(&c[int((key[base + k] >> shift) & (kDigits - 1))], 1);
  __syncthreads();
  if (threadIdx.x < kDigits) cnt[int64_t(threadIdx.x) * tiles + blockIdx.x] = c[threadIdx.x];
}

// Each thread owns kItems consecutive keys; its per-digit counts are scanned
// across the CTA (digit-major, thread-minor), so a key's place is: the
// digit's global offset for this tile + the counts of earlier threads + the
// earlier keys of the same thread.  Equal digits keep their input order.
__global__ void radix_scatter(const uint64_t *key, const int32_t *val, uint64_t *key2, int32_t *val2, int64_t n,
                              int shift, const int64_t *off, int64_t tiles) {
  __shared__ int cnt[kDigits * kT];
  const int t = threadIdx.x;
  const int64_t base = int64_t(blockIdx.x) * kTile + int64_t(t) * kItems;
  uint64_t k[kItems];
  int d[kItems];
#pragma unroll
  for (int u = 0; u < kItems; ++u) {
    k[u] = base + u < n ? key[base + u] : 0;
    d[u] = base + u < n ? int((k[u] >> shift) & (kDigits - 1)) : -1;
  }
  for (int q = 0; q < kDigits; ++q) cnt[q * kT + t] = 0;
#pragma unroll
  for (int u = 0; u < kItems; ++u)
    if (d[u] >= 0) cnt[d[u] * kT + t]++;
  __syncthreads();
  // exclusive scan of cnt[] (kDigits * kT entries; thread t owns kDigits
  // consecutive ones)
  int loc[kDigits], s = 0;
#pragma unroll
  for (int q = 0; q < kDigits; ++q) {
    loc[q] = cnt[t * kDigits + q];
    s += loc[q];
  }
  int64_t tot;
  const int64_t before = block_excl_scan(int64_t(s), &tot);
  int run = int(before);
#pragma unroll
  for (int q = 0; q < kDigits; ++q) {
    const int c = loc[q];
    cnt[t * kDigits + q] = run;
    run += c;
  }
  __syncthreads();
  // offset of digit q's first key of this tile within the tile: cnt[q * kT]
  int seen[kDigits];
#pragma unroll
  for (int q = 0; q < kDigits; ++q) seen[q] = 0;
#pragma unroll
  for (int u = 0; u < kItems; ++u) {
    if (d[u] < 0) continue;
    const int q = d[u];
    const int64_t pos = off[int64_t(q) * tiles + blockIdx.x] + (cnt[q * kT + t] - cnt[q * kT]) + seen[q];
    seen[q]++;
    key2[pos] = k[u];
    if (val) val2[pos] = val[base + u];
  }
}

// sorts key[0..n) (and val, may be null) in place by the low `bits` bits
cudaError_t radix_sort(uint64_t *key, int32_t *val, int64_t n, int bits, Scratch &S) {
  if (n <= 1 || bits <= 0) return cudaSuccess;
  const int64_t tiles = (n + kTile - 1) / kTile;
  uint64_t *k2 = S.get<uint64_t>(size_t(n));
  int32_t *v2 = val ? S.get<int32_t>(size_t(n)) : nullptr;
  int64_t *cnt = S.get<int64_t>(size_t(kDigits * tiles));
  if (S.err != cudaSuccess) return S.err;
  uint64_t *ka = key, *kb = k2;
  int32_t *va = val, *vb = v2;
  cudaError_t e = cudaSuccess;
  for (int shift = 0; shift < bits && e == cudaSuccess; shift += kDigitBits) {
    radix_count<<<unsigned(tiles), kT, 0, S.s>>>(ka, n, shift, cnt, tiles);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = scan(cnt, cnt, kDigits * tiles, S);
    if (e == cudaSuccess) {
      radix_scatter<<<unsigned(tiles), kT, 0, S.s>>>(ka, va, kb, vb, n, shift, cnt, tiles);
      e = cudaGetLastError();
    }
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (e == cudaSuccess && ka != key) {
    e = cudaMemcpyAsync(key, ka, size_t(n) * sizeof(uint64_t), cudaMemcpyDeviceToDevice, S.s);
    if (e == cudaSuccess && val) e = cudaMemcpyAsync(val, va, size_t(n) * sizeof(int32_t), cudaMemcpyDeviceToDevice, S.s);
  }
  return e;
}

inline int bits_for(uint64_t v) {   // bits to hold 0..v
  int b = 0;
  while (b < 64 && (v >> b) != 0) ++b;
  return std::max(b, 1);
}

// ---------------------------------------------------------------------------
// pairs (row, col) -> CSR with sorted, de-duplicated rows
// ---------------------------------------------------------------------------
// keys: row * ncol + col, or `none` for an unused slot; sorted ascending
__global__ void unique_flags(const uint64_t *key, int64_t n, uint64_t none, int64_t *flag) {
  for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x)
    flag[k] = (key[k] != none && (k == 0 || key[k] != key[k - 1])) ? 1 : 0;
}

__global__ void unique_emit(const uint64_t *key, const int64_t *flag, const int64_t *pos, int64_t n, uint64_t none,
                            uint64_t ncol, int32_t *adj, int64_t *rowcnt) {
  for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x)
    if (flag[k]) {
      adj[pos[k]] = int32_t(key[k] % ncol);
      atomicAdd(reinterpret_cast<unsigned long long *>(rowcnt + key[k] / ncol), 1ull);
    }
}

// sorts keys, writes ptr[nrow+1] and adj (capacity n), *m = entries (host)
cudaError_t pairs_to_csr(uint64_t *key, int64_t n, uint64_t nrow, uint64_t ncol, int64_t *ptr, int32_t *adj,
                         int64_t *m, Scratch &S) {
  const uint64_t none = nrow * ncol;
  cudaError_t e = radix_sort(key, nullptr, n, bits_for(none), S);
  int64_t *flag = S.get<int64_t>(size_t(n) + 1);
  int64_t *rowcnt = S.get<int64_t>(size_t(nrow) + 1);
  if (S.err != cudaSuccess) return S.err;
  if (e == cudaSuccess) e = cudaMemsetAsync(rowcnt, 0, (size_t(nrow) + 1) * sizeof(int64_t), S.s);
  if (e == cudaSuccess && n > 0) {
    unique_flags<<<grid_for(n), kT, 0, S.s>>>(key, n, none, flag);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = scan(flag, flag + 0, n, S);   // in place: positions
  // unique_emit needs the flags again: recompute them into rowcnt's neighbour
  int64_t *flag2 = S.get<int64_t>(size_t(n) + 1);
  if (S.err != cudaSuccess) return S.err;
  if (e == cudaSuccess && n > 0) {
    unique_flags<<<grid_for(n), kT, 0, S.s>>>(key, n, none, flag2);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && n > 0) {
    unique_emit<<<grid_for(n), kT, 0, S.s>>>(key, flag2, flag, n, none, ncol, adj, rowcnt);
    e = cudaGetLastError();
  }
  int64_t *tot = S.get<int64_t>(1);
  if (S.err != cudaSuccess) return S.err;
  if (e == cudaSuccess) e = scan(rowcnt, ptr, int64_t(nrow) + 1, S, tot);
  if (e == cudaSuccess) e = cudaMemcpyAsync(m, ptr + nrow, sizeof(int64_t), cudaMemcpyDeviceToHost, S.s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(S.s);
  return e;
}

// ---------------------------------------------------------------------------
// the graph
// ---------------------------------------------------------------------------
__global__ void graph_pairs(int32_t n, int64_t nnz, const int64_t *rowptr, const int32_t *colind, uint64_t *key,
                            int *bad) {
  const uint64_t un = uint64_t(n), none = un * un;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t a = rowptr[i], b = rowptr[i + 1];
    if (a > b || a < 0 || b > nnz || (i == 0 && a != 0) || (i == n - 1 && b != nnz)) {
      atomicExch(bad, 1);
      continue;
    }
    for (int64_t e = a; e < b; ++e) {
      const int32_t j = colind[e];
      if (j < 0 || j >= n) {
        atomicExch(bad, 1);
        key[2 * e] = key[2 * e + 1] = none;
        continue;
      }
      if (j == i) {
        key[2 * e] = key[2 * e + 1] = none;
      } else {
        key[2 * e] = uint64_t(i) * un + uint64_t(j);
        key[2 * e + 1] = uint64_t(j) * un + uint64_t(i);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// greedy block coloring (exact) and the ordering
// ---------------------------------------------------------------------------
// rows of the graph's entries, after checking gptr (monotone, 0 .. m) and
// the neighbours' range
__global__ void edge_rows(int32_t n, int64_t m, const int64_t *gptr, const int32_t *gadj, int32_t *row, int *bad) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t a = gptr[i], b = gptr[i + 1];
    if (a > b || a < 0 || b > m || (i == 0 && a != 0) || (i == n - 1 && b != m)) {
      atomicExch(bad, 1);
      continue;
    }
    for (int64_t e = a; e < b; ++e) {
      row[e] = int32_t(i);
      if (gadj[e] < 0 || gadj[e] >= n) atomicExch(bad, 1);
    }
  }
}

__global__ void edge_rows_unchecked(int32_t n, const int64_t *gptr, int32_t *row) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    for (int64_t e = gptr[i]; e < gptr[i + 1]; ++e) row[e] = int32_t(i);
}

__global__ void block_pairs(int64_t m, const int32_t *row, const int32_t *gadj, const int32_t *block_of, int32_t n_b,
                            uint64_t *key, int *bad) {
  const uint64_t nb = uint64_t(n_b), none = nb * nb;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < m; e += int64_t(gridDim.x) * blockDim.x) {
    const int32_t a = block_of[row[e]], b = block_of[gadj[e]];
    if (a < 0 || a >= n_b || b < 0 || b >= n_b) {
      atomicExch(bad, 1);
      key[e] = none;
      continue;
    }
    key[e] = a == b ? none : uint64_t(a) * nb + uint64_t(b);
  }
}

__global__ void check_blocks(int32_t n, const int32_t *block_of, int32_t n_b, int *bad) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    if (block_of[i] < 0 || block_of[i] >= n_b) atomicExch(bad, 1);
}

// lower[b] = number of neighbours with a smaller index (their colors come first)
__global__ void lower_counts(int32_t n_b, const int64_t *bptr, const int32_t *badj, int32_t *lower, int32_t *wave,
                             int32_t *wave_n, int32_t *color) {
  for (int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; b < n_b; b += int64_t(gridDim.x) * blockDim.x) {
    int32_t c = 0;
    for (int64_t e = bptr[b]; e < bptr[b + 1] && badj[e] < b; ++e) ++c;
    lower[b] = c;
    color[b] = -1;
    if (c == 0) wave[atomicAdd(wave_n, 1)] = int32_t(b);
  }
}

// One wave: every listed block has all smaller neighbours colored; its color
// is the smallest one none of them has.  Then each larger neighbour loses one
// pending smaller neighbour and joins the next wave when none is left.
__global__ void color_wave(const int32_t *wave, int32_t nw, const int64_t *bptr, const int32_t *badj, int32_t *lower,
                           int32_t *color, int32_t *next, int32_t *next_n, int32_t *ncolor) {
  for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < nw; k += int64_t(gridDim.x) * blockDim.x) {
    const int32_t b = wave[k];
    const int64_t e0 = bptr[b], e1 = bptr[b + 1];
    int32_t c = 0;
    for (int base = 0;; base += 64) {
      uint64_t used = 0;
      for (int64_t e = e0; e < e1 && badj[e] < b; ++e) {
        const int32_t q = color[badj[e]] - base;
        if (q >= 0 && q < 64) used |= 1ull << q;
      }
      if (~used != 0) {
        c = base + __ffsll(static_cast<long long>(~used)) - 1;
        break;
      }
    }
    color[b] = c;
    atomicMax(ncolor, c + 1);
    for (int64_t e = e0; e < e1; ++e) {
      const int32_t u = badj[e];
      if (u > b && atomicSub(lower + u, 1) == 1) next[atomicAdd(next_n, 1)] = u;
    }
  }
}

__global__ void keys_from(int64_t n, const int32_t *a, uint64_t *key, int32_t *val) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    key[i] = uint64_t(uint32_t(a[i]));
    val[i] = int32_t(i);
  }
}

__global__ void block_rank_size(int32_t n_b, const int32_t *order, int32_t *rank, const int32_t *color,
                                int32_t *color_cnt) {
  for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n_b; k += int64_t(gridDim.x) * blockDim.x) {
    rank[order[k]] = int32_t(k);
    atomicAdd(color_cnt + color[order[k]], 1);
  }
}

__global__ void row_keys(int32_t n, const int32_t *block_of, const int32_t *rank, uint64_t *key, int32_t *val,
                         int64_t *bsize) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const int32_t r = rank[block_of[i]];
    key[i] = uint64_t(r);
    val[i] = int32_t(i);
    atomicAdd(reinterpret_cast<unsigned long long *>(bsize + r), 1ull);
  }
}

__global__ void to_i32(int64_t n, const int64_t *a, int32_t *b) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    b[i] = int32_t(a[i]);
}

__global__ void i32_to_i64(int64_t n, const int32_t *a, int64_t *b) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    b[i] = a[i];
}

// ---------------------------------------------------------------------------
// Leiden block order: size descending, ties by smallest row
// ---------------------------------------------------------------------------
__global__ void size_first(int32_t n, const int32_t *block_of, int32_t *size, int32_t *first) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    atomicAdd(size + block_of[i], 1);
    atomicMin(first + block_of[i], int32_t(i));
  }
}

__global__ void size_keys(int32_t n_b, int32_t n, const int32_t *size, const int32_t *first, uint64_t *key,
                          int32_t *val) {
  for (int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; b < n_b; b += int64_t(gridDim.x) * blockDim.x) {
    key[b] = uint64_t(n - size[b]) * uint64_t(n + 1) + uint64_t(first[b]);
    val[b] = int32_t(b);
  }
}

__global__ void rank_of(int32_t n_b, const int32_t *order, int32_t *rank) {
  for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n_b; k += int64_t(gridDim.x) * blockDim.x)
    rank[order[k]] = int32_t(k);
}

__global__ void relabel(int32_t n, int32_t *block_of, const int32_t *rank) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    block_of[i] = rank[block_of[i]];
}

__global__ void fill_i32(int64_t n, int32_t *a, int32_t v) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) a[i] = v;
}

// ---------------------------------------------------------------------------
// Leiden on the device (Sec. 4; Traag, Waltman & van Eck 2019), a parallel
// restatement of the host's method with the same quality and gains:
// H = sum_c (e_c - gp W_c^2 / 2), the gain of placing node v (weight w) in
// community c being k_vc - gp w W_c (W_c without v).  All weights are
// integers (edge counts, node counts or degrees), so the sums are exact and
// the result does not depend on the order of the atomic additions.
//   - local moving in synchronous sub-rounds: every node takes its best
//     community (strictly better than staying, ties to the lowest label, a
//     free label of its own as the "new community"), moves in even sub-rounds
//     only to smaller labels and in odd ones only to larger ones, so no two
//     nodes swap; until two sub-rounds move nothing;
//   - refinement: inside each community, well-connected singleton nodes join
//     the well-connected sub-community of largest non-negative gain (the
//     greedy limit beta -> 0 of the randomized choice), same sub-round rule;
//   - aggregation on the refined partition (the unrefined one when the
//     refinement merged nothing), the aggregate's starting partition being
//     the unrefined one; until local moving merges nothing; n_iter passes;
//   - finally every community is split into its connected components.
// ---------------------------------------------------------------------------
struct DGraph {
  int32_t n = 0;
  int64_t m = 0;
  int64_t *ptr = nullptr;
  int32_t *adj = nullptr;
  int64_t *ew = nullptr;
  int64_t *vw = nullptr;
};

__global__ void init_unit_graph(int32_t n, const int64_t *gptr, int64_t m, int64_t *ew, int64_t *vw, int cpm) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < m; e += stride) ew[e] = 1;
  for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < n; v += stride)
    vw[v] = cpm ? 1 : gptr[v + 1] - gptr[v];
}

__global__ void community_weights(int32_t n, const int32_t *comm, const int64_t *vw, int64_t *W, int32_t *cnt) {
  for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < n; v += int64_t(gridDim.x) * blockDim.x) {
    atomicAdd(reinterpret_cast<unsigned long long *>(W + comm[v]), static_cast<unsigned long long>(vw[v]));
    atomicAdd(cnt + comm[v], 1);
  }
}

// Every floating-point operation of the Leiden decisions is one IEEE
// round-to-nearest step in a fixed order (no contraction into FMA), so a
// sequential restatement on the CPU takes exactly the same decisions.
__device__ __forceinline__ double penalty(double gp, int64_t w, int64_t W) {
  return __dmul_rn(__dmul_rn(gp, double(w)), double(W));
}
__device__ __forceinline__ double leiden_gain(int64_t k, int64_t w, int64_t W, double gp) {
  return __dsub_rn(double(k), penalty(gp, w, W));
}

// one local-moving sub-round: the decision of every node from the state at
// the sub-round's start
// proposal key: the gain over staying (positive; float bits order like the
// values) above, 0xffffffff - node below, so the largest gain wins and ties
// go to the smallest node
__device__ __forceinline__ unsigned long long join_key(double delta, int32_t v) {
  const float f = fmaxf(__double2float_rn(delta), 1e-30f);
  return (static_cast<unsigned long long>(__float_as_uint(f)) << 32) |
         static_cast<unsigned long long>(0xffffffffu - uint32_t(v));
}

__global__ void lm_decide(DGraph g, const int32_t *comm, const int64_t *W, const int32_t *cnt, double gp, int dir,
                          int32_t *newc, unsigned long long *join) {
  for (int64_t vv = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; vv < g.n;
       vv += int64_t(gridDim.x) * blockDim.x) {
    const int32_t v = int32_t(vv), C = comm[v];
    const int64_t wv = g.vw[v], e0 = g.ptr[v], e1 = g.ptr[v + 1];
    int64_t kC = 0;
    for (int64_t e = e0; e < e1; ++e)
      if (comm[g.adj[e]] == C) kC += g.ew[e];
    int32_t best = C;
    double bestg = leiden_gain(kC, wv, W[C] - wv, gp);
    for (int64_t e = e0; e < e1; ++e) {
      const int32_t c = comm[g.adj[e]];
      if (c == C || (dir == 0 ? c > C : c < C)) continue;
      bool dup = false;
      for (int64_t f = e0; f < e && !dup; ++f) dup = comm[g.adj[f]] == c;
      if (dup) continue;
      int64_t kc = g.ew[e];
      for (int64_t f = e + 1; f < e1; ++f)
        if (comm[g.adj[f]] == c) kc += g.ew[f];
      const double gc = leiden_gain(kc, wv, W[c], gp);
      if (gc > bestg || (gc == bestg && best != C && c < best)) {
        best = c;
        bestg = gc;
      }
    }
    // a new community: the node's own label when no node holds it
    const double stay = leiden_gain(kC, wv, W[C] - wv, gp);
    if (cnt[C] > 1 && cnt[v] == 0 && 0.0 > bestg) {
      best = v;
      bestg = 0.0;
    }
    newc[v] = best;
    if (best != C && best != v) atomicMax(join + best, join_key(__dsub_rn(bestg, stay), v));
  }
}

// a proposed move happens when it is the best proposal into its target (at
// most one node joins a community per sub-round) and no node joins the
// mover's own community; a move to a new community always happens
__global__ void lm_apply(int32_t n, const int32_t *comm, const int32_t *newc, const int32_t *cnt,
                         const unsigned long long *join, int32_t *out, int32_t *moved) {
  for (int64_t vv = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; vv < n; vv += int64_t(gridDim.x) * blockDim.x) {
    const int32_t v = int32_t(vv), C = comm[v], D = newc[v];
    int32_t r = C;
    if (D != C) {
      if (D == v && cnt[v] == 0) r = D;
      else if (join[C] == 0 && (join[D] & 0xffffffffull) == 0xffffffffull - uint32_t(v)) r = D;
    }
    out[v] = r;
    if (r != C) atomicAdd(moved, 1);
  }
}

// refinement: E(s, C - s) for every sub-community s (edges inside the
// community leaving s)
__global__ void sub_external(DGraph g, const int32_t *comm, const int32_t *sub, int64_t *subE) {
  for (int64_t vv = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; vv < g.n;
       vv += int64_t(gridDim.x) * blockDim.x) {
    const int32_t v = int32_t(vv), C = comm[v], s = sub[v];
    int64_t x = 0;
    for (int64_t e = g.ptr[v]; e < g.ptr[v + 1]; ++e) {
      const int32_t u = g.adj[e];
      if (comm[u] == C && sub[u] != s) x += g.ew[e];
    }
    if (x) atomicAdd(reinterpret_cast<unsigned long long *>(subE + s), static_cast<unsigned long long>(x));
  }
}

__global__ void refine_decide(DGraph g, const int32_t *comm, const int64_t *W, const int32_t *sub, const int64_t *SW,
                              const int32_t *subN, const int64_t *subE, double gp, int dir, int32_t *newsub,
                              unsigned long long *join) {
  for (int64_t vv = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; vv < g.n;
       vv += int64_t(gridDim.x) * blockDim.x) {
    const int32_t v = int32_t(vv), C = comm[v];
    newsub[v] = sub[v];
    if (sub[v] != v || subN[v] != 1) continue;   // only singletons move
    const int64_t wv = g.vw[v], e0 = g.ptr[v], e1 = g.ptr[v + 1], WC = W[C];
    int64_t inside = 0;
    for (int64_t e = e0; e < e1; ++e)
      if (comm[g.adj[e]] == C) inside += g.ew[e];
    if (!(double(inside) >= penalty(gp, wv, WC - wv))) continue;   // not well connected
    int32_t best = v;
    double bestg = 0.0;
    bool found = false;
    for (int64_t e = e0; e < e1; ++e) {
      const int32_t u = g.adj[e];
      if (comm[u] != C) continue;
      const int32_t t = sub[u];
      if (t == v || (dir == 0 ? t > v : t < v)) continue;
      bool dup = false;
      for (int64_t f = e0; f < e && !dup; ++f) dup = comm[g.adj[f]] == C && sub[g.adj[f]] == t;
      if (dup) continue;
      if (!(double(subE[t]) >= penalty(gp, SW[t], WC - SW[t]))) continue;
      int64_t kt = g.ew[e];
      for (int64_t f = e + 1; f < e1; ++f)
        if (comm[g.adj[f]] == C && sub[g.adj[f]] == t) kt += g.ew[f];
      const double gt = leiden_gain(kt, wv, SW[t], gp);
      if (gt >= 0.0 && (!found || gt > bestg || (gt == bestg && t < best))) {
        best = t;
        bestg = gt;
        found = true;
      }
    }
    if (found) {
      newsub[v] = best;
      atomicMax(join + best, join_key(__dadd_rn(bestg, 1.0), v));
    }
  }
}

__global__ void refine_apply(int32_t n, const int32_t *sub, const int32_t *newsub, const unsigned long long *join,
                             int32_t *out, int32_t *moved) {
  for (int64_t vv = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; vv < n; vv += int64_t(gridDim.x) * blockDim.x) {
    const int32_t v = int32_t(vv), s0 = sub[v], t = newsub[v];
    int32_t r = s0;
    if (t != s0 && join[v] == 0 && (join[t] & 0xffffffffull) == 0xffffffffull - uint32_t(v)) r = t;
    out[v] = r;
    if (r != s0) atomicAdd(moved, 1);
  }
}

__global__ void iota_i32(int64_t n, int32_t *a) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    a[i] = int32_t(i);
}

__global__ void used_flags(int64_t n, const int32_t *cnt, int64_t *flag) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    flag[i] = cnt[i] > 0 ? 1 : 0;
}

__global__ void remap(int64_t n, int32_t *a, const int64_t *id) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    a[i] = int32_t(id[a[i]]);
}

// the aggregate's nodes: weights, starting communities (the unrefined ones)
__global__ void agg_nodes(int32_t n, const int32_t *grp, const int32_t *comm, const int64_t *vw, int64_t *vw2,
                          int32_t *comm2) {
  for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < n; v += int64_t(gridDim.x) * blockDim.x) {
    atomicAdd(reinterpret_cast<unsigned long long *>(vw2 + grp[v]), static_cast<unsigned long long>(vw[v]));
    comm2[grp[v]] = comm[v];   // equal for every member
  }
}

__global__ void agg_keys(DGraph g, const int32_t *grp, uint64_t K, const int32_t *erow, uint64_t *key, int32_t *idx) {
  const uint64_t none = K * K;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < g.m; e += int64_t(gridDim.x) * blockDim.x) {
    const int32_t a = grp[erow[e]], b = grp[g.adj[e]];
    key[e] = a == b ? none : uint64_t(a) * K + uint64_t(b);
    idx[e] = int32_t(e);
  }
}

__global__ void agg_emit(int64_t m, const uint64_t *key, const int32_t *idx, const int64_t *flag, const int64_t *pos,
                         uint64_t K, const int64_t *ew, int32_t *adj2, int64_t *ew2, int64_t *rowcnt) {
  const uint64_t none = K * K;
  for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < m; k += int64_t(gridDim.x) * blockDim.x) {
    if (key[k] == none) continue;
    const int64_t s = pos[k] + flag[k] - 1;
    atomicAdd(reinterpret_cast<unsigned long long *>(ew2 + s), static_cast<unsigned long long>(ew[idx[k]]));
    if (flag[k]) {
      adj2[s] = int32_t(key[k] % K);
      atomicAdd(reinterpret_cast<unsigned long long *>(rowcnt + key[k] / K), 1ull);
    }
  }
}

__global__ void compose(int64_t n, int32_t *where, const int32_t *grp) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    where[i] = grp[where[i]];
}

__global__ void gather_i32(int64_t n, const int32_t *where, const int32_t *val, int32_t *out) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    out[i] = val[where[i]];
}

// connected components inside communities: min-label propagation with
// pointer jumping
__global__ void cc_hook(int32_t n, const int64_t *gptr, const int32_t *gadj, const int32_t *memb, int32_t *lab,
                        int32_t *changed) {
  for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < n; v += int64_t(gridDim.x) * blockDim.x) {
    int32_t l = lab[v];
    for (int64_t e = gptr[v]; e < gptr[v + 1]; ++e) {
      const int32_t u = gadj[e];
      if (memb[u] == memb[v]) l = min(l, lab[u]);
    }
    if (l < lab[v]) {
      atomicMin(lab + v, l);
      *changed = 1;
    }
  }
}

__global__ void cc_jump(int32_t n, int32_t *lab) {
  for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < n; v += int64_t(gridDim.x) * blockDim.x)
    lab[v] = lab[lab[v]];
}

__global__ void count_labels(int64_t n, const int32_t *lab, int32_t *cnt) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    atomicAdd(cnt + lab[i], 1);
}

constexpr int kSubRounds = 128;   // local-moving / refinement sub-rounds per level (bound)

struct LeidenRun {
  Scratch &S;
  cudaStream_t s;
  double gp;
  cudaError_t e = cudaSuccess;
  int32_t *dmoved = nullptr;

  int32_t read_i32(const int32_t *d) {
    int32_t h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return h;
  }
  template <typename... KA, typename... A>
  void go(void (*k)(KA...), int64_t work, A... args) {
    if (e != cudaSuccess || work <= 0) return;
    k<<<grid_for(work), kT, 0, s>>>(args...);
    e = cudaGetLastError();
  }

  // community weights and member counts of `comm` on g
  void weights(const DGraph &g, const int32_t *comm, int64_t *W, int32_t *cnt) {
    if (e == cudaSuccess) e = cudaMemsetAsync(W, 0, size_t(g.n) * sizeof(int64_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, size_t(g.n) * sizeof(int32_t), s);
    go(community_weights, g.n, g.n, comm, g.vw, W, cnt);
  }

  // relabels a[0..n) (labels < n, counts cnt) to 0..K-1; returns K
  int32_t compact(int64_t n, int32_t *a, const int32_t *cnt) {
    int64_t *flag = S.get<int64_t>(size_t(n) + 1);
    int64_t *tot = S.get<int64_t>(1);
    if (S.err != cudaSuccess) { e = S.err; return 0; }
    go(used_flags, n, n, cnt, flag);
    if (e == cudaSuccess) e = scan(flag, flag, n, S, tot);
    go(remap, n, n, a, flag);
    int64_t h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return int32_t(h);
  }

  void move_nodes(const DGraph &g, int32_t *comm, int64_t *W, int32_t *cnt, int32_t *tmp) {
    unsigned long long *join = S.get<unsigned long long>(size_t(g.n));
    int32_t *out = S.get<int32_t>(size_t(g.n));
    if (S.err != cudaSuccess) { e = S.err; return; }
    int idle = 0;
    for (int r = 0; r < kSubRounds && idle < 2 && e == cudaSuccess; ++r) {
      weights(g, comm, W, cnt);
      if (e == cudaSuccess) e = cudaMemsetAsync(dmoved, 0, sizeof(int32_t), s);
      if (e == cudaSuccess) e = cudaMemsetAsync(join, 0, size_t(g.n) * sizeof(unsigned long long), s);
      go(lm_decide, g.n, g, comm, W, cnt, gp, r & 1, tmp, join);
      go(lm_apply, g.n, g.n, comm, tmp, cnt, join, out, dmoved);
      if (e == cudaSuccess) e = cudaMemcpyAsync(comm, out, size_t(g.n) * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
      idle = read_i32(dmoved) == 0 ? idle + 1 : 0;
    }
    weights(g, comm, W, cnt);
  }

  void refine(const DGraph &g, const int32_t *comm, const int64_t *W, int32_t *sub, int64_t *SW, int32_t *subN,
              int64_t *subE, int32_t *tmp) {
    go(iota_i32, g.n, int64_t(g.n), sub);
    unsigned long long *join = S.get<unsigned long long>(size_t(g.n));
    int32_t *out = S.get<int32_t>(size_t(g.n));
    if (S.err != cudaSuccess) { e = S.err; return; }
    int idle = 0;
    for (int r = 0; r < kSubRounds && idle < 2 && e == cudaSuccess; ++r) {
      weights(g, sub, SW, subN);
      if (e == cudaSuccess) e = cudaMemsetAsync(subE, 0, size_t(g.n) * sizeof(int64_t), s);
      go(sub_external, g.n, g, comm, sub, subE);
      if (e == cudaSuccess) e = cudaMemsetAsync(dmoved, 0, sizeof(int32_t), s);
      if (e == cudaSuccess) e = cudaMemsetAsync(join, 0, size_t(g.n) * sizeof(unsigned long long), s);
      go(refine_decide, g.n, g, comm, W, sub, SW, subN, subE, gp, r & 1, tmp, join);
      go(refine_apply, g.n, g.n, sub, tmp, join, out, dmoved);
      if (e == cudaSuccess) e = cudaMemcpyAsync(sub, out, size_t(g.n) * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
      idle = read_i32(dmoved) == 0 ? idle + 1 : 0;
    }
  }

  // the aggregate of g by grp (labels 0..K-1)
  DGraph aggregate(const DGraph &g, const int32_t *grp, int32_t K, const int32_t *comm, int32_t *comm2) {
    DGraph a;
    a.n = K;
    a.ptr = S.get<int64_t>(size_t(K) + 1);
    a.vw = S.get<int64_t>(size_t(K));
    int32_t *erow = S.get<int32_t>(size_t(g.m));
    uint64_t *key = S.get<uint64_t>(size_t(g.m));
    int32_t *idx = S.get<int32_t>(size_t(g.m));
    int64_t *flag = S.get<int64_t>(size_t(g.m) + 1);
    int64_t *pos = S.get<int64_t>(size_t(g.m) + 1);
    int64_t *rowcnt = S.get<int64_t>(size_t(K) + 1);
    a.adj = S.get<int32_t>(size_t(g.m));
    a.ew = S.get<int64_t>(size_t(g.m));
    int64_t *tot = S.get<int64_t>(1);
    if (S.err != cudaSuccess) { e = S.err; return a; }
    if (e == cudaSuccess) e = cudaMemsetAsync(a.vw, 0, size_t(K) * sizeof(int64_t), s);
    go(agg_nodes, g.n, g.n, grp, comm, g.vw, a.vw, comm2);
    go(edge_rows_unchecked, g.n, g.n, g.ptr, erow);
    go(agg_keys, g.m, g, grp, uint64_t(K), erow, key, idx);
    if (e == cudaSuccess) e = radix_sort(key, idx, g.m, bits_for(uint64_t(K) * uint64_t(K)), S);
    go(unique_flags, g.m, key, g.m, uint64_t(K) * uint64_t(K), flag);
    if (e == cudaSuccess) e = cudaMemcpyAsync(pos, flag, size_t(g.m) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = scan(pos, pos, g.m, S);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.ew, 0, size_t(std::max<int64_t>(g.m, 1)) * sizeof(int64_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(rowcnt, 0, (size_t(K) + 1) * sizeof(int64_t), s);
    go(agg_emit, g.m, g.m, key, idx, flag, pos, uint64_t(K), g.ew, a.adj, a.ew, rowcnt);
    if (e == cudaSuccess) e = scan(rowcnt, a.ptr, int64_t(K) + 1, S, tot);
    int64_t hm = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hm, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    a.m = hm;
    return a;
  }

  // one multilevel pass from memb (labels on g0's nodes, < n); memb is
  // overwritten with the result's labels (compacted)
  void pass(const DGraph &g0, int32_t *memb) {
    const int32_t n0 = g0.n;
    int32_t *where = S.get<int32_t>(size_t(n0));
    if (S.err != cudaSuccess) { e = S.err; return; }
    go(iota_i32, n0, int64_t(n0), where);
    DGraph g = g0;
    int32_t *comm = S.get<int32_t>(size_t(n0));
    if (S.err != cudaSuccess) { e = S.err; return; }
    if (e == cudaSuccess) e = cudaMemcpyAsync(comm, memb, size_t(n0) * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    for (int level = 0; level < 64 && e == cudaSuccess; ++level) {
      const int32_t n = g.n;
      int64_t *W = S.get<int64_t>(size_t(n));
      int32_t *cnt = S.get<int32_t>(size_t(n));
      int32_t *tmp = S.get<int32_t>(size_t(n));
      int32_t *sub = S.get<int32_t>(size_t(n));
      int64_t *SW = S.get<int64_t>(size_t(n));
      int32_t *subN = S.get<int32_t>(size_t(n));
      int64_t *subE = S.get<int64_t>(size_t(n));
      if (S.err != cudaSuccess) { e = S.err; return; }
      move_nodes(g, comm, W, cnt, tmp);
      // communities after local moving
      if (e == cudaSuccess) e = cudaMemcpyAsync(tmp, comm, size_t(n) * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
      const int32_t ncomm = compact(n, tmp, cnt);
      if (e != cudaSuccess || ncomm == n) break;   // every node alone: done
      if (e == cudaSuccess) e = cudaMemcpyAsync(comm, tmp, size_t(n) * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
      weights(g, comm, W, cnt);
      refine(g, comm, W, sub, SW, subN, subE, tmp);
      weights(g, sub, SW, subN);
      int32_t K = compact(n, sub, subN);
      int32_t *comm2 = nullptr;
      if (K == n) {
        // the refinement merged nothing: aggregate on the communities
        if (e == cudaSuccess) e = cudaMemcpyAsync(sub, comm, size_t(n) * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
        K = ncomm;
        comm2 = S.get<int32_t>(size_t(K));
        DGraph a = aggregate(g, sub, K, comm, comm2);
        go(iota_i32, K, int64_t(K), comm2);
        go(compose, n0, int64_t(n0), where, sub);
        g = a;
      } else {
        comm2 = S.get<int32_t>(size_t(K));
        DGraph a = aggregate(g, sub, K, comm, comm2);
        go(compose, n0, int64_t(n0), where, sub);
        g = a;
      }
      if (S.err != cudaSuccess) { e = S.err; return; }
      comm = comm2;
    }
    // the result on g0's nodes
    go(gather_i32, n0, int64_t(n0), where, comm, memb);
    int32_t *cnt0 = S.get<int32_t>(size_t(n0));
    if (S.err != cudaSuccess) { e = S.err; return; }
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt0, 0, size_t(n0) * sizeof(int32_t), s);
    go(count_labels, n0, int64_t(n0), memb, cnt0);
    compact(n0, memb, cnt0);
  }
};

iccg_status status_of(cudaError_t e) { return e == cudaSuccess ? ICCG_OK : ICCG_ERR_CUDA; }

iccg_status read_flag(int *bad, Scratch &S, cudaError_t e) {
  if (e != cudaSuccess) return ICCG_ERR_CUDA;
  int h = 0;
  e = cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, S.s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(S.s);
  if (e != cudaSuccess) return ICCG_ERR_CUDA;
  return h ? ICCG_ERR_ARG : ICCG_OK;
}

}  // namespace iccg_dev

using namespace iccg_dev;

extern "C" iccg_status iccg_dev_graph(int32_t n, const int64_t *rowptr, const int32_t *colind, int64_t nnz,
                                      int64_t *gptr, int32_t *gadj, int64_t *m, iccg_stream_t stream) {
  if (n < 0 || nnz < 0 || !rowptr || !gptr || !m || (nnz > 0 && (!colind || !gadj))) return ICCG_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Scratch S(s);
  const int64_t np = 2 * nnz;
  uint64_t *key = S.get<uint64_t>(size_t(np));
  int *bad = S.get<int>(1);
  if (S.err != cudaSuccess) return ICCG_ERR_CUDA;
  cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int), s);
  if (e == cudaSuccess && n > 0) {
    graph_pairs<<<grid_for(n), kT, 0, s>>>(n, nnz, rowptr, colind, key, bad);
    e = cudaGetLastError();
  }
  iccg_status st = read_flag(bad, S, e);
  if (st != ICCG_OK) return st;
  return status_of(pairs_to_csr(key, np, uint64_t(n), uint64_t(n), gptr, gadj, m, S));
}

extern "C" iccg_status iccg_dev_color_order(int32_t n, const int64_t *gptr, const int32_t *gadj, int64_t m,
                                            int32_t n_b, const int32_t *block_of, int32_t *color_of, int32_t *n_c,
                                            int32_t *perm, int32_t *block_ptr, int32_t *color_ptr,
                                            iccg_stream_t stream) {
  if (n < 0 || n_b < 0 || m < 0 || !gptr || !block_of || !color_of || !n_c || !perm || !block_ptr || !color_ptr ||
      (m > 0 && !gadj))
    return ICCG_ERR_ARG;
  if (n_b == 0 && n > 0) return ICCG_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Scratch S(s);
  int *bad = S.get<int>(1);
  int32_t *row = S.get<int32_t>(size_t(m));
  uint64_t *key = S.get<uint64_t>(size_t(std::max<int64_t>(m, n)));
  int64_t *bptr = S.get<int64_t>(size_t(n_b) + 1);
  int32_t *badj = S.get<int32_t>(size_t(m));
  int32_t *lower = S.get<int32_t>(size_t(n_b));
  int32_t *waves = S.get<int32_t>(2 * size_t(n_b));
  int32_t *cnts = S.get<int32_t>(4);   // wave sizes (2), number of colors
  if (S.err != cudaSuccess) return ICCG_ERR_CUDA;
  cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int), s);
  if (e == cudaSuccess && n > 0) {
    check_blocks<<<grid_for(n), kT, 0, s>>>(n, block_of, n_b, bad);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && n > 0) {
    edge_rows<<<grid_for(n), kT, 0, s>>>(n, m, gptr, gadj, row, bad);
    e = cudaGetLastError();
  }
  iccg_status st = read_flag(bad, S, e);
  if (st != ICCG_OK) return st;
  if (m > 0) {
    block_pairs<<<grid_for(m), kT, 0, s>>>(m, row, gadj, block_of, n_b, key, bad);
    e = cudaGetLastError();
  }
  st = read_flag(bad, S, e);
  if (st != ICCG_OK) return st;
  int64_t mb = 0;
  e = pairs_to_csr(key, m, uint64_t(n_b), uint64_t(n_b), bptr, badj, &mb, S);
  // waves of the exact greedy coloring
  if (e == cudaSuccess) e = cudaMemsetAsync(cnts, 0, 4 * sizeof(int32_t), s);
  if (e == cudaSuccess && n_b > 0) {
    lower_counts<<<grid_for(n_b), kT, 0, s>>>(n_b, bptr, badj, lower, waves, cnts, color_of);
    e = cudaGetLastError();
  }
  int32_t h[4] = {0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, cnts, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  int cur = 0, done = 0;
  int32_t nw = h[0];
  while (e == cudaSuccess && nw > 0) {
    const int nx = cur ^ 1;
    e = cudaMemsetAsync(cnts + nx, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) break;
    color_wave<<<grid_for(nw), kT, 0, s>>>(waves + size_t(cur) * size_t(n_b), nw, bptr, badj, lower, color_of,
                                           waves + size_t(nx) * size_t(n_b), cnts + nx, cnts + 2);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h[nx], cnts + nx, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    done += nw;
    nw = h[nx];
    cur = nx;
  }
  if (e == cudaSuccess && done != n_b) return ICCG_ERR_CUDA;   // every block is colored exactly once
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h[2], cnts + 2, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return ICCG_ERR_CUDA;
  const int32_t ncol = h[2];
  *n_c = ncol;
  // blocks ordered by (color, index): a stable sort by color
  int32_t *order = S.get<int32_t>(size_t(n_b));
  int32_t *rank = S.get<int32_t>(size_t(n_b));
  int32_t *ccnt = S.get<int32_t>(size_t(ncol) + 1);
  int64_t *c64 = S.get<int64_t>(size_t(ncol) + 1);
  int64_t *bsz = S.get<int64_t>(size_t(n_b) + 1);
  int32_t *rv = S.get<int32_t>(size_t(n));
  if (S.err != cudaSuccess) return ICCG_ERR_CUDA;
  if (n_b > 0) {
    keys_from<<<grid_for(n_b), kT, 0, s>>>(n_b, color_of, key, order);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = radix_sort(key, order, n_b, bits_for(uint64_t(ncol)), S);
  if (e == cudaSuccess) e = cudaMemsetAsync(ccnt, 0, (size_t(ncol) + 1) * sizeof(int32_t), s);
  if (e == cudaSuccess && n_b > 0) {
    block_rank_size<<<grid_for(n_b), kT, 0, s>>>(n_b, order, rank, color_of, ccnt);
    e = cudaGetLastError();
  }
  // color_ptr = scan of the per-color block counts
  if (e == cudaSuccess) {
    i32_to_i64<<<grid_for(ncol + 1), kT, 0, s>>>(ncol + 1, ccnt, c64);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = scan(c64, c64, int64_t(ncol) + 1, S);
  if (e == cudaSuccess) {
    to_i32<<<grid_for(ncol + 1), kT, 0, s>>>(ncol + 1, c64, color_ptr);
    e = cudaGetLastError();
  }
  // rows ordered by (block rank, row): a stable sort by rank; block sizes
  if (e == cudaSuccess) e = cudaMemsetAsync(bsz, 0, (size_t(n_b) + 1) * sizeof(int64_t), s);
  if (e == cudaSuccess && n > 0) {
    row_keys<<<grid_for(n), kT, 0, s>>>(n, block_of, rank, key, rv, bsz);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = radix_sort(key, rv, n, bits_for(uint64_t(n_b)), S);
  if (e == cudaSuccess && n > 0) e = cudaMemcpyAsync(perm, rv, size_t(n) * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = scan(bsz, bsz, int64_t(n_b) + 1, S);
  if (e == cudaSuccess) {
    to_i32<<<grid_for(n_b + 1), kT, 0, s>>>(int64_t(n_b) + 1, bsz, block_ptr);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return status_of(e);
}

extern "C" iccg_status iccg_dev_sort_blocks_desc(int32_t n, int32_t n_b, int32_t *block_of, iccg_stream_t stream) {
  if (n < 0 || n_b < 0 || (n > 0 && !block_of) || (n > 0 && n_b == 0)) return ICCG_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Scratch S(s);
  int *bad = S.get<int>(1);
  int32_t *size = S.get<int32_t>(size_t(n_b));
  int32_t *first = S.get<int32_t>(size_t(n_b));
  uint64_t *key = S.get<uint64_t>(size_t(n_b));
  int32_t *order = S.get<int32_t>(size_t(n_b));
  int32_t *rank = S.get<int32_t>(size_t(n_b));
  if (S.err != cudaSuccess) return ICCG_ERR_CUDA;
  cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int), s);
  if (e == cudaSuccess && n > 0) {
    check_blocks<<<grid_for(n), kT, 0, s>>>(n, block_of, n_b, bad);
    e = cudaGetLastError();
  }
  iccg_status st = read_flag(bad, S, e);
  if (st != ICCG_OK || n == 0) return st;
  e = cudaMemsetAsync(size, 0, size_t(n_b) * sizeof(int32_t), s);
  if (e == cudaSuccess) {
    fill_i32<<<grid_for(n_b), kT, 0, s>>>(n_b, first, n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    size_first<<<grid_for(n), kT, 0, s>>>(n, block_of, size, first);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    size_keys<<<grid_for(n_b), kT, 0, s>>>(n_b, n, size, first, key, order);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = radix_sort(key, order, n_b, bits_for(uint64_t(n) * uint64_t(n + 1) + uint64_t(n)), S);
  if (e == cudaSuccess) {
    rank_of<<<grid_for(n_b), kT, 0, s>>>(n_b, order, rank);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    relabel<<<grid_for(n), kT, 0, s>>>(n, block_of, rank);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return status_of(e);
}

extern "C" iccg_status iccg_dev_block_leiden(int32_t n, const int64_t *gptr, const int32_t *gadj, int64_t m,
                                             int32_t quality, double gamma, int32_t n_iter, int32_t *block_of,
                                             int32_t *n_b, iccg_stream_t stream) {
  if (n < 0 || m < 0 || !gptr || !block_of || !n_b || (m > 0 && !gadj) || (quality != 0 && quality != 1) ||
      !(gamma >= 0.0) || n_iter < 0)
    return ICCG_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Scratch S(s);
  int *bad = S.get<int>(1);
  int32_t *row = S.get<int32_t>(size_t(m));
  DGraph g;
  g.n = n;
  g.m = m;
  g.ptr = const_cast<int64_t *>(gptr);
  g.adj = const_cast<int32_t *>(gadj);
  g.ew = S.get<int64_t>(size_t(m));
  g.vw = S.get<int64_t>(size_t(n));
  int32_t *moved = S.get<int32_t>(2);
  if (S.err != cudaSuccess) return ICCG_ERR_CUDA;
  if (n == 0) {
    *n_b = 0;
    return ICCG_OK;
  }
  cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    edge_rows<<<grid_for(n), kT, 0, s>>>(n, m, gptr, gadj, row, bad);
    e = cudaGetLastError();
  }
  iccg_status st = read_flag(bad, S, e);
  if (st != ICCG_OK) return st;
  init_unit_graph<<<grid_for(std::max<int64_t>(n, m)), kT, 0, s>>>(n, gptr, m, g.ew, g.vw, quality);
  e = cudaGetLastError();
  LeidenRun L{S, s, quality == 1 ? gamma : (m > 0 ? gamma / double(m) : 0.0)};
  L.e = e;
  L.dmoved = moved;
  L.go(iota_i32, n, int64_t(n), block_of);
  for (int it = 0; it < n_iter && L.e == cudaSuccess; ++it) L.pass(g, block_of);
  e = L.e;
  // connected components inside every community
  int32_t *lab = S.get<int32_t>(size_t(n));
  int32_t *cnt = S.get<int32_t>(size_t(n));
  if (S.err != cudaSuccess) return ICCG_ERR_CUDA;
  L.go(iota_i32, n, int64_t(n), lab);
  for (int r = 0; r < n && L.e == cudaSuccess; ++r) {
    if (L.e == cudaSuccess) L.e = cudaMemsetAsync(moved, 0, sizeof(int32_t), s);
    L.go(cc_hook, n, n, gptr, gadj, block_of, lab, moved);
    for (int j = 0; j < 4; ++j) L.go(cc_jump, n, n, lab);
    if (L.read_i32(moved) == 0) break;
  }
  if (L.e == cudaSuccess) L.e = cudaMemsetAsync(cnt, 0, size_t(n) * sizeof(int32_t), s);
  L.go(count_labels, n, int64_t(n), lab, cnt);
  const int32_t nb = L.compact(n, lab, cnt);
  if (L.e == cudaSuccess) L.e = cudaMemcpyAsync(block_of, lab, size_t(n) * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
  if (L.e == cudaSuccess) L.e = cudaStreamSynchronize(s);
  if (L.e != cudaSuccess) return ICCG_ERR_CUDA;
  *n_b = nb;
  return ICCG_OK;
}
