// iccg_spmv_dot_noalloc: q = A p and <p, q> without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need a
// sparse product: latency-critical loops that must not pay for the
// allocator's implicit device synchronisation, and host frameworks that own
// all device memory through their own pool and forbid raw cudaMalloc (an
// allocation behind their back would break their accounting or fail under
// their memory cap).  This entry point serves them: the caller passes every
// input and output as device pointers, and the only scratch the kernel needs
// (one partial sum per CTA plus the arrival counters of the deterministic
// two-level reduction) lives in a fixed file-scope __device__ array.
//
// That array is part of the module: every GPU that loads the library holds
// it until the process exits.  All calls share it, and it keeps the contents
// of the last call, so the counters that must start at zero are cleared at
// the start of every call (a memset on the caller's stream, not an
// allocation).  Two calls whose kernels overlap on the GPU (different streams,
// or different host threads) race on the array and give wrong results.
//
// The first call on each device looks up the array's device address with
// cudaGetSymbolAddress (with that device current) and caches it.  The stream
// must belong to the current device (the cached address is that device's
// copy of the array).
#include <mutex>

#include "iccg_internal.h"

namespace {

constexpr int kNaWarps = 8;                       // warps per CTA
constexpr int kNaRowsPerCta = kNaWarps * 32;      // one row per lane
constexpr int kNaMaxCtas = ICCG_NOALLOC_MAX_ROWS / kNaRowsPerCta;
constexpr int kNaGroup = 32;                      // CTAs per first-level group
constexpr int kNaMaxGroups = kNaMaxCtas / kNaGroup;

struct NaScratch {
  double part[kNaMaxCtas];        // per-CTA partial of <p, q>
  double gsum[kNaMaxGroups];      // per-group sums
  unsigned int gticket[kNaMaxGroups];
  unsigned int ticket;            // groups finished
};

static_assert(kNaMaxCtas * kNaRowsPerCta == ICCG_NOALLOC_MAX_ROWS, "row limit must split into CTAs");

static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NaScratch)];

__device__ __forceinline__ double na_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// one value per thread -> thread 0, fixed order
__device__ __forceinline__ double na_cta_sum(double v, double *red) {
  v = na_warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < int(blockDim.x >> 5); ++k) s += red[k];
  return s;
}

__device__ __forceinline__ bool na_last(unsigned int *ticket, unsigned int expected, int *flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    *flag = atomicAdd(ticket, 1u) == expected - 1 ? 1 : 0;
    if (*flag) __threadfence();
  }
  __syncthreads();
  return *flag != 0;
}

__global__ void __launch_bounds__(kNaRowsPerCta)
spmv_dot_noalloc_kernel(int n, const int64_t *__restrict__ rowptr, const int32_t *__restrict__ colind,
                        const double *__restrict__ val, const double *__restrict__ p, double *__restrict__ q,
                        double *__restrict__ pq, NaScratch *s) {
  __shared__ double red[kNaWarps];
  __shared__ int flag;
  const int i = blockIdx.x * kNaRowsPerCta + threadIdx.x;
  double acc = 0.0;
  if (i < n) {
    double sum = 0.0;
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) sum += val[e] * p[colind[e]];
    q[i] = sum;
    acc = p[i] * sum;
  }
  const double cta = na_cta_sum(acc, red);
  const int g = blockIdx.x / kNaGroup;
  const int g0 = g * kNaGroup;
  const int gs = min(kNaGroup, int(gridDim.x) - g0);
  if (threadIdx.x == 0) s->part[blockIdx.x] = cta;
  if (!na_last(&s->gticket[g], unsigned(gs), &flag)) return;
  const double gv = na_cta_sum(threadIdx.x < gs ? __ldcg(&s->part[g0 + threadIdx.x]) : 0.0, red);
  if (threadIdx.x == 0) s->gsum[g] = gv;
  const unsigned ng = (gridDim.x + kNaGroup - 1) / kNaGroup;
  if (!na_last(&s->ticket, ng, &flag)) return;
  double t = 0.0;
  for (unsigned k = threadIdx.x; k < ng; k += blockDim.x) t += __ldcg(&s->gsum[k]);
  const double total = na_cta_sum(t, red);
  if (threadIdx.x == 0) *pq = total;
}

std::mutex g_na_mutex;
NaScratch *g_na_ptr[64] = {nullptr};

}  // namespace

extern "C" iccg_status iccg_spmv_dot_noalloc(int32_t n, const int64_t *rowptr, const int32_t *colind,
                                             const double *val, const double *p, double *q, double *pq,
                                             iccg_stream_t stream) {
  if (n < 0 || n > ICCG_NOALLOC_MAX_ROWS) return ICCG_ERR_ARG;
  if (!pq || (n > 0 && (!rowptr || !colind || !val || !p || !q))) return ICCG_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return ICCG_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the scratch address below is the current device's copy: a stream of
  // another device would run the kernel against the wrong GPU's memory
  int sdev = -1;
  if (cudaStreamGetDevice(st, &sdev) != cudaSuccess) return ICCG_ERR_ARG;
  if (sdev != dev) return ICCG_ERR_ARG;
  NaScratch *s = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_na_mutex);
    if (!g_na_ptr[dev]) {
      void *addr = nullptr;
      if (cudaGetSymbolAddress(&addr, g_noalloc_scratch) != cudaSuccess || !addr) return ICCG_ERR_CUDA;
      g_na_ptr[dev] = static_cast<NaScratch *>(addr);
    }
    s = g_na_ptr[dev];
  }
  if (n == 0) return cudaMemsetAsync(pq, 0, sizeof(double), st) == cudaSuccess ? ICCG_OK : ICCG_ERR_CUDA;
  const int grid = (n + kNaRowsPerCta - 1) / kNaRowsPerCta;
  const int ngroups = (grid + kNaGroup - 1) / kNaGroup;
  // the arrival counters must start at zero; the previous call left them at
  // their final counts
  if (cudaMemsetAsync(s->gticket, 0, sizeof(unsigned int) * size_t(ngroups), st) != cudaSuccess ||
      cudaMemsetAsync(&s->ticket, 0, sizeof(unsigned int), st) != cudaSuccess)
    return ICCG_ERR_CUDA;
  // the launch's own status (cudaGetLastError would also report, and clear,
  // an error that earlier unrelated work of the caller left pending)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(grid));
  cfg.blockDim = dim3(unsigned(kNaRowsPerCta));
  cfg.stream = st;
  return cudaLaunchKernelEx(&cfg, spmv_dot_noalloc_kernel, n, rowptr, colind, val, p, q, pq, s) == cudaSuccess
             ? ICCG_OK
             : ICCG_ERR_CUDA;
}
