// MLP of the learned blocking: forward pass, loss gradient and Adam step as
// plain CUDA kernels (FP32; the network has ~6k parameters and batches of a
// few hundred matrices, so one thread per output element is the whole
// mapping; no tensor cores).  Layout of the flat parameter array:
//   W1 [nf][h], b1 [h], W2 [h][h], b2 [h], W3 [h][c+1], b3 [c+1]
// (c = ncls; the last output is the regression head).  Every sum runs in a
// fixed order, so results do not depend on the launch shape.
#include <cmath>

#include "iccg_internal.h"

namespace iccg {
namespace {

constexpr int kMlpThreads = 128;

struct MlpOff {
  int64_t w1, b1, w2, b2, w3, b3, total;
};

MlpOff mlp_off(int nf, int h, int c) {
  MlpOff o;
  o.w1 = 0;
  o.b1 = o.w1 + int64_t(nf) * h;
  o.w2 = o.b1 + h;
  o.b2 = o.w2 + int64_t(h) * h;
  o.w3 = o.b2 + h;
  o.b3 = o.w3 + int64_t(h) * (c + 1);
  o.total = o.b3 + (c + 1);
  return o;
}

int blocks_for(int64_t n) { return int((n + kMlpThreads - 1) / kMlpThreads); }

// out[b][o] = act(sum_i in[b][i] W[i][o] + bias[o]), i ascending
__global__ void dense_fwd(const float *in, int nin, const float *W, const float *bias, int nout, int batch,
                          float *out, int relu) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= batch * nout) return;
  const int b = idx / nout, o = idx % nout;
  float s = bias[o];
  for (int i = 0; i < nin; ++i) s = fmaf(in[b * nin + i], W[i * nout + o], s);
  out[idx] = relu ? fmaxf(s, 0.0f) : s;
}

// per sample: softmax cross entropy of z[b][0:c] against y[b] plus
// wreg (z[b][c] - yreg[b])^2; dz = d(loss / batch) / dz; lb[b] = sample loss
__global__ void head_grad(const float *z, int c, const int32_t *y, const float *yreg, float wreg, int batch,
                          float *dz, float *lb) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  const float *zb = z + b * (c + 1);
  float *db = dz + b * (c + 1);
  float mx = zb[0];
  for (int k = 1; k < c; ++k) mx = fmaxf(mx, zb[k]);
  float se = 0.0f;
  for (int k = 0; k < c; ++k) se += expf(zb[k] - mx);
  const float inv_b = 1.0f / float(batch);
  const int yb = y[b];
  for (int k = 0; k < c; ++k) {
    const float p = expf(zb[k] - mx) / se;
    db[k] = (p - (k == yb ? 1.0f : 0.0f)) * inv_b;
  }
  const float err = zb[c] - yreg[b];
  db[c] = 2.0f * wreg * err * inv_b;
  lb[b] = (logf(se) + mx - zb[yb]) + wreg * err * err;
}

__global__ void loss_sum(const float *lb, int batch, float *loss) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    float s = 0.0f;
    for (int b = 0; b < batch; ++b) s += lb[b];
    *loss = s / float(batch);
  }
}

// gW[i][o] = sum_b in[b][i] d[b][o]; gb[o] = sum_b d[b][o] (b ascending)
__global__ void dense_wgrad(const float *in, int nin, const float *d, int nout, int batch, float *gW, float *gb) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < nin * nout) {
    const int i = idx / nout, o = idx % nout;
    float s = 0.0f;
    for (int b = 0; b < batch; ++b) s = fmaf(in[b * nin + i], d[b * nout + o], s);
    gW[idx] = s;
  } else if (idx < nin * nout + nout) {
    const int o = idx - nin * nout;
    float s = 0.0f;
    for (int b = 0; b < batch; ++b) s += d[b * nout + o];
    gb[o] = s;
  }
}

// dx[b][i] = (sum_o d[b][o] W[i][o]) * (act[b][i] > 0), o ascending
__global__ void dense_bwd_in(const float *d, const float *W, int nin, int nout, const float *act, int batch,
                             float *dx) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= batch * nin) return;
  const int b = idx / nin, i = idx % nin;
  float s = 0.0f;
  for (int o = 0; o < nout; ++o) s = fmaf(d[b * nout + o], W[i * nout + o], s);
  dx[idx] = act[idx] > 0.0f ? s : 0.0f;
}

__global__ void adam_step(float *p, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2,
                          float eps, float c1, float c2) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float gk = g[k];
  const float mk = b1 * m[k] + (1.0f - b1) * gk;
  const float vk = b2 * v[k] + (1.0f - b2) * gk * gk;
  m[k] = mk;
  v[k] = vk;
  p[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
}

bool shape_ok(int nf, int h, int c, int batch) {
  return nf >= 1 && h >= 1 && c >= 1 && batch >= 1 && nf <= 4096 && h <= 4096 && c <= 4096 &&
         int64_t(batch) * std::max(std::max(nf, h), c + 1) < (int64_t(1) << 31);
}

iccg_status launched(cudaError_t e) { return e == cudaSuccess ? ICCG_OK : ICCG_ERR_CUDA; }

void forward(const float *P, int nf, int h, int c, const float *X, int batch, float *h1, float *h2, float *z,
             cudaStream_t s) {
  const MlpOff o = mlp_off(nf, h, c);
  dense_fwd<<<blocks_for(int64_t(batch) * h), kMlpThreads, 0, s>>>(X, nf, P + o.w1, P + o.b1, h, batch, h1, 1);
  dense_fwd<<<blocks_for(int64_t(batch) * h), kMlpThreads, 0, s>>>(h1, h, P + o.w2, P + o.b2, h, batch, h2, 1);
  dense_fwd<<<blocks_for(int64_t(batch) * (c + 1)), kMlpThreads, 0, s>>>(h2, h, P + o.w3, P + o.b3, c + 1, batch, z,
                                                                          0);
}

}  // namespace
}  // namespace iccg

using namespace iccg;

extern "C" {

int64_t iccg_mlp_nparams(int32_t nf, int32_t hidden, int32_t ncls) {
  if (nf < 1 || hidden < 1 || ncls < 1) return -1;
  return mlp_off(nf, hidden, ncls).total;
}

iccg_status iccg_mlp_forward(const float *params, int32_t nf, int32_t hidden, int32_t ncls, const float *X,
                             int32_t batch, float *out, float *act, iccg_stream_t stream) {
  if (!params || !X || !out || !shape_ok(nf, hidden, ncls, batch)) return ICCG_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float *h1 = act, *tmp = nullptr;
  if (!h1) {
    if (cudaMallocAsync(reinterpret_cast<void **>(&tmp), sizeof(float) * 2 * size_t(batch) * hidden, s) != cudaSuccess)
      return ICCG_ERR_CUDA;
    h1 = tmp;
  }
  forward(params, nf, hidden, ncls, X, batch, h1, h1 + size_t(batch) * hidden, out, s);
  cudaError_t e = cudaGetLastError();
  if (tmp) cudaFreeAsync(tmp, s);
  return launched(e);
}

iccg_status iccg_mlp_grad(const float *params, int32_t nf, int32_t hidden, int32_t ncls, const float *X,
                          const int32_t *ycls, const float *yreg, float wreg, int32_t batch, float *grad,
                          float *loss, float *work, iccg_stream_t stream) {
  if (!params || !X || !ycls || !yreg || !grad || !loss || !work || !shape_ok(nf, hidden, ncls, batch))
    return ICCG_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int h = hidden, c = ncls;
  const size_t B = size_t(batch);
  float *h1 = work, *h2 = h1 + B * h, *d1 = h2 + B * h, *d2 = d1 + B * h, *z = d2 + B * h, *lb = z + B * (c + 1);
  float *dz = lb + B;
  // work layout: h1, h2, dh1, dh2 [batch][h]; z [batch][c+1]; sample losses
  // [batch]; dz [batch][c+1]
  const MlpOff o = mlp_off(nf, h, c);
  forward(params, nf, h, c, X, batch, h1, h2, z, s);
  head_grad<<<blocks_for(batch), kMlpThreads, 0, s>>>(z, c, ycls, yreg, wreg, batch, dz, lb);
  loss_sum<<<1, 32, 0, s>>>(lb, batch, loss);
  dense_wgrad<<<blocks_for(int64_t(h) * (c + 1) + c + 1), kMlpThreads, 0, s>>>(h2, h, dz, c + 1, batch,
                                                                               grad + o.w3, grad + o.b3);
  dense_bwd_in<<<blocks_for(int64_t(batch) * h), kMlpThreads, 0, s>>>(dz, params + o.w3, h, c + 1, h2, batch, d2);
  dense_wgrad<<<blocks_for(int64_t(h) * h + h), kMlpThreads, 0, s>>>(h1, h, d2, h, batch, grad + o.w2, grad + o.b2);
  dense_bwd_in<<<blocks_for(int64_t(batch) * h), kMlpThreads, 0, s>>>(d2, params + o.w2, h, h, h1, batch, d1);
  dense_wgrad<<<blocks_for(int64_t(nf) * h + h), kMlpThreads, 0, s>>>(X, nf, d1, h, batch, grad + o.w1, grad + o.b1);
  return launched(cudaGetLastError());
}

iccg_status iccg_mlp_adam(float *params, const float *grad, float *m, float *v, int64_t nparams, float lr,
                          float beta1, float beta2, float eps, int32_t step, iccg_stream_t stream) {
  if (!params || !grad || !m || !v || nparams < 1 || step < 1 || !(beta1 >= 0.f && beta1 < 1.f) ||
      !(beta2 >= 0.f && beta2 < 1.f))
    return ICCG_ERR_ARG;
  const float c1 = 1.0f - std::pow(beta1, float(step)), c2 = 1.0f - std::pow(beta2, float(step));
  adam_step<<<blocks_for(nparams), kMlpThreads, 0, static_cast<cudaStream_t>(stream)>>>(params, grad, m, v, nparams,
                                                                                         lr, beta1, beta2, eps, c1, c2);
  return launched(cudaGetLastError());
}

}  // extern "C"
