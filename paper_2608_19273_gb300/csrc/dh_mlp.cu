// Training and inference kernels of the FP32 MLP pressure seed (layout and
// inputs in dh_mlp.cuh).  Loss: mean squared error on y = ln(p/E).
//
// Gradients are deterministic: each CTA of 64 threads takes 64 samples
// (one per thread), runs forward and backward per sample, keeps the
// per-sample activations and back-propagated errors in shared memory, and
// sums every one of the 1217 gradient entries over its samples in a fixed
// order into one row of a partial-gradient table; a second kernel sums the
// rows in a fixed order.  No floating-point atomics anywhere.
#include <cmath>

#include "dh_internal.cuh"
#include "dh_mlp.cuh"

namespace dh {

constexpr int GB = 64;  // samples per gradient CTA

// Raw invariants x (n x 3, row-major) and, if p is given, targets y = ln(p/E)
// from conserved states in SoA layout with the given stride.
__global__ void k_mlp_features(const double* __restrict__ cons, const double* __restrict__ p, int64_t n,
                               int64_t stride, float* __restrict__ x, float* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double q[5], xd[3];
#pragma unroll
    for (int v = 0; v < 5; ++v) q[v] = cons[v * stride + i];
    srhd_invariants(q, xd);
#pragma unroll
    for (int j = 0; j < 3; ++j) x[3 * i + j] = (float)xd[j];
    if (y) y[i] = (float)log(p[i] / (q[4] + q[0]));
  }
}

// Mean and standard deviation of the three inputs, in two deterministic passes:
// per-CTA FP64 partial sums (fixed order), then one CTA sums the partial rows.
__global__ void k_mlp_stats_partial(const float* __restrict__ x, int64_t n, double* __restrict__ part) {
  __shared__ double s[256][6];
  double a[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const double v = x[3 * i + j];
      a[j] += v;
      a[3 + j] = fma(v, v, a[3 + j]);
    }
  }
#pragma unroll
  for (int j = 0; j < 6; ++j) s[threadIdx.x][j] = a[j];
  __syncthreads();
  if (threadIdx.x < 6) {
    double t = 0.0;
    for (int i = 0; i < (int)blockDim.x; ++i) t += s[i][threadIdx.x];
    part[blockIdx.x * 6 + threadIdx.x] = t;
  }
}

__global__ void k_mlp_stats_final(const double* __restrict__ part, int nb, int64_t n, float* __restrict__ w) {
  if (threadIdx.x < 3) {
    const int j = threadIdx.x;
    double s1 = 0.0, s2 = 0.0;
    for (int b = 0; b < nb; ++b) { s1 += part[b * 6 + j]; s2 += part[b * 6 + 3 + j]; }
    const double mean = s1 / (double)n;
    double var = s2 / (double)n - mean * mean;
    if (!(var > 1e-30)) var = 1.0;
    w[MLP_MEAN + j] = (float)mean;
    w[MLP_STD + j] = (float)sqrt(var);
  }
}

// Forward pass on raw inputs (z-scored with the statistics in w).
__global__ void k_mlp_forward(const float* __restrict__ wg, const float* __restrict__ x, int64_t n,
                              float* __restrict__ y) {
  __shared__ __align__(16) float w[MLP_LEN];
  for (int i = threadIdx.x; i < MLP_LEN; i += blockDim.x) w[i] = wg[i];
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double xd[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
    float xn[3], h1[32], h2[32];
    mlp_normalize(w, xd, xn);
    y[i] = mlp_forward(w, xn, h1, h2);
  }
}

// Per-CTA partial gradient of (1/B) sum (y_i - t_i)^2 over samples [off, off + B).
// part row layout: 1217 gradient entries, then the partial sum of squared residuals.
__global__ void __launch_bounds__(GB) k_mlp_grad(const float* __restrict__ wg, const float* __restrict__ x,
                                                 const float* __restrict__ t, int64_t off, int B,
                                                 float* __restrict__ part) {
  __shared__ __align__(16) float w[MLP_LEN];
  __shared__ float sh1[GB][33], sh2[GB][33], sg1[GB][33], sg2[GB][33];
  __shared__ float sx[GB][3], sgy[GB], sr2[GB];
  for (int i = threadIdx.x; i < MLP_LEN; i += blockDim.x) w[i] = wg[i];
  __syncthreads();
  const int k = threadIdx.x;
  const int64_t i = (int64_t)blockIdx.x * GB + k;
  const bool valid = i < B;
  float h1[32], h2[32], xn[3] = {0.f, 0.f, 0.f};
  float gy = 0.f, r2 = 0.f;
  if (valid) {
    const int64_t s = off + i;
    double xd[3] = {x[3 * s], x[3 * s + 1], x[3 * s + 2]};
    mlp_normalize(w, xd, xn);
    const float y = mlp_forward(w, xn, h1, h2);
    const float r = y - t[s];
    r2 = r * r;
    gy = 2.0f * r / (float)B;
  } else {
#pragma unroll
    for (int j = 0; j < 32; ++j) { h1[j] = 0.f; h2[j] = 0.f; }
  }
  // back-propagation
  float g2[32];
#pragma unroll
  for (int a = 0; a < 32; ++a) g2[a] = gy * w[MLP_W3 + a] * (1.0f - h2[a] * h2[a]);
#pragma unroll 4
  for (int j = 0; j < 32; ++j) {
    float s = 0.f;
#pragma unroll
    for (int a = 0; a < 32; ++a) s = fmaf(w[MLP_W2 + 32 * a + j], g2[a], s);
    sg1[k][j] = s * (1.0f - h1[j] * h1[j]);
  }
#pragma unroll
  for (int j = 0; j < 32; ++j) { sh1[k][j] = h1[j]; sh2[k][j] = h2[j]; sg2[k][j] = g2[j]; }
  sx[k][0] = xn[0]; sx[k][1] = xn[1]; sx[k][2] = xn[2];
  sgy[k] = gy;
  sr2[k] = r2;
  __syncthreads();
  // gradient entries, each summed over the CTA's samples in order
  float* row = part + (int64_t)blockIdx.x * MLP_LEN;
  for (int e = threadIdx.x; e <= MLP_NW; e += blockDim.x) {
    float s = 0.f;
    if (e < MLP_B1) {                 // W1[a][j] += g1[a] x[j]
      const int a = e / 3, j = e % 3;
      for (int m = 0; m < GB; ++m) s = fmaf(sg1[m][a], sx[m][j], s);
    } else if (e < MLP_W2) {          // b1[a] += g1[a]
      const int a = e - MLP_B1;
      for (int m = 0; m < GB; ++m) s += sg1[m][a];
    } else if (e < MLP_B2) {          // W2[a][j] += g2[a] h1[j]
      const int a = (e - MLP_W2) / 32, j = (e - MLP_W2) % 32;
      for (int m = 0; m < GB; ++m) s = fmaf(sg2[m][a], sh1[m][j], s);
    } else if (e < MLP_W3) {          // b2[a] += g2[a]
      const int a = e - MLP_B2;
      for (int m = 0; m < GB; ++m) s += sg2[m][a];
    } else if (e < MLP_B3) {          // W3[a] += gy h2[a]
      const int a = e - MLP_W3;
      for (int m = 0; m < GB; ++m) s = fmaf(sgy[m], sh2[m][a], s);
    } else if (e == MLP_B3) {         // b3 += gy
      for (int m = 0; m < GB; ++m) s += sgy[m];
    } else {                          // squared residuals
      for (int m = 0; m < GB; ++m) s += sr2[m];
    }
    row[e] = s;
  }
}

// Sum the partial rows in order: grad[e] = sum_b part[b][e]; grad[1217] = loss.
__global__ void k_mlp_reduce(const float* __restrict__ part, int nb, int B, float* __restrict__ grad) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e > MLP_NW) return;
  float s = 0.f;
  for (int b = 0; b < nb; ++b) s += part[(int64_t)b * MLP_LEN + e];
  grad[e] = e == MLP_NW ? s / (float)B : s;
}

// Adam (Kingma & Ba 2015): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
// w -= lr (m / c1) / (sqrt(v / c2) + eps), c1 = 1 - b1^t, c2 = 1 - b2^t.
__global__ void k_mlp_adam(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                           const float* __restrict__ g, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= MLP_NW) return;
  const float ge = g[e];
  const float me = fmaf(b1, m[e], (1.0f - b1) * ge);
  const float ve = fmaf(b2, v[e], (1.0f - b2) * ge * ge);
  m[e] = me;
  v[e] = ve;
  w[e] -= lr * (me / c1) / (sqrtf(ve / c2) + eps);
}

static int grid_for(int64_t n) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (n + 255) / 256;
  return (int)std::min<int64_t>(std::max<int64_t>(want, 1), (int64_t)sms * 8);
}

}  // namespace dh

using namespace dh;

extern "C" {

dh_status dh_mlp_features(const double* cons, const double* p, int64_t n, int64_t stride, float* x, float* y,
                          void* stream) {
  if (!cons || !x || n <= 0 || stride < n || (y && !p)) { set_error("dh_mlp_features: bad arguments"); return DH_EINVAL; }
  k_mlp_features<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(cons, p, n, stride, x, y);
  return cuda_error(cudaGetLastError(), "dh_mlp_features launch");
}

dh_status dh_mlp_standardize(const float* x, int64_t n, float* w, double* scratch, int32_t scratch_len,
                             void* stream) {
  if (!x || !w || !scratch || n <= 1) { set_error("dh_mlp_standardize: bad arguments"); return DH_EINVAL; }
  const int nb = std::min(grid_for(n), scratch_len / 6);
  if (nb < 1) { set_error("dh_mlp_standardize: scratch must hold at least 6 doubles"); return DH_EINVAL; }
  cudaStream_t s = (cudaStream_t)stream;
  k_mlp_stats_partial<<<nb, 256, 0, s>>>(x, n, scratch);
  k_mlp_stats_final<<<1, 32, 0, s>>>(scratch, nb, n, w);
  return cuda_error(cudaGetLastError(), "dh_mlp_standardize launch");
}

dh_status dh_mlp_forward(const float* w, const float* x, int64_t n, float* y, void* stream) {
  if (!w || !x || !y || n <= 0) { set_error("dh_mlp_forward: bad arguments"); return DH_EINVAL; }
  k_mlp_forward<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(w, x, n, y);
  return cuda_error(cudaGetLastError(), "dh_mlp_forward launch");
}

dh_status dh_mlp_grad(const float* w, const float* x, const float* t, int64_t offset, int32_t B, float* partials,
                      float* grad, void* stream) {
  if (!w || !x || !t || !partials || !grad || B <= 0 || offset < 0) { set_error("dh_mlp_grad: bad arguments"); return DH_EINVAL; }
  const int nb = (B + GB - 1) / GB;
  cudaStream_t s = (cudaStream_t)stream;
  k_mlp_grad<<<nb, GB, 0, s>>>(w, x, t, offset, B, partials);
  k_mlp_reduce<<<(MLP_NW + 1 + 255) / 256, 256, 0, s>>>(partials, nb, B, grad);
  return cuda_error(cudaGetLastError(), "dh_mlp_grad launch");
}

dh_status dh_mlp_adam(float* w, float* m, float* v, const float* g, int32_t t, float lr, float b1, float b2,
                      float eps, void* stream) {
  if (!w || !m || !v || !g || t < 1) { set_error("dh_mlp_adam: bad arguments"); return DH_EINVAL; }
  const float c1 = (float)(1.0 - std::pow((double)b1, t)), c2 = (float)(1.0 - std::pow((double)b2, t));
  k_mlp_adam<<<(MLP_NW + 255) / 256, 256, 0, (cudaStream_t)stream>>>(w, m, v, g, lr, b1, b2, eps, c1, c2);
  return cuda_error(cudaGetLastError(), "dh_mlp_adam launch");
}

dh_status dh_mlp_train(float* w, float* m, float* v, const float* x, const float* t, int64_t n, int32_t batch,
                       int32_t steps, int32_t t0, float lr, float* partials, float* grad, float* loss_log,
                       void* stream) {
  if (!w || !m || !v || !x || !t || !partials || !grad || n <= 0 || batch <= 0 || batch > n || steps < 0 || t0 < 0) {
    set_error("dh_mlp_train: bad arguments");
    return DH_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t nbatch = n / batch;
  for (int k = 0; k < steps; ++k) {
    const int64_t off = (int64_t)(k % nbatch) * batch;
    dh_status st = dh_mlp_grad(w, x, t, off, batch, partials, grad, stream);
    if (st != DH_OK) return st;
    if (loss_log) {
      cudaError_t e = cudaMemcpyAsync(loss_log + k, grad + MLP_NW, sizeof(float), cudaMemcpyDeviceToDevice, s);
      if (e != cudaSuccess) return cuda_error(e, "dh_mlp_train loss copy");
    }
    st = dh_mlp_adam(w, m, v, grad, t0 + k + 1, lr, 0.9f, 0.999f, 1e-8f, stream);
    if (st != DH_OK) return st;
  }
  return DH_OK;
}

}  // extern "C"
