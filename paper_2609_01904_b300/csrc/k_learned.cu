// Learned rank proposal and the randomised rounding of the learned form.
//
// The MLP (3 linear layers, width 128, ReLU, FP32) reads 40 features of a
// bond's singular-value spectrum at step k and proposes the bond's rank at
// step k+1; it is trained here with mean squared error and Adam (Kingma & Ba
// 2015, Algorithm 1).  Every product is an FP32 tile kernel with a fixed
// reduction order, so training is deterministic.
//
// The round's SVD of a bond with a proposal r_hat first tries the range
// finder of width ks = r_hat + p (Halko, Martinsson & Tropp 2011, Algorithm
// 4.1 and Sec. 5.1).  The kernels below compute the FP64 residual
// rho = ||X - X Q Q^T||_F and decide, on the device, whether the sketch meets
// the rounding rule of Sec. 4.3: uncapped, rho <= eps sigma_1; capped at chi,
// rho^2 <= ((1+tau)^2 - 1) sum_{i>=chi} sigma_i(B)^2, which keeps the
// discarded weight within (1+tau)^2 of the optimum (X X^T = A A^T + E E^T
// with A = X Q Q^T, E = X - A, and Ky Fan's maximum principle bound the top
// chi energy of X by that of A plus rho^2).  The host falls back to the full
// SVD otherwise.
#include <cmath>

#include "k_learned.cuh"
#include "qtt_internal.cuh"

namespace qtt {

namespace {

constexpr int TS = 16;  // output tile of the FP32 product

// C[i][j] = act(alpha sum_k A(i,k) B(k,j) + bias[j]) + beta C[i][j], row-major C
__global__ void __launch_bounds__(TS * TS) sgemm_kernel(int M, int N, int K, const float* __restrict__ A,
                                                         long long sai, long long sak, const float* __restrict__ B,
                                                         long long sbk, long long sbj, float* C, long long ldc,
                                                         const float* __restrict__ bias, int relu, float beta) {
  __shared__ float As[TS][TS + 1];
  __shared__ float Bs[TS][TS + 1];
  const int tx = threadIdx.x % TS, ty = threadIdx.x / TS;
  const int i = blockIdx.y * TS + ty, j = blockIdx.x * TS + tx;
  float acc = 0.f;
  for (int k0 = 0; k0 < K; k0 += TS) {
    const int ka = k0 + tx, kb = k0 + ty;
    const int ia = blockIdx.y * TS + ty, jb = blockIdx.x * TS + tx;
    As[ty][tx] = (ia < M && ka < K) ? A[ia * sai + ka * sak] : 0.f;
    Bs[ty][tx] = (kb < K && jb < N) ? B[kb * sbk + jb * sbj] : 0.f;
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TS; ++kk) acc = fmaf(As[ty][kk], Bs[kk][tx], acc);
    __syncthreads();
  }
  if (i < M && j < N) {
    float v = acc + (bias ? bias[j] : 0.f);
    if (relu) v = fmaxf(v, 0.f);
    float* c = C + (long long)i * ldc + j;
    *c = beta != 0.f ? v + beta * (*c) : v;
  }
}

cudaError_t sgemm(int M, int N, int K, const float* A, long long sai, long long sak, const float* B, long long sbk,
                  long long sbj, float* C, long long ldc, const float* bias, int relu, float beta, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  dim3 grid((N + TS - 1) / TS, (M + TS - 1) / TS);
  if (grid.y > 65535) return cudaErrorInvalidConfiguration;
  sgemm_kernel<<<grid, TS * TS, 0, st>>>(M, N, K, A, sai, sak, B, sbk, sbj, C, ldc, bias, relu, beta);
  return cudaGetLastError();
}

// dy = 2 (y - t) / n; loss = mean (y - t)^2 (FP64 accumulation, one CTA)
__global__ void __launch_bounds__(1024) mse_kernel(const float* y, const float* t, int n, float* dy, float* loss) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float d = y[i] - t[i];
    dy[i] = 2.f * d / (float)n;
    s += (double)d * (double)d;
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0 && loss) *loss = (float)(s / n);
}

// dA = dH * (A > 0), elementwise over count entries
__global__ void relu_back_kernel(const float* dH, const float* A, float* dA, long long count) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count; e += (long long)gridDim.x * blockDim.x)
    dA[e] = A[e] > 0.f ? dH[e] : 0.f;
}

// db[j] = sum_i dA[i][j] (dA row-major n x cols), one block per column
__global__ void colsum_kernel(const float* dA, int n, int cols, float* db) {
  __shared__ float red[32];
  for (int j = blockIdx.x; j < cols; j += gridDim.x) {
    float s = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += dA[(long long)i * cols + j];
    s = block_sum(s, red);
    if (threadIdx.x == 0) db[j] = s;
  }
}

__global__ void adam_kernel(float* p, const float* g, float* m, float* v, long long count, float lr, float b1,
                            float b2, float eps, float bc1, float bc2) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count; e += (long long)gridDim.x * blockDim.x) {
    const float ge = g[e];
    const float me = b1 * m[e] + (1.f - b1) * ge;
    const float ve = b2 * v[e] + (1.f - b2) * ge * ge;
    m[e] = me;
    v[e] = ve;
    const float mh = me / bc1, vh = ve / bc2;
    p[e] -= lr * mh / (sqrtf(vh) + eps);
  }
}

// 40 features of bond k = 1..nb (row k-1 of X); S row k (ld lds) holds the
// descending singular values, L[k] of them, r[k] kept.
__global__ void features_kernel(const double* S, long long lds, const int* L, const int* r, int nb, double eps,
                                int chi, int d, float* X) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
    const int k = b + 1;
    const double* s = S + (long long)k * lds;
    const int len = L[k], rk = r[k];
    float* f = X + (long long)b * kFeat;
    const double s0 = len > 0 ? s[0] : 0.0;
    for (int j = 0; j < kSpec; ++j) {
      const int p = len > 1 ? (j * (len - 1)) / (kSpec - 1) : 0;
      double v = -1.0;
      if (s0 > 0.0 && s[p] > 0.0) v = fmin(fmax(log10(s[p] / s0), -16.0), 0.0) / 16.0;
      f[j] = (float)v;
    }
    double disc = 0.0;
    int cnt = 0;
    for (int i = 0; i < len; ++i) {
      if (i >= rk) disc += s[i] * s[i];
      if (s0 > 0.0 && s[i] >= eps * s0) ++cnt;
    }
    f[32] = (float)((double)rk / chi);
    f[33] = (float)((s0 > 0.0 && disc > 0.0) ? fmin(fmax(log10(disc / (s0 * s0)), -32.0), 0.0) / 32.0 : -1.0);
    f[34] = (float)(eps > 0.0 ? log10(eps) / 16.0 : -1.0);
    f[35] = (float)((double)k / d);
    const long long capk = min(min(1LL << k, 1LL << (d - k)), (long long)chi);
    f[36] = (float)((double)capk / chi);
    f[37] = (float)((double)cnt / chi);
    f[38] = (float)((double)len / (2.0 * chi));
    f[39] = 1.f;
  }
}

// prop[k] = clamp(ceil(chi y[k-1]), 1, chi), k = 1..nb; prop[0] = 0
__global__ void propose_kernel(const float* y, int nb, int chi, int* prop) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b <= nb; b += gridDim.x * blockDim.x) {
    if (b == 0) {
      prop[0] = 0;
      continue;
    }
    const double v = ceil((double)chi * (double)y[b - 1]);
    prop[b] = (int)fmin(fmax(v, 1.0), (double)chi);
  }
}

// out = sum of squares of the rows x cols block of X (row i at X + i*ld), FP64, one CTA
__global__ void __launch_bounds__(1024) sumsq_kernel(const double* X, Dim ld_d, Dim rows_d, Dim cols_d, double* out) {
  __shared__ double red[32];
  const long long ld = dv(ld_d), rows = dv(rows_d), cols = dv(cols_d);
  double s = 0.0;
  for (long long e = threadIdx.x; e < rows * cols; e += blockDim.x) {
    const double x = X[(e / cols) * ld + e % cols];
    s = fma(x, x, s);
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) *out = s;
}

// Acceptance of the range finder (see the file comment).  sig: the nsv
// descending singular values of the sketch; the kept rank r was written by
// the rounding rule.  flag: 1 accepted, 0 rejected, 2 not attempted (the
// sketch is not narrower than the matrix).
__global__ void rf_accept_kernel(const double* sig, const int* nsv_p, const int* r_p, int ks, const int* nv_p,
                                 const int* ell_p, int nv_mul, double eps, int chi, double tau, const double* rho2_p,
                                 const double* nx2_p, int* flag, double* disc_out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const long long nv = (long long)nv_mul * nv_p[0], ell = ell_p[0];
  if (ks >= nv || ks >= ell) {
    *flag = 2;
    return;
  }
  const int nsv = *nsv_p, r = *r_p;
  const double rho2 = fmax(*rho2_p, 0.0), rho = sqrt(rho2);
  (void)nx2_p;
  const double s0 = nsv > 0 ? sig[0] : 0.0;
  int c = 0;
  if (s0 > 0.0)
    for (int i = 0; i < nsv; ++i) c += sig[i] >= eps * s0;
  int ok;
  if (s0 == 0.0) {
    ok = rho2 == 0.0;
  } else if (c >= ks) {
    ok = 0;
  } else if (c < chi) {
    ok = rho <= eps * s0;
  } else {
    // Ky Fan: the optimal tail is at least the sketch's own tail beyond chi
    double tail = 0.0;
    for (int i = chi; i < nsv; ++i) tail += sig[i] * sig[i];
    ok = rho2 <= ((1.0 + tau) * (1.0 + tau) - 1.0) * tail;
  }
  *flag = ok;
  if (ok && disc_out) {
    double tail = 0.0;
    for (int i = r; i < nsv; ++i) tail += sig[i] * sig[i];
    *disc_out = tail + rho2;
  }
}

inline int eg(long long total) {
  long long g = (total + 255) / 256;
  return (int)std::max(1LL, std::min(g, device_sms() * 8LL));
}

}  // namespace

// ------------------------------------------------------------------ MLP
cudaError_t mlp_forward(const MlpDev& m, const float* X, int n, float* y, cudaStream_t st) {
  cudaError_t e;
  if ((e = sgemm(n, kWidth, kFeat, X, kFeat, 1, m.W1(), 1, kFeat, m.a1, kWidth, m.b1(), 1, 0.f, st)) != cudaSuccess)
    return e;
  if ((e = sgemm(n, kWidth, kWidth, m.a1, kWidth, 1, m.W2(), 1, kWidth, m.a2, kWidth, m.b2(), 1, 0.f, st)) !=
      cudaSuccess)
    return e;
  return sgemm(n, 1, kWidth, m.a2, kWidth, 1, m.W3(), 1, kWidth, y, 1, m.b3(), 0, 0.f, st);
}

// With ReLU applied in place, a1/a2 hold h1/h2 = relu(a); relu'(a) = [h > 0].
cudaError_t mlp_grad(const MlpDev& m, const float* X, const float* t, int n, float* loss, cudaStream_t st) {
  cudaError_t e;
  if ((e = mlp_forward(m, X, n, m.y, st)) != cudaSuccess) return e;
  mse_kernel<<<1, 1024, 0, st>>>(m.y, t, n, m.dy, loss);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // layer 3: gW3 (1 x W) = dy^T h2, gb3 = sum dy
  if ((e = sgemm(1, kWidth, n, m.dy, 0, 1, m.a2, kWidth, 1, m.gW3(), kWidth, nullptr, 0, 0.f, st)) != cudaSuccess)
    return e;
  colsum_kernel<<<1, 256, 0, st>>>(m.dy, n, 1, m.gb3());
  // dh2 (n x W) = dy W3, masked by relu'
  if ((e = sgemm(n, kWidth, 1, m.dy, 1, 1, m.W3(), kWidth, 1, m.d2, kWidth, nullptr, 0, 0.f, st)) != cudaSuccess)
    return e;
  relu_back_kernel<<<eg((long long)n * kWidth), 256, 0, st>>>(m.d2, m.a2, m.d2, (long long)n * kWidth);
  // layer 2: gW2 = da2^T h1, gb2 = colsum da2, dh1 = da2 W2 masked
  if ((e = sgemm(kWidth, kWidth, n, m.d2, 1, kWidth, m.a1, kWidth, 1, m.gW2(), kWidth, nullptr, 0, 0.f, st)) !=
      cudaSuccess)
    return e;
  colsum_kernel<<<kWidth, 256, 0, st>>>(m.d2, n, kWidth, m.gb2());
  if ((e = sgemm(n, kWidth, kWidth, m.d2, kWidth, 1, m.W2(), kWidth, 1, m.d1, kWidth, nullptr, 0, 0.f, st)) !=
      cudaSuccess)
    return e;
  relu_back_kernel<<<eg((long long)n * kWidth), 256, 0, st>>>(m.d1, m.a1, m.d1, (long long)n * kWidth);
  // layer 1: gW1 = da1^T X, gb1 = colsum da1
  if ((e = sgemm(kWidth, kFeat, n, m.d1, 1, kWidth, X, kFeat, 1, m.gW1(), kFeat, nullptr, 0, 0.f, st)) !=
      cudaSuccess)
    return e;
  colsum_kernel<<<kWidth, 256, 0, st>>>(m.d1, n, kWidth, m.gb1());
  return cudaGetLastError();
}

cudaError_t mlp_adam(const MlpDev& m, int t, float lr, float b1, float b2, float eps, cudaStream_t st) {
  const float bc1 = (float)(1.0 - std::pow((double)b1, t)), bc2 = (float)(1.0 - std::pow((double)b2, t));
  adam_kernel<<<eg(kParams), 256, 0, st>>>(m.p, m.g, m.m, m.v, kParams, lr, b1, b2, eps, bc1, bc2);
  return cudaGetLastError();
}

cudaError_t rank_features(const double* S, long long lds, const int* L, const int* r, int nb, double eps, int chi,
                          int d, float* X, cudaStream_t st) {
  if (nb <= 0) return cudaSuccess;
  features_kernel<<<(nb + 63) / 64, 64, 0, st>>>(S, lds, L, r, nb, eps, chi, d, X);
  return cudaGetLastError();
}

cudaError_t propose(const float* y, int nb, int chi, int* prop, cudaStream_t st) {
  propose_kernel<<<(nb + 256) / 256, 256, 0, st>>>(y, nb, chi, prop);
  return cudaGetLastError();
}

cudaError_t sumsq(const double* X, Dim ld, Dim rows, Dim cols, double* out, cudaStream_t st) {
  sumsq_kernel<<<1, 1024, 0, st>>>(X, ld, rows, cols, out);
  return cudaGetLastError();
}

cudaError_t rf_accept(const double* sig, const int* nsv, const int* r, int ks, const int* nv, const int* ell,
                      int nv_mul, double eps, int chi, double tau, const double* rho2, const double* nx2, int* flag,
                      double* disc_out, cudaStream_t st) {
  rf_accept_kernel<<<1, 32, 0, st>>>(sig, nsv, r, ks, nv, ell, nv_mul, eps, chi, tau, rho2, nx2, flag, disc_out);
  return cudaGetLastError();
}

}  // namespace qtt
