// Learned rank proposal (MLP) and range-finder helpers (k_learned.cu).
#pragma once

#include "qtt_internal.cuh"

namespace qtt {

constexpr int kFeat = 40;    // features of one bond's spectrum
constexpr int kSpec = 32;    // spectrum samples among them
constexpr int kWidth = 128;  // hidden width
// W1 (kWidth x kFeat), b1, W2 (kWidth x kWidth), b2, W3 (1 x kWidth), b3
constexpr long long kParams = (long long)kWidth * kFeat + kWidth + (long long)kWidth * kWidth + kWidth + kWidth + 1;

// Device state of one network: parameters, gradient, Adam moments and the
// activations of up to max_batch samples.
struct MlpDev {
  float* p = nullptr;
  float* g = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  float* a1 = nullptr;  // relu(W1 x + b1), max_batch x kWidth
  float* a2 = nullptr;  // relu(W2 h1 + b2)
  float* d1 = nullptr;  // gradients at the hidden layers
  float* d2 = nullptr;
  float* y = nullptr;   // outputs, max_batch
  float* dy = nullptr;
  int max_batch = 0;
  static constexpr long long oW1 = 0, ob1 = oW1 + (long long)kWidth * kFeat, oW2 = ob1 + kWidth,
                             ob2 = oW2 + (long long)kWidth * kWidth, oW3 = ob2 + kWidth, ob3 = oW3 + kWidth;
  const float* W1() const { return p + oW1; }
  const float* b1() const { return p + ob1; }
  const float* W2() const { return p + oW2; }
  const float* b2() const { return p + ob2; }
  const float* W3() const { return p + oW3; }
  const float* b3() const { return p + ob3; }
  float* gW1() const { return g + oW1; }
  float* gb1() const { return g + ob1; }
  float* gW2() const { return g + oW2; }
  float* gb2() const { return g + ob2; }
  float* gW3() const { return g + oW3; }
  float* gb3() const { return g + ob3; }
};

// y (n) = MLP(X (n x kFeat, row-major))
cudaError_t mlp_forward(const MlpDev& m, const float* X, int n, float* y, cudaStream_t st);
// loss (device float, may be null) = mean (y - t)^2 and the gradient into m.g
cudaError_t mlp_grad(const MlpDev& m, const float* X, const float* t, int n, float* loss, cudaStream_t st);
// one Adam update of m.p from m.g; t counts from 1
cudaError_t mlp_adam(const MlpDev& m, int t, float lr, float b1, float b2, float eps, cudaStream_t st);
// features of bonds 1..nb (rows 0..nb-1 of X) from spectra S (row k, ld lds),
// their lengths L[k] and kept ranks r[k]
cudaError_t rank_features(const double* S, long long lds, const int* L, const int* r, int nb, double eps, int chi,
                          int d, float* X, cudaStream_t st);
// prop[k] = clamp(ceil(chi y[k-1]), 1, chi) for k = 1..nb, prop[0] = 0
cudaError_t propose(const float* y, int nb, int chi, int* prop, cudaStream_t st);
// *out = sum of squares of a rows x cols block (row stride ld)
cudaError_t sumsq(const double* X, Dim ld, Dim rows, Dim cols, double* out, cudaStream_t st);
// acceptance of one range-finder attempt (flag: 1 accept, 0 reject, 2 not attempted)
cudaError_t rf_accept(const double* sig, const int* nsv, const int* r, int ks, const int* nv, const int* ell,
                      int nv_mul, double eps, int chi, double tau, const double* rho2, const double* nx2, int* flag,
                      double* disc_out, cudaStream_t st);

}  // namespace qtt
