// FP64 strided, batched GEMM with device-side sizes.
//
// Every contraction of the step (zip-up core contractions, absorption of R
// and U*S factors into neighbouring cores, the Hadamard contraction with the
// c^2 cores) is a small GEMM whose sizes are bond ranks held in device
// memory.  The kernel evaluates M, N, K, strides and batch offsets from
// device ints, so a step needs no host synchronisation.  Tiles are 32x32 so
// that the FP64 work spreads over all SMs (the FP64 pipe, not bandwidth,
// bounds these products on this part).
#include "qtt_internal.cuh"

namespace qtt {

namespace {

constexpr int BM = 32, BN = 32, BK = 16, NT = 256;

struct GemmKArgs {
  GemmArgs a;
  long long nb2max;
};

__global__ void __launch_bounds__(NT) gemm_f64_kernel(GemmKArgs ka) {
  const GemmArgs& a = ka.a;
  const long long M = dv(a.M), N = dv(a.N), K = dv(a.K);
  const long long bz = blockIdx.z;
  const long long b1 = bz / ka.nb2max, b2 = bz % ka.nb2max;
  const long long i0 = (long long)blockIdx.y * BM, j0 = (long long)blockIdx.x * BN;
  if (i0 >= M || j0 >= N || b1 >= dv(a.nb1) || b2 >= dv(a.nb2)) return;

  const long long sai = dv(a.sai), sak = dv(a.sak), sbk = dv(a.sbk), sbj = dv(a.sbj);
  const long long sci = dv(a.sci), scj = dv(a.scj);
  const double* A = a.A + b1 * dv(a.sa1) + b2 * dv(a.sa2);
  const double* B = a.B + b1 * dv(a.sb1) + b2 * dv(a.sb2);
  double* C = a.C + b1 * dv(a.sc1) + b2 * dv(a.sc2);

  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc00 = 0.0, acc01 = 0.0, acc10 = 0.0, acc11 = 0.0;
  const bool a_k_fast = (sak == 1);
  const bool b_j_fast = (sbj == 1);

  for (long long k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
    for (int e2 = 0; e2 < 2; ++e2) {
      int e = tid + e2 * NT;
      int r, kk;
      if (a_k_fast) { kk = e & (BK - 1); r = e >> 4; } else { r = e & (BM - 1); kk = e >> 5; }
      long long gi = i0 + r, gk = k0 + kk;
      As[kk][r] = (gi < M && gk < K) ? A[gi * sai + gk * sak] : 0.0;
      int c;
      if (b_j_fast) { c = e & (BN - 1); kk = e >> 5; } else { kk = e & (BK - 1); c = e >> 4; }
      long long gj = j0 + c;
      gk = k0 + kk;
      Bs[kk][c] = (gj < N && gk < K) ? B[gk * sbk + gj * sbj] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a0 = As[kk][ty], a1 = As[kk][ty + 16];
      double c0 = Bs[kk][tx], c1 = Bs[kk][tx + 16];
      acc00 = fma(a0, c0, acc00);
      acc01 = fma(a0, c1, acc01);
      acc10 = fma(a1, c0, acc10);
      acc11 = fma(a1, c1, acc11);
    }
    __syncthreads();
  }
  const double al = a.alpha, be = a.beta;
  double accs[2][2] = {{acc00, acc01}, {acc10, acc11}};
#pragma unroll
  for (int ii = 0; ii < 2; ++ii) {
    long long gi = i0 + ty + ii * 16;
    if (gi >= M) continue;
#pragma unroll
    for (int jj = 0; jj < 2; ++jj) {
      long long gj = j0 + tx + jj * 16;
      if (gj >= N) continue;
      double* cp = C + gi * sci + gj * scj;
      double v = al * accs[ii][jj];
      if (be != 0.0) v += be * (*cp);
      *cp = v;
    }
  }
}

}  // namespace

cudaError_t gemm_f64(const GemmArgs& a, long long Mmax, long long Nmax, long long nb1max, long long nb2max,
                     cudaStream_t st) {
  if (Mmax <= 0 || Nmax <= 0 || nb1max <= 0 || nb2max <= 0) return cudaSuccess;
  long long gx = (Nmax + BN - 1) / BN, gy = (Mmax + BM - 1) / BM, gz = nb1max * nb2max;
  if (gx > 2147483647LL || gy > 65535 || gz > 65535) return cudaErrorInvalidConfiguration;
  GemmKArgs ka{a, nb2max};
  gemm_f64_kernel<<<dim3((unsigned)gx, (unsigned)gy, (unsigned)gz), NT, 0, st>>>(ka);
  return cudaGetLastError();
}

}  // namespace qtt
