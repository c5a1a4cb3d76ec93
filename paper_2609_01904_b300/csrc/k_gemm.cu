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

constexpr int BK = 16, NT = 256;

struct GemmKArgs {
  GemmArgs a;
  long long nb2max;
  double* flops;  // algorithmic FLOP counter of the launch's class (null: not counting)
};

// T: arithmetic of the products and the accumulation (double, or float for
// the reduced-precision form); operands and result stay FP64 in memory.
// TM x TN output tile per CTA, each of the 256 threads owns (TM/16)x(TN/16).
template <typename T, int TM, int TN>
__global__ void __launch_bounds__(NT) gemm_kernel(GemmKArgs ka) {
  constexpr int RI = TM / 16, RJ = TN / 16;
  const GemmArgs& a = ka.a;
  const long long M = dv(a.M), N = dv(a.N), K = dv(a.K);
  const long long bz = blockIdx.z;
  const long long b1 = bz / ka.nb2max, b2 = bz % ka.nb2max;
  const long long i0 = (long long)blockIdx.y * TM, j0 = (long long)blockIdx.x * TN;
  if (ka.flops && bz == 0 && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0)
    atomicAdd(ka.flops, 2.0 * (double)M * (double)N * (double)K * (double)dv(a.nb1) * (double)dv(a.nb2));
  if (i0 >= M || j0 >= N || b1 >= dv(a.nb1) || b2 >= dv(a.nb2)) return;

  const long long sai = dv(a.sai), sak = dv(a.sak), sbk = dv(a.sbk), sbj = dv(a.sbj);
  const long long sci = dv(a.sci), scj = dv(a.scj);
  const double* A = a.A + b1 * dv(a.sa1) + b2 * dv(a.sa2);
  const double* B = a.B + b1 * dv(a.sb1) + b2 * dv(a.sb2);
  double* C = a.C + b1 * dv(a.sc1) + b2 * dv(a.sc2);

  __shared__ T As[BK][TM + 1];
  __shared__ T Bs[BK][TN + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  T acc[RI][RJ];
#pragma unroll
  for (int ii = 0; ii < RI; ++ii)
#pragma unroll
    for (int jj = 0; jj < RJ; ++jj) acc[ii][jj] = T(0);
  const bool a_k_fast = (sak == 1);
  const bool b_j_fast = (sbj == 1);

  for (long long k0 = 0; k0 < K; k0 += BK) {
    for (int e = tid; e < BK * TM; e += NT) {
      int r, kk;
      if (a_k_fast) { kk = e % BK; r = e / BK; } else { r = e % TM; kk = e / TM; }
      const long long gi = i0 + r, gk = k0 + kk;
      As[kk][r] = (gi < M && gk < K) ? T(A[gi * sai + gk * sak]) : T(0);
    }
    for (int e = tid; e < BK * TN; e += NT) {
      int c, kk;
      if (b_j_fast) { c = e % TN; kk = e / TN; } else { kk = e % BK; c = e / BK; }
      const long long gj = j0 + c, gk = k0 + kk;
      Bs[kk][c] = (gj < N && gk < K) ? T(B[gk * sbk + gj * sbj]) : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T av[RI], bv[RJ];
#pragma unroll
      for (int ii = 0; ii < RI; ++ii) av[ii] = As[kk][ty + ii * 16];
#pragma unroll
      for (int jj = 0; jj < RJ; ++jj) bv[jj] = Bs[kk][tx + jj * 16];
#pragma unroll
      for (int ii = 0; ii < RI; ++ii)
#pragma unroll
        for (int jj = 0; jj < RJ; ++jj) acc[ii][jj] = fma(av[ii], bv[jj], acc[ii][jj]);
    }
    __syncthreads();
  }
  const double al = a.alpha, be = a.beta;
#pragma unroll
  for (int ii = 0; ii < RI; ++ii) {
    const long long gi = i0 + ty + ii * 16;
    if (gi >= M) continue;
#pragma unroll
    for (int jj = 0; jj < RJ; ++jj) {
      const long long gj = j0 + tx + jj * 16;
      if (gj >= N) continue;
      double* cp = C + gi * sci + gj * scj;
      double v = al * (double)acc[ii][jj];
      if (be != 0.0) v += be * (*cp);
      *cp = v;
    }
  }
}

template <typename T>
cudaError_t gemm_launch(const GemmArgs& a, long long Mmax, long long Nmax, long long nb1max, long long nb2max,
                        cudaStream_t st, int tile) {
  if (Mmax <= 0 || Nmax <= 0 || nb1max <= 0 || nb2max <= 0) return cudaSuccess;
  const long long gz = nb1max * nb2max;
  if (gz > 65535) return cudaErrorInvalidConfiguration;
  GemmKArgs ka{a, nb2max, g_flop_ctr};
  // 32x32 tiles when they already cover the SMs, else 16x16 tiles (4x the CTAs)
  const long long big = ((Nmax + 31) / 32) * ((Mmax + 31) / 32) * gz;
  if (tile == 0) tile = big >= device_sms() ? 32 : 16;
  if (tile != 16 && tile != 32) return cudaErrorInvalidValue;
  if (tile == 32) {
    const long long gx = (Nmax + 31) / 32, gy = (Mmax + 31) / 32;
    if (gx > 2147483647LL || gy > 65535) return cudaErrorInvalidConfiguration;
    gemm_kernel<T, 32, 32><<<dim3((unsigned)gx, (unsigned)gy, (unsigned)gz), NT, 0, st>>>(ka);
  } else {
    const long long gx = (Nmax + 15) / 16, gy = (Mmax + 15) / 16;
    if (gx > 2147483647LL || gy > 65535) return cudaErrorInvalidConfiguration;
    gemm_kernel<T, 16, 16><<<dim3((unsigned)gx, (unsigned)gy, (unsigned)gz), NT, 0, st>>>(ka);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t gemm_f64(const GemmArgs& a, long long Mmax, long long Nmax, long long nb1max, long long nb2max,
                     cudaStream_t st, int tile) {
  return gemm_launch<double>(a, Mmax, Nmax, nb1max, nb2max, st, tile);
}

cudaError_t gemm_f32(const GemmArgs& a, long long Mmax, long long Nmax, long long nb1max, long long nb2max,
                     cudaStream_t st, int tile) {
  return gemm_launch<float>(a, Mmax, Nmax, nb1max, nb2max, st, tile);
}

}  // namespace qtt
