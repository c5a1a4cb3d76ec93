// FP64 strided, batched GEMM with device-side sizes.
//
// Every contraction of the step (zip-up core contractions, absorption of R
// and U*S factors into neighbouring cores, the Hadamard contraction with the
// c^2 cores) is a small GEMM whose sizes are bond ranks held in device
// memory.  The kernel evaluates M, N, K, strides and batch offsets from
// device ints, so a step needs no host synchronisation.  Tiles are 32x32 so
// that the FP64 work spreads over all SMs (the FP64 pipe, not bandwidth,
// bounds these products on this part).
#include <algorithm>

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

// Gram matrix G = X X^T of nv vectors X_i (vector-major, X_i at X + i*ldx,
// length ell), FP64, split over the vector length: chunk s of the launch adds
// the products over its part of the length into P[s] (nvmax x nvmax), upper
// 32 x 32 tiles only (the matrix is symmetric); gram_reduce sums the chunks
// in a fixed order (the result does not depend on scheduling) and mirrors.
constexpr int GT = 32, GK = 16;

__global__ void __launch_bounds__(NT) gram_part_kernel(const double* __restrict__ X, Dim ldx_d, Dim nv_d, Dim ell_d,
                                                       long long nvmax, int chunks, double* __restrict__ P,
                                                       double* flops) {
  const long long nv = dv(nv_d), ell = dv(ell_d), ldx = dv(ldx_d);
  // upper tile (ti, tj), ti <= tj, from the linear index
  const int T = (int)((nvmax + GT - 1) / GT);
  int lin = blockIdx.x, ti = 0;
  while (lin >= T - ti) {
    lin -= T - ti;
    ++ti;
  }
  const int tj = ti + lin;
  const int sidx = blockIdx.y;
  if (flops && blockIdx.x == 0 && sidx == 0 && threadIdx.x == 0)
    atomicAdd(flops, (double)nv * (double)(nv + 1) * (double)ell);  // the triangle, 2 flops per product
  const long long i0 = (long long)ti * GT, j0 = (long long)tj * GT;
  if (i0 >= nv || j0 >= nv) return;
  const long long kc = ((ell + chunks - 1) / chunks + GK - 1) / GK * GK;
  const long long k_lo = (long long)sidx * kc, k_hi = k_lo + kc < ell ? k_lo + kc : ell;
  __shared__ double As[GK][GT + 1];
  __shared__ double Bs[GK][GT + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (long long k0 = k_lo; k0 < k_hi; k0 += GK) {
    for (int e = tid; e < GK * GT; e += NT) {
      const int kk = e % GK, r = e / GK;  // consecutive threads along the vector
      const long long gk = k0 + kk;
      As[kk][r] = (i0 + r < nv && gk < k_hi) ? X[(i0 + r) * ldx + gk] : 0.0;
      Bs[kk][r] = (j0 + r < nv && gk < k_hi) ? X[(j0 + r) * ldx + gk] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      const double a0 = As[kk][ty], a1 = As[kk][ty + 16], b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
      acc[0][0] = fma(a0, b0, acc[0][0]);
      acc[0][1] = fma(a0, b1, acc[0][1]);
      acc[1][0] = fma(a1, b0, acc[1][0]);
      acc[1][1] = fma(a1, b1, acc[1][1]);
    }
    __syncthreads();
  }
  double* Ps = P + (long long)sidx * nvmax * nvmax;
#pragma unroll
  for (int ii = 0; ii < 2; ++ii)
#pragma unroll
    for (int jj = 0; jj < 2; ++jj) {
      const long long gi = i0 + ty + 16 * ii, gj = j0 + tx + 16 * jj;
      if (gi < nv && gj < nv) Ps[gi * nvmax + gj] = acc[ii][jj];
    }
}

__global__ void gram_reduce_kernel(const double* __restrict__ P, Dim nv_d, long long nvmax, int chunks,
                                   double* __restrict__ G, long long ldg) {
  const long long nv = dv(nv_d);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nv * nv;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / nv, j = e % nv;
    // the chunks hold the upper tiles: (i, j) or its mirror
    const bool upper = (i / GT) <= (j / GT);
    const long long src = upper ? i * nvmax + j : j * nvmax + i;
    double v = 0.0;
    for (int s = 0; s < chunks; ++s) v += P[(long long)s * nvmax * nvmax + src];
    G[i * ldg + j] = v;
  }
}

}  // namespace

cudaError_t gram_f64(const double* X, Dim ldx, Dim nv, Dim ell, long long nvmax, long long ellmax, double* G,
                     long long ldg, double* P, int max_chunks, cudaStream_t st) {
  if (nvmax <= 0) return cudaSuccess;
  const long long T = (nvmax + GT - 1) / GT;
  // enough chunks for about four CTAs per SM, each at least 4 K-steps long
  const long long want = (4LL * device_sms() + T * (T + 1) / 2 - 1) / (T * (T + 1) / 2);
  int chunks = (int)std::max<long long>(1, std::min<long long>({(long long)max_chunks, want, (ellmax + 63) / 64}));
  gram_part_kernel<<<dim3((unsigned)(T * (T + 1) / 2), (unsigned)chunks), NT, 0, st>>>(X, ldx, nv, ell, nvmax, chunks,
                                                                                      P, g_flop_ctr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long tot = nvmax * nvmax;
  const int grid = (int)std::max<long long>(1, std::min<long long>((tot + 255) / 256, device_sms() * 4LL));
  gram_reduce_kernel<<<grid, 256, 0, st>>>(P, nv, nvmax, chunks, G, ldg);
  return cudaGetLastError();
}

cudaError_t gemm_f64(const GemmArgs& a, long long Mmax, long long Nmax, long long nb1max, long long nb2max,
                     cudaStream_t st, int tile) {
  return gemm_launch<double>(a, Mmax, Nmax, nb1max, nb2max, st, tile);
}

cudaError_t gemm_f32(const GemmArgs& a, long long Mmax, long long Nmax, long long nb1max, long long nb2max,
                     cudaStream_t st, int tile) {
  return gemm_launch<float>(a, Mmax, Nmax, nb1max, nb2max, st, tile);
}

}  // namespace qtt
