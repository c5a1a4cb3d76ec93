// MPS-level kernels: the MPO contraction of the zip-up, the block-diagonal
// MPS sum with the rank-1 source (Sec. 4.3, Eq. 17), receiver sampling and
// the dense reconstruction (Eq. 8), the grid -> site-tensor permutation
// (Eq. 3, Eq. 12 order), the dense FDTD update (Eq. 2) and small helpers.
#include "qtt_internal.cuh"

#include "k_mps.cuh"

namespace qtt {

namespace {

__device__ __forceinline__ int site_bit(long long ix, long long iz, int k, int n, int order) {
  if (order == QTT_ORDER_SEQUENTIAL) return k < n ? (int)((ix >> k) & 1) : (int)((iz >> (k - n)) & 1);
  return (k & 1) ? (int)((iz >> (k >> 1)) & 1) : (int)((ix >> (k >> 1)) & 1);
}

// T[(a,t)][(w',b')] = sum_{w,s} W[w][t][s][w'] X[(a,w)][(s,b')]
__global__ void mpo_apply_lr_kernel(const double* __restrict__ X, double* __restrict__ T,
                                    const double* __restrict__ W, int w, int w2, const int* a_p,
                                    const int* b2_p) {
  const long long a = *a_p, B2 = *b2_p, ell = (long long)w2 * B2;
  const long long total = a * 2 * ell;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long e = idx % ell, row = idx / ell;
    const int t = (int)(row & 1);
    const long long ai = row >> 1;
    const int wp = (int)(e / B2);
    const long long bp = e % B2;
    double acc = 0.0;
    for (int wi = 0; wi < w; ++wi) {
      const double* xr = X + ((ai * w + wi) * 2) * B2 + bp;
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const double c = W[((wi * 2 + t) * 2 + s) * w2 + wp];
        if (c != 0.0) acc = fma(c, xr[s * B2], acc);
      }
    }
    T[row * ell + e] = acc;
  }
}

__global__ void mps_sum_kernel(SumArgs a) {
  const int k = blockIdx.y, d = a.d;
  // bond sums
  __shared__ long long offL[kMaxTerms + 1], offR[kMaxTerms + 1];
  if (threadIdx.x == 0) {
    offL[0] = 0;
    offR[0] = 0;
    for (int t = 0; t < a.nterms; ++t) {
      offL[t + 1] = offL[t] + (k == 0 ? 1 : a.ranks[t][k]);
      offR[t + 1] = offR[t] + (k == d - 1 ? 1 : a.ranks[t][k + 1]);
    }
    if (a.has_src) {
      offL[a.nterms + 1] = offL[a.nterms] + 1;
      offR[a.nterms + 1] = offR[a.nterms] + 1;
    }
  }
  __syncthreads();
  const int nt = a.nterms + (a.has_src ? 1 : 0);
  const long long Dl = (k == 0) ? 1 : offL[nt];
  const long long Dr = (k == d - 1) ? 1 : offR[nt];
  if (k == 0 && blockIdx.x == 0) {
    for (int kk = threadIdx.x; kk <= d; kk += blockDim.x) {
      int s = 0;
      if (kk == 0 || kk == d) s = 1;
      else {
        for (int t = 0; t < a.nterms; ++t) s += a.ranks[t][kk];
        s += a.has_src ? 1 : 0;
      }
      a.out_ranks[kk] = s;
    }
  }
  double* out = a.out[k];
  const long long total = Dl * 2 * Dr;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / (2 * Dr), s = (e / Dr) & 1, j = e % Dr;
    // term owning this row (k > 0) or column (k == 0)
    int t = 0;
    if (k == 0) {
      while (t < nt - 1 && j >= offR[t + 1]) ++t;
    } else {
      while (t < nt - 1 && i >= offL[t + 1]) ++t;
    }
    double v = 0.0;
    const long long li = (k == 0) ? 0 : i - offL[t];
    const long long lj = (k == d - 1) ? 0 : j - offR[t];
    const bool inside = (k == 0 || k == d - 1) ? true : (j >= offR[t] && j < offR[t + 1]);
    if (k == d - 1 && !(i >= offL[t] && i < offL[t + 1])) {
      v = 0.0;
    } else if (inside) {
      if (t < a.nterms) {
        const long long rr = (k == d - 1) ? 1 : a.ranks[t][k + 1];
        v = a.core[t][k][(li * 2 + s) * rr + lj];
        if (k == 0) v *= a.coef[t];
      } else {  // rank-1 source: one-hot on the source's bits
        v = (s == a.src_bits[k]) ? 1.0 : 0.0;
        if (k == 0) v *= a.src_amp_dev ? *a.src_amp_dev : a.src_amp;
      }
    }
    out[e] = v;
  }
}

__global__ void sample_kernel(SampleArgs a) {
  extern __shared__ double sh[];
  double* v = sh;
  double* v2 = sh + a.rmax;
  for (long long p = blockIdx.x; p < a.count; p += gridDim.x) {
    const long long ix = a.ix[p], iz = a.iz[p];
    if (threadIdx.x == 0) v[0] = 1.0;
    __syncthreads();
    int rl = 1;
    for (int k = 0; k < a.d; ++k) {
      const int bit = site_bit(ix, iz, k, a.n, a.order);
      const int rr = a.ranks[k + 1];
      const double* c = a.core[k];
      for (int j = threadIdx.x; j < rr; j += blockDim.x) {
        double acc = 0.0;
        for (int i = 0; i < rl; ++i) acc = fma(v[i], c[((long long)i * 2 + bit) * rr + j], acc);
        v2[j] = acc;
      }
      __syncthreads();
      for (int j = threadIdx.x; j < rr; j += blockDim.x) v[j] = v2[j];
      __syncthreads();
      rl = rr;
    }
    if (threadIdx.x == 0) a.out[p] = v[0];
    __syncthreads();
  }
}

// left partial products: Lm[L][j] = (A_0[s_0] ... A_{h-1}[s_{h-1}])_j, s_k = bit k of L
__global__ void left_chain_kernel(ChainArgs a) {
  extern __shared__ double sh[];
  double* v = sh;
  double* v2 = sh + a.rmax;
  const long long nL = 1LL << a.h;
  for (long long L = blockIdx.x; L < nL; L += gridDim.x) {
    if (threadIdx.x == 0) v[0] = 1.0;
    __syncthreads();
    int rl = 1;
    for (int k = 0; k < a.h; ++k) {
      const int bit = (int)((L >> k) & 1);
      const int rr = a.ranks[k + 1];
      const double* c = a.core[k];
      for (int j = threadIdx.x; j < rr; j += blockDim.x) {
        double acc = 0.0;
        for (int i = 0; i < rl; ++i) acc = fma(v[i], c[((long long)i * 2 + bit) * rr + j], acc);
        v2[j] = acc;
      }
      __syncthreads();
      for (int j = threadIdx.x; j < rr; j += blockDim.x) v[j] = v2[j];
      __syncthreads();
      rl = rr;
    }
    for (int j = threadIdx.x; j < rl; j += blockDim.x) a.out[L * rl + j] = v[j];
    __syncthreads();
  }
}

// right partial products: Rm[i][R] = (A_h[s_h] ... A_{d-1}[s_{d-1}])_i, s_{h+k} = bit k of R
__global__ void right_chain_kernel(ChainArgs a) {
  extern __shared__ double sh[];
  double* v = sh;
  double* v2 = sh + a.rmax;
  const int nr = a.d - a.h;
  const long long nR = 1LL << nr;
  const int rh = a.ranks[a.h];
  for (long long R = blockIdx.x; R < nR; R += gridDim.x) {
    if (threadIdx.x == 0) v[0] = 1.0;
    __syncthreads();
    int rr = 1;
    for (int k = a.d - 1; k >= a.h; --k) {
      const int bit = (int)((R >> (k - a.h)) & 1);
      const int rl = a.ranks[k];
      const double* c = a.core[k];
      for (int i = threadIdx.x; i < rl; i += blockDim.x) {
        double acc = 0.0;
        const double* ci = c + ((long long)i * 2 + bit) * rr;
        for (int j = 0; j < rr; ++j) acc = fma(ci[j], v[j], acc);
        v2[i] = acc;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < rl; i += blockDim.x) v[i] = v2[i];
      __syncthreads();
      rr = rl;
    }
    for (int i = threadIdx.x; i < rh; i += blockDim.x) a.out[(long long)i * nR + R] = v[i];
    __syncthreads();
  }
}

// dense[x*N+z] = S[L][R] with (L, R) the site bits of (x, z)
__global__ void scatter_dense_kernel(const double* __restrict__ S, double* __restrict__ out, int n, int order,
                                     int h) {
  const long long N = 1LL << n, total = N * N;
  const int d = 2 * n;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long x = idx / N, z = idx % N;
    long long L = 0, R = 0;
    for (int k = 0; k < d; ++k) {
      long long b = site_bit(x, z, k, n, order);
      if (k < h) L |= b << k;
      else R |= b << (k - h);
    }
    out[idx] = S[L * (1LL << (d - h)) + R];
  }
}

// site tensor t[Lin], Lin = sum_k s_k 2^(d-1-k) (site 0 slowest), from u[x*N+z]
__global__ void site_permute_kernel(const double* __restrict__ u, double* __restrict__ t, int n, int order,
                                    int square) {
  const int d = 2 * n;
  const long long N = 1LL << n, total = N * N;
  for (long long lin = blockIdx.x * (long long)blockDim.x + threadIdx.x; lin < total;
       lin += (long long)gridDim.x * blockDim.x) {
    long long x = 0, z = 0;
    for (int k = 0; k < d; ++k) {
      const long long s = (lin >> (d - 1 - k)) & 1;
      if (order == QTT_ORDER_SEQUENTIAL) {
        if (k < n) x |= s << k;
        else z |= s << (k - n);
      } else {
        if (k & 1) z |= s << (k >> 1);
        else x |= s << (k >> 1);
      }
    }
    double v = u[x * N + z];
    t[lin] = square ? v * v : v;
  }
}

__global__ void fdtd_kernel(const double* __restrict__ c2, double lambda2, const double* __restrict__ up,
                            const double* __restrict__ uc, double* __restrict__ un, int n, int bc, long long sx,
                            long long sz, double amp) {
  const long long N = 1LL << n, total = N * N;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long x = idx >> n, z = idx & (N - 1);  // N = 2^n
    const double c = uc[idx];
    double nb;
    if (bc == QTT_BC_PERIODIC) {
      nb = uc[((x + 1) & (N - 1)) * N + z] + uc[((x - 1) & (N - 1)) * N + z] + uc[x * N + ((z + 1) & (N - 1))] +
           uc[x * N + ((z - 1) & (N - 1))];
    } else {
      nb = (x + 1 < N ? uc[(x + 1) * N + z] : 0.0) + (x > 0 ? uc[(x - 1) * N + z] : 0.0) +
           (z + 1 < N ? uc[x * N + z + 1] : 0.0) + (z > 0 ? uc[x * N + z - 1] : 0.0);
    }
    double v = 2.0 * c - up[idx] + lambda2 * c2[idx] * (nb - 4.0 * c);
    if (x == sx && z == sz) v += amp;
    un[idx] = v;
  }
}

__global__ void copy2d_kernel(const double* __restrict__ src, double* __restrict__ dst, Dim R, Dim C, Dim ssi,
                              Dim ssj, Dim dsi, Dim dsj, double alpha) {
  const long long r = dv(R), c = dv(C);
  const long long a = dv(ssi), b = dv(ssj), e = dv(dsi), f = dv(dsj);
  const long long total = r * c;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long i = idx / c, j = idx % c;
    dst[i * e + j * f] = alpha * src[i * a + j * b];
  }
}

__global__ void init_kernel(double* carry, int* ranks, int d, const int* copy_src, int* copy_dst, int ncopy) {
  if (threadIdx.x == 0) {
    if (carry) carry[0] = 1.0;
    if (ranks) {
      ranks[0] = 1;
      ranks[d] = 1;
    }
  }
  for (int i = threadIdx.x; i < ncopy; i += blockDim.x) copy_dst[i] = copy_src[i];
}

// rows j < r of M (ld ldm) scaled by 1/sigma_j (0 where sigma_j == 0)
__global__ void scale_rows_kernel(double* M, long long ldm, Dim ncols, const int* r_p, const double* sigma) {
  const long long r = *r_p, nc = dv(ncols);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < r * nc;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long j = idx / nc, c = idx % nc;
    const double s = sigma[j];
    M[j * ldm + c] = s > 0.0 ? M[j * ldm + c] / s : 0.0;
  }
}

inline int grid_for(long long total, int nt) {
  long long g = (total + nt - 1) / nt;
  if (g < 1) g = 1;
  if (g > 148 * 32) g = 148 * 32;
  return (int)g;
}

}  // namespace

cudaError_t mpo_apply_lr(const double* X, double* T, const double* W, int w, int w2, const int* a_p, const int* b2_p,
                         long long total_max, cudaStream_t st) {
  mpo_apply_lr_kernel<<<grid_for(total_max, 256), 256, 0, st>>>(X, T, W, w, w2, a_p, b2_p);
  return cudaGetLastError();
}

cudaError_t mps_sum(const SumArgs& a, long long max_core_elems, cudaStream_t st) {
  dim3 g(grid_for(max_core_elems, 256) / 4 + 1, a.d);
  mps_sum_kernel<<<g, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t sample(const SampleArgs& a, cudaStream_t st) {
  int g = (int)std::min<long long>(a.count, 148 * 8);
  if (g < 1) return cudaSuccess;
  sample_kernel<<<g, 128, 2 * a.rmax * sizeof(double), st>>>(a);
  return cudaGetLastError();
}

cudaError_t chains(const ChainArgs& left, const ChainArgs& right, cudaStream_t st) {
  long long nL = 1LL << left.h, nR = 1LL << (right.d - right.h);
  left_chain_kernel<<<(int)std::min<long long>(nL, 148 * 8), 128, 2 * left.rmax * sizeof(double), st>>>(left);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  right_chain_kernel<<<(int)std::min<long long>(nR, 148 * 8), 128, 2 * right.rmax * sizeof(double), st>>>(right);
  return cudaGetLastError();
}

cudaError_t scatter_dense(const double* S, double* out, int n, int order, int h, cudaStream_t st) {
  long long total = 1LL << (2 * n);
  scatter_dense_kernel<<<grid_for(total, 256), 256, 0, st>>>(S, out, n, order, h);
  return cudaGetLastError();
}

cudaError_t site_permute(const double* u, double* t, int n, int order, bool square, cudaStream_t st) {
  long long total = 1LL << (2 * n);
  site_permute_kernel<<<grid_for(total, 256), 256, 0, st>>>(u, t, n, order, square ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t fdtd(const double* c2, double lambda2, const double* up, const double* uc, double* un, int n, int bc,
                 long long sx, long long sz, double amp, cudaStream_t st) {
  long long total = 1LL << (2 * n);
  fdtd_kernel<<<grid_for(total, 256), 256, 0, st>>>(c2, lambda2, up, uc, un, n, bc, sx, sz, amp);
  return cudaGetLastError();
}

cudaError_t copy2d(const double* src, double* dst, Dim R, Dim C, Dim ssi, Dim ssj, Dim dsi, Dim dsj,
                   long long total_max, double alpha, cudaStream_t st) {
  copy2d_kernel<<<grid_for(total_max, 256), 256, 0, st>>>(src, dst, R, C, ssi, ssj, dsi, dsj, alpha);
  return cudaGetLastError();
}

cudaError_t init_zip(double* carry, int* ranks, int d, const int* copy_src, int* copy_dst, int ncopy,
                     cudaStream_t st) {
  init_kernel<<<1, 64, 0, st>>>(carry, ranks, d, copy_src, copy_dst, ncopy);
  return cudaGetLastError();
}

cudaError_t scale_rows(double* M, long long ldm, Dim ncols, const int* r_p, const double* sigma, long long total_max,
                       cudaStream_t st) {
  scale_rows_kernel<<<grid_for(total_max, 256), 256, 0, st>>>(M, ldm, ncols, r_p, sigma);
  return cudaGetLastError();
}

}  // namespace qtt
