// MPS-level kernels: the MPO contraction of the zip-up, the block-diagonal
// MPS sum with the rank-1 source (Sec. 4.3, Eq. 17), receiver sampling and
// the dense reconstruction (Eq. 8), the grid -> site-tensor permutation
// (Eq. 3, Eq. 12 order), the dense FDTD update (Eq. 2) and small helpers.
#include "qtt_internal.cuh"

#include "k_mps.cuh"

namespace qtt {

namespace {


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
        if (k == 0) v *= (a.src_amp_dev ? *a.src_amp_dev : a.src_amp) * (a.amp_scale ? *a.amp_scale : 1.0);
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
    const long long N = 1LL << a.n;
    long long lin = a.ix[p];
    if (a.dims == 3) lin = lin * N + a.iy[p];
    lin = lin * N + a.iz[p];
    if (threadIdx.x == 0) v[0] = 1.0;
    __syncthreads();
    int rl = 1;
    for (int k = 0; k < a.d; ++k) {
      const int bit = (int)((lin >> a.sp.pos[k]) & 1);
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

// dense[i] = S[L][R] with (L, R) the site bits of dense index i: sites below h
// give L, the others R
__global__ void scatter_dense_kernel(const double* __restrict__ S, double* __restrict__ out, SitePos sp, int h) {
  const int d = sp.d;
  const long long total = 1LL << d;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    long long L = 0, R = 0;
    for (int k = 0; k < d; ++k) {
      const long long b = (idx >> sp.pos[k]) & 1;
      if (k < h) L |= b << k;
      else R |= b << (k - h);
    }
    out[idx] = S[L * (1LL << (d - h)) + R];
  }
}

// site tensor t[Lin], Lin = sum_k s_k 2^(d-1-k) (site 0 slowest), from the dense u
__global__ void site_permute_kernel(const double* __restrict__ u, double* __restrict__ t, SitePos sp, int square) {
  const int d = sp.d;
  const long long total = 1LL << d;
  for (long long lin = blockIdx.x * (long long)blockDim.x + threadIdx.x; lin < total;
       lin += (long long)gridDim.x * blockDim.x) {
    long long idx = 0;
    for (int k = 0; k < d; ++k) idx |= ((lin >> (d - 1 - k)) & 1) << sp.pos[k];
    const double v = u[idx];
    t[lin] = square ? v * v : v;
  }
}

// Eq. 2 with the 7-point stencil (the 3D extension)
__global__ void fdtd3_kernel(const double* __restrict__ c2, double lambda2, const double* __restrict__ up,
                             const double* __restrict__ uc, double* __restrict__ un, int n, int bc, long long sx,
                             long long sy, long long sz, double amp) {
  const long long N = 1LL << n, M = N - 1, total = N * N * N;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long x = idx >> (2 * n), y = (idx >> n) & M, z = idx & M;
    const double c = uc[idx];
    double nb;
    if (bc == QTT_BC_PERIODIC) {
      nb = uc[((((x + 1) & M) * N + y) << n) + z] + uc[((((x - 1) & M) * N + y) << n) + z] +
           uc[((x * N + ((y + 1) & M)) << n) + z] + uc[((x * N + ((y - 1) & M)) << n) + z] +
           uc[((x * N + y) << n) + ((z + 1) & M)] + uc[((x * N + y) << n) + ((z - 1) & M)];
    } else {
      nb = (x + 1 < N ? uc[idx + N * N] : 0.0) + (x > 0 ? uc[idx - N * N] : 0.0) + (y + 1 < N ? uc[idx + N] : 0.0) +
           (y > 0 ? uc[idx - N] : 0.0) + (z + 1 < N ? uc[idx + 1] : 0.0) + (z > 0 ? uc[idx - 1] : 0.0);
    }
    double v = 2.0 * c - up[idx] + lambda2 * c2[idx] * (nb - 6.0 * c);
    if (x == sx && y == sy && z == sz) v += amp;
    un[idx] = v;
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

__global__ void __launch_bounds__(256) state_scale_prepare_kernel(const double* a, const int* ra, const double* b,
                                                                 const int* rb, double* scale) {
  __shared__ double red[32];
  double m = 0.0;
  const long long na = 2LL * *ra, nb = 2LL * *rb;
  for (long long i = threadIdx.x; i < na; i += blockDim.x) m = fmax(m, fabs(a[i]));
  for (long long i = threadIdx.x; i < nb; i += blockDim.x) m = fmax(m, fabs(b[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
    m = fmax(m, red[0]);
    int e = 0;
    if (m > 0.0 && isfinite(m)) frexp(m, &e);  // m = f 2^e, f in [0.5, 1)
    scale[0] = ldexp(1.0, -e);
    scale[1] = ldexp(1.0, e);
  }
}

__global__ void state_scale_apply_kernel(double* core, const int* r, const double* scale, int which) {
  const long long n = 2LL * *r;
  const double f = scale[which];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    core[i] *= f;
}

inline int grid_for(long long total, int nt) {
  long long g = (total + nt - 1) / nt;
  if (g < 1) g = 1;
  if (g > device_sms() * 32LL) g = device_sms() * 32LL;
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
  int g = (int)std::min<long long>(a.count, device_sms() * 8LL);
  if (g < 1) return cudaSuccess;
  sample_kernel<<<g, 128, 2 * a.rmax * sizeof(double), st>>>(a);
  return cudaGetLastError();
}

cudaError_t chains(const ChainArgs& left, const ChainArgs& right, cudaStream_t st) {
  long long nL = 1LL << left.h, nR = 1LL << (right.d - right.h);
  left_chain_kernel<<<(int)std::min<long long>(nL, device_sms() * 8LL), 128, 2 * left.rmax * sizeof(double), st>>>(left);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  right_chain_kernel<<<(int)std::min<long long>(nR, device_sms() * 8LL), 128, 2 * right.rmax * sizeof(double), st>>>(right);
  return cudaGetLastError();
}

cudaError_t state_scale_prepare(const double* a, const int* ra, const double* b, const int* rb, long long rmax,
                                double* scale, cudaStream_t st) {
  (void)rmax;
  state_scale_prepare_kernel<<<1, 256, 0, st>>>(a, ra, b, rb, scale);
  return cudaGetLastError();
}

cudaError_t state_scale_apply(double* core, const int* r, long long rmax, const double* scale, int which,
                              cudaStream_t st) {
  state_scale_apply_kernel<<<grid_for(2 * rmax, 256), 256, 0, st>>>(core, r, scale, which);
  return cudaGetLastError();
}

cudaError_t scatter_dense(const double* S, double* out, const SitePos& sp, int h, cudaStream_t st) {
  scatter_dense_kernel<<<grid_for(1LL << sp.d, 256), 256, 0, st>>>(S, out, sp, h);
  return cudaGetLastError();
}

cudaError_t site_permute(const double* u, double* t, const SitePos& sp, bool square, cudaStream_t st) {
  site_permute_kernel<<<grid_for(1LL << sp.d, 256), 256, 0, st>>>(u, t, sp, square ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t fdtd3(const double* c2, double lambda2, const double* up, const double* uc, double* un, int n, int bc,
                  long long sx, long long sy, long long sz, double amp, cudaStream_t st) {
  fdtd3_kernel<<<grid_for(1LL << (3 * n), 256), 256, 0, st>>>(c2, lambda2, up, uc, un, n, bc, sx, sy, sz, amp);
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
