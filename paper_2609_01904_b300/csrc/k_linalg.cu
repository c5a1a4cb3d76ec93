// FP64 factorisations of the bond matrices (Sec. 4.3): Householder QR and
// one-sided (Hestenes) Jacobi SVD, each one cooperative launch over the SMs,
// plus the sort / truncation / gather that applies the Sec. 4.3 rule.
//
// Matrices are held "vector-major": column j of the factorised matrix is a
// contiguous run of doubles.  The QR gives each CTA a fixed set of columns;
// reflector j is formed by its owner and applied by every CTA after one grid
// barrier.  The Jacobi SVD rotates pairs of vectors in the round-robin
// (circle) order, one pair per CTA per round, one grid barrier per round,
// until a sweep performs no rotation.
#include "qtt_internal.cuh"

#include <algorithm>

namespace qtt {

namespace {

constexpr int NT = 256;

__device__ __forceinline__ void block_sum3(double& a, double& b, double& c, double* red /* 96 */) {
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) { red[w] = a; red[32 + w] = b; red[64 + w] = c; }
  __syncthreads();
  if (w == 0) {
    double x = l < nw ? red[l] : 0.0, y = l < nw ? red[32 + l] : 0.0, z = l < nw ? red[64 + l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      x += __shfl_xor_sync(0xffffffffu, x, o);
      y += __shfl_xor_sync(0xffffffffu, y, o);
      z += __shfl_xor_sync(0xffffffffu, z, o);
    }
    if (l == 0) { red[0] = x; red[32] = y; red[64] = z; }
  }
  __syncthreads();
  a = red[0]; b = red[32]; c = red[64];
  __syncthreads();
}

// --------------------------------------------------------------------- QR
__global__ void __launch_bounds__(NT) qr_kernel(const double* __restrict__ Ain, Dim lda_d, double* W, long long ldw,
                                                Dim m_d, Dim n_d, double* tau, double* Rout, int r_rowmajor,
                                                long long ldr, double* Qout, int* kq_out, DevSync* sync) {
  __shared__ double red[32];
  extern __shared__ double ysh[];
  const long long m = dv(m_d), n = dv(n_d), lda = dv(lda_d);
  const long long kq = m < n ? m : n;
  const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x;

  for (long long c = b; c < n; c += G)
    for (long long i = tid; i < m; i += NT) W[c * ldw + i] = Ain[c * lda + i];
  __syncthreads();

  for (long long j = 0; j < kq; ++j) {
    if (j % G == b) {
      double* x = W + j * ldw;
      double s = 0.0;
      for (long long i = j + 1 + tid; i < m; i += NT) s = fma(x[i], x[i], s);
      s = block_sum(s, red);
      const double alpha = x[j];
      double tj = 0.0, beta = alpha;
      if (s != 0.0) {
        double nrm = sqrt(alpha * alpha + s);
        beta = alpha >= 0.0 ? -nrm : nrm;
        tj = (beta - alpha) / beta;
        double sc = 1.0 / (alpha - beta);
        for (long long i = j + 1 + tid; i < m; i += NT) x[i] *= sc;
      }
      __syncthreads();
      if (tid == 0) {
        x[j] = beta;
        tau[j] = tj;
      }
    }
    if (!grid_sync(sync)) return;
    const double tj = tau[j];
    if (tj == 0.0) continue;
    const double* v = W + j * ldw;
    long long c0 = b + ((j + 1 - b + G - 1) / G) * G;  // first owned column > j
    if (j + 1 <= b) c0 = b;
    for (long long c = c0; c < n; c += G) {
      double* y = W + c * ldw;
      double s = 0.0;
      for (long long i = j + 1 + tid; i < m; i += NT) s = fma(v[i], y[i], s);
      s = block_sum(s, red);
      const double w = tj * (y[j] + s);
      __syncthreads();
      if (tid == 0) y[j] -= w;
      for (long long i = j + 1 + tid; i < m; i += NT) y[i] = fma(-w, v[i], y[i]);
    }
  }
  __syncthreads();

  // R: rows 0..kq-1 of the owned columns
  for (long long c = b; c < n; c += G) {
    for (long long i = tid; i < kq; i += NT) {
      double r = i <= c ? W[c * ldw + i] : 0.0;
      if (r_rowmajor) Rout[i * ldr + c] = r;
      else Rout[c * ldr + i] = r;
    }
  }
  if (kq_out && b == 0 && tid == 0) *kq_out = (int)kq;
  if (!Qout) return;

  // thin Q (m x kq, row-major): column c = H_0 ... H_c e_c, built in shared memory
  for (long long c = b; c < kq; c += G) {
    for (long long i = tid; i < m; i += NT) ysh[i] = (i == c) ? 1.0 : 0.0;
    __syncthreads();
    for (long long i = c; i >= 0; --i) {
      const double ti = tau[i];
      if (ti == 0.0) continue;
      const double* v = W + i * ldw;
      double s = 0.0;
      for (long long l = i + 1 + tid; l < m; l += NT) s = fma(v[l], ysh[l], s);
      s = block_sum(s, red);
      const double w = ti * (ysh[i] + s);
      __syncthreads();
      if (tid == 0) ysh[i] -= w;
      for (long long l = i + 1 + tid; l < m; l += NT) ysh[l] = fma(-w, v[l], ysh[l]);
      __syncthreads();
    }
    for (long long i = tid; i < m; i += NT) Qout[i * kq + c] = ysh[i];
    __syncthreads();
  }
}

// ----------------------------------------------------------------- Jacobi
__device__ __forceinline__ void circle_pair(long long rd, long long q, long long P, long long& i, long long& j) {
  const long long R = P - 1;
  if (q == 0) {
    i = R;
    j = rd;
  } else {
    i = (rd + q) % R;
    j = (rd - q + R) % R;
  }
}

__global__ void __launch_bounds__(NT) jacobi_kernel(double* V, long long ldv, Dim nv_d, Dim m_d, double* J,
                                                    long long ldj, double* norms, DevSync* sync, int max_sweeps,
                                                    double tol, double tol_abs, int* log) {
  __shared__ double red[96];
  const long long nv = dv(nv_d), m = dv(m_d);
  if (log && blockIdx.x == 0 && threadIdx.x == 0) {
    log[0] = (int)nv;
    log[1] = (int)m;
  }
  const long long P = nv + (nv & 1);
  const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x;

  for (long long c = b; c < nv; c += G)
    for (long long i = tid; i < nv; i += NT) J[c * ldj + i] = (i == c) ? 1.0 : 0.0;
  if (b == 0 && tid == 0) {
    sync->counters[0] = 0;
    sync->counters[1] = 0;
  }
  if (!grid_sync(sync)) return;

  int sweep = 0;
  if (nv >= 2) {
    for (sweep = 0; sweep < max_sweeps; ++sweep) {
      int local = 0;
      for (long long rd = 0; rd < P - 1; ++rd) {
        for (long long q = b; q < P / 2; q += G) {
          long long i, j;
          circle_pair(rd, q, P, i, j);
          if (i >= nv || j >= nv) continue;
          double* vi = V + i * ldv;
          double* vj = V + j * ldv;
          double a = 0.0, bb = 0.0, g = 0.0;
          for (long long l = tid; l < m; l += NT) {
            double x = vi[l], y = vj[l];
            a = fma(x, x, a);
            bb = fma(y, y, bb);
            g = fma(x, y, g);
          }
          block_sum3(a, bb, g, red);
          // rotate unless the pair is orthogonal to working precision, measured
          // against both vectors and against the larger one alone (a pair whose
          // norms differ by more than 1/tol cannot be made more orthogonal)
          if (g != 0.0 && fabs(g) > tol * sqrt(a) * sqrt(bb) && fabs(g) > tol_abs * fmax(a, bb)) {
            const double zeta = (bb - a) / (2.0 * g);
            const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
            for (long long l = tid; l < m; l += NT) {
              double x = vi[l], y = vj[l];
              vi[l] = cs * x - sn * y;
              vj[l] = sn * x + cs * y;
            }
            double* Ji = J + i * ldj;
            double* Jj = J + j * ldj;
            for (long long l = tid; l < nv; l += NT) {
              double x = Ji[l], y = Jj[l];
              Ji[l] = cs * x - sn * y;
              Jj[l] = sn * x + cs * y;
            }
            ++local;
          }
        }
        if (!grid_sync(sync)) return;
        if (rd == 0 && b == 0 && tid == 0) sync->counters[(sweep + 1) & 1] = 0;
      }
      if (tid == 0 && local) atomicAdd(&sync->counters[sweep & 1], local);
      if (!grid_sync(sync)) return;
      int total = *(volatile int*)&sync->counters[sweep & 1];
      if (total == 0) break;
    }
    if (sweep >= max_sweeps && b == 0 && tid == 0) set_status(sync, QTT_ENOCONV);
  }
  // final norms
  for (long long c = b; c < nv; c += G) {
    const double* vc = V + c * ldv;
    double s = 0.0;
    for (long long l = tid; l < m; l += NT) s = fma(vc[l], vc[l], s);
    s = block_sum(s, red);
    if (tid == 0) norms[c] = sqrt(s);
  }
}

// ------------------------------------------------------ sort + truncation
__global__ void __launch_bounds__(1024) svd_post_kernel(const double* norms, Dim cnt_d, Dim len_d, Dim jlen_d,
                                                        const double* J, long long ldj, double eps, int chi,
                                                        int rank_cap, int* rank_out, double* sigma_out,
                                                        double* disc_out, double* Jp, double* Jt, DevSync* sync) {
  extern __shared__ double sh[];
  // cnt rotated vectors (norms), each a combination of jlen input vectors
  // (row perm_j of J has jlen entries); they span min(cnt, len) directions
  const int nv = (int)dv(cnt_d);
  const long long len = dv(len_d);
  const int jl = (int)dv(jlen_d);
  const int nsv = (int)(len < nv ? len : nv);
  double* s = sh;
  double* ss = sh + nv;
  int* perm = (int*)(sh + 2 * nv);
  __shared__ int s_r;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < nv; i += nt) {
    double v = norms[i];
    if (!isfinite(v)) set_status(sync, QTT_ENONFINITE);
    s[i] = isfinite(v) ? v : 0.0;
  }
  __syncthreads();
  for (int i = tid; i < nv; i += nt) {
    const double si = s[i];
    int r = 0;
    for (int j = 0; j < nv; ++j) {
      const double sj = s[j];
      r += (sj > si) || (sj == si && j < i);
    }
    perm[r] = i;
  }
  __syncthreads();
  for (int i = tid; i < nv; i += nt) ss[i] = s[perm[i]];
  __syncthreads();
  if (tid == 0) {
    int r = 1;
    if (nv > 0 && ss[0] > 0.0) {
      const double thr = eps * ss[0];
      r = 0;
      while (r < nv && ss[r] >= thr) ++r;
    }
    if (chi > 0 && r > chi) r = chi;
    if (r > nsv) r = nsv;
    if (r < 1) r = 1;
    if (r > rank_cap) {  // never write past the destination core
      set_status(sync, QTT_EINVAL);
      r = rank_cap;
    }
    double dsum = 0.0;
    for (int i = r; i < nv; ++i) dsum += ss[i] * ss[i];
    s_r = r;
    if (rank_out) *rank_out = r;
    if (disc_out) *disc_out = dsum;
  }
  __syncthreads();
  const int r = s_r;
  if (sigma_out)
    for (int i = tid; i < nv; i += nt) sigma_out[i] = ss[i];
  for (long long e = tid; e < (long long)r * jl; e += nt) {
    const int j = (int)(e / jl), i = (int)(e % jl);
    const double v = J[(long long)perm[j] * ldj + i];
    if (Jp) Jp[e] = v;
    if (Jt) Jt[(long long)i * r + j] = v;
  }
}

}  // namespace

static cudaError_t coop_launch(const void* fn, int grid, int block, void** args, size_t smem, cudaStream_t st) {
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(block), args, smem, st);
}

cudaError_t qr_f64(qtt_ctx* ctx, const double* Ain, Dim lda, double* W, long long ldw, Dim m, Dim n, long long nmax,
                   double* Rout, bool r_rowmajor, double* Qout, int* kq_out, long long ldr, long long qm_max) {
  int grid = (int)std::min<long long>(ctx->coop_blocks, std::max<long long>(nmax, 1));
  size_t smem = 0;
  if (Qout) smem = (size_t)qm_max * sizeof(double);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  double* tau = ctx->ws.d_tau;
  int rrm = r_rowmajor ? 1 : 0;
  DevSync* sync = ctx->ws.d_sync;
  void* args[] = {(void*)&Ain, (void*)&lda, (void*)&W, (void*)&ldw, (void*)&m, (void*)&n, (void*)&tau,
                  (void*)&Rout, (void*)&rrm, (void*)&ldr, (void*)&Qout, (void*)&kq_out, (void*)&sync};
  return coop_launch((const void*)qr_kernel, grid, NT, args, smem, ctx->stream);
}

cudaError_t jacobi_f64(qtt_ctx* ctx, double* V, long long ldv, Dim nv, Dim m, long long nvmax, double* J,
                       long long ldj, double* norms) {
  long long pairs = (nvmax + 1) / 2;
  int grid = (int)std::min<long long>(ctx->coop_blocks, std::max<long long>(pairs, 1));
  DevSync* sync = ctx->ws.d_sync;
  int max_sweeps = 100;
  // a pair counts as orthogonal when |v_i.v_j| <= 1e-13 |v_i||v_j| (above the
  // rounding floor of accumulated rotations) or <= 1e-15 max(|v_i|^2, |v_j|^2)
  double tol = 1e-13, tol_abs = 1e-15;
  int* log = jacobi_log_slot(ctx);
  void* args[] = {(void*)&V, (void*)&ldv, (void*)&nv, (void*)&m, (void*)&J, (void*)&ldj, (void*)&norms,
                  (void*)&sync, (void*)&max_sweeps, (void*)&tol, (void*)&tol_abs, (void*)&log};
  return coop_launch((const void*)jacobi_kernel, grid, NT, args, 0, ctx->stream);
}

cudaError_t svd_post(qtt_ctx* ctx, const double* norms, Dim cnt, Dim len, Dim jlen, const double* J, long long ldj,
                     double eps, int chi, int rank_cap, int* rank_out, double* sigma_out, double* disc_out,
                     double* Jp, double* Jt) {
  long long nvmax = ldj;
  size_t smem = (size_t)nvmax * (2 * sizeof(double) + sizeof(int)) + 16;
  svd_post_kernel<<<1, 1024, smem, ctx->stream>>>(norms, cnt, len, jlen, J, ldj, eps, chi, rank_cap, rank_out,
                                                  sigma_out, disc_out, Jp, Jt, ctx->ws.d_sync);
  return cudaGetLastError();
}

int* jacobi_log_slot(qtt_ctx* ctx) {
  Prof& p = ctx->prof;
  if (!p.d_log || p.log_used >= p.log_cap) return nullptr;
  return p.d_log + 2 * (p.log_used++);
}

cudaError_t linalg_init(int device) {
  cudaError_t e = cudaFuncSetAttribute((const void*)qr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       200 * 1024);
  if (e != cudaSuccess) return e;
  return cudaSuccess;
}

int coop_max_blocks(int num_sms) {
  int a = 0, b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, (const void*)jacobi_kernel, NT, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, (const void*)qr_kernel, NT, 200 * 1024);
  int per = std::min(std::max(a, 1), std::max(b, 1));
  (void)per;
  // one CTA per SM: the FP64 pipe is per SM, more CTAs only add barrier traffic
  return num_sms;
}

}  // namespace qtt
