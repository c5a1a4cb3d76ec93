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
constexpr int kQrQCols = 4;  // columns of the thin Q a CTA forms together
constexpr int kRegE = 2;  // register-resident Jacobi pairs up to NT * kRegE = 512 elements

// Block-wide sums of N values per thread (red: 32 N entries).
template <typename T, int N>
__device__ __forceinline__ void block_sum_n(T (&v)[N], T* red) {
#pragma unroll
  for (int k = 0; k < N; ++k)
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0)
#pragma unroll
    for (int k = 0; k < N; ++k) red[32 * k + w] = v[k];
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      T t = l < nw ? red[32 * k + l] : T(0);
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (l == 0) red[32 * k] = t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < N; ++k) v[k] = red[32 * k];
  __syncthreads();
}

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
// Column c belongs to CTA c % G for the whole factorisation.  Reflector j is
// formed by the owner of column j and published through flag[j]; a CTA
// applies reflector j to its columns as soon as the flag is set.  The owner
// of column j+1 applies reflector j to that column first and then forms
// reflector j+1 (lookahead), so the critical path per column is one flag
// hand-over plus one apply and one formation.
template <typename T>
__device__ __forceinline__ T sqrt_t(T x) { return sqrt(x); }

template <typename T, int B>
__device__ __forceinline__ void qr_form(T* x, long long j, long long m, T* tau, T* red) {
  const int tid = threadIdx.x;
  T s = T(0);
  for (long long i = j + 1 + tid; i < m; i += B) s = fma(x[i], x[i], s);
  s = block_sum(s, red);
  const T alpha = x[j];
  T tj = T(0), beta = alpha;
  if (s != T(0)) {
    const T nrm = sqrt_t(alpha * alpha + s);
    beta = alpha >= T(0) ? -nrm : nrm;
    tj = (beta - alpha) / beta;
    const T sc = T(1) / (alpha - beta);
    for (long long i = j + 1 + tid; i < m; i += B) x[i] *= sc;
  }
  __syncthreads();
  if (tid == 0) {
    x[j] = beta;
    tau[j] = tj;
  }
}

// y <- (I - tau v v^T) y on rows j..m-1 (v_j = 1 implicit); v is another CTA's
// column, read through L2 once: up to kApplyRegs entries per thread stay in
// registers between the dot product and the update (the update is on the
// reflector chain's critical path), longer columns are read twice
constexpr int kApplyRegs = 4;
template <typename T, int B>
__device__ __forceinline__ void qr_apply(const T* v, T tj, T* y, long long j, long long m, T* red) {
  const int tid = threadIdx.x;
  // every thread reads y[j] before the barriers of block_sum: thread 0
  // overwrites it below, and no thread may see the new value
  const T yj = y[j];
  T s = T(0);
  if (m - (j + 1) <= (long long)kApplyRegs * B) {
    T vr[kApplyRegs];
#pragma unroll
    for (int u = 0; u < kApplyRegs; ++u) {
      const long long i = j + 1 + tid + (long long)u * B;
      vr[u] = i < m ? __ldcg(v + i) : T(0);
    }
#pragma unroll
    for (int u = 0; u < kApplyRegs; ++u) {
      const long long i = j + 1 + tid + (long long)u * B;
      if (i < m) s = fma(vr[u], y[i], s);
    }
    s = block_sum(s, red);
    const T w = tj * (yj + s);
    if (tid == 0) y[j] = yj - w;
#pragma unroll
    for (int u = 0; u < kApplyRegs; ++u) {
      const long long i = j + 1 + tid + (long long)u * B;
      if (i < m) y[i] = fma(-w, vr[u], y[i]);
    }
  } else {
    for (long long i = j + 1 + tid; i < m; i += B) s = fma(__ldcg(v + i), y[i], s);
    s = block_sum(s, red);
    const T w = tj * (yj + s);
    if (tid == 0) y[j] = yj - w;
    for (long long i = j + 1 + tid; i < m; i += B) y[i] = fma(-w, __ldcg(v + i), y[i]);
  }
  __syncthreads();
}

template <typename T, int B>
__global__ void __launch_bounds__(B) qr_kernel(const double* __restrict__ Ain, Dim lda_d, T* W, long long ldw,
                                                Dim m_d, Dim n_d, T* tau, double* Rout, int r_rowmajor,
                                                long long ldr, double* Qout, int* kq_out, int* flag,
                                                DevSync* sync, double* flops, int qcols) {
  __shared__ T red[32 * kQrQCols];
  __shared__ int s_ok;
  extern __shared__ unsigned char ysh_raw[];
  T* ysh = reinterpret_cast<T*>(ysh_raw);
  const long long m = dv(m_d), n = dv(n_d), lda = dv(lda_d);
  const long long kq = m < n ? m : n;
  const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
  if (flops && b == 0 && tid == 0) {  // Householder R: 2 p k^2 - 2k^3/3; thin Q: 2 m k^2 - 2k^3/3
    const double p = (double)(m > n ? m : n), k = (double)kq;
    double f = 2.0 * p * k * k - 2.0 * k * k * k / 3.0;
    if (Qout) f += 2.0 * (double)m * k * k - 2.0 * k * k * k / 3.0;
    atomicAdd(flops, f);
  }

  // the rank of R is known from the sizes: written first, so that a launch
  // that gives up on a wait still leaves its consumers a size in range
  if (kq_out && b == 0 && tid == 0) *kq_out = (int)kq;
  for (long long c = b; c < n; c += G)
    for (long long i = tid; i < m; i += B) W[c * ldw + i] = T(Ain[c * lda + i]);
  for (long long j = (long long)b * B + tid; j < kq; j += (long long)G * B) flag[j] = 0;
  if (!grid_sync(sync)) return;

  if (kq > 0 && b == 0) {  // column 0 is owned by CTA 0
    qr_form<T, B>(W, 0, m, tau, red);
    if (tid == 0) {
      __threadfence();
      st_release(flag + 0, 1);
    }
  }
  for (long long j = 0; j < kq; ++j) {
    // last owned column: nothing left to apply once j reaches it
    const long long last_owned = b + ((n - 1 - b) / G) * G;
    if (b >= n || last_owned <= j) break;
    if (tid == 0) s_ok = (j % G == b) ? 1 : (wait_geq(flag + j, 1, sync) ? 1 : 0);
    __syncthreads();
    if (!s_ok) return;
    const T tj = __ldcg(tau + j);
    const T* v = W + j * ldw;
    const long long nx = j + 1;
    if (nx < n && nx % G == b) {
      T* y = W + nx * ldw;
      if (tj != T(0)) qr_apply<T, B>(v, tj, y, j, m, red);
      if (nx < kq) {
        qr_form<T, B>(y, nx, m, tau, red);
        if (tid == 0) {
          __threadfence();
          st_release(flag + nx, 1);
        }
      }
    }
    if (tj != T(0)) {
      long long c0 = b + ((j + 2 - b + G - 1) / G) * G;  // first owned column > j+1
      if (j + 2 <= b) c0 = b;
      for (long long c = c0; c < n; c += G) qr_apply<T, B>(v, tj, W + c * ldw, j, m, red);
    }
  }
  __syncthreads();

  // R: rows 0..kq-1 of the owned columns
  for (long long c = b; c < n; c += G) {
    for (long long i = tid; i < kq; i += B) {
      const double r = i <= c ? (double)W[c * ldw + i] : 0.0;
      if (r_rowmajor) Rout[i * ldr + c] = r;
      else Rout[c * ldr + i] = r;
    }
  }
  if (!Qout || kq == 0) return;

  // thin Q (m x kq, row-major): column c = H_0 ... H_c e_c, built in shared
  // memory, kQrQCols columns of a CTA at a time: H_i is read once for all of
  // them (its entries kept in registers between the dot products and the
  // updates), so a CTA's time is its largest column's chain, not the sum
  if (tid == 0) s_ok = wait_geq(flag + kq - 1, 1, sync) ? 1 : 0;
  __syncthreads();
  if (!s_ok) return;
  constexpr int QC = kQrQCols;
  for (long long c0 = b; c0 < kq; c0 += (long long)G * qcols) {
    long long cols[QC];
    int nc = 0;
#pragma unroll
    for (int u = 0; u < QC; ++u) {
      cols[u] = c0 + (long long)u * G;
      if (u < qcols && cols[u] < kq) nc = u + 1;
    }
    for (int u = 0; u < nc; ++u)
      for (long long i = tid; i < m; i += B) ysh[u * m + i] = (i == cols[u]) ? T(1) : T(0);
    __syncthreads();
    for (long long i = cols[nc - 1]; i >= 0; --i) {
      const T ti = __ldcg(tau + i);
      if (ti == T(0)) continue;
      const T* v = W + i * ldw;
      T yi[QC], dot[QC];
#pragma unroll
      for (int u = 0; u < QC; ++u) {  // read before the reduction's barriers (thread 0 overwrites them)
        yi[u] = (u < nc && cols[u] >= i) ? ysh[u * m + i] : T(0);
        dot[u] = T(0);
      }
      const bool regs = m - (i + 1) <= (long long)kApplyRegs * B;
      T vr[kApplyRegs];
      if (regs) {
#pragma unroll
        for (int e = 0; e < kApplyRegs; ++e) {
          const long long l = i + 1 + tid + (long long)e * B;
          vr[e] = l < m ? __ldcg(v + l) : T(0);
        }
#pragma unroll
        for (int e = 0; e < kApplyRegs; ++e) {
          const long long l = i + 1 + tid + (long long)e * B;
          if (l < m)
#pragma unroll
            for (int u = 0; u < QC; ++u)
              if (u < nc && cols[u] >= i) dot[u] = fma(vr[e], ysh[u * m + l], dot[u]);
        }
      } else {
        for (long long l = i + 1 + tid; l < m; l += B) {
          const T vl = __ldcg(v + l);
#pragma unroll
          for (int u = 0; u < QC; ++u)
            if (u < nc && cols[u] >= i) dot[u] = fma(vl, ysh[u * m + l], dot[u]);
        }
      }
      block_sum_n<T, QC>(dot, red);
      T w[QC];
#pragma unroll
      for (int u = 0; u < QC; ++u) w[u] = ti * (yi[u] + dot[u]);
      if (tid == 0)
#pragma unroll
        for (int u = 0; u < QC; ++u)
          if (u < nc && cols[u] >= i) ysh[u * m + i] = yi[u] - w[u];
      if (regs) {
#pragma unroll
        for (int e = 0; e < kApplyRegs; ++e) {
          const long long l = i + 1 + tid + (long long)e * B;
          if (l < m)
#pragma unroll
            for (int u = 0; u < QC; ++u)
              if (u < nc && cols[u] >= i) ysh[u * m + l] = fma(-w[u], vr[e], ysh[u * m + l]);
        }
      } else {
        for (long long l = i + 1 + tid; l < m; l += B) {
          const T vl = __ldcg(v + l);
#pragma unroll
          for (int u = 0; u < QC; ++u)
            if (u < nc && cols[u] >= i) ysh[u * m + l] = fma(-w[u], vl, ysh[u * m + l]);
        }
      }
      __syncthreads();
    }
    for (int u = 0; u < nc; ++u)
      for (long long i = tid; i < m; i += B) Qout[i * kq + cols[u]] = (double)ysh[u * m + i];
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

// Pairs follow the circle schedule; column c carries ver[c], the number of
// rounds it has been through.  The CTA rotating (i, j) in global round t waits
// until both columns reached t and then publishes t+1: no grid barrier per
// round, only the two predecessors.  At the end of a sweep every CTA adds its
// rotation count and waits for the others; a sweep without rotations ends it.
__global__ void __launch_bounds__(NT) jacobi_kernel(double* V, long long ldv, Dim nv_d, Dim m_d, double* J,
                                                    long long ldj, double* norms, DevSync* sync, int max_sweeps,
                                                    double tol, double tol_abs, int* log, int* ver) {
  __shared__ double red[96];
  __shared__ int s_ok, s_total;
  const long long nv = dv(nv_d), m = dv(m_d);
  const long long P = nv + (nv & 1);
  const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x;

  for (long long c = b; c < nv; c += G)
    for (long long i = tid; i < nv; i += NT) J[c * ldj + i] = (i == c) ? 1.0 : 0.0;
  for (long long c = (long long)b * NT + tid; c < P; c += (long long)G * NT) ver[c] = 0;
  if (b == 0 && tid < 4) {
    sync->counters[tid] = 0;
    sync->done[tid] = 0;
  }
  if (!grid_sync(sync)) return;

  int sweep = 0;
  if (nv >= 2) {
    for (sweep = 0; sweep < max_sweeps; ++sweep) {
      int local = 0;
      for (long long rd = 0; rd < P - 1; ++rd) {
        const int t = (int)(sweep * (P - 1) + rd);
        for (long long q = b; q < P / 2; q += G) {
          long long i, j;
          circle_pair(rd, q, P, i, j);
          if (tid == 0) s_ok = (wait_geq(ver + i, t, sync) && wait_geq(ver + j, t, sync)) ? 1 : 0;
          __syncthreads();
          if (!s_ok) return;
          if (i < nv && j < nv) {
            double* vi = V + i * ldv;
            double* vj = V + j * ldv;
            double* Ji = J + i * ldj;
            double* Jj = J + j * ldj;
            if (m <= NT * kRegE && nv <= NT * kRegE) {
              // one L2 pass: the pair and its rotation columns live in registers
              double x[kRegE], y[kRegE], jx[kRegE], jy[kRegE];
              double a = 0.0, bb = 0.0, g = 0.0;
#pragma unroll
              for (int e = 0; e < kRegE; ++e) {
                const long long l = tid + (long long)e * NT;
                x[e] = l < m ? __ldcg(vi + l) : 0.0;
                y[e] = l < m ? __ldcg(vj + l) : 0.0;
                jx[e] = l < nv ? __ldcg(Ji + l) : 0.0;
                jy[e] = l < nv ? __ldcg(Jj + l) : 0.0;
                a = fma(x[e], x[e], a);
                bb = fma(y[e], y[e], bb);
                g = fma(x[e], y[e], g);
              }
              block_sum3(a, bb, g, red);
              // rotate unless the pair is orthogonal to working precision, measured
              // against both vectors and against the larger one alone (a pair whose
              // norms differ by more than 1/tol cannot be made more orthogonal)
              if (g != 0.0 && fabs(g) > tol * sqrt(a) * sqrt(bb) && fabs(g) > tol_abs * fmax(a, bb)) {
                const double zeta = (bb - a) / (2.0 * g);
                const double tt = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                const double cs = 1.0 / sqrt(1.0 + tt * tt), sn = cs * tt;
#pragma unroll
                for (int e = 0; e < kRegE; ++e) {
                  const long long l = tid + (long long)e * NT;
                  if (l < m) {
                    vi[l] = cs * x[e] - sn * y[e];
                    vj[l] = sn * x[e] + cs * y[e];
                  }
                  if (l < nv) {
                    Ji[l] = cs * jx[e] - sn * jy[e];
                    Jj[l] = sn * jx[e] + cs * jy[e];
                  }
                }
                ++local;
              }
            } else {
              double a = 0.0, bb = 0.0, g = 0.0;
              for (long long l = tid; l < m; l += NT) {
                const double x = __ldcg(vi + l), y = __ldcg(vj + l);
                a = fma(x, x, a);
                bb = fma(y, y, bb);
                g = fma(x, y, g);
              }
              block_sum3(a, bb, g, red);
              if (g != 0.0 && fabs(g) > tol * sqrt(a) * sqrt(bb) && fabs(g) > tol_abs * fmax(a, bb)) {
                const double zeta = (bb - a) / (2.0 * g);
                const double tt = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                const double cs = 1.0 / sqrt(1.0 + tt * tt), sn = cs * tt;
                for (long long l = tid; l < m; l += NT) {
                  const double x = __ldcg(vi + l), y = __ldcg(vj + l);
                  vi[l] = cs * x - sn * y;
                  vj[l] = sn * x + cs * y;
                }
                for (long long l = tid; l < nv; l += NT) {
                  const double x = __ldcg(Ji + l), y = __ldcg(Jj + l);
                  Ji[l] = cs * x - sn * y;
                  Jj[l] = sn * x + cs * y;
                }
                ++local;
              }
            }
          }
          __syncthreads();
          if (tid == 0) {  // publish the CTA's writes (bar.sync, then fence + release)
            __threadfence();
            st_release(ver + i, t + 1);
            st_release(ver + j, t + 1);
          }
        }
      }
      // end of sweep: total rotations over all CTAs
      const int slot = sweep & 3;
      if (tid == 0) {
        if (local) atomicAdd(&sync->counters[slot], local);
        __threadfence();
        atomicAdd(&sync->done[slot], 1);
        s_ok = wait_geq(&sync->done[slot], G, sync) ? 1 : 0;
        s_total = ld_acquire(&sync->counters[slot]);
        if (b == 0) {  // slot of sweep+2 is free: every CTA has read sweep-2's
          sync->counters[(sweep + 2) & 3] = 0;
          sync->done[(sweep + 2) & 3] = 0;
        }
      }
      __syncthreads();
      if (!s_ok) return;
      if (s_total == 0) break;
    }
    if (sweep >= max_sweeps && b == 0 && tid == 0) set_status(sync, QTT_ENOCONV);
  }
  if (log && b == 0 && tid == 0) {
    log[0] = (int)nv;
    log[1] = (int)m;
    log[2] = sweep + 1;
  }
  // final norms
  for (long long c = b; c < nv; c += G) {
    const double* vc = V + c * ldv;
    double s = 0.0;
    for (long long l = tid; l < m; l += NT) {
      const double x = __ldcg(vc + l);
      s = fma(x, x, s);
    }
    s = block_sum(s, red);
    if (tid == 0) norms[c] = sqrt(s);
  }
}

// ------------------------------------------------------ sort + truncation
__global__ void __launch_bounds__(1024) svd_post_kernel(const double* norms, Dim cnt_d, Dim len_d, Dim jlen_d,
                                                        const double* J, long long ldj, double eps, int chi,
                                                        int rank_cap, int* rank_out, double* sigma_out,
                                                        double* disc_out, double* Jp, double* Jt, DevSync* sync,
                                                        int* nsv_out) {
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
    if (nsv_out) *nsv_out = nsv;
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

template <typename T>
static cudaError_t qr_launch(qtt_ctx* ctx, const double* Ain, Dim lda, double* Wd, long long ldw, Dim m, Dim n,
                             long long nmax, double* Rout, bool r_rowmajor, double* Qout, int* kq_out, long long ldr,
                             long long qm_max, int block) {
  int grid = (int)std::min<long long>(ctx->coop_blocks, std::max<long long>(nmax, 1));
  size_t smem = 0;
  int qcols = 1;  // columns of Q formed together: as many as fit in shared memory, at most kQrQCols
  if (Qout) {
    while (qcols < kQrQCols && (size_t)(qcols + 1) * qm_max * sizeof(T) <= 200 * 1024) ++qcols;
    smem = (size_t)qcols * qm_max * sizeof(T);
  }
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  T* W = reinterpret_cast<T*>(Wd);
  T* tau = reinterpret_cast<T*>(ctx->ws.d_tau);
  int rrm = r_rowmajor ? 1 : 0;
  DevSync* sync = ctx->ws.d_sync;
  int* flag = ctx->ws.d_flags;
  double* flops = g_flop_ctr;
  void* args[] = {(void*)&Ain, (void*)&lda, (void*)&W, (void*)&ldw, (void*)&m, (void*)&n, (void*)&tau,
                  (void*)&Rout, (void*)&rrm, (void*)&ldr, (void*)&Qout, (void*)&kq_out, (void*)&flag,
                  (void*)&sync, (void*)&flops, (void*)&qcols};
  // long columns (ldw bounds the rows): 1024 threads shorten each pass over a
  // column, which the reflector chain waits on
  if (block == 0) block = ldw >= 2048 ? 1024 : NT;
  if (block == 1024) return coop_launch((const void*)qr_kernel<T, 1024>, grid, 1024, args, smem, ctx->stream);
  if (block != NT) return cudaErrorInvalidValue;
  return coop_launch((const void*)qr_kernel<T, NT>, grid, NT, args, smem, ctx->stream);
}

cudaError_t qr_f64(qtt_ctx* ctx, const double* Ain, Dim lda, double* W, long long ldw, Dim m, Dim n, long long nmax,
                   double* Rout, bool r_rowmajor, double* Qout, int* kq_out, long long ldr, long long qm_max,
                   int block) {
  return qr_launch<double>(ctx, Ain, lda, W, ldw, m, n, nmax, Rout, r_rowmajor, Qout, kq_out, ldr, qm_max, block);
}

cudaError_t qr_f32(qtt_ctx* ctx, const double* Ain, Dim lda, double* W, long long ldw, Dim m, Dim n, long long nmax,
                   double* Rout, bool r_rowmajor, double* Qout, int* kq_out, long long ldr, long long qm_max,
                   int block) {
  return qr_launch<float>(ctx, Ain, lda, W, ldw, m, n, nmax, Rout, r_rowmajor, Qout, kq_out, ldr, qm_max, block);
}

cudaError_t jacobi_f64(qtt_ctx* ctx, double* V, long long ldv, Dim nv, Dim m, long long nvmax, double* J,
                       long long ldj, double* norms) {
  long long pairs = (nvmax + 1) / 2;
  int grid = (int)std::min<long long>(ctx->coop_blocks, std::max<long long>(pairs, 1));
  DevSync* sync = ctx->ws.d_sync;
  int max_sweeps = ctx->max_sweeps;
  // a pair counts as orthogonal when |v_i.v_j| <= 1e-13 |v_i||v_j| (above the
  // rounding floor of accumulated rotations) or <= 1e-15 max(|v_i|^2, |v_j|^2)
  double tol = 1e-13, tol_abs = 1e-15;
  int* log = jacobi_log_slot(ctx);
  int* ver = ctx->ws.d_flags;
  void* args[] = {(void*)&V, (void*)&ldv, (void*)&nv, (void*)&m, (void*)&J, (void*)&ldj, (void*)&norms,
                  (void*)&sync, (void*)&max_sweeps, (void*)&tol, (void*)&tol_abs, (void*)&log, (void*)&ver};
  return coop_launch((const void*)jacobi_kernel, grid, NT, args, 0, ctx->stream);
}

cudaError_t svd_post(qtt_ctx* ctx, const double* norms, Dim cnt, Dim len, Dim jlen, const double* J, long long ldj,
                     double eps, int chi, int rank_cap, int* rank_out, double* sigma_out, double* disc_out,
                     double* Jp, double* Jt, int* nsv_out) {
  long long nvmax = ldj;
  size_t smem = (size_t)nvmax * (2 * sizeof(double) + sizeof(int)) + 16;
  svd_post_kernel<<<1, 1024, smem, ctx->stream>>>(norms, cnt, len, jlen, J, ldj, eps, chi, rank_cap, rank_out,
                                                  sigma_out, disc_out, Jp, Jt, ctx->ws.d_sync, nsv_out);
  return cudaGetLastError();
}

int* jacobi_log_slot(qtt_ctx* ctx) {
  Prof& p = ctx->prof;
  if (!p.d_log || p.log_used >= p.log_cap) return nullptr;
  return p.d_log + 3 * (p.log_used++);
}

cudaError_t linalg_init(int device) {
  const void* ks[] = {(const void*)qr_kernel<double, NT>, (const void*)qr_kernel<float, NT>,
                      (const void*)qr_kernel<double, 1024>, (const void*)qr_kernel<float, 1024>};
  for (const void* k : ks) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int coop_max_blocks(int num_sms) {
  int a = 0, b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, (const void*)jacobi_kernel, NT, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, (const void*)qr_kernel<double, NT>, NT, 200 * 1024);
  int per = std::min(std::max(a, 1), std::max(b, 1));
  (void)per;
  // one CTA per SM: the FP64 pipe is per SM, more CTAs only add barrier traffic
  return num_sms;
}

}  // namespace qtt
