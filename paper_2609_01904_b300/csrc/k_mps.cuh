// Launchers of the MPS-level kernels (k_mps.cu).
#pragma once

#include "qtt_internal.cuh"

namespace qtt {

constexpr int kMaxSites = 32;
constexpr int kMaxTerms = 4;

struct SumArgs {
  int d;
  int nterms;  // MPS terms (the rank-1 source is extra)
  const double* core[kMaxTerms][kMaxSites];
  const int* ranks[kMaxTerms];
  double coef[kMaxTerms];
  double* out[kMaxSites];
  int* out_ranks;
  int has_src;
  int src_bits[kMaxSites];
  double src_amp;
  const double* src_amp_dev;  // when set, the amplitude is read from here (graph replays)
  const double* amp_scale;    // when set, the amplitude is multiplied by *amp_scale (state scaling)
};

// Encoding (Eq. 3, Eq. 12 order, Eq. 14-15): site k carries bit pos[k] of the
// linear dense index ((x N + y) N + z in 3D, x N + z in 2D); see site_pos().
struct SitePos {
  int d;
  int pos[kMaxSites];
};

struct SampleArgs {
  int d, n, dims, rmax;
  SitePos sp;
  const double* core[kMaxSites];
  const int* ranks;
  const long* ix;
  const long* iy;  // 3D only
  const long* iz;
  long long count;
  double* out;
};

struct ChainArgs {
  int d, h, rmax;
  const double* core[kMaxSites];
  const int* ranks;
  double* out;
};

cudaError_t mpo_apply_lr(const double* X, double* T, const double* W, int w, int w2, const int* a_p, const int* b2_p,
                         long long total_max, cudaStream_t st);
cudaError_t mps_sum(const SumArgs& a, long long max_core_elems, cudaStream_t st);
cudaError_t sample(const SampleArgs& a, cudaStream_t st);
cudaError_t chains(const ChainArgs& left, const ChainArgs& right, cudaStream_t st);
cudaError_t scatter_dense(const double* S, double* out, const SitePos& sp, int h, cudaStream_t st);
cudaError_t site_permute(const double* u, double* t, const SitePos& sp, bool square, cudaStream_t st);
// dense 7-point update of the 3D extension: arrays N^3, u[(x N + y) N + z]
cudaError_t fdtd3(const double* c2, double lambda2, const double* up, const double* uc, double* un, int n, int bc,
                  long long sx, long long sy, long long sz, double amp, cudaStream_t st);
cudaError_t fdtd(const double* c2, double lambda2, const double* up, const double* uc, double* un, int n, int bc,
                 long long sx, long long sz, double amp, cudaStream_t st);
cudaError_t copy2d(const double* src, double* dst, Dim R, Dim C, Dim ssi, Dim ssj, Dim dsi, Dim dsj,
                   long long total_max, double alpha, cudaStream_t st);
cudaError_t init_zip(double* carry, int* ranks, int d, const int* copy_src, int* copy_dst, int ncopy,
                     cudaStream_t st);
cudaError_t scale_rows(double* M, long long ldm, Dim ncols, const int* r_p, const double* sigma, long long total_max,
                       cudaStream_t st);
// Power-of-two state scaling of the reduced-precision step: scale[0] = 2^s,
// scale[1] = 2^-s with 2^s max(|a|, |b|) in [0.5, 1) over the first cores
// a, b (1 x 2 x r, r = *ra / *rb) of two states (s = 0 for zero states);
// then core <- core * scale[which] for a first core of rank *r (exact).
cudaError_t state_scale_prepare(const double* a, const int* ra, const double* b, const int* rb, long long rmax,
                                double* scale, cudaStream_t st);
cudaError_t state_scale_apply(double* core, const int* r, long long rmax, const double* scale, int which,
                              cudaStream_t st);

// k_linalg.cu
cudaError_t linalg_init(int device);
int coop_max_blocks(int num_sms);

// k_mixed.cu
cudaError_t jacobi32_cluster(qtt_ctx* ctx, const double* V, long long ldv, Dim nv, Dim m, long long nvmax,
                             long long mmax, double* J, long long ldj);
cudaError_t ns_factor(const double* G, double* H, long long ld, Dim n, long long nmax, cudaStream_t st);
// rs: nmax doubles of scratch (row sums of |Omega|)
cudaError_t omega_factor(const double* G, double* rs, double* M, long long ld, Dim n, long long nmax,
                         cudaStream_t st);
// QR with column pivoting of A (nr x nc, A[a][i] = Ain[a*lda + i], nr and
// nc <= nmax <= 256) in one cluster, FP32: R1 (k1 x nc) row-major (stride
// ldr1), thin Q1 (nr x k1) row-major (stride ldq), k1 = min(nr, nc) to
// *k1_out.  Vg: k1 * 256 floats of scratch.
cudaError_t qrcp_cluster(qtt_ctx* ctx, const double* Ain, long long lda, Dim nr, Dim nc, long long nmax, double* R1,
                         long long ldr1, double* Q1, long long ldq, float* Vg, int* k1_out);
// Cholesky with diagonal pivoting of a symmetric positive semidefinite G
// (n x n, ld ldg, n <= nmax <= 256) in one cluster, FP64: R (k x n, row-major,
// row stride ldr, columns in their original order) with R^T R = G, k <= kcap
// rows (fewer once the remaining pivots reach the rounding level of G), k at
// *k_out.
cudaError_t pchol_cluster(qtt_ctx* ctx, const double* G, long long ldg, Dim n, Dim kcap, long long nmax, double* R,
                          long long ldr, int* k_out);
// J[c][a] = W[c][a] / norms[c] for c < rows, a < cols (0 where norms[c] = 0)
cudaError_t scale_rows(const double* W, long long ldw, const double* norms, Dim rows, Dim cols, long long rmax,
                       long long cmax, double* J, long long ldj, cudaStream_t st);
cudaError_t row_norms(const double* W, long long ldw, Dim n, Dim m, long long nmax, double* norms, cudaStream_t st);
cudaError_t mixed_init();

}  // namespace qtt
