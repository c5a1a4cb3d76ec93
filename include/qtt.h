/*
 * qtt.h -- C ABI of the B300 (sm_103a) MPS / quantized-tensor-train stepper
 * for the explicit 2D acoustic FDTD scheme.
 *
 * Paper: "Quantum Circuit and Tensor Network Implementation of the 2D Acoustic
 * Wave Equation" (Nemeth & Vattay).  One time step (Eq. 17, Table 1) is
 *
 *     phi       = L psi^k                  (Laplacian MPO, Eq. 16, by zip-up)
 *     eta       = C^2 phi                  (diagonal MPO of c^2, Eq. 4, Sec. 4.3)
 *     theta     = 2 psi^k - psi^{k-1} + lambda^2 eta [+ s_k e_src]
 *     psi^{k+1} = round(theta)             (QR sweep, then truncated-SVD sweep,
 *                                           Sec. 4.3)
 *
 * Conventions shared by every call:
 *   - Grid: N = 2^n points per axis; dense fields are double, row-major
 *     u[x * N + z] with x horizontal and z depth (Sec. 2, Eq. 2).
 *   - Sites: d = 2n binary sites in the tensor-product order of Eq. 12, the
 *     least significant bit first.  QTT_ORDER_SEQUENTIAL: x_0..x_{n-1} then
 *     z_0..z_{n-1} (Eq. 14-15); QTT_ORDER_INTERLEAVED: x_0, z_0, x_1, z_1, ...
 *   - MPS core k (k = 0..d-1) is a double array [r_k][2][r_{k+1}], row-major,
 *     r_0 = r_d = 1 (Eq. 8).  MPO core k is [w_k][2 out][2 in][w_{k+1}].
 *   - Truncation (Sec. 4.3): keep sigma_i >= eps * sigma_1, at most chi_max
 *     values, at least one.
 *   - Every function returns a qtt_status; nothing throws across the ABI.
 *     QTT_EINVAL is returned before any launch for bad arguments; the text of
 *     the last error of the calling thread is given by qtt_last_error().
 *   - Work is queued asynchronously on the context's CUDA stream.  Failures
 *     detected on the device (a Jacobi sweep limit, a grid-barrier timeout, a
 *     non-finite value) are recorded in a device status word and returned by
 *     the next call that synchronises (qtt_ctx_sync, qtt_mps_ranks,
 *     qtt_mps_get_cores).
 *   - Ownership: handles and their device buffers belong to the library and
 *     are released by the matching *_destroy.  Caller buffers marked "device"
 *     are device pointers on the context's device (e.g. torch tensors); they
 *     are read or written on the context stream.
 *   - There is no CPU fallback: every call needs a CUDA device.
 */
#ifndef QTT_H
#define QTT_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  QTT_OK = 0,
  QTT_EINVAL = 1,      /* bad argument, nothing launched */
  QTT_ENOMEM = 2,      /* device allocation failed */
  QTT_ECUDA = 3,       /* a CUDA runtime call failed */
  QTT_ENOCONV = 4,     /* Jacobi SVD hit its sweep limit */
  QTT_ETIMEOUT = 5,    /* a bounded device wait gave up */
  QTT_ENONFINITE = 6   /* NaN/Inf met in a singular-value spectrum */
} qtt_status;

typedef enum { QTT_ORDER_SEQUENTIAL = 0, QTT_ORDER_INTERLEAVED = 1 } qtt_order;
typedef enum { QTT_BC_PERIODIC = 0, QTT_BC_ZERO = 1 } qtt_bc;
typedef enum { QTT_FP64 = 0, QTT_TF32 = 1, QTT_BF16 = 2, QTT_FP32 = 3, QTT_TF32X3 = 4 } qtt_precision;

/* Solver parameters.  n: bits per axis (1..14).  order: qtt_order.  bc:
 * qtt_bc; PERIODIC is the cyclic shift |x> -> |(x+1) mod 2^n> of Sec. 3.1 and
 * Sec. 4.2, ZERO is the terminal tensor of Eq. 11 as printed (the overflow is
 * dropped, i.e. u = 0 outside the grid).  prec: arithmetic of the
 * contractions (qtt_precision): QTT_FP64 is the plain form; QTT_FP32 runs
 * the contractions and QR updates in FP32 and the truncation SVD of each
 * bond factor as an FP32 Jacobi refined to FP64 accuracy in FP64 (the
 * singular values, the rank decision and the discarded weight are FP64).
 * QTT_TF32, QTT_TF32X3 and QTT_BF16 are QTT_FP32 with the core contractions
 * (zip-up site contractions, the Hadamard contraction with c^2, the
 * absorption of R and U S factors; Sec. 4.3) on the tensor cores (tcgen05,
 * FP32 accumulation in tensor memory): TF32 operands, TF32 operands split
 * x = hi + lo with the products hi*hi + hi*lo + lo*hi (about FP32
 * accuracy), or BF16 operands.  chi_max, eps:
 * truncation of the state (Sec. 4.3).  chi_zip, eps_zip: truncation inside
 * the two zip-up applications (0 = use chi_max / eps).  chi_c, eps_c:
 * truncation of the c^2 MPS (the paper does not say; 0 = chi_max / 1e-8).
 * use_learned_rank: 1 enables the learned rounding (qtt_set_rank_model).
 * dims: 2 (or 0) for the 2D scheme of Eq. 2; 3 for its 3D extension (the
 * paper's discussion section): an N^3 grid u[(x N + y) N + z] on d = 3n
 * sites (n <= 9), SEQUENTIAL = x, y, z registers one after another,
 * INTERLEAVED = x_0, y_0, z_0, x_1, ..., the 7-point Laplacian; every call
 * that takes a grid point then takes three coordinates (src_ixiz of the
 * step calls holds {ix, iy, iz}; the *_3d calls below). */
typedef struct {
  int n;
  int order;
  int bc;
  int prec;
  int chi_max;
  double eps;
  int chi_zip;
  double eps_zip;
  int chi_c;
  double eps_c;
  int use_learned_rank;
  int dims;
} qtt_params;

typedef struct qtt_ctx qtt_ctx;
typedef struct qtt_mps qtt_mps;
typedef struct qtt_mpo qtt_mpo;

/* Create a context on the current CUDA device.  cuda_stream is a
 * cudaStream_t (NULL = the legacy default stream); the caller keeps it alive
 * until qtt_ctx_destroy.  The context owns its workspace. */
qtt_status qtt_ctx_create(const qtt_params* params, void* cuda_stream, qtt_ctx** out);
void qtt_ctx_destroy(qtt_ctx* ctx);

/* Text of the last error raised on the calling thread ("" if none). */
const char* qtt_last_error(void);

/* Wait for the context stream and return (then clear) the device status. */
qtt_status qtt_ctx_sync(qtt_ctx* ctx);

/* Failure-detection limits of the context (the bounded waits and sweep
 * limit behind QTT_ETIMEOUT and QTT_ENOCONV).  wait_limit_s: how long a
 * kernel waits on another CTA of its launch (a grid barrier, a published
 * reflector or Jacobi round) before it records QTT_ETIMEOUT and returns;
 * <= 0 restores the default of 2 s.  max_sweeps: sweeps of the FP64 Jacobi
 * SVD before it records QTT_ENOCONV; <= 0 restores the default of 100.  A
 * kernel that gave up leaves its outputs undefined; the next synchronising
 * call reports the status and resets the device status word, after which the
 * context is usable again.  Captured step graphs are dropped (they are
 * captured again on the next qtt_step_graph). */
qtt_status qtt_set_limits(qtt_ctx* ctx, double wait_limit_s, int max_sweeps);

/* ------------------------------------------------------------------ states */

/* Rank-1 MPS of the zero field (the zero initial condition). */
qtt_status qtt_mps_create_zero(qtt_ctx* ctx, qtt_mps** out);

/* MPS of a dense field: sequential truncated SVDs (TT-SVD, Eq. 8) with
 * (chi_max, eps), then the compression of Sec. 4.3 (QR sweep, SVD sweep),
 * so that cores 1..d-1 are right-orthonormal as qtt_step expects.  grid: N*N
 * doubles u[x*N+z] (3D: N^3, u[(x*N+y)*N+z]), device memory if on_device
 * else host memory (copied; the call waits for it).  Synchronises. */
qtt_status qtt_mps_from_dense(qtt_ctx* ctx, const double* grid, int on_device, qtt_mps** out);

/* MPS from explicit cores.  ranks: d+1 host ints (ranks[0] = ranks[d] = 1,
 * each rank >= 1 and <= the context's capacity min(2^k, 2^(d-k), chi_max));
 * cores: host doubles, core 0..d-1 concatenated, each [r_k][2][r_{k+1}]. */
qtt_status qtt_mps_from_cores(qtt_ctx* ctx, const int* ranks, const double* cores, qtt_mps** out);

/* Copy an MPS to the host: ranks (d+1 ints) and, if cores is not NULL, the
 * concatenated cores (capacity given in doubles by cores_capacity; the
 * needed size is sum_k r_k*2*r_{k+1}).  Synchronises the stream. */
qtt_status qtt_mps_get_cores(qtt_ctx* ctx, const qtt_mps* psi, int* ranks, double* cores,
                             long cores_capacity);

/* Current bond dimensions r_0..r_d (d+1 host ints).  Synchronises. */
qtt_status qtt_mps_ranks(qtt_ctx* ctx, const qtt_mps* psi, int* ranks_out);
void qtt_mps_destroy(qtt_mps* psi);

/* MPS of the squared velocity c^2(x,z) (the diagonal operator C^2 of Eq. 4,
 * used as a diagonal MPO in Sec. 4.3), by TT-SVD (Eq. 8) with
 * (chi_c, eps_c).  c_grid: N*N velocities (m/s, > 0; N^3 in 3D), device if
 * on_device else host.  Synchronises (the c^2 ranks are fixed for the run). */
qtt_status qtt_velocity_mps(qtt_ctx* ctx, const double* c_grid, int on_device, qtt_mps** c2_out);

/* Laplacian MPO S_x^+ + S_x^- + S_z^+ + S_z^- - 4I (Eq. 16) built from the
 * carry tensors of Eq. 9-13 as one five-state carry automaton, for the
 * context's order and boundary condition (3D: the 7-point operator with the
 * y shifts, a seven-state automaton).  Built on the host, copied once. */
qtt_status qtt_laplacian_mpo(qtt_ctx* ctx, qtt_mpo** out);
/* Bond dimensions w_0..w_d of an MPO (d+1 host ints). */
qtt_status qtt_mpo_bonds(const qtt_mpo* L, int* bonds_out);
void qtt_mpo_destroy(qtt_mpo* L);

/* Checkpoint of a state: file = 8 bytes "QTTMPS1\0", int32 d, int32
 * ranks[d+1], then the cores [r_k][2][r_{k+1}] as FP64, little-endian.  Load
 * returns QTT_EINVAL for another grid size or a rank above the context's
 * capacity. */
qtt_status qtt_mps_save(qtt_ctx* ctx, const qtt_mps* psi, const char* path);
qtt_status qtt_mps_load(qtt_ctx* ctx, const char* path, qtt_mps** out);

/* ------------------------------------------------------------------- step */

/* psi <- round(psi + amp * e_(ix,iz)): a rank-1 product-state add (the
 * impulsive source of Sec. 5) followed by the Sec. 4.3 compression. */
qtt_status qtt_inject_source(qtt_ctx* ctx, qtt_mps* psi, long ix, long iz, double amp);
/* The same at (ix, iy, iz) of a 3D context. */
qtt_status qtt_inject_source_3d(qtt_ctx* ctx, qtt_mps* psi, long ix, long iy, long iz, double amp);

/* One time step of Eq. 17.  On entry psi_prev = u^{k-1}, psi_cur = u^k; on
 * return psi_prev = u^k and psi_cur = u^{k+1} (the handles exchange their
 * buffers; nothing is reallocated).  lambda2 = (dt/dh)^2 (Eq. 2).
 * src_ixiz: NULL for no source, else a host pair {ix, iz} ({ix, iy, iz} in
 * 3D) where src_amp is added to u^{k+1} as a rank-1 product state.  psi_cur must be right-
 * orthonormal in cores 1..d-1 (as every state this library returns is) for
 * the zip-up truncation to measure the right norm.  Stability is the
 * caller's: the leapfrog of Eq. 2 needs lambda2 * max(c^2) <= 1/2 (2D;
 * 1/3 in 3D), which the paper does not state and the step does not check
 * (the maximum of the c^2 MPS is not known without a dense evaluation). */
qtt_status qtt_step(qtt_ctx* ctx, const qtt_mpo* L, const qtt_mps* c2, double lambda2,
                    qtt_mps* psi_prev, qtt_mps* psi_cur, const long* src_ixiz, double src_amp);

/* The same step as qtt_step, replayed from a CUDA graph: the first call
 * for a given (L, c2, lambda2, source position, pair of state buffers)
 * captures the step's launches twice (once for each role of the two state
 * buffers, which exchange roles every step) on the context stream; later
 * calls write the source sample to the device and launch the matching graph,
 * one launch instead of ~2000.  Any other argument, or a workspace that had
 * to grow, makes it capture again.  Not for contexts with use_learned_rank
 * (the learned rounding synchronises with the host) nor while per-kernel
 * timing is on (QTT_EINVAL).  Results are those of qtt_step. */
qtt_status qtt_step_graph(qtt_ctx* ctx, const qtt_mpo* L, const qtt_mps* c2, double lambda2, qtt_mps* psi_prev,
                          qtt_mps* psi_cur, const long* src_ixiz, double src_amp);

/* Autotuner of the step's launch shapes.  Runs one dry-run step (no source)
 * on copies of (psi_prev, psi_cur), recording every contraction GEMM (the
 * core contractions of Sec. 4.3 and the FP64 products of the SVD
 * refinement) and every Householder QR; groups them by bucket (kind and
 * operand precision, the host-side size bounds, batch count); times every
 * candidate on all launches of a bucket with their own arguments and
 * device-side sizes, reps times after a warm-up (CUDA events on the context
 * stream); and keeps the fastest for later steps of the context: the output
 * tile (16 or 32) of the SIMT GEMMs, the tile width (64, 128 or 256 columns)
 * of the tensor-core contractions, the threads per CTA (256 or 1024) of the
 * QR.  cache_path (may be NULL): a JSON file; if it holds the choices for
 * this device, form and shape (a header line), they are loaded instead of
 * measured, else the measured choices are written there.  *entries_out
 * (may be NULL): the number of buckets tuned.  The states are not changed.
 * Captured step graphs are dropped.  Synchronises.  The paper has no
 * counterpart; the choices change no result beyond rounding. */
qtt_status qtt_autotune(qtt_ctx* ctx, const qtt_mpo* L, const qtt_mps* c2, double lambda2, const qtt_mps* psi_prev,
                        const qtt_mps* psi_cur, const char* cache_path, int reps, int* entries_out);

/* The transition operator of Eq. 7, A = 2I + lambda^2 C^2 L, as one MPO:
 * the product of the diagonal MPO of the c^2 MPS (Sec. 4.3) and the
 * Laplacian MPO (Eq. 16) plus twice the identity, bond r_c w + 1 (r_c the
 * c^2 ranks, w the Laplacian bonds).  The norm nu of the last c^2 core is
 * carried by the coefficient of the product term (lambda^2 nu on the first
 * core, the last c^2 core divided by nu), so that both terms are of order one
 * at every bond.  Built on the host (the c^2 cores are copied back; the call
 * synchronises), copied to the device once; released by qtt_mpo_destroy. */
qtt_status qtt_a_operator_mpo(qtt_ctx* ctx, const qtt_mpo* L, const qtt_mps* c2, double lambda2, qtt_mpo** out);

/* One time step of Eq. 7 with A applied as one operator (the fused variant
 * of qtt_step): phi = A psi^k by one zip-up (sites 1 -> d, truncated with
 * chi_zip / eps_zip), theta = phi - psi^{k-1} [+ src_amp e_src], psi^{k+1} =
 * round(theta) (Sec. 4.3).  In exact arithmetic the step of qtt_step; one
 * truncated zip-up instead of two.  A: from qtt_a_operator_mpo (any MPO is
 * accepted: the step then advances psi^{k+1} = round(A psi^k - psi^{k-1})).
 * Handles rotate as in qtt_step.  The workspace is sized for A's bonds (a
 * context alternating this and qtt_step regrows it). */
qtt_status qtt_step_fused(qtt_ctx* ctx, const qtt_mpo* A, qtt_mps* psi_prev, qtt_mps* psi_cur, const long* src_ixiz,
                          double src_amp);

/* Batched shots.  A batch holds one context per shot (each with its own
 * chi_max and workspace, all on `cuda_stream`) and a pool of min(nshots, 8)
 * internal streams; qtt_step_batched advances every shot by one step
 * (Eq. 17), shot i on pool stream i mod 8, so that shots of different pool
 * streams run concurrently on the GPU; one host thread per pool stream
 * issues the launches.  The cooperative grids of each shot are capped so
 * that the pool's grids fit on the device together.  The batched step is
 * ordered after earlier work on `cuda_stream`, and later work on it waits for
 * every shot.  Shot i's states are created in qtt_batch_ctx(batch, i) (owned
 * by the batch: never passed to qtt_ctx_destroy).  chi_per_shot: nshots host
 * ints, 0 = base->chi_max; NULL = all base->chi_max.  qtt_batch_destroy
 * frees the contexts: destroy the shots' states first. */
typedef struct qtt_batch qtt_batch;
qtt_status qtt_batch_create(const qtt_params* base, int nshots, const int* chi_per_shot, void* cuda_stream,
                            qtt_batch** out);
qtt_ctx* qtt_batch_ctx(qtt_batch* batch, int shot);
/* L and c2 are shared by all shots (created in any context of the same n,
 * order and boundary condition).  prev, cur: nshots handles each, created in
 * the shots' contexts; they rotate as in qtt_step.  src_ixiz: NULL, or
 * 2*nshots host longs {ix_0, iz_0, ix_1, ...} (3*nshots in 3D);
 * src_amp: nshots doubles. */
qtt_status qtt_step_batched(qtt_batch* batch, const qtt_mpo* L, const qtt_mps* c2, double lambda2, qtt_mps** prev,
                            qtt_mps** cur, const long* src_ixiz, const double* src_amp);
void qtt_batch_destroy(qtt_batch* batch);
/* on != 0: qtt_step_batched steps every shot through qtt_step_graph (one
 * graph launch per shot and step instead of ~2000 kernel launches). */
qtt_status qtt_batch_set_graphs(qtt_batch* batch, int on);

/* ------------------------------------------------------------ learned form
 * The rounding rule of Sec. 4.3 still decides every truncation; a learned model only
 * proposes, per bond, the rank of the next step's round, whose SVD then first
 * tries a randomised range finder of width proposal + oversample (Halko,
 * Martinsson & Tropp 2011, Algorithm 4.1 with the direct SVD of Sec. 5.1):
 * Y = X^T Omega, Y = QR, B = Q^T X^T, SVD of B, for X the bond matrix
 * (q_k x 2 r_{k+1}) and Omega the top-left block of a caller-provided
 * Gaussian matrix.  An exact check in FP64 accepts the sketch only if the rule
 * is met: with rho = ||X - X Q Q^T||_F and c = #{sigma_i(B) >= eps sigma_1(B)},
 * c < chi needs rho <= eps sigma_1(B); c >= chi needs
 * rho^2 <= ((1 + 0.05)^2 - 1) sum_{i>=chi} sigma_i(B)^2, which keeps the
 * discarded weight within (1.05)^2 of the optimum (Ky Fan's maximum
 * principle on X X^T = A A^T + E E^T, A = X Q Q^T, E = X - A); c >= width
 * rejects.
 * A rejected bond takes the full SVD.  Each attempt costs one host
 * synchronisation (the flag decides which kernels follow).
 *
 * The model: an MLP of 3 linear layers (40 -> 128 -> 128 -> 1, ReLU, FP32)
 * reading 40 features of a bond's spectrum at step k (qtt_rank_features) and
 * returning the bond's rank at step k+1 divided by chi_max; proposal =
 * clamp(ceil(chi_max * y), 1, chi_max).  Parameters are one flat float array
 * of qtt_mlp_param_count() values: W1 (128 x 40, row-major), b1 (128),
 * W2 (128 x 128), b2 (128), W3 (1 x 128), b3 (1).  Training: mean squared
 * error, Adam (Kingma & Ba 2015, Algorithm 1), on `cuda_stream` of the
 * network. */
typedef struct qtt_mlp qtt_mlp;
int qtt_mlp_param_count(void);
/* params: host, qtt_mlp_param_count() floats (copied).  max_batch: the most
 * samples one forward or gradient call takes (>= 2n to serve a context). */
qtt_status qtt_mlp_create(const float* params, int max_batch, void* cuda_stream, qtt_mlp** out);
void qtt_mlp_destroy(qtt_mlp* mlp);
/* X: device, n x 40 row-major floats; y: device, n floats. */
qtt_status qtt_mlp_forward(qtt_mlp* mlp, const float* X, int n, float* y);
/* Mean squared error against t (device, n floats) into *loss (device float,
 * may be NULL) and its gradient, kept for qtt_mlp_adam_step and copied to
 * grad (device, qtt_mlp_param_count() floats) when grad is not NULL. */
qtt_status qtt_mlp_grad(qtt_mlp* mlp, const float* X, const float* t, int n, float* loss, float* grad);
/* One Adam update from the last gradient (step count kept by the network). */
qtt_status qtt_mlp_adam_step(qtt_mlp* mlp, float lr, float beta1, float beta2, float eps);
qtt_status qtt_mlp_get_params(qtt_mlp* mlp, float* params);
/* Features of bonds 1..nb (row k-1 of X, 40 floats each) from descending
 * singular values S (device; row k at S + k*lds holds len[k] values) and the
 * kept ranks ranks[k] (device ints), for rule parameters eps, chi and d sites:
 * 0..31 log10(S_p/S_0) at p = floor(j (len-1)/31), clipped to [-16, 0], / 16;
 * 32 rank/chi; 33 log10(discarded weight / S_0^2) clipped to [-32, 0], / 32;
 * 34 log10(eps)/16; 35 k/d; 36 min(2^k, 2^(d-k), chi)/chi;
 * 37 #{S_i >= eps S_0}/chi; 38 len/(2 chi); 39 1 (-1 for undefined logs). */
qtt_status qtt_rank_features(const double* S, int lds, const int* len, const int* ranks, int nb, double eps, int chi,
                             int d, float* X, void* cuda_stream);
/* Features of bonds 1..d-1 of the last step's round (its logged spectra and
 * the ranks of psi, the state that step produced), on the context stream. */
qtt_status qtt_step_features(qtt_ctx* ctx, const qtt_mps* psi, float* X);
/* Learned rounding for a context created with use_learned_rank = 1: sketch
 * (device, rows x cols row-major doubles, not copied, kept alive by the
 * caller) and oversample p; mlp (may be NULL) proposes the ranks after every
 * step.  sketch = NULL turns the learned rounding off. */
qtt_status qtt_set_rank_model(qtt_ctx* ctx, qtt_mlp* mlp, const double* sketch, int rows, int cols, int oversample);
/* Proposals (host, d+1 ints; 0 = none) for the next step only, instead of
 * the model's. */
qtt_status qtt_set_proposals(qtt_ctx* ctx, const int* prop);
/* The proposals the model made after the last step (host, d+1 ints). */
qtt_status qtt_get_proposals(qtt_ctx* ctx, int* prop);
/* Range-finder attempts and accepted attempts since the context was made. */
qtt_status qtt_learned_stats(qtt_ctx* ctx, long* attempts, long* accepts);

/* ---------------------------------------------------------------- readout */

/* Receiver readout: out[p] = A_0[s_0] A_1[s_1] ... A_{d-1}[s_{d-1}] (Eq. 8)
 * at grid points (ix[p], iz[p]), p < count.  ix, iz, out: device arrays of
 * count int64 / int64 / double.  Indices are not range-checked on the
 * device; the caller keeps them in [0, N).  An index outside that range
 * still reads only the state's cores: the kernel takes the 2n low bits of
 * ix N + iz, so the value returned is that of another grid point. */
qtt_status qtt_sample(qtt_ctx* ctx, const qtt_mps* psi, const long* ix_dev, const long* iz_dev,
                      long count, double* out_dev);

/* Receiver readout of a 3D context: out[p] at (ix[p], iy[p], iz[p]). */
qtt_status qtt_sample_3d(qtt_ctx* ctx, const qtt_mps* psi, const long* ix_dev, const long* iy_dev,
                         const long* iz_dev, long count, double* out_dev);

/* Full contraction to the dense grid: out_dev[x*N+z], N*N device doubles
 * (3D: out_dev[(x*N+y)*N+z], N^3 device doubles). */
qtt_status qtt_to_dense(qtt_ctx* ctx, const qtt_mps* psi, double* out_dev);

/* ------------------------------------------------------- linear algebra */

/* Truncated SVD of one bond matrix with the Sec. 4.3 rule, the factorisation
 * every truncation in the step uses: M = U S V^T, M an (m x n) row-major
 * device matrix (not modified).  Writes r = kept rank to *rank_out (host)
 * and, on the device, U (m x r, row-major, ld r), S (r values, descending)
 * and Vt (r x n, row-major, ld n); out buffers hold at least m*min(m,n),
 * min(m,n) and min(m,n)*n doubles.  chi <= 0 means no cap.  Synchronises. */
qtt_status qtt_svd_trunc(qtt_ctx* ctx, const double* M_dev, int m, int n, double eps, int chi,
                         double* U_dev, double* S_dev, double* Vt_dev, int* rank_out);

/* Truncated SVD with the same arithmetic and outputs as qtt_svd_trunc, for
 * callers that cannot allocate device memory: code whose device memory is
 * owned by another allocator (a framework's caching pool, an arena sized at
 * start-up) and latency-critical loops that cannot take the implicit
 * synchronisation of cudaMalloc/cudaFree.  It needs no context and calls no
 * allocator: its scratch is one file-scope device array of about 3.2 MB,
 * present on every GPU that loads the library until the process exits.
 * The paper has no counterpart of this call.
 *   M_dev: m x n row-major device matrix (not modified); U_dev (m x min(m,n)),
 *   S_dev (min(m,n)), Vt_dev (min(m,n) x n): device outputs laid out as for
 *   qtt_svd_trunc; *rank_out: kept rank (host).  cuda_stream: cudaStream_t
 *   (NULL = legacy default stream); the call synchronises it.
 * Limits: max(m,n) <= 512 and min(m,n) <= 128, else QTT_EINVAL (message in
 * qtt_last_error).  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress).  Every call shares the array: calls whose
 * work overlaps on the GPU (two streams, two threads) race and corrupt each
 * other's results. */
qtt_status qtt_svd_trunc_noalloc(const double* M_dev, int m, int n, double eps, int chi, double* U_dev,
                                 double* S_dev, double* Vt_dev, int* rank_out, void* cuda_stream);

/* One core contraction on its own, the kernel every contraction of a step
 * uses (the zip-up site contractions, the Hadamard contraction with the c^2
 * cores and the absorption of R and U S factors into neighbouring cores,
 * Sec. 4.3): C = alpha op(A) op(B) + beta C on the context stream, with
 * op(A) m x k, op(B) k x n, all device FP64 row-major: A is m x k (lda) or,
 * if a_trans, k x m; B is k x n (ldb) or, if b_trans, n x k; C is m x n
 * (ldc).  kind: 0 FP64, 1 FP32 (SIMT kernels); 2 TF32, 3 3xTF32 (x split
 * into two TF32 parts, three products), 4 BF16 (tensor cores, tcgen05 with
 * the FP32 accumulator in tensor memory).  tile_n: columns per CTA of the
 * tensor-core kinds (64, 128 or 256; 0 = the library's choice).  QTT_EINVAL
 * for bad sizes or leading dimensions; asynchronous (qtt_ctx_sync reports
 * device failures). */
qtt_status qtt_gemm(qtt_ctx* ctx, int kind, int a_trans, int b_trans, int m, int n, int k, const double* A, int lda,
                    const double* B, int ldb, double* C, int ldc, double alpha, double beta, int tile_n);

/* ------------------------------------------------------------- context */

/* Dense FDTD update of Eq. 2 on the device (the scheme the MPS step
 * reproduces; used for comparison runs):
 * u_next = 2 u_cur - u_prev + lambda2 * c2 * (4-neighbour sum - 4 u_cur),
 * plus amp at (src_ix, src_iz) when src_ix >= 0.  All arrays N*N device
 * doubles; boundary rule from the context. */
qtt_status qtt_fdtd_step(qtt_ctx* ctx, const double* c2_dev, double lambda2, const double* u_prev_dev,
                         const double* u_cur_dev, double* u_next_dev, long src_ix, long src_iz,
                         double amp);
/* The 7-point update of a 3D context (arrays N^3, u[(x*N+y)*N+z]): six face
 * neighbours, - 6 u_cur, the context's boundary rule; amp at the source
 * when every coordinate is in range. */
qtt_status qtt_fdtd_step_3d(qtt_ctx* ctx, const double* c2_dev, double lambda2, const double* u_prev_dev,
                            const double* u_cur_dev, double* u_next_dev, long src_ix, long src_iy, long src_iz,
                            double amp);

/* Singular values, kept ranks and discarded weights of the last step, for
 * diagnostics.  discarded: 3*(d-1) host doubles (zip-up L bonds 1..d-1,
 * zip-up C^2 bonds 1..d-1, rounding bonds 1..d-1).  Synchronises. */
qtt_status qtt_last_step_discarded(qtt_ctx* ctx, double* discarded);

/* --------------------------------------------------------- measurement */

/* Kernel classes counted by qtt_profile: 0 GEMM contraction, 1 Householder
 * QR, 2 Jacobi SVD, 3 sort/truncate (Sec. 4.3 rule), 4 MPO application,
 * 5 MPS sum, 6 copy/transpose, 7 dense FDTD, 8 FP64 refinement of the
 * mixed-precision SVD, 9 other, 10 the pivoted factor that preconditions the
 * mixed SVD's Jacobi (Gram matrix and pivoted Cholesky, or pivoted QR of the
 * small R factor). */
#define QTT_KCLASSES 11

typedef struct {
  long launches[QTT_KCLASSES]; /* kernels launched since qtt_profile_start */
  double ms[QTT_KCLASSES];     /* device time of those launches (timing on) */
  long svd_logged;             /* Jacobi launches whose size was logged */
  double svd_flops;            /* sum of 6 m n^2 + 20 n^3 over them (n <= m:
                                  the two sizes of the rotated problem) */
  long svd_sweeps;             /* Jacobi sweeps over them (the last one finds
                                  no pair to rotate) */
  double flops[QTT_KCLASSES];  /* algorithmic FLOPs of the launches of each
                                  class while work logging is on (log_svd),
                                  counted by the kernels from their device-side
                                  sizes: 2 M N K per GEMM (batches included),
                                  2 p k^2 - 2k^3/3 per Householder QR of a
                                  p x q matrix (k = min(p, q)) and the same again
                                  for its thin Q; the cluster factorisations
                                  and the Jacobi sweeps are not counted here
                                  (svd_flops holds the SVD work) */
} qtt_profile;

/* Reset the counters of the context.  timing != 0 brackets every launch with
 * CUDA events on the context stream (adds a little host work per launch);
 * log_svd != 0 records the size of up to 65536 Jacobi launches and counts
 * the algorithmic FLOPs per class (qtt_profile.flops).  Counting launches is
 * always on.  qtt_step_graph refuses to capture while timing or logging is
 * on. */
qtt_status qtt_profile_start(qtt_ctx* ctx, int timing, int log_svd);

/* Read the counters (synchronises the stream). */
qtt_status qtt_profile_read(qtt_ctx* ctx, qtt_profile* out);

/* Measured ALU peak of the current device: kind 0 = FP32 FMA, 1 = FP64 FMA.
 * Runs an FMA-chain kernel (8 independent chains per thread, 32 warps per
 * SM) for about 60 ms on cuda_stream (a cudaStream_t, NULL = legacy default
 * stream) and writes 2 x FMAs / elapsed time in TFLOP/s to *tflops.  These
 * are the roofline peaks of the SIMT kernels (the FP32 Jacobi, the FP64
 * refinement and Jacobi).  Synchronises; allocates a small device buffer. */
qtt_status qtt_peak_probe(int kind, double* tflops, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* QTT_H */
