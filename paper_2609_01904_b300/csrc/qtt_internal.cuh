// Internal declarations of the QTT stepper library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda/atomic>

#include <cstdint>
#include <functional>
#include <map>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "../../include/qtt.h"

namespace qtt {

// ---------------------------------------------------------------------------
// Device-side dimensions.  Bond ranks change every step and live in device
// memory, so kernels evaluate their sizes and strides on the device:
//   value = add + mul * (p1 ? *p1 : 1) * (p2 ? *p2 : 1)
// A pure constant has mul = 0.  The host sizes grids from capacities.
// ---------------------------------------------------------------------------
struct Dim {
  const int* p1;
  const int* p2;
  long long mul;
  long long add;
};

inline Dim dconst(long long v) { return Dim{nullptr, nullptr, 0, v}; }
inline Dim dptr(const int* p, long long mul = 1, long long add = 0) { return Dim{p, nullptr, mul, add}; }
inline Dim dptr2(const int* p, const int* q, long long mul = 1, long long add = 0) {
  return Dim{p, q, mul, add};
}

__device__ __forceinline__ long long dv(const Dim& d) {
  long long v = d.mul;
  if (d.mul != 0) {
    if (d.p1) v *= (long long)(*d.p1);
    if (d.p2) v *= (long long)(*d.p2);
  }
  return d.add + v;
}

// ---------------------------------------------------------------------------
// Device status word and grid barrier with bounded waits.  A wait that runs
// out records QTT_ETIMEOUT and returns false; the kernel then unwinds.
// ---------------------------------------------------------------------------
struct DevSync {
  unsigned int bar_count;
  unsigned int bar_gen;
  int counters[4];   // rotations per sweep (4 rotating slots)
  int status;
  int done[4];       // CTAs that finished a sweep (same slots)
  int pad;
  unsigned long long limit_ns;  // wait limit of this context (0 = kWaitLimitNs)
  int pad2[2];
};

constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s

__device__ __forceinline__ unsigned long long wait_limit(const DevSync* s) {
  const unsigned long long l = s->limit_ns;
  return l ? l : kWaitLimitNs;
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void set_status(DevSync* s, int code) {
  atomicCAS(&s->status, 0, code);
}

// bounded waits on a counter written by another CTA of the same launch
__device__ __forceinline__ int ld_acquire(const int* p) {
  return cuda::atomic_ref<const int, cuda::thread_scope_device>(*p).load(cuda::memory_order_acquire);
}
__device__ __forceinline__ void st_release(int* p, int v) {
  cuda::atomic_ref<int, cuda::thread_scope_device>(*p).store(v, cuda::memory_order_release);
}
// thread 0 waits until *p >= target; false (status set) on timeout or error
__device__ __forceinline__ bool wait_geq(const int* p, int target, DevSync* s) {
  if (ld_acquire(p) >= target) return true;
  const unsigned long long t0 = globaltimer_ns(), lim = wait_limit(s);
  while (ld_acquire(p) < target) {
    if (ld_acquire(&s->status) != 0) return false;
    if (globaltimer_ns() - t0 > lim) {
      set_status(s, QTT_ETIMEOUT);
      return false;
    }
    __nanosleep(20);
  }
  return true;
}

// All CTAs of a cooperative launch call this the same number of times.
__device__ __forceinline__ bool grid_sync(DevSync* s) {
  __shared__ int s_ok;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    cuda::atomic_ref<unsigned int, cuda::thread_scope_device> gen(s->bar_gen);
    cuda::atomic_ref<unsigned int, cuda::thread_scope_device> cnt(s->bar_count);
    cuda::atomic_ref<int, cuda::thread_scope_device> st(s->status);
    unsigned int g = gen.load(cuda::memory_order_acquire);
    unsigned int nb = gridDim.x * gridDim.y * gridDim.z;
    unsigned int arrived = cnt.fetch_add(1u, cuda::memory_order_acq_rel);
    int ok = 1;
    if (arrived == nb - 1) {
      cnt.store(0u, cuda::memory_order_relaxed);
      gen.fetch_add(1u, cuda::memory_order_release);
    } else {
      const unsigned long long t0 = globaltimer_ns(), lim = wait_limit(s);
      while (gen.load(cuda::memory_order_acquire) == g) {
        if (st.load(cuda::memory_order_relaxed) != 0) { ok = 0; break; }
        if (globaltimer_ns() - t0 > lim) {
          set_status(s, QTT_ETIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(40);
      }
    }
    if (st.load(cuda::memory_order_relaxed) != 0) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Block-wide sum of one value per thread (blockDim.x a multiple of 32, <= 1024).
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red /* >= 32 */) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  int nw = blockDim.x >> 5;
  if (w == 0) {
    T t = (l < nw) ? red[l] : T(0);
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (l == 0) red[0] = t;
  }
  __syncthreads();
  T r = red[0];
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------------------
// Handles
// ---------------------------------------------------------------------------
struct Mps {
  qtt_ctx* ctx = nullptr;
  int d = 0;
  std::vector<int> cap;        // capacity of bonds 0..d
  std::vector<long long> off;  // element offset of core k in data (capacity layout)
  long long total = 0;         // capacity in doubles
  double* data = nullptr;      // device
  int* ranks = nullptr;        // device, d+1
  std::vector<int> host_ranks; // host copy when the ranks are fixed (c^2)
  double* core(int k) const { return data + off[k]; }
};

struct Mpo {
  int d = 0;
  std::vector<int> w;           // bonds 0..d
  std::vector<long long> off;   // offset of core k
  std::vector<double> host;     // cores, [w_k][2][2][w_{k+1}]
  double* data = nullptr;       // device copy
};

}  // namespace qtt

struct qtt_mps : qtt::Mps {};
struct qtt_mpo : qtt::Mpo {};

namespace qtt {

// Workspace: every scratch buffer of the step, sized from capacities once.
struct Workspace {
  long long carry = 0, xbuf = 0, tv = 0, tq = 0, rv = 0, jv = 0, jp = 0, w1 = 0, vec = 0;
  double* d_carry = nullptr;  // zip-up carried tensor
  double* d_x = nullptr;      // contraction intermediate
  double* d_tv = nullptr;     // SVD input: nv vectors (vector-major)
  double* d_tq = nullptr;     // QR working copy
  double* d_rv = nullptr;     // R factor, vector-major (nv vectors)
  double* d_jv = nullptr;     // Jacobi rotations, vector-major (nv x nv)
  double* d_jp = nullptr;     // kept rotations, row-major (r x nv)
  double* d_w1 = nullptr;     // absorption intermediate
  double* d_tt = nullptr;     // transposed vectors (wide SVDs)
  double* d_qt = nullptr;     // thin Q of a wide SVD
  double* d_jh = nullptr;     // Jacobi rotations of the reduced problem
  int* d_flags = nullptr;     // per-column round counters / reflector flags
  double* d_rg = nullptr;     // FP64 refinement of the mixed-precision SVD:
  double* d_rh = nullptr;     //   Gram, Newton-Schulz / correction factor,
  double* d_rt = nullptr;     //   product, rotated vectors (ws_nvmax^2 each)
  double* d_rw = nullptr;
  double* d_tau = nullptr;    // Householder scalars
  double* d_sig = nullptr;    // singular values (sorted)
  double* d_norm = nullptr;   // vector norms from the Jacobi sweeps
  double* d_disc = nullptr;   // discarded weights per (phase, bond)
  double* d_scale = nullptr;  // power-of-two state scaling of a reduced-precision step (2^s, 2^-s)
  double* d_gpart = nullptr;  // partial Gram products (kGramChunks x gnv^2) of the mixed SVD
  long long gnv = 0;          // vectors the partial buffer holds
  int* d_ints = nullptr;      // scratch ints (ranks of temporaries)
  DevSync* d_sync = nullptr;
  // learned form: spectra of the last round (row k = bond k, ws_nvmax wide),
  // their lengths, the proposed ranks, features and network outputs
  double* d_spec = nullptr;
  int* d_spec_len = nullptr;
  int* d_prop = nullptr;
  float* d_feat = nullptr;
  float* d_y = nullptr;
  // range finder (allocated when the context uses learned ranks): sketch Y,
  // its thin Q, B = Q^T X^T, residual E, kept rotations, scalars, flags
  double* d_rfy = nullptr;
  double* d_rfq = nullptr;
  double* d_rfb = nullptr;
  double* d_rfe = nullptr;
  double* d_rfjp = nullptr;
  double* d_rfs = nullptr;
  int* d_rff = nullptr;
  Mps* phi = nullptr;
  Mps* eta = nullptr;
  Mps* theta = nullptr;
  Mps* spare = nullptr;
};

}  // namespace qtt

namespace qtt {
enum { KC_GEMM = 0, KC_QR, KC_JACOBI, KC_POST, KC_MPO, KC_SUM, KC_COPY, KC_FDTD, KC_REFINE, KC_OTHER, KC_PIVOT, KC_N };

struct Prof {
  int timing = 0;
  int used = 0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
  std::vector<int> cls;
  long long launches[KC_N] = {0};
  int* d_log = nullptr;     // (nv, m) of each Jacobi launch while profiling
  int log_cap = 0;
  int log_used = 0;
  double* d_flops = nullptr;  // algorithmic FLOPs per class, counted by the kernels while logging
};

// Counter of the class whose launch is being issued on this thread (set by
// the launch bracket while work logging is on, else null).  Launchers pass
// it to their kernels, which add the algorithmic FLOP count of the launch
// from their device-side sizes.
extern thread_local double* g_flop_ctr;

// Multiprocessor count of the current device (queried once per device).
int device_sms();
}  // namespace qtt

namespace qtt {
// Autotuning.  A launch recorded during a dry-run step, re-launchable with
// any candidate choice: op 0 = a contraction GEMM (kind 0 FP64, 1 FP32 SIMT,
// 2 TF32, 3 3xTF32, 4 BF16 tensor cores; bucket a, b, c = Mmax, Nmax,
// batches; choice = output tile 16 / 32 or tensor-core columns 64 / 128 /
// 256), op 1 = a Householder QR (kind 0 FP64, 1 FP32; bucket = rows of the
// working columns, columns, thin Q formed; choice = threads per CTA 256 /
// 1024).  Choice 0 is the built-in heuristic.
struct TuneRec {
  int op;
  int kind;
  long long a, b, c;
  std::function<cudaError_t(int)> launch;
};
using TuneKey = std::tuple<int, int, long long, long long, long long>;
}  // namespace qtt

struct qtt_mlp;

struct qtt_ctx {
  qtt_params p{};
  int d = 0;
  int dims = 2;          // 2: Eq. 2 on an N x N grid; 3: the 3D extension, N^3
  int site_pos[32] = {0};  // bit of the linear dense index carried by site k
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 0;
  int coop_blocks = 0;  // co-resident CTAs for the cooperative kernels
  qtt::Workspace ws;
  bool ws_ready = false;
  qtt::Prof prof;
  bool use_mp = false;      // inside a reduced-precision step: FP32 contractions and QR, mixed SVD
  int ckind = -1;           // contractions of a reduced-precision step: -1 FP32 SIMT, else gemm_tc kind
  long long ws_nvmax = 0;   // widest SVD (vectors) the workspace holds
  long long ws_ellmax = 0;  // longest vector of a step SVD
  // learned form (the Sec. 4.3 rule still decides every truncation)
  qtt_mlp* mlp = nullptr;          // rank model (not owned)
  const double* sketch = nullptr;  // Gaussian test matrix, row-major rows x cols (not owned)
  long long sketch_rows = 0, sketch_cols = 0;
  int oversample = 16;
  double tau = 0.05;
  bool have_prop = false;          // d_prop holds proposals from the previous step
  std::vector<int> pending_prop;   // proposals set by the caller for the next step
  long long rf_attempts = 0, rf_accepts = 0;
  // CUDA-graph form of the step: two graphs (the two roles of the pair of
  // state buffers), their keys, the launches one replay makes per class
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  const void* gkey[2][4] = {{nullptr, nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr, nullptr}};
  double gkey_lam = 0.0;
  long gkey_src[4] = {0, 0, 0, 0};
  long long glaunches[16] = {0};
  double* d_amp = nullptr;  // source sample of the step being replayed
  cudaStream_t gstream = nullptr;  // capture stream (the legacy stream cannot be captured)
  bool capturing = false;   // inside a capture: the sum reads d_amp
  // failure-detection limits: device waits give up after wait_limit_ns
  // (QTT_ETIMEOUT), the FP64 Jacobi after max_sweeps sweeps (QTT_ENOCONV)
  unsigned long long wait_limit_ns = 0;  // 0: the default, 2 s
  int max_sweeps = 100;
  // autotuned choice per launch bucket (qtt_autotune), and the launches of
  // a dry-run step while one is being recorded
  std::map<qtt::TuneKey, int> tune;
  std::vector<qtt::TuneRec>* tune_rec = nullptr;
};

namespace qtt {

// ---------------------------------------------------------------- kernels
// (defined in the .cu files; all launch on ctx->stream)

struct GemmArgs {
  const double* A;
  const double* B;
  double* C;
  Dim M, N, K;
  Dim sai, sak, sbk, sbj, sci, scj;  // element strides
  Dim nb1, nb2;                      // two-level batch counts
  Dim sa1, sa2, sb1, sb2, sc1, sc2;  // batch strides
  double alpha, beta;
};
// C[b1,b2](i,j) = alpha * sum_k A(i,k) B(k,j) + beta * C(i,j); Mmax/Nmax/nbmax size the grid;
// tile: 16 or 32 (square output tile per CTA), 0 = by the number of tiles
cudaError_t gemm_f64(const GemmArgs& a, long long Mmax, long long Nmax, long long nb1max,
                     long long nb2max, cudaStream_t st, int tile = 0);
// the same product with FP32 arithmetic (the reduced-precision form)
cudaError_t gemm_f32(const GemmArgs& a, long long Mmax, long long Nmax, long long nb1max,
                     long long nb2max, cudaStream_t st, int tile = 0);
// G (ld ldg) = X X^T for nv vectors X_i at X + i*ldx of length ell, FP64,
// split over the length into at most max_chunks partial products in P
// (max_chunks * nvmax * nvmax doubles), upper tiles only, reduced in a fixed
// order
cudaError_t gram_f64(const double* X, Dim ldx, Dim nv, Dim ell, long long nvmax, long long ellmax, double* G,
                     long long ldg, double* P, int max_chunks, cudaStream_t st);
constexpr int kGramChunks = 16;
// the same product on the tensor cores (tcgen05, accumulator in TMEM): kind
// 0 = TF32, 1 = 3xTF32 (hi/lo split, ~FP32 accuracy), 2 = BF16; FP32
// accumulation; bn = 64, 128 or 256 columns per CTA (128 rows); waits
// bounded by the limit in *sync (QTT_ETIMEOUT recorded there)
cudaError_t gemm_tc(const GemmArgs& a, long long Mmax, long long Nmax, long long nb1max, long long nb2max, int kind,
                    int bn, DevSync* sync, cudaStream_t st);
cudaError_t tc_init();

// Householder QR of the m x n matrix whose column j is Ain + j*lda (length m).
// R (kq x n, kq = min(m,n)) is written to Rout row-major (R[i][c] at i*ldr+c)
// if r_rowmajor else column-major (c*ldr+i); Q (m x kq) row-major to Qout if
// not null; kq to *kq_out if not null.  Work: column j at W + j*ldw.
// ldr: leading dimension of a column-major R.  Q formation needs m <= qm_max
// (the column is built in shared memory).
// block: threads per CTA (256 or 1024; 0 = 1024 for columns of 2048 rows or more)
cudaError_t qr_f64(qtt_ctx* ctx, const double* Ain, Dim lda, double* W, long long ldw, Dim m, Dim n,
                   long long nmax, double* Rout, bool r_rowmajor, double* Qout, int* kq_out, long long ldr,
                   long long qm_max = 0, int block = 0);
// the same factorisation with FP32 arithmetic on an FP32 working copy (W is
// reinterpreted as float storage); R and Q are written as doubles
cudaError_t qr_f32(qtt_ctx* ctx, const double* Ain, Dim lda, double* W, long long ldw, Dim m, Dim n,
                   long long nmax, double* Rout, bool r_rowmajor, double* Qout, int* kq_out, long long ldr,
                   long long qm_max = 0, int block = 0);

// One-sided Jacobi on nv vectors V + i*ldv of length m; J (nv x nv,
// vector-major, ld ldj) accumulates the rotations; norms[i] = |v_i| at the end.
cudaError_t jacobi_f64(qtt_ctx* ctx, double* V, long long ldv, Dim nv, Dim m, long long nvmax, double* J,
                       long long ldj, double* norms);
int* jacobi_log_slot(qtt_ctx* ctx);

// Sort, truncate, write rank, sigma, discarded weight and the kept rotations:
// Jp[j*nv + i] = J[perm_j][i] (j < r), and Jt[i*r + j] the same if Jt != null.
// cnt rotated vectors with norms; len: their length (min(cnt, len) singular
// values exist); jlen: length of a row of J (the number of input vectors);
// rank_cap: the destination capacity (a larger rank is clamped and reported).
// nsv_out (optional): min(cnt, len), the number of singular values.
cudaError_t svd_post(qtt_ctx* ctx, const double* norms, Dim cnt, Dim len, Dim jlen, const double* J, long long ldj,
                     double eps, int chi, int rank_cap, int* rank_out, double* sigma_out, double* disc_out,
                     double* Jp, double* Jt, int* nsv_out = nullptr);

}  // namespace qtt
