// C ABI of the QTT stepper: handles, workspace and the orchestration of one
// time step (Eq. 17) as a sequence of launches on the context stream with
// every bond rank kept in device memory (no host synchronisation per step).
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "k_learned.cuh"
#include "k_mps.cuh"
#include "qtt_internal.cuh"

namespace qtt {
void build_laplacian(int n, int order, int bc, int dims, Mpo* mpo);
int site_pos(int k, int n, int order, int dims);
void build_a_operator(const Mpo& L, const std::vector<std::vector<double>>& c2, const std::vector<int>& rc,
                      double lambda2, Mpo* A);
}

using namespace qtt;

namespace {

thread_local std::string g_err;

qtt_status fail(qtt_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

}  // namespace

namespace qtt {
void set_last_error(const std::string& msg) { g_err = msg; }

thread_local double* g_flop_ctr = nullptr;

int device_sms() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 1;
  if (dev < 64 && cache[dev] > 0) return cache[dev];
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
  if (dev < 64) cache[dev] = n;
  return n;
}
}  // namespace qtt

namespace {

#define CK(call)                                                                               \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return fail(e_ == cudaErrorMemoryAllocation ? QTT_ENOMEM : QTT_ECUDA,                    \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                         \
  } while (0)

// Every kernel launch goes through KL: it counts the launch and, when kernel
// timing is on, brackets it with events on the context stream.
#define KL_N(cls, nk, call)                                                                    \
  do {                                                                                         \
    prof_begin(ctx, cls);                                                                      \
    cudaError_t e_ = (call);                                                                   \
    g_flop_ctr = nullptr;                                                                      \
    if (e_ != cudaSuccess)                                                                     \
      return fail(e_ == cudaErrorMemoryAllocation ? QTT_ENOMEM : QTT_ECUDA,                    \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                         \
    prof_end(ctx, cls, nk);                                                                    \
  } while (0)
#define KL(cls, call) KL_N(cls, 1, call)
#define KL2(cls, call) KL_N(cls, 2, call)

void prof_begin(qtt_ctx* ctx, int cls) {
  Prof& p = ctx->prof;
  g_flop_ctr = p.d_flops ? p.d_flops + cls : nullptr;
  if (!p.timing) return;
  if (p.used >= (int)p.ev.size()) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
      p.timing = 0;
      return;
    }
    p.ev.push_back({a, b});
  }
  cudaEventRecord(p.ev[p.used].first, ctx->stream);
  p.cls.resize(p.ev.size());
  p.cls[p.used] = cls;
}

void prof_end(qtt_ctx* ctx, int cls, int nk) {
  Prof& p = ctx->prof;
  p.launches[cls] += nk;
  if (!p.timing) return;
  cudaEventRecord(p.ev[p.used].second, ctx->stream);
  ++p.used;
}

#define CKS(expr)                  \
  do {                             \
    qtt_status s_ = (expr);        \
    if (s_ != QTT_OK) return s_;   \
  } while (0)

inline long long p2(int e) { return e >= 62 ? (1LL << 62) : (1LL << e); }

// -------------------------------------------------------------- MPS memory
std::vector<int> psi_caps(int d, int chi) {
  std::vector<int> c(d + 1);
  for (int k = 0; k <= d; ++k) c[k] = (int)std::min<long long>({p2(k), p2(d - k), (long long)chi});
  return c;
}

qtt_status mps_alloc(qtt_ctx* ctx, const std::vector<int>& cap, Mps* m) {
  m->ctx = ctx;
  m->d = ctx->d;
  m->cap = cap;
  m->off.assign(m->d, 0);
  long long tot = 0;
  for (int k = 0; k < m->d; ++k) {
    m->off[k] = tot;
    tot += (long long)cap[k] * 2 * cap[k + 1];
  }
  m->total = tot;
  CK(cudaMalloc(&m->data, std::max<long long>(tot, 1) * sizeof(double)));
  CK(cudaMalloc(&m->ranks, (m->d + 1) * sizeof(int)));
  CK(cudaMemsetAsync(m->data, 0, std::max<long long>(tot, 1) * sizeof(double), ctx->stream));
  std::vector<int> ones(m->d + 1, 1);
  CK(cudaMemcpyAsync(m->ranks, ones.data(), (m->d + 1) * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return QTT_OK;
}

void mps_free(Mps* m) {
  if (!m) return;
  if (m->data) cudaFree(m->data);
  if (m->ranks) cudaFree(m->ranks);
  m->data = nullptr;
  m->ranks = nullptr;
}

// --------------------------------------------------------------- workspace
struct Caps {
  std::vector<int> psi, phi, eta, theta;
};

Caps step_caps(const qtt_ctx* ctx, const std::vector<int>& w, const std::vector<int>& rc) {
  const int d = ctx->d, chi = ctx->p.chi_max, chz = ctx->p.chi_zip;
  Caps c;
  c.psi = psi_caps(d, chi);
  c.phi.assign(d + 1, 1);
  c.eta.assign(d + 1, 1);
  c.theta.assign(d + 1, 1);
  for (int k = 1; k < d; ++k)
    c.phi[k] = (int)std::min<long long>({(long long)chz, p2(k), (long long)w[k] * c.psi[k]});
  for (int k = 1; k < d; ++k)
    c.eta[k] = (int)std::min<long long>({(long long)chz, p2(d - k), (long long)c.phi[k] * rc[k]});
  for (int k = 1; k < d; ++k) c.theta[k] = 2 * c.psi[k] + c.eta[k] + 1;
  return c;
}

void ws_free(qtt_ctx* ctx) {
  Workspace& s = ctx->ws;
  double** bufs[] = {&s.d_carry, &s.d_x, &s.d_tv, &s.d_tq, &s.d_rv, &s.d_jv, &s.d_jp, &s.d_w1,
                     &s.d_tt, &s.d_qt, &s.d_jh, &s.d_rg, &s.d_rh, &s.d_rt, &s.d_rw, &s.d_tau,
                     &s.d_sig, &s.d_norm, &s.d_disc, &s.d_scale, &s.d_gpart};
  for (double** b : bufs)
    if (*b) {
      cudaFree(*b);
      *b = nullptr;
    }
  if (s.d_ints) cudaFree(s.d_ints);
  s.d_ints = nullptr;
  if (s.d_flags) cudaFree(s.d_flags);
  s.d_flags = nullptr;
  if (s.d_sync) cudaFree(s.d_sync);
  s.d_sync = nullptr;
  void** lbufs[] = {(void**)&s.d_spec, (void**)&s.d_spec_len, (void**)&s.d_prop, (void**)&s.d_feat, (void**)&s.d_y,
                    (void**)&s.d_rfy, (void**)&s.d_rfq, (void**)&s.d_rfb, (void**)&s.d_rfe, (void**)&s.d_rfjp,
                    (void**)&s.d_rfs, (void**)&s.d_rff};
  for (void** b : lbufs)
    if (*b) {
      cudaFree(*b);
      *b = nullptr;
    }
  ctx->have_prop = false;
  Mps* ms[] = {s.phi, s.eta, s.theta, s.spare};
  for (Mps* m : ms)
    if (m) {
      mps_free(m);
      delete m;
    }
  s.phi = s.eta = s.theta = s.spare = nullptr;
  ctx->ws_ready = false;
  for (auto& g : ctx->gexec)  // graphs point into the workspace
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
}

struct Sizes {
  long long carry = 1, x = 1, tv = 1, rv = 1, jv = 1, jp = 1, w1 = 1, vec = 1;
  long long nvmax = 2, ellmax = 1;
};

// Largest buffer each phase needs, from the per-bond capacities.
Sizes step_sizes(const qtt_ctx* ctx, const Caps& c, const std::vector<int>& w, const std::vector<int>& rc) {
  const int d = ctx->d;
  Sizes z;
  auto upd = [](long long& a, long long b) { a = std::max(a, b); };
  // zip-up L: site k, a = phi[k], w = w[k], b = psi[k], b' = psi[k+1], w' = w[k+1]
  for (int k = 0; k < d; ++k) {
    long long a = c.phi[k], b2 = c.psi[k + 1], wl = w[k], wr = w[k + 1];
    upd(z.x, a * wl * 2 * b2);
    upd(z.tv, 2 * a * wr * b2);
    upd(z.carry, (long long)c.phi[k + 1] * wr * b2);
    upd(z.nvmax, 2 * a);
    upd(z.ellmax, wr * b2);
  }
  // zip-up C^2: site k, B = phi[k], B' = phi[k+1], R = rc[k], R' = rc[k+1], A' = eta[k+1]
  for (int k = d - 1; k >= 0; --k) {
    long long B = c.phi[k], B2 = c.phi[k + 1], R = rc[k], R2 = rc[k + 1], A2 = c.eta[k + 1];
    upd(z.x, 2 * B * R2 * A2);
    upd(z.tv, 2 * A2 * B * R);
    upd(z.carry, B2 * R2 * A2);
    upd(z.carry, B * R * (long long)c.eta[k]);
    upd(z.nvmax, 2 * A2);
    upd(z.ellmax, B * R);
  }
  // round: QR of (2 q_k) x D_{k+1}; SVD of q_k x 2 r_{k+1}
  for (int k = 0; k < d; ++k) {
    long long q = c.theta[k], D2 = c.theta[k + 1];
    upd(z.tv, 2 * q * D2);
    upd(z.rv, std::min(2 * q, D2) * D2);
    upd(z.w1, (long long)c.psi[k] * q);
    upd(z.nvmax, 2 * (long long)c.psi[k + 1]);
    upd(z.ellmax, std::max(2 * q, q));
    upd(z.vec, D2);
    upd(z.vec, 2 * q);
  }
  // TT-SVD of a dense grid (c^2 with chi_c, states with chi_max)
  upd(z.nvmax, 2LL * std::max(ctx->p.chi_max, ctx->p.chi_c));
  upd(z.vec, z.nvmax);
  upd(z.jv, z.nvmax * z.nvmax);
  upd(z.jp, z.nvmax * z.nvmax);
  upd(z.rv, z.nvmax * z.nvmax);
  return z;
}

qtt_status ws_alloc(qtt_ctx* ctx, const Sizes& z, const Caps& c) {
  Workspace& s = ctx->ws;
  const int d = ctx->d;
  const long long N2 = p2(ctx->d);
  // TT-SVD of a dense grid and to_dense use N^dims-sized scratch
  long long tv = std::max(z.tv, N2), carry = std::max(z.carry, N2), x = std::max(z.x, N2);
  s.carry = carry;
  s.xbuf = x;
  s.tv = tv;
  s.tq = tv;
  s.rv = z.rv;
  s.jv = z.jv;
  s.jp = z.jp;
  s.w1 = std::max(z.w1, 1LL);
  s.vec = std::max(z.vec, 64LL);
  CK(cudaMalloc(&s.d_carry, carry * sizeof(double)));
  CK(cudaMalloc(&s.d_x, x * sizeof(double)));
  CK(cudaMalloc(&s.d_tv, tv * sizeof(double)));
  CK(cudaMalloc(&s.d_tq, tv * sizeof(double)));
  CK(cudaMalloc(&s.d_rv, s.rv * sizeof(double)));
  CK(cudaMalloc(&s.d_jv, s.jv * sizeof(double)));
  CK(cudaMalloc(&s.d_jp, s.jp * sizeof(double)));
  CK(cudaMalloc(&s.d_w1, s.w1 * sizeof(double)));
  CK(cudaMalloc(&s.d_tt, tv * sizeof(double)));
  CK(cudaMalloc(&s.d_qt, tv * sizeof(double)));
  CK(cudaMalloc(&s.d_jh, s.jv * sizeof(double)));
  CK(cudaMalloc(&s.d_rg, s.jv * sizeof(double)));
  CK(cudaMalloc(&s.d_rh, s.jv * sizeof(double)));
  CK(cudaMalloc(&s.d_rt, s.jv * sizeof(double)));
  CK(cudaMalloc(&s.d_rw, s.jv * sizeof(double)));
  CK(cudaMalloc(&s.d_tau, s.vec * sizeof(double)));
  CK(cudaMalloc(&s.d_sig, s.vec * sizeof(double)));
  CK(cudaMalloc(&s.d_norm, s.vec * sizeof(double)));
  CK(cudaMalloc(&s.d_disc, 3 * (d + 1) * sizeof(double)));
  CK(cudaMalloc(&s.d_scale, 2 * sizeof(double)));
  s.gnv = std::min<long long>(z.nvmax, 256);
  CK(cudaMalloc(&s.d_gpart, (size_t)kGramChunks * s.gnv * s.gnv * sizeof(double)));
  CK(cudaMalloc(&s.d_ints, 4 * (d + 8) * sizeof(int)));
  CK(cudaMalloc(&s.d_flags, (s.vec + 64) * sizeof(int)));
  CK(cudaMalloc(&s.d_sync, sizeof(DevSync)));
  CK(cudaMemsetAsync(s.d_sync, 0, sizeof(DevSync), ctx->stream));
  CK(cudaMemcpyAsync(&s.d_sync->limit_ns, &ctx->wait_limit_ns, sizeof(unsigned long long), cudaMemcpyHostToDevice,
                     ctx->stream));
  CK(cudaMemsetAsync(s.d_disc, 0, 3 * (d + 1) * sizeof(double), ctx->stream));
  CK(cudaMalloc(&s.d_spec, (d + 1) * z.nvmax * sizeof(double)));
  CK(cudaMalloc(&s.d_spec_len, (d + 1) * sizeof(int)));
  CK(cudaMalloc(&s.d_prop, (d + 1) * sizeof(int)));
  CK(cudaMalloc(&s.d_feat, (d + 1) * (size_t)kFeat * sizeof(float)));
  CK(cudaMalloc(&s.d_y, (d + 1) * sizeof(float)));
  CK(cudaMemsetAsync(s.d_spec_len, 0, (d + 1) * sizeof(int), ctx->stream));
  CK(cudaMemsetAsync(s.d_prop, 0, (d + 1) * sizeof(int), ctx->stream));
  if (ctx->p.use_learned_rank) {
    CK(cudaMalloc(&s.d_rfy, tv * sizeof(double)));
    CK(cudaMalloc(&s.d_rfq, tv * sizeof(double)));
    CK(cudaMalloc(&s.d_rfb, tv * sizeof(double)));
    CK(cudaMalloc(&s.d_rfe, tv * sizeof(double)));
    CK(cudaMalloc(&s.d_rfjp, z.nvmax * z.nvmax * sizeof(double)));
    CK(cudaMalloc(&s.d_rfs, 4 * sizeof(double)));
    CK(cudaMalloc(&s.d_rff, 4 * sizeof(int)));
  }
  s.phi = new Mps();
  s.eta = new Mps();
  s.theta = new Mps();
  CKS(mps_alloc(ctx, c.phi, s.phi));
  CKS(mps_alloc(ctx, c.eta, s.eta));
  CKS(mps_alloc(ctx, c.theta, s.theta));
  ctx->ws_nvmax = z.nvmax;
  ctx->ws_ellmax = z.ellmax;
  ctx->ws_ready = true;
  return QTT_OK;
}

// Capacities of the fused step (Eq. 7 applied as one MPO A of bonds w):
// theta = phi - psi^{k-1} (+ source) needs phi + psi + 1 at every bond.
Caps fused_caps(const qtt_ctx* ctx, const std::vector<int>& w) {
  Caps c = step_caps(ctx, w, std::vector<int>(ctx->d + 1, 1));
  for (int k = 1; k < ctx->d; ++k) c.theta[k] = std::max(c.theta[k], c.phi[k] + c.psi[k] + 1);
  return c;
}

qtt_status ensure_ws_caps(qtt_ctx* ctx, const std::vector<int>& w, const std::vector<int>& rc, const Caps& c);

// Workspace for a step with MPO bonds w and c^2 ranks rc (grown if needed).
qtt_status ensure_ws(qtt_ctx* ctx, const std::vector<int>& w, const std::vector<int>& rc) {
  return ensure_ws_caps(ctx, w, rc, step_caps(ctx, w, rc));
}

qtt_status ensure_ws_caps(qtt_ctx* ctx, const std::vector<int>& w, const std::vector<int>& rc, const Caps& c) {
  Sizes z = step_sizes(ctx, c, w, rc);
  if (ctx->ws_ready) {
    const Workspace& s = ctx->ws;
    bool ok = s.tv >= z.tv && s.carry >= z.carry && s.xbuf >= z.x && s.rv >= z.rv && s.jv >= z.jv &&
              s.w1 >= z.w1 && s.vec >= z.vec && ctx->ws_nvmax >= z.nvmax && s.theta->cap == c.theta &&
              s.phi->cap == c.phi && s.eta->cap == c.eta;
    if (ok) return QTT_OK;
    CK(cudaStreamSynchronize(ctx->stream));
    ws_free(ctx);
  }
  return ws_alloc(ctx, z, c);
}

// workspace for setup-only work (no MPO / c^2 known yet)
qtt_status ensure_ws_basic(qtt_ctx* ctx) {
  if (ctx->ws_ready) return QTT_OK;
  std::vector<int> w(ctx->d + 1, 5), rc(ctx->d + 1, 1);
  w[0] = w[ctx->d] = 1;
  return ensure_ws(ctx, w, rc);
}

qtt_status device_status(qtt_ctx* ctx) {
  int st = 0;
  CK(cudaMemcpyAsync(&st, &ctx->ws.d_sync->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (st != 0) {
    // a kernel that gave up leaves barrier counters and flags mid-way: reset
    // the whole word (keeping the context's wait limit) before the next launch
    CK(cudaMemsetAsync(ctx->ws.d_sync, 0, sizeof(DevSync), ctx->stream));
    CK(cudaMemcpyAsync(&ctx->ws.d_sync->limit_ns, &ctx->wait_limit_ns, sizeof(unsigned long long),
                       cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    const char* what = st == QTT_ENOCONV ? "Jacobi SVD reached its sweep limit"
                       : st == QTT_ETIMEOUT ? "a grid barrier wait timed out"
                       : st == QTT_ENONFINITE ? "non-finite singular value"
                                              : "device error";
    return fail((qtt_status)st, what);
  }
  return QTT_OK;
}

// Site positions of the context (Eq. 3, Eq. 12, Eq. 14-15; 3D extension).
SitePos site_positions(const qtt_ctx* ctx) {
  SitePos sp;
  std::memset(&sp, 0, sizeof(sp));
  sp.d = ctx->d;
  for (int k = 0; k < ctx->d; ++k) sp.pos[k] = ctx->site_pos[k];
  return sp;
}

// A grid point given as dims coordinates, each in [0, N).
qtt_status check_point(const qtt_ctx* ctx, const long* p) {
  const long N = 1L << ctx->p.n;
  for (int a = 0; a < ctx->dims; ++a)
    if (p[a] < 0 || p[a] >= N) return fail(QTT_EINVAL, "point outside the grid");
  return QTT_OK;
}

qtt_status inject_impl(qtt_ctx* ctx, qtt_mps* psi, const long* src, double amp);

// ------------------------------------------------------------- SVD helper
// Truncated SVD of nv vectors (rows of the vector-major array Tv, ld ell,
// not modified).  Jacobi rotations J satisfy: the rotated vectors
// J^T Tv have orthogonal rows.  Writes the kept rank to rank_out and
// Jp (r x nv) / Jt (nv x r).
qtt_status svd_vm(qtt_ctx* ctx, const double* Tv, Dim nv, Dim ell, long long nvmax, long long ellmax, double eps,
                  int chi, int rank_cap, int* rank_out, double* Jp, double* Jt, double* disc_out,
                  double* sigma_out, int* nsv_out = nullptr);

GemmArgs gemm0();

}  // namespace

namespace {

// columns per CTA of a tensor-core contraction: the widest tile that still
// gives every SM a CTA, else the narrowest
int tc_tile_n(const qtt_ctx* ctx, long long Mmax, long long Nmax, long long nb) {
  const long long tiles_m = (Mmax + 127) / 128 * nb;
  for (int bn : {256, 128}) {
    if (Nmax <= bn / 2) continue;
    if (tiles_m * ((Nmax + bn - 1) / bn) >= ctx->num_sms) return bn;
  }
  return Nmax <= 64 ? 64 : (Nmax <= 128 && tiles_m * 2 < ctx->num_sms ? 64 : 128);
}

int tune_choice(const qtt_ctx* ctx, int op, int kind, long long a, long long b, long long c) {
  if (ctx->tune.empty()) return 0;
  auto it = ctx->tune.find(TuneKey{op, kind, a, b, c});
  return it == ctx->tune.end() ? 0 : it->second;
}

// A contraction GEMM of the given kind (0 FP64, 1 FP32 SIMT, 2.. tensor
// cores) with the autotuned tile of its bucket; recorded when a dry-run step
// is being recorded.
cudaError_t gemm_k(qtt_ctx* ctx, int kind, const GemmArgs& g, long long Mmax, long long Nmax, long long b1,
                   long long b2) {
  const long long nb = b1 * b2;
  auto run = [ctx, kind, g, Mmax, Nmax, b1, b2, nb](int ch) -> cudaError_t {
    if (kind == 0) return gemm_f64(g, Mmax, Nmax, b1, b2, ctx->stream, ch);
    if (kind == 1) return gemm_f32(g, Mmax, Nmax, b1, b2, ctx->stream, ch);
    return gemm_tc(g, Mmax, Nmax, b1, b2, kind - 2, ch ? ch : tc_tile_n(ctx, Mmax, Nmax, nb), ctx->ws.d_sync,
                   ctx->stream);
  };
  if (ctx->tune_rec) ctx->tune_rec->push_back(TuneRec{0, kind, Mmax, Nmax, nb, run});
  return run(tune_choice(ctx, 0, kind, Mmax, Nmax, nb));
}

// contractions and QR in the step's precision; setup work is always FP64
cudaError_t gemm_any(qtt_ctx* ctx, const GemmArgs& g, long long Mmax, long long Nmax, long long b1, long long b2) {
  return gemm_k(ctx, !ctx->use_mp ? 0 : (ctx->ckind < 0 ? 1 : ctx->ckind + 2), g, Mmax, Nmax, b1, b2);
}

// an FP64 GEMM of the refinement or the Gram matrix (autotuned like the rest)
cudaError_t gemm_d(qtt_ctx* ctx, const GemmArgs& g, long long Mmax, long long Nmax, long long b1, long long b2,
                   cudaStream_t) {
  return gemm_k(ctx, 0, g, Mmax, Nmax, b1, b2);
}

cudaError_t qr_any(qtt_ctx* ctx, const double* Ain, Dim lda, double* W, long long ldw, Dim m, Dim n, long long nmax,
                   double* Rout, bool r_rowmajor, double* Qout, int* kq_out, long long ldr, long long qm_max) {
  const int kind = ctx->use_mp ? 1 : 0;
  auto run = [=](int ch) -> cudaError_t {
    return kind ? qr_f32(ctx, Ain, lda, W, ldw, m, n, nmax, Rout, r_rowmajor, Qout, kq_out, ldr, qm_max, ch)
                : qr_f64(ctx, Ain, lda, W, ldw, m, n, nmax, Rout, r_rowmajor, Qout, kq_out, ldr, qm_max, ch);
  };
  const long long withq = Qout ? 1 : 0;
  if (ctx->tune_rec) ctx->tune_rec->push_back(TuneRec{1, kind, ldw, nmax, withq, run});
  return run(tune_choice(ctx, 1, kind, ldw, nmax, withq));
}

// C (ld ldc) = A B with A (M x K, ld lda) and B (K x N, ld ldb), FP64
GemmArgs mm(const double* A, long long lda, const double* B, long long ldb, double* C, long long ldc, Dim M, Dim K,
            Dim N) {
  GemmArgs g = gemm0();
  g.A = A;
  g.B = B;
  g.C = C;
  g.M = M;
  g.N = N;
  g.K = K;
  g.sai = dconst(lda);
  g.sak = dconst(1);
  g.sbk = dconst(ldb);
  g.sbj = dconst(1);
  g.sci = dconst(ldc);
  g.scj = dconst(1);
  return g;
}

// G (ld ldg) = X X^T for X (rows x cols, ld ldx), FP64
GemmArgs gram(const double* X, long long ldx, double* G, long long ldg, Dim rows, Dim cols) {
  GemmArgs g = mm(X, ldx, X, ldx, G, ldg, rows, cols, rows);
  g.sbk = dconst(1);
  g.sbj = dconst(ldx);
  return g;
}

// One-sided Jacobi of nv vectors V (length m) in the step's precision.  The
// mixed form: FP32 Jacobi in one cluster, then FP64 refinement (two damped
// first-order corrections from the Gram of W = J V with a Newton-Schulz step
// between them, one final Newton-Schulz step), sigma = |W_c|.
qtt_status jacobi_any(qtt_ctx* ctx, double* V, long long ldv, Dim nv, Dim m, long long nvmax, long long mmax,
                      double* J, long long ldj, double* norms) {
  if (!ctx->use_mp) {
    KL(KC_JACOBI, jacobi_f64(ctx, V, ldv, nv, m, nvmax, J, ldj, norms));
    return QTT_OK;
  }
  Workspace& s = ctx->ws;
  const long long ld = ctx->ws_nvmax;
  if (mmax > ld || nvmax > ld) return fail(QTT_EINVAL, "internal: mixed SVD wider than the workspace");
  KL(KC_JACOBI, jacobi32_cluster(ctx, V, ldv, nv, m, nvmax, mmax, J, ldj));
  auto ns = [&]() -> qtt_status {  // J <- (3I - J J^T)/2 J  (rows of J are the columns of the rotation)
    KL(KC_REFINE, gemm_d(ctx, gram(J, ldj, s.d_rg, ld, nv, nv), nvmax, nvmax, 1, 1, ctx->stream));
    KL(KC_REFINE, ns_factor(s.d_rg, s.d_rh, ld, nv, nvmax, ctx->stream));
    KL(KC_REFINE, gemm_d(ctx, mm(s.d_rh, ld, J, ldj, s.d_rt, ld, nv, nv, nv), nvmax, nvmax, 1, 1, ctx->stream));
    KL(KC_REFINE, copy2d(s.d_rt, J, nv, nv, dconst(ld), dconst(1), dconst(ldj), dconst(1), nvmax * nvmax, 1.0,
                         ctx->stream));
    return QTT_OK;
  };
  for (int it = 0; it < 2; ++it) {
    // the FP32 rotation is orthogonal to ~1e-6: the first correction takes
    // that in with the off-diagonal part, the Newton-Schulz step before the
    // second one restores orthogonality to ~|Omega|^2
    if (it > 0) CKS(ns());
    KL(KC_REFINE, gemm_d(ctx, mm(J, ldj, V, ldv, s.d_rw, ld, nv, nv, m), nvmax, mmax, 1, 1, ctx->stream));
    KL(KC_REFINE, gemm_d(ctx, gram(s.d_rw, ld, s.d_rg, ld, nv, m), nvmax, nvmax, 1, 1, ctx->stream));
    KL2(KC_REFINE, omega_factor(s.d_rg, norms, s.d_rh, ld, nv, nvmax, ctx->stream));  // two kernels; norms: scratch
    KL(KC_REFINE, gemm_d(ctx, mm(s.d_rh, ld, J, ldj, s.d_rt, ld, nv, nv, nv), nvmax, nvmax, 1, 1, ctx->stream));
    KL(KC_REFINE, copy2d(s.d_rt, J, nv, nv, dconst(ld), dconst(1), dconst(ldj), dconst(1), nvmax * nvmax, 1.0,
                         ctx->stream));
  }
  // after the second correction J is orthogonal to ~|Omega|^2 (FP64
  // rounding once the FP32 stage reached its 1e-4 stop): one Newton-Schulz
  // step takes it to rounding
  CKS(ns());
  KL(KC_REFINE, gemm_d(ctx, mm(J, ldj, V, ldv, s.d_rw, ld, nv, nv, m), nvmax, mmax, 1, 1, ctx->stream));
  KL(KC_REFINE, row_norms(s.d_rw, ld, nv, m, nvmax, norms, ctx->stream));
  return QTT_OK;
}

// Rows of J (rows x cols, row stride ldj) made orthonormal to FP64 rounding
// when they already are to FP32 rounding: J <- (3I - J J^T)/2 J, FP64.
qtt_status ns_rows(qtt_ctx* ctx, double* J, long long ldj, Dim rows, Dim cols, long long rowsmax, long long colsmax) {
  Workspace& s = ctx->ws;
  const long long ld = ctx->ws_nvmax;
  KL(KC_REFINE, gemm_d(ctx, gram(J, ldj, s.d_rg, ld, rows, cols), rowsmax, rowsmax, 1, 1, ctx->stream));
  KL(KC_REFINE, ns_factor(s.d_rg, s.d_rh, ld, rows, rowsmax, ctx->stream));
  KL(KC_REFINE, gemm_d(ctx, mm(s.d_rh, ld, J, ldj, s.d_rt, ld, rows, rows, cols), rowsmax, colsmax, 1, 1, ctx->stream));
  KL(KC_REFINE, copy2d(s.d_rt, J, rows, cols, dconst(ld), dconst(1), dconst(ldj), dconst(1), rowsmax * colsmax, 1.0,
                       ctx->stream));
  return QTT_OK;
}

// Truncated SVD of nv vectors (rows of the vector-major array Tv, ld ell,
// not modified).  J (nv x r) holds the kept right singular vectors of the
// matrix M whose columns are the vectors: M J = U S.  Writes the kept rank
// to rank_out, Jp = J^T (r x nv) and Jt = J (nv x r).  The Jacobi sweeps
// always run on a square problem of size at most min(nv, ell):
//   reduced-precision form, ell > nv (nv <= 256): the rows of a pivoted
//     triangular factor R of M (from the Gram matrix, or from a QR and a
//     pivoted QR of the small R0^T), rotated in FP32 and refined in FP64;
//   ell >= nv: M = Q R, rotate the columns of R (Q never formed);
//   ell <  nv: M^T = Q R, rotate the rows of R, J = Q J_R.
qtt_status svd_vm(qtt_ctx* ctx, const double* Tv, Dim nv, Dim ell, long long nvmax, long long ellmax, double eps,
                  int chi, int rank_cap, int* rank_out, double* Jp, double* Jt, double* disc_out,
                  double* sigma_out, int* nsv_out) {
  Workspace& s = ctx->ws;
  const long long ldv = ctx->ws_nvmax;  // R / J leading dimension
  if (nvmax > ldv || ellmax * nvmax > s.tv)
    return fail(QTT_EINVAL, "internal: SVD larger than the workspace");
  double* sig = sigma_out ? sigma_out : s.d_sig;
  int* kq = s.d_ints + 0;
  // The Gram matrix costs nv^2 ell / 2 FP64 FMAs spread over all SMs (split
  // over the vector length), the QR about 4 us per column (its chain of
  // reflectors) plus the pivoted QR of R0^T: up to nv ell = 2^25 (every bond
  // of the 1024x1024 and 2048x2048 workloads' mixed SVDs) the Gram route is
  // the cheaper, and on the tall zip-up bonds of diag(c^2) it is also the more
  // accurate of the two (the QR route rounds M itself in FP32).
  if (ellmax > nvmax && ctx->use_mp && nvmax <= 256 && nvmax <= s.gnv && ldv * nvmax <= s.tv &&
      nvmax * ellmax <= (1LL << 25)) {
    // Preconditioned Jacobi (Drmac & Veselic 2008) on the rows of the
    // triangular factor of a QR with column pivoting of M, formed without
    // touching M again: G = M^T M in FP64, G = R^T R by Cholesky with
    // diagonal pivoting (R graded, k rows: the numerical rank), one-sided
    // Jacobi on the rows of R (~7 sweeps instead of ~25), J R = W with
    // orthogonal rows.  M = Q R = (Q J^T) W, so sigma = |W_c| and the right
    // singular vectors of M are the rows of W / |W_c|, re-orthonormalised in
    // FP64.
    int* kr = s.d_ints + 1;
    // G[a][c] = sum_l Tv[a][l] Tv[c][l]
    KL2(KC_PIVOT, gram_f64(Tv, ell, nv, ell, nvmax, ellmax, s.d_tt, ldv, s.d_gpart, kGramChunks, ctx->stream));
    KL(KC_PIVOT, pchol_cluster(ctx, s.d_tt, ldv, nv, ell, nvmax, s.d_rv, ldv, kr));
    CKS(jacobi_any(ctx, s.d_rv, ldv, dptr(kr), nv, nvmax, nvmax, s.d_jv, ldv, s.d_norm));
    // jacobi_any leaves W = J R in the refinement buffer
    KL(KC_REFINE, scale_rows(s.d_rw, ldv, s.d_norm, dptr(kr), nv, nvmax, nvmax, s.d_jh, ldv, ctx->stream));
    CKS(ns_rows(ctx, s.d_jh, ldv, dptr(kr), nv, nvmax, nvmax));
    KL(KC_POST, svd_post(ctx, s.d_norm, dptr(kr), nv, nv, s.d_jh, ldv, eps, chi, rank_cap, rank_out, sig, disc_out,
                         Jp, Jt, nsv_out));
    return QTT_OK;
  }
  if (ellmax > nvmax && ctx->use_mp && nvmax <= 256 && ldv * nvmax <= s.tv && nvmax * 128 <= s.tv) {
    // Preconditioned Jacobi (Drmac & Veselic 2008): M = Q R0 (R0 only),
    // R0^T P = Q1 R1 with column pivoting in one cluster, one-sided Jacobi
    // on the rows of R1 (graded by the pivoting: ~7 sweeps instead of ~25).
    // The rotation J of R1's rows gives R1's left singular vectors, so the
    // right singular vectors of M are the rows of J Q1^T: products of
    // orthogonal factors, re-orthonormalised in FP64.
    int* k1 = s.d_ints + 1;
    KL(KC_QR, qr_any(ctx, Tv, ell, s.d_tq, ellmax, ell, nv, nvmax, s.d_rv, false, nullptr, kq, ldv, 0));
    KL(KC_PIVOT, qrcp_cluster(ctx, s.d_rv, ldv, nv, dptr(kq), nvmax, s.d_tt, ldv, s.d_qt, ldv,
                           reinterpret_cast<float*>(s.d_tq), k1));
    CKS(jacobi_any(ctx, s.d_tt, ldv, dptr(k1), dptr(kq), nvmax, nvmax, s.d_jv, ldv, s.d_norm));
    GemmArgs g = gemm0();  // J_M[c][a] = sum_k J[c][k] Q1[a][k]
    g.A = s.d_jv;
    g.B = s.d_qt;
    g.C = s.d_jh;
    g.M = dptr(k1);
    g.N = nv;
    g.K = dptr(k1);
    g.sai = dconst(ldv);
    g.sak = dconst(1);
    g.sbk = dconst(1);
    g.sbj = dconst(ldv);
    g.sci = dconst(ldv);
    g.scj = dconst(1);
    KL(KC_REFINE, gemm_d(ctx, g, nvmax, nvmax, 1, 1, ctx->stream));
    CKS(ns_rows(ctx, s.d_jh, ldv, dptr(k1), nv, nvmax, nvmax));
    KL(KC_POST, svd_post(ctx, s.d_norm, dptr(k1), dptr(kq), nv, s.d_jh, ldv, eps, chi, rank_cap, rank_out, sig,
                         disc_out, Jp, Jt, nsv_out));
    return QTT_OK;
  }
  if (ellmax >= nvmax) {
    Dim len = ell;
    if (ellmax > nvmax) {
      // M (ell x nv, column i = vector i) = Q R;  R column-major with ld ldv
      KL(KC_QR, qr_any(ctx, Tv, ell, s.d_tq, ellmax, ell, nv, nvmax, s.d_rv, false, nullptr, kq, ldv, 0));
      CKS(jacobi_any(ctx, s.d_rv, ldv, nv, dptr(kq), nvmax, nvmax, s.d_jv, ldv, s.d_norm));
      len = dptr(kq);
    } else {
      KL(KC_COPY, copy2d(Tv, s.d_tq, nv, ell, ell, dconst(1), dconst(ellmax), dconst(1), nvmax * ellmax, 1.0,
                         ctx->stream));
      CKS(jacobi_any(ctx, s.d_tq, ellmax, nv, ell, nvmax, ellmax, s.d_jv, ldv, s.d_norm));
    }
    KL(KC_POST, svd_post(ctx, s.d_norm, nv, len, nv, s.d_jv, ldv, eps, chi, rank_cap, rank_out, sig, disc_out, Jp, Jt,
                         nsv_out));
    return QTT_OK;
  }
  if (ellmax > ldv) return fail(QTT_EINVAL, "internal: SVD larger than the workspace");
  // M^T (nv x ell): its columns are the ell components, stored contiguously
  KL(KC_COPY, copy2d(Tv, s.d_tt, nv, ell, ell, dconst(1), dconst(1), dconst(nvmax), nvmax * ellmax, 1.0, ctx->stream));
  KL(KC_QR, qr_any(ctx, s.d_tt, dconst(nvmax), s.d_tq, nvmax, nv, ell, ellmax, s.d_rv, true, s.d_qt, kq, ellmax,
                   nvmax));
  // rows of R (kq x ell, ld ellmax) are the vectors of the reduced problem
  CKS(jacobi_any(ctx, s.d_rv, ellmax, dptr(kq), ell, ellmax, ellmax, s.d_jh, ldv, s.d_norm));
  // J_v[c][i] = sum_j J_R[c][j] Q[i][j]
  GemmArgs g = gemm0();
  g.A = s.d_jh;
  g.B = s.d_qt;
  g.C = s.d_jv;
  g.M = dptr(kq);
  g.N = nv;
  g.K = dptr(kq);
  g.sai = dconst(ldv);
  g.sak = dconst(1);
  g.sbk = dconst(1);
  g.sbj = dptr(kq);
  g.sci = dconst(ldv);
  g.scj = dconst(1);
  KL(KC_GEMM, gemm_any(ctx, g, ellmax, nvmax, 1, 1));
  KL(KC_POST, svd_post(ctx, s.d_norm, dptr(kq), ell, nv, s.d_jv, ldv, eps, chi, rank_cap, rank_out, sig, disc_out, Jp, Jt,
                       nsv_out));
  return QTT_OK;
}

GemmArgs gemm0() {
  GemmArgs g;
  std::memset(&g, 0, sizeof(g));
  g.nb1 = dconst(1);
  g.nb2 = dconst(1);
  g.sa1 = g.sa2 = g.sb1 = g.sb2 = g.sc1 = g.sc2 = dconst(0);
  g.alpha = 1.0;
  g.beta = 0.0;
  return g;
}

// ---------------------------------------------------------------- zip-ups
// phi = L psi, sweeping sites 0 -> d-1 (with the carry of Eq. 9-12).
qtt_status zipup_L(qtt_ctx* ctx, const Mpo* L, const Mps* psi, Mps* phi, const Caps& c) {
  Workspace& s = ctx->ws;
  const int d = ctx->d;
  const double eps = ctx->p.eps_zip;
  const int chi = ctx->p.chi_zip;
  KL(KC_OTHER, init_zip(s.d_carry, phi->ranks, d, nullptr, nullptr, 0, ctx->stream));
  for (int k = 0; k < d; ++k) {
    const int w = L->w[k], w2 = L->w[k + 1];
    const int* a_p = phi->ranks + k;
    const int* b_p = psi->ranks + k;
    const int* b2_p = psi->ranks + k + 1;
    // X[(a,w)][(s,b')] = C[(a,w)][b] A_k[b][(s,b')]
    GemmArgs g = gemm0();
    g.A = s.d_carry;
    g.B = psi->core(k);
    g.C = s.d_x;
    g.M = dptr(a_p, w);
    g.N = dptr(b2_p, 2);
    g.K = dptr(b_p);
    g.sai = dptr(b_p);
    g.sak = dconst(1);
    g.sbk = dptr(b2_p, 2);
    g.sbj = dconst(1);
    g.sci = dptr(b2_p, 2);
    g.scj = dconst(1);
    KL(KC_GEMM, gemm_any(ctx, g, (long long)c.phi[k] * w, 2LL * c.psi[k + 1], 1, 1));
    const double* Wk = L->data + L->off[k];
    const long long tot = 2LL * c.phi[k] * w2 * c.psi[k + 1];
    if (k == d - 1) {  // w' = b' = 1: T is the last core
      KL(KC_MPO, mpo_apply_lr(s.d_x, phi->core(k), Wk, w, w2, a_p, b2_p, tot, ctx->stream));
      break;
    }
    KL(KC_MPO, mpo_apply_lr(s.d_x, s.d_tv, Wk, w, w2, a_p, b2_p, tot, ctx->stream));
    int* r_p = phi->ranks + k + 1;
    const Dim nv = dptr(a_p, 2), ell = dptr(b2_p, w2);
    CKS(svd_vm(ctx, s.d_tv, nv, ell, 2LL * c.phi[k], (long long)w2 * c.psi[k + 1], eps, chi, c.phi[k + 1], r_p,
               s.d_jp, phi->core(k), s.d_disc + 0 * (d + 1) + k + 1, nullptr));
    // carry C'[j][(w',b')] = sum_i Jp[j][i] T[i][(w',b')]
    GemmArgs h = gemm0();
    h.A = s.d_jp;
    h.B = s.d_tv;
    h.C = s.d_carry;
    h.M = dptr(r_p);
    h.N = ell;
    h.K = nv;
    h.sai = nv;
    h.sak = dconst(1);
    h.sbk = ell;
    h.sbj = dconst(1);
    h.sci = ell;
    h.scj = dconst(1);
    KL(KC_GEMM, gemm_any(ctx, h, c.phi[k + 1], (long long)w2 * c.psi[k + 1], 1, 1));
  }
  return QTT_OK;
}

// eta = C^2 phi, the diagonal MPO of the c^2 MPS, sweeping sites d-1 -> 0.
qtt_status zipup_C(qtt_ctx* ctx, const Mps* c2, const std::vector<int>& rc, const Mps* phi, Mps* eta,
                   const Caps& c) {
  Workspace& s = ctx->ws;
  const int d = ctx->d;
  const double eps = ctx->p.eps_zip;
  const int chi = ctx->p.chi_zip;
  KL(KC_OTHER, init_zip(s.d_carry, eta->ranks, d, nullptr, nullptr, 0, ctx->stream));
  for (int k = d - 1; k >= 0; --k) {
    const int R = rc[k], R2 = rc[k + 1];
    const int* B_p = phi->ranks + k;
    const int* B2_p = phi->ranks + k + 1;
    const int* A2_p = eta->ranks + k + 1;
    // Z[t][b][(r',a')] = sum_b' phi_k[b][t][b'] C[b'][(r',a')]
    GemmArgs g = gemm0();
    g.A = phi->core(k);
    g.B = s.d_carry;
    g.C = s.d_x;
    g.M = dptr(B_p);
    g.N = dptr(A2_p, R2);
    g.K = dptr(B2_p);
    g.sai = dptr(B2_p, 2);
    g.sak = dconst(1);
    g.sbk = dptr(A2_p, R2);
    g.sbj = dconst(1);
    g.sci = dptr(A2_p, R2);
    g.scj = dconst(1);
    g.nb1 = dconst(2);
    g.sa1 = dptr(B2_p);
    g.sb1 = dconst(0);
    g.sc1 = dptr2(B_p, A2_p, R2);
    KL(KC_GEMM, gemm_any(ctx, g, c.phi[k], (long long)R2 * c.eta[k + 1], 2, 1));
    // T[(t,a')][(b,r)] = sum_r' B_k[r][t][r'] Z[t][b][r'][a']
    double* Tdst = (k == 0) ? eta->core(0) : s.d_tv;
    GemmArgs h = gemm0();
    h.A = c2->core(k);
    h.B = s.d_x;
    h.C = Tdst;
    h.M = dconst(R);
    h.N = dptr(A2_p);
    h.K = dconst(R2);
    h.sai = dconst(2LL * R2);
    h.sak = dconst(1);
    h.sbk = dptr(A2_p);
    h.sbj = dconst(1);
    h.sci = dconst(1);
    h.scj = dptr(B_p, R);
    h.nb1 = dconst(2);
    h.nb2 = dptr(B_p);
    h.sa1 = dconst(R2);
    h.sa2 = dconst(0);
    h.sb1 = dptr2(B_p, A2_p, R2);
    h.sb2 = dptr(A2_p, R2);
    h.sc1 = dptr2(A2_p, B_p, R);
    h.sc2 = dconst(R);
    KL(KC_GEMM, gemm_any(ctx, h, R, c.eta[k + 1], 2, c.phi[k]));
    if (k == 0) break;
    int* r_p = eta->ranks + k;
    const Dim nv = dptr(A2_p, 2), ell = dptr(B_p, R);
    CKS(svd_vm(ctx, s.d_tv, nv, ell, 2LL * c.eta[k + 1], (long long)c.phi[k] * R, eps, chi, c.eta[k], r_p,
               eta->core(k), nullptr, s.d_disc + 1 * (d + 1) + k, nullptr));
    // carry C'[(b,r)][j] = sum_i T[i][(b,r)] Jp[j][i]  (Jp = eta core k)
    GemmArgs q = gemm0();
    q.A = s.d_tv;
    q.B = eta->core(k);
    q.C = s.d_carry;
    q.M = ell;
    q.N = dptr(r_p);
    q.K = nv;
    q.sai = dconst(1);
    q.sak = ell;
    q.sbk = dconst(1);
    q.sbj = nv;
    q.sci = dptr(r_p);
    q.scj = dconst(1);
    KL(KC_GEMM, gemm_any(ctx, q, (long long)c.phi[k] * R, c.eta[k], 1, 1));
  }
  return QTT_OK;
}

// -------------------------------------------------------------------- sum
qtt_status form_sum(qtt_ctx* ctx, const std::vector<std::pair<double, const Mps*>>& terms, const long* src,
                    double amp, Mps* out, const double* amp_scale = nullptr) {
  const int d = ctx->d;
  SumArgs a;
  std::memset(&a, 0, sizeof(a));
  a.d = d;
  a.nterms = (int)terms.size();
  for (int t = 0; t < a.nterms; ++t) {
    a.coef[t] = terms[t].first;
    a.ranks[t] = terms[t].second->ranks;
    for (int k = 0; k < d; ++k) a.core[t][k] = terms[t].second->core(k);
  }
  for (int k = 0; k < d; ++k) a.out[k] = out->core(k);
  a.out_ranks = out->ranks;
  a.has_src = src ? 1 : 0;
  a.src_amp = amp;
  a.src_amp_dev = ctx->capturing ? ctx->d_amp : nullptr;
  a.amp_scale = amp_scale;
  if (src) {  // the point's linear dense index, then the bit each site carries
    long long lin = 0;
    for (int a_ = 0; a_ < ctx->dims; ++a_) lin = (lin << ctx->p.n) | src[a_];
    for (int k = 0; k < d; ++k) a.src_bits[k] = (int)((lin >> ctx->site_pos[k]) & 1);
  }
  long long mx = 1;
  for (int k = 0; k < d; ++k) mx = std::max(mx, (long long)out->cap[k] * 2 * out->cap[k + 1]);
  KL(KC_SUM, mps_sum(a, mx, ctx->stream));
  return QTT_OK;
}

// ------------------------------------------------------------------ round
// Range finder for bond k of the round's SVD sweep (the learned form).  The
// matrix X (l x m, l = q_k, m = 2 r_{k+1}) is held as m vectors of length l
// in Tv.  With Omega = the top-left l x ks block of the sketch matrix:
//   Y = X^T Omega (ks vectors of length m), Y = Q R (thin Q, m x ks),
//   B = Q^T X^T (ks vectors of length l), rho^2 = ||X^T - Q B||_F^2 (FP64),
//   SVD of B by the rounding rule: B^T J = U S with J = the left singular
//   vectors of B; the new core k is (Q J_r)^T.
// Writes the accept flag to d_rff[0] (1 accept, 0 reject, 2 not attempted);
// the core and rank are only meaningful when accepted.
qtt_status rf_bond(qtt_ctx* ctx, const Mps* th, Mps* out, int k, int ks, long long nvmax, long long ellmax) {
  Workspace& s = ctx->ws;
  const int d = ctx->d;
  const int* q_p = th->ranks + k;
  const int* r2_p = out->ranks + k + 1;
  int* r_p = out->ranks + k;
  const Dim nv = dptr(r2_p, 2), ell = dptr(q_p);
  const long long ld_om = ctx->sketch_cols;
  // Y[j][c] = sum_l Omega[l][j] Tv[c][l]
  GemmArgs g = gemm0();
  g.A = ctx->sketch;
  g.B = s.d_tv;
  g.C = s.d_rfy;
  g.M = dconst(ks);
  g.N = nv;
  g.K = ell;
  g.sai = dconst(1);
  g.sak = dconst(ld_om);
  g.sbk = dconst(1);
  g.sbj = ell;
  g.sci = nv;
  g.scj = dconst(1);
  KL(KC_GEMM, gemm_any(ctx, g, ks, nvmax, 1, 1));
  // thin Q of Y (m x ks, row-major); R is not needed
  KL(KC_QR, qr_any(ctx, s.d_rfy, nv, s.d_tq, nvmax, nv, dconst(ks), ks, s.d_rv, false, s.d_rfq, s.d_rff + 1, ks,
                   nvmax));
  // B[j][l] = sum_c Q[c][j] Tv[c][l]
  GemmArgs b = gemm0();
  b.A = s.d_rfq;
  b.B = s.d_tv;
  b.C = s.d_rfb;
  b.M = dconst(ks);
  b.N = ell;
  b.K = nv;
  b.sai = dconst(1);
  b.sak = dconst(ks);
  b.sbk = ell;
  b.sbj = dconst(1);
  b.sci = ell;
  b.scj = dconst(1);
  KL(KC_GEMM, gemm_any(ctx, b, ks, ellmax, 1, 1));
  // E = Tv - Q B in FP64, rho^2 = |E|^2, |X|^2
  KL(KC_COPY, copy2d(s.d_tv, s.d_rfe, nv, ell, ell, dconst(1), ell, dconst(1), nvmax * ellmax, 1.0, ctx->stream));
  GemmArgs e = gemm0();
  e.A = s.d_rfq;
  e.B = s.d_rfb;
  e.C = s.d_rfe;
  e.M = nv;
  e.N = ell;
  e.K = dconst(ks);
  e.sai = dconst(ks);
  e.sak = dconst(1);
  e.sbk = ell;
  e.sbj = dconst(1);
  e.sci = ell;
  e.scj = dconst(1);
  e.alpha = -1.0;
  e.beta = 1.0;
  KL(KC_GEMM, gemm_f64(e, nvmax, ellmax, 1, 1, ctx->stream));
  KL(KC_OTHER, sumsq(s.d_rfe, ell, nv, ell, s.d_rfs + 0, ctx->stream));
  KL(KC_OTHER, sumsq(s.d_tv, ell, nv, ell, s.d_rfs + 1, ctx->stream));
  // SVD of B (ks vectors of length l) by the rounding rule
  double* sig = s.d_spec + (long long)k * ctx->ws_nvmax;
  CKS(svd_vm(ctx, s.d_rfb, dconst(ks), ell, ks, ellmax, ctx->p.eps, ctx->p.chi_max, out->cap[k], r_p, s.d_rfjp,
             nullptr, nullptr, sig, s.d_spec_len + k));
  KL(KC_OTHER, rf_accept(sig, s.d_spec_len + k, r_p, ks, r2_p, q_p, 2, ctx->p.eps, ctx->p.chi_max, ctx->tau,
                         s.d_rfs + 0, s.d_rfs + 1, s.d_rff, s.d_disc + 2 * (d + 1) + k, ctx->stream));
  // core k (r x m) = J_r^T Q^T: core[i][c] = sum_j Jp[i][j] Q[c][j]
  GemmArgs c = gemm0();
  c.A = s.d_rfjp;
  c.B = s.d_rfq;
  c.C = out->core(k);
  c.M = dptr(r_p);
  c.N = nv;
  c.K = dconst(ks);
  c.sai = dconst(ks);
  c.sak = dconst(1);
  c.sbk = dconst(1);
  c.sbj = dconst(ks);
  c.sci = nv;
  c.scj = dconst(1);
  KL(KC_GEMM, gemm_any(ctx, c, std::min<long long>(out->cap[k], ks), nvmax, 1, 1));
  return QTT_OK;
}

// out = round(theta): QR sweep 0 -> d-1, then truncated-SVD sweep d-1 -> 1
// (Sec. 4.3).  theta is overwritten.  Every bond's singular values go to the
// spectrum log.  In the learned form, a bond with a proposed rank first tries
// the range finder (rf_bond) and keeps its result when the exact check
// accepts it; otherwise it takes the full SVD.
qtt_status tt_round(qtt_ctx* ctx, Mps* th, Mps* out) {
  Workspace& s = ctx->ws;
  const int d = ctx->d;
  const std::vector<int>& cap = th->cap;
  int* Dsave = s.d_ints + 8;  // original theta ranks, d+1 ints
  KL(KC_OTHER, init_zip(nullptr, out->ranks, d, th->ranks, Dsave, d + 1, ctx->stream));
  // theta_0 (1 x 2 x D_1) -> vector-major columns: M[y][s]
  KL(KC_COPY, copy2d(th->core(0), s.d_tv, dconst(2), dptr(Dsave + 1), dptr(Dsave + 1), dconst(1), dconst(1), dconst(2),
            2LL * cap[1], 1.0, ctx->stream));
  for (int k = 0; k < d - 1; ++k) {
    int* q_p = th->ranks + k;       // q_k (rows / 2 of the matrix)
    int* kq_p = th->ranks + k + 1;  // becomes min(2 q_k, D_{k+1})
    const Dim m = dptr(q_p, 2), n = dptr(Dsave + k + 1);
    const long long ldw = 2LL * cap[k];
    KL(KC_QR, qr_any(ctx, s.d_tv, m, s.d_tq, ldw, m, n, cap[k + 1], s.d_rv, true, th->core(k), kq_p, cap[k + 1], ldw));
    // next core (kq x 2 x D_{k+2}) = R (kq x D_{k+1}) theta_{k+1}
    GemmArgs g = gemm0();
    g.A = s.d_rv;
    g.B = th->core(k + 1);
    g.C = s.d_tv;
    g.M = dptr(kq_p);
    g.N = dptr(Dsave + k + 2);
    g.K = dptr(Dsave + k + 1);
    g.sai = dconst(cap[k + 1]);
    g.sak = dconst(1);
    g.sbk = dptr(Dsave + k + 2, 2);
    g.sbj = dconst(1);
    g.nb1 = dconst(2);
    g.sa1 = dconst(0);
    g.sb1 = dptr(Dsave + k + 2);
    if (k + 1 < d - 1) {  // QR layout: column y holds (x', s)
      g.sci = dconst(2);
      g.scj = dptr(kq_p, 2);
      g.sc1 = dconst(1);
    } else {  // SVD layout of the last core: vector s holds x'
      g.sci = dconst(1);
      g.scj = dptr(kq_p);
      g.sc1 = dptr(kq_p);
    }
    KL(KC_GEMM, gemm_any(ctx, g, std::min<long long>(2LL * cap[k], cap[k + 1]), cap[k + 2], 2, 1));
  }
  const bool learned = ctx->p.use_learned_rank && ctx->sketch && ctx->have_prop && s.d_rfy;
  std::vector<int> prop;
  if (learned) {
    prop.resize(d + 1);
    CK(cudaMemcpyAsync(prop.data(), s.d_prop, (d + 1) * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  for (int k = d - 1; k >= 1; --k) {
    const int* q_p = th->ranks + k;  // rows of core k
    const int* r2_p = out->ranks + k + 1;
    int* r_p = out->ranks + k;
    const Dim nv = dptr(r2_p, 2), ell = dptr(q_p);
    const long long nvmax = 2LL * out->cap[k + 1];
    const long long ellmax = std::min<long long>(cap[k], p2(k));  // q_k <= 2^k after the QR sweep
    bool done = false;
    if (learned && prop[k] > 0) {
      const int ks = prop[k] + ctx->oversample;
      if (ks < std::min(nvmax, ellmax) && ks <= ctx->sketch_cols && ellmax <= ctx->sketch_rows) {
        CKS(rf_bond(ctx, th, out, k, ks, nvmax, ellmax));
        int flag = 0;
        CK(cudaMemcpyAsync(&flag, s.d_rff, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        if (flag != 2) ++ctx->rf_attempts;
        if (flag == 1) {
          ++ctx->rf_accepts;
          done = true;
        }
      }
    }
    if (!done)
      CKS(svd_vm(ctx, s.d_tv, nv, ell, nvmax, ellmax, ctx->p.eps, ctx->p.chi_max, out->cap[k], r_p, out->core(k),
                 nullptr, s.d_disc + 2 * (d + 1) + k, s.d_spec + (long long)k * ctx->ws_nvmax, s.d_spec_len + k));
    // W1 (r x q_k) = Jp Tv
    GemmArgs g = gemm0();
    g.A = out->core(k);
    g.B = s.d_tv;
    g.C = s.d_w1;
    g.M = dptr(r_p);
    g.N = ell;
    g.K = nv;
    g.sai = nv;
    g.sak = dconst(1);
    g.sbk = ell;
    g.sbj = dconst(1);
    g.sci = ell;
    g.scj = dconst(1);
    KL(KC_GEMM, gemm_any(ctx, g, out->cap[k], cap[k], 1, 1));
    // core_{k-1} (q_{k-1} x 2 x r) = Q_{k-1} (q_{k-1} x 2 x q_k) W1^T
    const int* ql_p = th->ranks + k - 1;
    GemmArgs h = gemm0();
    h.A = th->core(k - 1);
    h.B = s.d_w1;
    h.M = dptr(ql_p);
    h.N = dptr(r_p);
    h.K = dptr(q_p);
    h.sai = dptr(q_p, 2);
    h.sak = dconst(1);
    h.sbk = dconst(1);
    h.sbj = dptr(q_p);
    h.nb1 = dconst(2);
    h.sa1 = dptr(q_p);
    h.sb1 = dconst(0);
    if (k - 1 >= 1) {  // SVD layout for the next bond: vector (s', j) holds w
      h.C = s.d_tv;
      h.sci = dconst(1);
      h.scj = dptr(ql_p);
      h.sc1 = dptr2(r_p, ql_p);
    } else {  // final core 0: [1][2][r]
      h.C = out->core(0);
      h.sci = dconst(0);
      h.scj = dconst(1);
      h.sc1 = dptr(r_p);
    }
    KL(KC_GEMM, gemm_any(ctx, h, cap[k - 1], out->cap[k], 2, 1));
  }
  return QTT_OK;
}

// ------------------------------------------------------------------ TT-SVD
// MPS of a dense grid (site tensor built on the device), truncated (eps, chi).
qtt_status tt_svd(qtt_ctx* ctx, const double* grid_dev, bool square, double eps, int chi, Mps* out) {
  Workspace& s = ctx->ws;
  const int d = ctx->d, n = ctx->p.n;
  double* cur = s.d_carry;
  double* nxt = s.d_x;
  (void)n;
  KL(KC_OTHER, site_permute(grid_dev, cur, site_positions(ctx), square, ctx->stream));
  KL(KC_OTHER, init_zip(nullptr, out->ranks, d, nullptr, nullptr, 0, ctx->stream));
  for (int k = 0; k < d - 1; ++k) {
    const long long ell = p2(d - k - 1);
    const int* rl_p = out->ranks + k;
    int* r_p = out->ranks + k + 1;
    // rank of bond k is at most min(2^k, 2^(d-k), chi) whatever the buffer holds
    const long long capk = std::min<long long>({(long long)out->cap[k], p2(k), p2(d - k), (long long)chi});
    const long long capk1 = std::min<long long>({(long long)out->cap[k + 1], p2(k + 1), p2(d - k - 1), (long long)chi});
    const long long nvmax = 2 * capk;
    CKS(svd_vm(ctx, cur, dptr(rl_p, 2), dconst(ell), nvmax, ell, eps, chi, (int)capk1, r_p, s.d_jp, out->core(k),
               nullptr, nullptr));
    GemmArgs g = gemm0();
    g.A = s.d_jp;
    g.B = cur;
    g.C = nxt;
    g.M = dptr(r_p);
    g.N = dconst(ell);
    g.K = dptr(rl_p, 2);
    g.sai = dptr(rl_p, 2);
    g.sak = dconst(1);
    g.sbk = dconst(ell);
    g.sbj = dconst(1);
    g.sci = dconst(ell);
    g.scj = dconst(1);
    KL(KC_GEMM, gemm_any(ctx, g, capk1, ell, 1, 1));
    std::swap(cur, nxt);
  }
  // last core (r_{d-1} x 2 x 1) is the remainder
  KL(KC_COPY, copy2d(cur, out->core(d - 1), dptr(out->ranks + d - 1, 2), dconst(1), dconst(1), dconst(1), dconst(1), dconst(1),
            2LL * out->cap[d - 1], 1.0, ctx->stream));
  return QTT_OK;
}

}  // namespace

struct qtt_mlp {
  qtt::MlpDev dev;
  cudaStream_t stream = nullptr;
  int t = 0;  // Adam steps taken
};

namespace {

// Features of bonds 1..d-1 from the last round's spectra and the ranks of
// psi (its result), the network's outputs, and the proposals for the next
// step's round.
qtt_status propose_ranks(qtt_ctx* ctx, const Mps* psi) {
  Workspace& s = ctx->ws;
  const int nb = ctx->d - 1;
  if (nb < 1) return QTT_OK;
  KL(KC_OTHER, rank_features(s.d_spec, ctx->ws_nvmax, s.d_spec_len, psi->ranks, nb, ctx->p.eps, ctx->p.chi_max,
                             ctx->d, s.d_feat, ctx->stream));
  KL(KC_OTHER, mlp_forward(ctx->mlp->dev, s.d_feat, nb, s.d_y, ctx->stream));
  KL(KC_OTHER, propose(s.d_y, nb, ctx->p.chi_max, s.d_prop, ctx->stream));
  ctx->have_prop = true;
  return QTT_OK;
}

bool cuda_ok_device() {
  int n = 0;
  return cudaGetDeviceCount(&n) == cudaSuccess && n > 0;
}

}  // namespace

// =================================================================== ABI
extern "C" {

const char* qtt_last_error(void) { return g_err.c_str(); }

qtt_status qtt_ctx_create(const qtt_params* p, void* stream, qtt_ctx** out) {
  if (!p || !out) return fail(QTT_EINVAL, "null argument");
  *out = nullptr;
  if (p->dims != 0 && p->dims != 2 && p->dims != 3) return fail(QTT_EINVAL, "dims must be 2 or 3 (0 = 2)");
  if (p->n < 1 || p->n > 14) return fail(QTT_EINVAL, "n must be in 1..14");
  if (p->dims == 3 && p->n > 9) return fail(QTT_EINVAL, "n must be in 1..9 in 3D (3n <= 27 sites)");
  if (p->order != QTT_ORDER_SEQUENTIAL && p->order != QTT_ORDER_INTERLEAVED) return fail(QTT_EINVAL, "bad order");
  if (p->bc != QTT_BC_PERIODIC && p->bc != QTT_BC_ZERO) return fail(QTT_EINVAL, "bad boundary condition");
  if (p->prec != QTT_FP64 && p->prec != QTT_FP32 && p->prec != QTT_TF32 && p->prec != QTT_TF32X3 &&
      p->prec != QTT_BF16)
    return fail(QTT_EINVAL, "prec must be one of QTT_FP64, QTT_FP32, QTT_TF32, QTT_TF32X3, QTT_BF16");
  if (p->chi_max < 1 || p->chi_max > 1024) return fail(QTT_EINVAL, "chi_max must be in 1..1024");
  if (!(p->eps >= 0.0 && p->eps < 1.0)) return fail(QTT_EINVAL, "eps must be in [0, 1)");
  if (p->chi_zip < 0 || p->chi_zip > 1024 || p->chi_c < 0 || p->chi_c > 1024)
    return fail(QTT_EINVAL, "chi_zip / chi_c must be in 0..1024");
  if (p->use_learned_rank != 0 && p->use_learned_rank != 1) return fail(QTT_EINVAL, "use_learned_rank must be 0 or 1");
  if (!cuda_ok_device()) return fail(QTT_ECUDA, "no CUDA device");
  qtt_ctx* c = new qtt_ctx();
  c->p = *p;
  if (c->p.chi_zip == 0) c->p.chi_zip = c->p.chi_max;
  if (!(c->p.eps_zip > 0.0)) c->p.eps_zip = c->p.eps;
  if (c->p.chi_c == 0) c->p.chi_c = c->p.chi_max;
  if (!(c->p.eps_c > 0.0)) c->p.eps_c = 1e-8;
  c->dims = p->dims == 3 ? 3 : 2;
  c->p.dims = c->dims;
  c->d = c->dims * p->n;
  for (int k = 0; k < c->d; ++k) c->site_pos[k] = site_pos(k, p->n, p->order, c->dims);
  c->stream = (cudaStream_t)stream;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e == cudaSuccess) e = linalg_init(c->device);
  if (e == cudaSuccess) e = mixed_init();
  if (e == cudaSuccess) e = tc_init();
  c->ckind = p->prec == QTT_TF32 ? 0 : p->prec == QTT_TF32X3 ? 1 : p->prec == QTT_BF16 ? 2 : -1;
  if (e != cudaSuccess) {
    delete c;
    return fail(QTT_ECUDA, std::string("device query: ") + cudaGetErrorString(e));
  }
  c->coop_blocks = coop_max_blocks(c->num_sms);
  *out = c;
  return QTT_OK;
}

void qtt_ctx_destroy(qtt_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  ws_free(ctx);
  for (auto& e : ctx->prof.ev) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  if (ctx->prof.d_log) cudaFree(ctx->prof.d_log);
  if (ctx->prof.d_flops) cudaFree(ctx->prof.d_flops);
  if (ctx->d_amp) cudaFree(ctx->d_amp);
  if (ctx->gstream) cudaStreamDestroy(ctx->gstream);
  delete ctx;
}

qtt_status qtt_set_limits(qtt_ctx* ctx, double wait_limit_s, int max_sweeps) {
  if (!ctx) return fail(QTT_EINVAL, "null context");
  if (!(wait_limit_s <= 3600.0)) return fail(QTT_EINVAL, "wait_limit_s must be <= 3600 (<= 0: the default)");
  if (max_sweeps > 100000) return fail(QTT_EINVAL, "max_sweeps must be <= 100000 (<= 0: the default)");
  ctx->wait_limit_ns = wait_limit_s > 0.0 ? std::max(1ULL, (unsigned long long)(wait_limit_s * 1e9)) : 0ULL;
  ctx->max_sweeps = max_sweeps > 0 ? max_sweeps : 100;
  for (auto& g : ctx->gexec)  // the sweep limit is a launch argument of the captured kernels
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  if (ctx->ws_ready) {
    CK(cudaMemcpyAsync(&ctx->ws.d_sync->limit_ns, &ctx->wait_limit_ns, sizeof(unsigned long long),
                       cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  return QTT_OK;
}

qtt_status qtt_ctx_sync(qtt_ctx* ctx) {
  if (!ctx) return fail(QTT_EINVAL, "null context");
  CK(cudaStreamSynchronize(ctx->stream));
  if (!ctx->ws_ready) return QTT_OK;
  return device_status(ctx);
}

qtt_status qtt_mps_create_zero(qtt_ctx* ctx, qtt_mps** out) {
  if (!ctx || !out) return fail(QTT_EINVAL, "null argument");
  qtt_mps* m = new qtt_mps();
  qtt_status s = mps_alloc(ctx, psi_caps(ctx->d, ctx->p.chi_max), m);
  if (s != QTT_OK) {
    mps_free(m);
    delete m;
    return s;
  }
  *out = m;
  return QTT_OK;
}

void qtt_mps_destroy(qtt_mps* m) {
  if (!m) return;
  if (m->ctx) cudaStreamSynchronize(m->ctx->stream);
  mps_free(m);
  delete m;
}

qtt_status qtt_mps_from_cores(qtt_ctx* ctx, const int* ranks, const double* cores, qtt_mps** out) {
  if (!ctx || !ranks || !cores || !out) return fail(QTT_EINVAL, "null argument");
  const int d = ctx->d;
  std::vector<int> cap = psi_caps(d, ctx->p.chi_max);
  if (ranks[0] != 1 || ranks[d] != 1) return fail(QTT_EINVAL, "ranks[0] and ranks[d] must be 1");
  for (int k = 0; k <= d; ++k)
    if (ranks[k] < 1 || ranks[k] > cap[k]) return fail(QTT_EINVAL, "rank outside 1..capacity");
  qtt_mps* m = nullptr;
  CKS(qtt_mps_create_zero(ctx, &m));
  long long src = 0;
  for (int k = 0; k < d; ++k) {
    long long sz = (long long)ranks[k] * 2 * ranks[k + 1];
    cudaError_t e = cudaMemcpyAsync(m->core(k), cores + src, sz * sizeof(double), cudaMemcpyHostToDevice,
                                    ctx->stream);
    if (e != cudaSuccess) {
      qtt_mps_destroy(m);
      return fail(QTT_ECUDA, cudaGetErrorString(e));
    }
    src += sz;
  }
  CK(cudaMemcpyAsync(m->ranks, ranks, (d + 1) * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  *out = m;
  return QTT_OK;
}

qtt_status qtt_mps_ranks(qtt_ctx* ctx, const qtt_mps* psi, int* ranks_out) {
  if (!ctx || !psi || !ranks_out) return fail(QTT_EINVAL, "null argument");
  CK(cudaMemcpyAsync(ranks_out, psi->ranks, (psi->d + 1) * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (ctx->ws_ready) CKS(device_status(ctx));
  return QTT_OK;
}

qtt_status qtt_mps_get_cores(qtt_ctx* ctx, const qtt_mps* psi, int* ranks, double* cores, long cap) {
  CKS(qtt_mps_ranks(ctx, psi, ranks));
  if (!cores) return QTT_OK;
  long long need = 0;
  for (int k = 0; k < psi->d; ++k) need += (long long)ranks[k] * 2 * ranks[k + 1];
  if (need > cap) return fail(QTT_EINVAL, "cores buffer too small");
  long long dst = 0;
  for (int k = 0; k < psi->d; ++k) {
    long long sz = (long long)ranks[k] * 2 * ranks[k + 1];
    CK(cudaMemcpyAsync(cores + dst, psi->core(k), sz * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    dst += sz;
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return QTT_OK;
}

// File layout: 8 bytes "QTTMPS1\0", int32 d, int32 ranks[d+1], then the
// cores k = 0..d-1 ([r_k][2][r_{k+1}], FP64), all little-endian.
qtt_status qtt_mps_save(qtt_ctx* ctx, const qtt_mps* psi, const char* path) {
  if (!ctx || !psi || !path) return fail(QTT_EINVAL, "null argument");
  const int d = psi->d;
  std::vector<int> r(d + 1);
  CKS(qtt_mps_ranks(ctx, psi, r.data()));
  long long need = 0;
  for (int k = 0; k < d; ++k) need += (long long)r[k] * 2 * r[k + 1];
  std::vector<double> cores(std::max(need, 1LL));
  CKS(qtt_mps_get_cores(ctx, psi, r.data(), cores.data(), (long)need));
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(QTT_EINVAL, std::string("cannot open ") + path + " for writing");
  const char magic[8] = {'Q', 'T', 'T', 'M', 'P', 'S', '1', '\0'};
  const int32_t d32 = d;
  bool ok = std::fwrite(magic, 1, 8, f) == 8 && std::fwrite(&d32, 4, 1, f) == 1;
  for (int k = 0; ok && k <= d; ++k) {
    const int32_t v = r[k];
    ok = std::fwrite(&v, 4, 1, f) == 1;
  }
  if (ok && need > 0) ok = std::fwrite(cores.data(), sizeof(double), need, f) == (size_t)need;
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) return fail(QTT_EINVAL, std::string("write failed: ") + path);
  return QTT_OK;
}

qtt_status qtt_mps_load(qtt_ctx* ctx, const char* path, qtt_mps** out) {
  if (!ctx || !path || !out) return fail(QTT_EINVAL, "null argument");
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(QTT_EINVAL, std::string("cannot open ") + path);
  char magic[8];
  int32_t d32 = 0;
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "QTTMPS1\0", 8) == 0 &&
            std::fread(&d32, 4, 1, f) == 1 && d32 == ctx->d;
  std::vector<int> r(ctx->d + 1);
  for (int k = 0; ok && k <= ctx->d; ++k) {
    int32_t v = 0;
    ok = std::fread(&v, 4, 1, f) == 1 && v >= 1 && v <= (1 << 20);
    r[k] = v;
  }
  long long need = 0;
  for (int k = 0; ok && k < ctx->d; ++k) need += (long long)r[k] * 2 * r[k + 1];
  std::vector<double> cores(std::max(need, 1LL));
  if (ok && need > 0) ok = std::fread(cores.data(), sizeof(double), need, f) == (size_t)need;
  std::fclose(f);
  if (!ok) return fail(QTT_EINVAL, std::string("not an MPS file of this grid size: ") + path);
  return qtt_mps_from_cores(ctx, r.data(), cores.data(), out);
}

static qtt_status from_dense_impl(qtt_ctx* ctx, const double* grid, int on_device, bool square, double eps, int chi,
                                  qtt_mps** out) {
  if (!ctx || !grid || !out) return fail(QTT_EINVAL, "null argument");
  CKS(ensure_ws_basic(ctx));
  const long long N2 = p2(ctx->d);
  const double* g = grid;
  double* tmp = nullptr;
  if (!on_device) {
    CK(cudaMalloc(&tmp, N2 * sizeof(double)));
    CK(cudaMemcpyAsync(tmp, grid, N2 * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    g = tmp;
  }
  qtt_mps* m = new qtt_mps();
  qtt_status s = mps_alloc(ctx, psi_caps(ctx->d, chi), m);
  if (square) {  // c^2: the TT-SVD itself, cores 0..d-2 left-orthonormal
    if (s == QTT_OK) s = tt_svd(ctx, g, square, eps, chi, m);
  } else {  // a state: TT-SVD, then the Sec. 4.3 round (right-orthonormal cores 1..d-1)
    if (s == QTT_OK) s = tt_svd(ctx, g, square, eps, chi, ctx->ws.theta);
    if (s == QTT_OK) s = tt_round(ctx, ctx->ws.theta, m);
  }
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (tmp) cudaFree(tmp);
  if (s == QTT_OK && e != cudaSuccess) s = fail(QTT_ECUDA, cudaGetErrorString(e));
  if (s == QTT_OK) s = device_status(ctx);
  if (s == QTT_OK) {
    m->host_ranks.assign(ctx->d + 1, 1);
    if (cudaMemcpy(m->host_ranks.data(), m->ranks, (ctx->d + 1) * sizeof(int), cudaMemcpyDeviceToHost) !=
        cudaSuccess)
      s = fail(QTT_ECUDA, "rank read-back");
  }
  if (s != QTT_OK) {
    mps_free(m);
    delete m;
    return s;
  }
  *out = m;
  return QTT_OK;
}

qtt_status qtt_mps_from_dense(qtt_ctx* ctx, const double* grid, int on_device, qtt_mps** out) {
  if (!ctx) return fail(QTT_EINVAL, "null context");
  CKS(ensure_ws_basic(ctx));
  return from_dense_impl(ctx, grid, on_device, false, ctx->p.eps, ctx->p.chi_max, out);
}

qtt_status qtt_velocity_mps(qtt_ctx* ctx, const double* c_grid, int on_device, qtt_mps** c2_out) {
  if (!ctx) return fail(QTT_EINVAL, "null context");
  return from_dense_impl(ctx, c_grid, on_device, true, ctx->p.eps_c, ctx->p.chi_c, c2_out);
}

qtt_status qtt_laplacian_mpo(qtt_ctx* ctx, qtt_mpo** out) {
  if (!ctx || !out) return fail(QTT_EINVAL, "null argument");
  qtt_mpo* m = new qtt_mpo();
  build_laplacian(ctx->p.n, ctx->p.order, ctx->p.bc, ctx->dims, m);
  cudaError_t e = cudaMalloc(&m->data, m->host.size() * sizeof(double));
  if (e == cudaSuccess)
    e = cudaMemcpy(m->data, m->host.data(), m->host.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    if (m->data) cudaFree(m->data);
    delete m;
    return fail(QTT_ECUDA, cudaGetErrorString(e));
  }
  *out = m;
  return QTT_OK;
}

qtt_status qtt_mpo_bonds(const qtt_mpo* L, int* bonds_out) {
  if (!L || !bonds_out) return fail(QTT_EINVAL, "null argument");
  for (int k = 0; k <= L->d; ++k) bonds_out[k] = L->w[k];
  return QTT_OK;
}

void qtt_mpo_destroy(qtt_mpo* L) {
  if (!L) return;
  if (L->data) cudaFree(L->data);
  delete L;
}

qtt_status qtt_inject_source(qtt_ctx* ctx, qtt_mps* psi, long ix, long iz, double amp) {
  if (!ctx || !psi) return fail(QTT_EINVAL, "null argument");
  if (ctx->dims != 2) return fail(QTT_EINVAL, "3D context: use qtt_inject_source_3d");
  const long src[3] = {ix, iz, 0};
  return inject_impl(ctx, psi, src, amp);
}

qtt_status qtt_inject_source_3d(qtt_ctx* ctx, qtt_mps* psi, long ix, long iy, long iz, double amp) {
  if (!ctx || !psi) return fail(QTT_EINVAL, "null argument");
  if (ctx->dims != 3) return fail(QTT_EINVAL, "2D context: use qtt_inject_source");
  const long src[3] = {ix, iy, iz};
  return inject_impl(ctx, psi, src, amp);
}

}  // extern "C"

namespace {
qtt_status inject_impl(qtt_ctx* ctx, qtt_mps* psi, const long* src_in, double amp) {
  CKS(check_point(ctx, src_in));
  CKS(ensure_ws_basic(ctx));
  Workspace& s = ctx->ws;
  // theta needs room for psi + 1
  for (int k = 1; k < ctx->d; ++k)
    if (s.theta->cap[k] < psi->cap[k] + 1) return fail(QTT_EINVAL, "internal: sum workspace too small");
  CKS(form_sum(ctx, {{1.0, psi}}, src_in, amp, s.theta));
  CKS(tt_round(ctx, s.theta, psi));
  return QTT_OK;
}
}  // namespace

namespace {

// Reduced-precision steps only: the step is linear and its truncation rule
// relative, so both states (their first cores carry the norm) and the source
// sample are scaled by an exact power of two that brings the field to order
// one before the FP32 / tensor-core arithmetic (whose exponent range ends at
// ~1e-38: a field of 1e-10 with components kept down to 1e-10 of it would
// underflow in the squared norms), and the result is scaled back.
// phase 0: choose 2^s and scale u^{k-1}, u^k; phase 1: unscale the result
// (in prev) and restore u^k.  Exact in FP64.
qtt_status scale_states(qtt_ctx* ctx, Mps* prev, Mps* cur, int phase) {
  if (!ctx->use_mp) return QTT_OK;
  Workspace& s = ctx->ws;
  const long long r1 = std::max(prev->cap[1], cur->cap[1]);
  if (phase == 0)
    KL(KC_OTHER, state_scale_prepare(cur->core(0), cur->ranks + 1, prev->core(0), prev->ranks + 1, r1, s.d_scale,
                                     ctx->stream));
  KL(KC_OTHER, state_scale_apply(prev->core(0), prev->ranks + 1, r1, s.d_scale, phase, ctx->stream));
  KL(KC_OTHER, state_scale_apply(cur->core(0), cur->ranks + 1, r1, s.d_scale, phase, ctx->stream));
  return QTT_OK;
}

// The launches of one step (Eq. 17): zip-up of L, zip-up of diag(c^2), the
// sum with the source, the round into prev.  No host synchronisation.
qtt_status step_body(qtt_ctx* ctx, const Mpo* L, const Mps* c2, const std::vector<int>& rc, const Caps& c,
                     double lambda2, Mps* prev, Mps* cur, const long* src, double amp) {
  Workspace& s = ctx->ws;
  struct MpScope {  // the reduced-precision form applies inside the step only
    qtt_ctx* c;
    explicit MpScope(qtt_ctx* x) : c(x) { c->use_mp = (c->p.prec != QTT_FP64); }
    ~MpScope() { c->use_mp = false; }
  } mp_scope(ctx);
  CKS(scale_states(ctx, prev, cur, 0));
  CKS(zipup_L(ctx, L, cur, s.phi, c));
  CKS(zipup_C(ctx, c2, rc, s.phi, s.eta, c));
  CKS(form_sum(ctx, {{2.0, cur}, {-1.0, prev}, {lambda2, s.eta}}, src, amp, s.theta,
               ctx->use_mp ? s.d_scale : nullptr));
  CKS(tt_round(ctx, s.theta, prev));
  CKS(scale_states(ctx, prev, cur, 1));
  return QTT_OK;
}

qtt_status step_checks(qtt_ctx* ctx, const qtt_mpo* L, const qtt_mps* c2, double lambda2, qtt_mps* prev,
                       qtt_mps* cur, const long* src) {
  if (!ctx || !L || !c2 || !prev || !cur) return fail(QTT_EINVAL, "null argument");
  if (L->d != ctx->d || c2->d != ctx->d || prev->d != ctx->d || cur->d != ctx->d)
    return fail(QTT_EINVAL, "handle from another grid size");
  if (prev == cur) return fail(QTT_EINVAL, "psi_prev and psi_cur must differ");
  if (!(lambda2 >= 0.0) || !std::isfinite(lambda2)) return fail(QTT_EINVAL, "lambda2 must be finite, >= 0");
  if (src) CKS(check_point(ctx, src));
  return QTT_OK;
}

void swap_roles(Mps* a, Mps* b) {
  std::swap(a->data, b->data);
  std::swap(a->ranks, b->ranks);
}

void drop_graphs(qtt_ctx* ctx) {
  for (auto& e : ctx->gexec)
    if (e) {
      cudaGraphExecDestroy(e);
      e = nullptr;
    }
}

}  // namespace

extern "C" {

qtt_status qtt_step_graph(qtt_ctx* ctx, const qtt_mpo* L, const qtt_mps* c2, double lambda2, qtt_mps* prev,
                          qtt_mps* cur, const long* src, double amp) {
  CKS(step_checks(ctx, L, c2, lambda2, prev, cur, src));
  if (ctx->p.use_learned_rank) return fail(QTT_EINVAL, "the learned rounding synchronises with the host: use qtt_step");
  if (ctx->prof.timing) return fail(QTT_EINVAL, "per-kernel timing is on: use qtt_step");
  if (ctx->prof.d_log || ctx->prof.d_flops)
    return fail(QTT_EINVAL, "work logging is on (qtt_profile_start log_svd): use qtt_step");
  std::vector<int> rc = c2->cap;
  if (c2->host_ranks.size() == (size_t)ctx->d + 1) rc = c2->host_ranks;
  CKS(ensure_ws(ctx, L->w, rc));
  Caps c = step_caps(ctx, L->w, rc);
  if (!ctx->d_amp) CK(cudaMalloc(&ctx->d_amp, sizeof(double)));
  const long sk[4] = {src ? 1L : 0L, src ? src[0] : 0L, src ? src[1] : 0L,
                      (src && ctx->dims == 3) ? src[2] : 0L};
  auto same = [&](int g) {
    return ctx->gexec[g] && ctx->gkey[g][0] == L && ctx->gkey[g][1] == c2 && ctx->gkey[g][2] == prev->data &&
           ctx->gkey[g][3] == cur->data && ctx->gkey_lam == lambda2 && ctx->gkey_src[0] == sk[0] &&
           ctx->gkey_src[1] == sk[1] && ctx->gkey_src[2] == sk[2] && ctx->gkey_src[3] == sk[3];
  };
  int g = same(0) ? 0 : (same(1) ? 1 : -1);
  if (g < 0) {  // capture the step for both roles of the pair of state buffers
    drop_graphs(ctx);
    if (!ctx->gstream) CK(cudaStreamCreateWithFlags(&ctx->gstream, cudaStreamNonBlocking));
    long long before[KC_N];
    for (int r = 0; r < 2; ++r) {
      for (int k = 0; k < KC_N; ++k) before[k] = ctx->prof.launches[k];
      // capture on the context's own capture stream: recording runs nothing,
      // and the replays go to the caller's stream
      CK(cudaStreamBeginCapture(ctx->gstream, cudaStreamCaptureModeThreadLocal));
      const cudaStream_t user = ctx->stream;
      ctx->stream = ctx->gstream;
      ctx->capturing = true;
      const qtt_status st = step_body(ctx, L, c2, rc, c, lambda2, prev, cur, src, amp);
      ctx->capturing = false;
      ctx->stream = user;
      cudaGraph_t graph = nullptr;
      const cudaError_t e = cudaStreamEndCapture(ctx->gstream, &graph);
      cudaError_t ei = cudaErrorUnknown;
      if (st == QTT_OK && e == cudaSuccess) ei = cudaGraphInstantiate(&ctx->gexec[r], graph, 0);
      if (graph) cudaGraphDestroy(graph);
      for (int k = 0; k < KC_N; ++k) {
        ctx->glaunches[k] = ctx->prof.launches[k] - before[k];
        ctx->prof.launches[k] = before[k];
      }
      if (st != QTT_OK || e != cudaSuccess || ei != cudaSuccess) {
        if (r == 1) swap_roles(prev, cur);
        ctx->gexec[r] = nullptr;
        drop_graphs(ctx);
        if (st != QTT_OK) return st;
        return fail(QTT_ECUDA, std::string("step capture: ") + cudaGetErrorString(e != cudaSuccess ? e : ei));
      }
      ctx->gkey[r][0] = L;
      ctx->gkey[r][1] = c2;
      ctx->gkey[r][2] = prev->data;
      ctx->gkey[r][3] = cur->data;
      swap_roles(prev, cur);  // the second graph serves the exchanged roles
    }
    ctx->gkey_lam = lambda2;
    for (int k = 0; k < 4; ++k) ctx->gkey_src[k] = sk[k];
    g = 0;
  }
  CK(cudaMemcpyAsync(ctx->d_amp, &amp, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaGraphLaunch(ctx->gexec[g], ctx->stream));
  for (int k = 0; k < KC_N; ++k) ctx->prof.launches[k] += ctx->glaunches[k];
  swap_roles(prev, cur);
  return QTT_OK;
}

}  // extern "C"

namespace {

// Cache file of qtt_autotune: a small JSON document, one entry per line.
std::string tune_header(const qtt_ctx* ctx, const std::vector<int>& rc) {
  cudaDeviceProp prop{};
  cudaGetDeviceProperties(&prop, ctx->device);
  const int rcmax = rc.empty() ? 1 : *std::max_element(rc.begin(), rc.end());
  char buf[512];
  std::snprintf(buf, sizeof(buf), "device=%s sms=%d prec=%d n=%d chi=%d chi_zip=%d order=%d bc=%d rc_max=%d",
                prop.name, ctx->num_sms, ctx->p.prec, ctx->p.n, ctx->p.chi_max, ctx->p.chi_zip, ctx->p.order,
                ctx->p.bc, rcmax);
  return buf;
}

bool tune_load(const char* path, const std::string& header, std::map<TuneKey, int>* out) {
  FILE* f = std::fopen(path, "r");
  if (!f) return false;
  std::string text;
  char buf[4096];
  size_t got;
  while ((got = std::fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, got);
  std::fclose(f);
  if (text.find("\"header\": \"" + header + "\"") == std::string::npos) return false;
  std::map<TuneKey, int> m;
  size_t pos = 0;
  while ((pos = text.find("{\"op\": ", pos)) != std::string::npos) {
    int op = 0, kind = 0, choice = 0;
    long long a = 0, b = 0, c = 0;
    if (std::sscanf(text.c_str() + pos, "{\"op\": %d, \"kind\": %d, \"a\": %lld, \"b\": %lld, \"c\": %lld, \"choice\": %d",
                    &op, &kind, &a, &b, &c, &choice) == 6)
      m[TuneKey{op, kind, a, b, c}] = choice;
    pos += 8;
  }
  if (m.empty()) return false;
  *out = m;
  return true;
}

}  // namespace

extern "C" {

qtt_status qtt_autotune(qtt_ctx* ctx, const qtt_mpo* L, const qtt_mps* c2, double lambda2, const qtt_mps* prev,
                        const qtt_mps* cur, const char* cache_path, int reps, int* entries_out) {
  CKS(step_checks(ctx, L, c2, lambda2, const_cast<qtt_mps*>(prev), const_cast<qtt_mps*>(cur), nullptr));
  if (reps < 1 || reps > 1000) return fail(QTT_EINVAL, "reps must be in 1..1000");
  if (ctx->prof.timing || ctx->prof.d_log) return fail(QTT_EINVAL, "profiling is on: stop it before autotuning");
  if (ctx->p.use_learned_rank) return fail(QTT_EINVAL, "autotune a context without the learned rounding");
  std::vector<int> rc = c2->cap;
  if (c2->host_ranks.size() == (size_t)ctx->d + 1) rc = c2->host_ranks;
  CKS(ensure_ws(ctx, L->w, rc));
  const Caps caps = step_caps(ctx, L->w, rc);
  const std::string header = tune_header(ctx, rc);
  drop_graphs(ctx);  // the choices are launch parameters of captured graphs
  if (cache_path && tune_load(cache_path, header, &ctx->tune)) {
    if (entries_out) *entries_out = (int)ctx->tune.size();
    return QTT_OK;
  }
  ctx->tune.clear();
  // dry-run step on copies of the states, recording every tunable launch
  Mps tp, tc;
  CKS(mps_alloc(ctx, prev->cap, &tp));
  qtt_status st = mps_alloc(ctx, cur->cap, &tc);
  auto cleanup = [&]() {
    cudaStreamSynchronize(ctx->stream);
    mps_free(&tp);
    mps_free(&tc);
  };
  if (st == QTT_OK) {
    const cudaError_t e1 = cudaMemcpyAsync(tp.data, prev->data, prev->total * sizeof(double), cudaMemcpyDeviceToDevice,
                                           ctx->stream);
    const cudaError_t e2 = cudaMemcpyAsync(tc.data, cur->data, cur->total * sizeof(double), cudaMemcpyDeviceToDevice,
                                           ctx->stream);
    const cudaError_t e3 = cudaMemcpyAsync(tp.ranks, prev->ranks, (ctx->d + 1) * sizeof(int), cudaMemcpyDeviceToDevice,
                                           ctx->stream);
    const cudaError_t e4 = cudaMemcpyAsync(tc.ranks, cur->ranks, (ctx->d + 1) * sizeof(int), cudaMemcpyDeviceToDevice,
                                           ctx->stream);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess || e4 != cudaSuccess)
      st = fail(QTT_ECUDA, "autotune: state copy");
  }
  std::vector<TuneRec> recs;
  if (st == QTT_OK) {
    ctx->tune_rec = &recs;
    st = step_body(ctx, L, c2, rc, caps, lambda2, &tp, &tc, nullptr, 0.0);
    ctx->tune_rec = nullptr;
  }
  if (st == QTT_OK && cudaStreamSynchronize(ctx->stream) != cudaSuccess) st = fail(QTT_ECUDA, "autotune: dry run");
  if (st == QTT_OK) st = device_status(ctx);
  if (st != QTT_OK) {
    cleanup();
    return st;
  }
  // time every candidate on all launches of its bucket (the step's own
  // arguments and device-side sizes), keep the fastest
  std::map<TuneKey, std::vector<const TuneRec*>> buckets;
  for (const TuneRec& r : recs) buckets[TuneKey{r.op, r.kind, r.a, r.b, r.c}].push_back(&r);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  std::string body;
  for (const auto& kv : buckets) {
    const int op = std::get<0>(kv.first), kind = std::get<1>(kv.first);
    std::vector<int> cand;
    if (op == 1) cand = {256, 1024};
    else if (kind <= 1) cand = {16, 32};
    else cand = {64, 128, 256};
    int best = 0;
    double best_us = 1e300;
    std::string times;
    for (int ch : cand) {
      bool ok = true;
      for (const TuneRec* r : kv.second) ok = ok && r->launch(ch) == cudaSuccess;  // warm-up
      cudaEventRecord(e0, ctx->stream);
      for (int it = 0; it < reps && ok; ++it)
        for (const TuneRec* r : kv.second) ok = ok && r->launch(ch) == cudaSuccess;
      cudaEventRecord(e1, ctx->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) ok = false;
      cudaGetLastError();  // a refused candidate is skipped, not an error
      float ms = 0.f;
      if (ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) {
        const double us = 1e3 * ms / reps / kv.second.size();
        char tb[64];
        std::snprintf(tb, sizeof(tb), "%s\"%d\": %.2f", times.empty() ? "" : ", ", ch, us);
        times += tb;
        if (us < best_us) {
          best_us = us;
          best = ch;
        }
      }
    }
    if (best == 0) continue;
    ctx->tune[kv.first] = best;
    char line[512];
    std::snprintf(line, sizeof(line),
                  "%s  {\"op\": %d, \"kind\": %d, \"a\": %lld, \"b\": %lld, \"c\": %lld, \"choice\": %d, "
                  "\"launches_per_step\": %zu, \"us_per_launch\": {%s}}",
                  body.empty() ? "" : ",\n", op, kind, std::get<2>(kv.first), std::get<3>(kv.first),
                  std::get<4>(kv.first), best, kv.second.size(), times.c_str());
    body += line;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cleanup();
  st = device_status(ctx);
  if (st != QTT_OK) {
    ctx->tune.clear();
    return st;
  }
  if (cache_path) {
    FILE* f = std::fopen(cache_path, "w");
    if (!f) return fail(QTT_EINVAL, std::string("cannot write ") + cache_path);
    std::fprintf(f, "{\"qtt_autotune\": 1, \"header\": \"%s\", \"reps\": %d,\n \"entries\": [\n%s\n]}\n",
                 header.c_str(), reps, body.c_str());
    std::fclose(f);
  }
  if (entries_out) *entries_out = (int)ctx->tune.size();
  return QTT_OK;
}

qtt_status qtt_step(qtt_ctx* ctx, const qtt_mpo* L, const qtt_mps* c2, double lambda2, qtt_mps* prev, qtt_mps* cur,
                    const long* src, double amp) {
  CKS(step_checks(ctx, L, c2, lambda2, prev, cur, src));
  std::vector<int> rc = c2->cap;  // c^2 ranks are fixed; capacities bound them
  if (c2->host_ranks.size() == (size_t)ctx->d + 1) rc = c2->host_ranks;
  CKS(ensure_ws(ctx, L->w, rc));
  Caps c = step_caps(ctx, L->w, rc);
  Workspace& s = ctx->ws;
  if (!ctx->pending_prop.empty()) {
    CK(cudaMemcpyAsync(s.d_prop, ctx->pending_prop.data(), (ctx->d + 1) * sizeof(int), cudaMemcpyHostToDevice,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->pending_prop.clear();
    ctx->have_prop = true;
  }
  CKS(step_body(ctx, L, c2, rc, c, lambda2, prev, cur, src, amp));
  ctx->have_prop = false;  // proposals are for one step
  if (ctx->p.use_learned_rank && ctx->mlp) CKS(propose_ranks(ctx, prev));
  // prev now holds u^{k+1}: exchange buffers so that prev = u^k, cur = u^{k+1}
  std::swap(prev->data, cur->data);
  std::swap(prev->ranks, cur->ranks);
  return QTT_OK;
}

qtt_status qtt_a_operator_mpo(qtt_ctx* ctx, const qtt_mpo* L, const qtt_mps* c2, double lambda2, qtt_mpo** out) {
  if (!ctx || !L || !c2 || !out) return fail(QTT_EINVAL, "null argument");
  *out = nullptr;
  if (L->d != ctx->d || c2->d != ctx->d) return fail(QTT_EINVAL, "handle from another grid size");
  if (!(lambda2 >= 0.0) || !std::isfinite(lambda2)) return fail(QTT_EINVAL, "lambda2 must be finite, >= 0");
  const int d = ctx->d;
  std::vector<int> rc(d + 1);
  CK(cudaMemcpyAsync(rc.data(), c2->ranks, (d + 1) * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  std::vector<std::vector<double>> cores(d);
  for (int k = 0; k < d; ++k) {
    cores[k].resize((size_t)rc[k] * 2 * rc[k + 1]);
    CK(cudaMemcpyAsync(cores[k].data(), c2->core(k), cores[k].size() * sizeof(double), cudaMemcpyDeviceToHost,
                       ctx->stream));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  qtt_mpo* m = new qtt_mpo();
  build_a_operator(*L, cores, rc, lambda2, m);
  cudaError_t e = cudaMalloc(&m->data, m->host.size() * sizeof(double));
  if (e == cudaSuccess)
    e = cudaMemcpy(m->data, m->host.data(), m->host.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    if (m->data) cudaFree(m->data);
    delete m;
    return fail(e == cudaErrorMemoryAllocation ? QTT_ENOMEM : QTT_ECUDA, cudaGetErrorString(e));
  }
  *out = m;
  return QTT_OK;
}

qtt_status qtt_step_fused(qtt_ctx* ctx, const qtt_mpo* A, qtt_mps* prev, qtt_mps* cur, const long* src, double amp) {
  if (!ctx || !A || !prev || !cur) return fail(QTT_EINVAL, "null argument");
  if (A->d != ctx->d || prev->d != ctx->d || cur->d != ctx->d) return fail(QTT_EINVAL, "handle from another grid size");
  if (prev == cur) return fail(QTT_EINVAL, "psi_prev and psi_cur must differ");
  if (src) CKS(check_point(ctx, src));
  const Caps c = fused_caps(ctx, A->w);
  CKS(ensure_ws_caps(ctx, A->w, std::vector<int>(ctx->d + 1, 1), c));
  Workspace& s = ctx->ws;
  {
    struct MpScope {
      qtt_ctx* c;
      explicit MpScope(qtt_ctx* x) : c(x) { c->use_mp = (c->p.prec != QTT_FP64); }
      ~MpScope() { c->use_mp = false; }
    } mp_scope(ctx);
    CKS(scale_states(ctx, prev, cur, 0));
    CKS(zipup_L(ctx, A, cur, s.phi, c));
    CKS(form_sum(ctx, {{1.0, s.phi}, {-1.0, prev}}, src, amp, s.theta, ctx->use_mp ? s.d_scale : nullptr));
    CKS(tt_round(ctx, s.theta, prev));
    CKS(scale_states(ctx, prev, cur, 1));
  }
  std::swap(prev->data, cur->data);
  std::swap(prev->ranks, cur->ranks);
  return QTT_OK;
}

// ------------------------------------------------------------ learned form
int qtt_mlp_param_count(void) { return (int)kParams; }

void qtt_mlp_destroy(qtt_mlp* m) {
  if (!m) return;
  cudaStreamSynchronize(m->stream);
  float* bufs[] = {m->dev.p, m->dev.g, m->dev.m, m->dev.v, m->dev.a1, m->dev.a2, m->dev.d1, m->dev.d2, m->dev.y, m->dev.dy};
  for (float* b : bufs)
    if (b) cudaFree(b);
  delete m;
}

qtt_status qtt_mlp_create(const float* params, int max_batch, void* stream, qtt_mlp** out) {
  if (!params || !out || max_batch < 1) return fail(QTT_EINVAL, "bad MLP arguments");
  *out = nullptr;
  if (!cuda_ok_device()) return fail(QTT_ECUDA, "no CUDA device");
  qtt_mlp* m = new qtt_mlp();
  m->stream = (cudaStream_t)stream;
  m->dev.max_batch = max_batch;
  const size_t pb = kParams * sizeof(float), ab = (size_t)max_batch * kWidth * sizeof(float);
  cudaError_t e = cudaSuccess;
  float** pbufs[] = {&m->dev.p, &m->dev.g, &m->dev.m, &m->dev.v};
  for (float** b : pbufs)
    if (e == cudaSuccess) e = cudaMalloc(b, pb);
  float** abufs[] = {&m->dev.a1, &m->dev.a2, &m->dev.d1, &m->dev.d2};
  for (float** b : abufs)
    if (e == cudaSuccess) e = cudaMalloc(b, ab);
  if (e == cudaSuccess) e = cudaMalloc(&m->dev.y, max_batch * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->dev.dy, max_batch * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpyAsync(m->dev.p, params, pb, cudaMemcpyHostToDevice, m->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->dev.g, 0, pb, m->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->dev.m, 0, pb, m->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->dev.v, 0, pb, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) {
    qtt_mlp_destroy(m);
    return fail(e == cudaErrorMemoryAllocation ? QTT_ENOMEM : QTT_ECUDA, cudaGetErrorString(e));
  }
  *out = m;
  return QTT_OK;
}

qtt_status qtt_mlp_forward(qtt_mlp* m, const float* X, int n, float* y) {
  if (!m || !X || !y || n < 0) return fail(QTT_EINVAL, "bad MLP forward arguments");
  if (n > m->dev.max_batch) return fail(QTT_EINVAL, "batch larger than the network's max_batch");
  if (n == 0) return QTT_OK;
  CK(mlp_forward(m->dev, X, n, y, m->stream));
  return QTT_OK;
}

qtt_status qtt_mlp_grad(qtt_mlp* m, const float* X, const float* t, int n, float* loss, float* grad) {
  if (!m || !X || !t || n < 1) return fail(QTT_EINVAL, "bad MLP gradient arguments");
  if (n > m->dev.max_batch) return fail(QTT_EINVAL, "batch larger than the network's max_batch");
  CK(mlp_grad(m->dev, X, t, n, loss, m->stream));
  if (grad) CK(cudaMemcpyAsync(grad, m->dev.g, kParams * sizeof(float), cudaMemcpyDeviceToDevice, m->stream));
  return QTT_OK;
}

qtt_status qtt_mlp_adam_step(qtt_mlp* m, float lr, float beta1, float beta2, float eps) {
  if (!m) return fail(QTT_EINVAL, "null network");
  if (!(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
    return fail(QTT_EINVAL, "bad Adam hyper-parameters");
  ++m->t;
  CK(mlp_adam(m->dev, m->t, lr, beta1, beta2, eps, m->stream));
  return QTT_OK;
}

qtt_status qtt_mlp_get_params(qtt_mlp* m, float* params) {
  if (!m || !params) return fail(QTT_EINVAL, "null argument");
  CK(cudaMemcpyAsync(params, m->dev.p, kParams * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
  CK(cudaStreamSynchronize(m->stream));
  return QTT_OK;
}

qtt_status qtt_rank_features(const double* S, int lds, const int* len, const int* ranks, int nb, double eps, int chi,
                             int d, float* X, void* stream) {
  if (!S || !len || !ranks || !X || nb < 0 || nb > d - 1 || lds < 1 || chi < 1 || d < 2)
    return fail(QTT_EINVAL, "bad feature arguments");
  CK(rank_features(S, lds, len, ranks, nb, eps, chi, d, X, (cudaStream_t)stream));
  return QTT_OK;
}

qtt_status qtt_step_features(qtt_ctx* ctx, const qtt_mps* psi, float* X) {
  if (!ctx || !psi || !X) return fail(QTT_EINVAL, "null argument");
  if (!ctx->ws_ready) return fail(QTT_EINVAL, "no step has run on this context");
  CK(rank_features(ctx->ws.d_spec, ctx->ws_nvmax, ctx->ws.d_spec_len, psi->ranks, ctx->d - 1, ctx->p.eps,
                   ctx->p.chi_max, ctx->d, X, ctx->stream));
  return QTT_OK;
}

qtt_status qtt_set_rank_model(qtt_ctx* ctx, qtt_mlp* m, const double* sketch, int rows, int cols, int oversample) {
  if (!ctx) return fail(QTT_EINVAL, "null context");
  if (!sketch) {
    ctx->mlp = nullptr;
    ctx->sketch = nullptr;
    ctx->have_prop = false;
    return QTT_OK;
  }
  if (!ctx->p.use_learned_rank) return fail(QTT_EINVAL, "the context was created with use_learned_rank = 0");
  if (rows < 1 || cols < 1 || oversample < 0) return fail(QTT_EINVAL, "bad sketch arguments");
  if (m && m->dev.max_batch < ctx->d) return fail(QTT_EINVAL, "the network's max_batch must be >= 2n");
  ctx->mlp = m;
  ctx->sketch = sketch;
  ctx->sketch_rows = rows;
  ctx->sketch_cols = cols;
  ctx->oversample = oversample;
  ctx->have_prop = false;
  return QTT_OK;
}

qtt_status qtt_get_proposals(qtt_ctx* ctx, int* prop) {
  if (!ctx || !prop) return fail(QTT_EINVAL, "null argument");
  if (!ctx->ws_ready || !ctx->have_prop) {
    for (int k = 0; k <= ctx->d; ++k) prop[k] = 0;
    return QTT_OK;
  }
  CK(cudaMemcpyAsync(prop, ctx->ws.d_prop, (ctx->d + 1) * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return QTT_OK;
}

qtt_status qtt_set_proposals(qtt_ctx* ctx, const int* prop) {
  if (!ctx || !prop) return fail(QTT_EINVAL, "null argument");
  if (!ctx->p.use_learned_rank) return fail(QTT_EINVAL, "the context was created with use_learned_rank = 0");
  for (int k = 0; k <= ctx->d; ++k)
    if (prop[k] < 0 || prop[k] > ctx->p.chi_max) return fail(QTT_EINVAL, "proposals must be in 0..chi_max");
  ctx->pending_prop.assign(prop, prop + ctx->d + 1);
  return QTT_OK;
}

qtt_status qtt_learned_stats(qtt_ctx* ctx, long* attempts, long* accepts) {
  if (!ctx || !attempts || !accepts) return fail(QTT_EINVAL, "null argument");
  *attempts = (long)ctx->rf_attempts;
  *accepts = (long)ctx->rf_accepts;
  return QTT_OK;
}

}  // extern "C"

struct qtt_batch {
  std::vector<qtt_ctx*> ctx;
  std::vector<cudaStream_t> pool;
  std::vector<cudaEvent_t> done;
  cudaEvent_t start = nullptr;
  cudaStream_t user = nullptr;
  bool graphs = false;  // shots step through qtt_step_graph
};

extern "C" {

void qtt_batch_destroy(qtt_batch* b) {
  if (!b) return;
  for (cudaStream_t st : b->pool) cudaStreamSynchronize(st);
  for (qtt_ctx* c : b->ctx) qtt_ctx_destroy(c);
  for (cudaEvent_t e : b->done) cudaEventDestroy(e);
  if (b->start) cudaEventDestroy(b->start);
  for (cudaStream_t st : b->pool) cudaStreamDestroy(st);
  delete b;
}

qtt_status qtt_batch_create(const qtt_params* base, int nshots, const int* chi_per_shot, void* stream,
                            qtt_batch** out) {
  if (!base || !out || nshots < 1) return fail(QTT_EINVAL, "bad batch arguments");
  *out = nullptr;
  qtt_batch* b = new qtt_batch();
  b->user = (cudaStream_t)stream;
  const int S = std::min(nshots, 8);
  for (int i = 0; i < S; ++i) {
    cudaStream_t st;
    cudaEvent_t ev;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      qtt_batch_destroy(b);
      return fail(QTT_ECUDA, "stream pool");
    }
    b->pool.push_back(st);
    b->done.push_back(ev);
  }
  if (cudaEventCreateWithFlags(&b->start, cudaEventDisableTiming) != cudaSuccess) {
    qtt_batch_destroy(b);
    return fail(QTT_ECUDA, "event");
  }
  for (int i = 0; i < nshots; ++i) {
    qtt_params p = *base;
    if (chi_per_shot && chi_per_shot[i] > 0) p.chi_max = chi_per_shot[i];
    qtt_ctx* c = nullptr;
    qtt_status st = qtt_ctx_create(&p, b->user, &c);
    if (st != QTT_OK) {
      qtt_batch_destroy(b);
      return st;
    }
    // the pool's cooperative grids must be co-resident together
    c->coop_blocks = std::max(8, c->num_sms / S);
    b->ctx.push_back(c);
  }
  *out = b;
  return QTT_OK;
}

qtt_status qtt_batch_set_graphs(qtt_batch* b, int on) {
  if (!b) return fail(QTT_EINVAL, "null batch");
  b->graphs = on != 0;
  return QTT_OK;
}

qtt_ctx* qtt_batch_ctx(qtt_batch* b, int shot) {
  if (!b || shot < 0 || shot >= (int)b->ctx.size()) return nullptr;
  return b->ctx[shot];
}

qtt_status qtt_step_batched(qtt_batch* b, const qtt_mpo* L, const qtt_mps* c2, double lambda2, qtt_mps** prev,
                            qtt_mps** cur, const long* src, const double* amp) {
  if (!b || !L || !c2 || !prev || !cur) return fail(QTT_EINVAL, "null argument");
  if (src && !amp) return fail(QTT_EINVAL, "source positions without amplitudes");
  const int n = (int)b->ctx.size(), S = (int)b->pool.size();
  for (int i = 0; i < n; ++i)
    if (!prev[i] || !cur[i] || prev[i]->ctx != b->ctx[i] || cur[i]->ctx != b->ctx[i])
      return fail(QTT_EINVAL, "state " + std::to_string(i) + " does not belong to its shot's context");
  CK(cudaEventRecord(b->start, b->user));
  for (int s = 0; s < S; ++s) CK(cudaStreamWaitEvent(b->pool[s], b->start, 0));
  // each shot's step runs on its pool stream; every other call on a shot's
  // context stays on the batch's stream
  for (int i = 0; i < n; ++i) b->ctx[i]->stream = b->pool[i % S];
  std::vector<qtt_status> st(S, QTT_OK);
  std::vector<std::string> msg(S);
  auto worker = [&](int s) {
    for (int i = s; i < n; i += S) {
      qtt_status r = (b->graphs ? qtt_step_graph : qtt_step)(b->ctx[i], L, c2, lambda2, prev[i], cur[i],
                                                             src ? src + b->ctx[0]->dims * i : nullptr,
                                                             src ? amp[i] : 0.0);
      if (r != QTT_OK) {
        st[s] = r;
        msg[s] = g_err;
        return;
      }
    }
  };
  std::vector<std::thread> th;
  for (int s = 1; s < S; ++s) th.emplace_back(worker, s);
  worker(0);
  for (auto& t : th) t.join();
  for (int i = 0; i < n; ++i) b->ctx[i]->stream = b->user;
  for (int s = 0; s < S; ++s) {
    CK(cudaEventRecord(b->done[s], b->pool[s]));
    CK(cudaStreamWaitEvent(b->user, b->done[s], 0));
  }
  for (int s = 0; s < S; ++s)
    if (st[s] != QTT_OK) return fail(st[s], "shot on pool stream " + std::to_string(s) + ": " + msg[s]);
  return QTT_OK;
}

}  // extern "C"

namespace {
qtt_status sample_impl(qtt_ctx* ctx, const qtt_mps* psi, const long* ix, const long* iy, const long* iz, long count,
                       double* out) {
  if (count < 0) return fail(QTT_EINVAL, "negative count");
  if (count == 0) return QTT_OK;
  SampleArgs a;
  std::memset(&a, 0, sizeof(a));
  a.d = ctx->d;
  a.n = ctx->p.n;
  a.dims = ctx->dims;
  a.sp = site_positions(ctx);
  a.rmax = *std::max_element(psi->cap.begin(), psi->cap.end());
  for (int k = 0; k < ctx->d; ++k) a.core[k] = psi->core(k);
  a.ranks = psi->ranks;
  a.ix = ix;
  a.iy = iy;
  a.iz = iz;
  a.count = count;
  a.out = out;
  KL(KC_OTHER, sample(a, ctx->stream));
  return QTT_OK;
}
}  // namespace

extern "C" {

qtt_status qtt_sample(qtt_ctx* ctx, const qtt_mps* psi, const long* ix, const long* iz, long count, double* out) {
  if (!ctx || !psi || (count > 0 && (!ix || !iz || !out))) return fail(QTT_EINVAL, "null argument");
  if (ctx->dims != 2) return fail(QTT_EINVAL, "3D context: use qtt_sample_3d");
  return sample_impl(ctx, psi, ix, nullptr, iz, count, out);
}

qtt_status qtt_sample_3d(qtt_ctx* ctx, const qtt_mps* psi, const long* ix, const long* iy, const long* iz, long count,
                         double* out) {
  if (!ctx || !psi || (count > 0 && (!ix || !iy || !iz || !out))) return fail(QTT_EINVAL, "null argument");
  if (ctx->dims != 3) return fail(QTT_EINVAL, "2D context: use qtt_sample");
  return sample_impl(ctx, psi, ix, iy, iz, count, out);
}

qtt_status qtt_to_dense(qtt_ctx* ctx, const qtt_mps* psi, double* out) {
  if (!ctx || !psi || !out) return fail(QTT_EINVAL, "null argument");
  CKS(ensure_ws_basic(ctx));
  Workspace& s = ctx->ws;
  const int d = ctx->d, h = d / 2;
  const long long nL = p2(h), nR = p2(d - h);
  const int rmax = *std::max_element(psi->cap.begin(), psi->cap.end());
  const long long rh = psi->cap[h];
  if (nL * rh > s.xbuf || rh * nR > s.carry || nL * nR > s.tv) return fail(QTT_EINVAL, "internal: to_dense scratch");
  ChainArgs l, r;
  std::memset(&l, 0, sizeof(l));
  l.d = d;
  l.h = h;
  l.rmax = rmax;
  for (int k = 0; k < d; ++k) l.core[k] = psi->core(k);
  l.ranks = psi->ranks;
  r = l;
  l.out = s.d_x;      // Lm: nL x r_h
  r.out = s.d_carry;  // Rm: r_h x nR
  KL2(KC_OTHER, chains(l, r, ctx->stream));
  GemmArgs g = gemm0();
  g.A = s.d_x;
  g.B = s.d_carry;
  g.C = s.d_tv;
  g.M = dconst(nL);
  g.N = dconst(nR);
  g.K = dptr(psi->ranks + h);
  g.sai = dptr(psi->ranks + h);
  g.sak = dconst(1);
  g.sbk = dconst(nR);
  g.sbj = dconst(1);
  g.sci = dconst(nR);
  g.scj = dconst(1);
  KL(KC_GEMM, gemm_f64(g, nL, nR, 1, 1, ctx->stream));
  KL(KC_OTHER, scatter_dense(s.d_tv, out, site_positions(ctx), h, ctx->stream));
  return QTT_OK;
}

qtt_status qtt_svd_trunc(qtt_ctx* ctx, const double* M, int m, int n, double eps, int chi, double* U, double* S,
                         double* Vt, int* rank_out) {
  if (!ctx || !M || !U || !S || !Vt || !rank_out) return fail(QTT_EINVAL, "null argument");
  if (m < 1 || n < 1) return fail(QTT_EINVAL, "empty matrix");
  if (!(eps >= 0.0)) return fail(QTT_EINVAL, "eps must be >= 0");
  CKS(ensure_ws_basic(ctx));
  Workspace& s = ctx->ws;
  const long long nv = std::min(m, n), ell = std::max(m, n);
  if (nv > ctx->ws_nvmax || nv * ell > s.tv || ell > ctx->ws_ellmax * 64)
    return fail(QTT_EINVAL, "matrix larger than the context workspace");
  int* r_d = s.d_ints + 4;
  const int chic = chi <= 0 ? (int)nv : chi;
  if (m <= n) {
    // vectors = rows of M; U = J (m x r), Vt = S^-1 Jp M
    CKS(svd_vm(ctx, M, dconst(m), dconst(n), m, n, eps, chic, (int)nv, r_d, s.d_jp, U, nullptr, S));
    GemmArgs g = gemm0();
    g.A = s.d_jp;
    g.B = M;
    g.C = Vt;
    g.M = dptr(r_d);
    g.N = dconst(n);
    g.K = dconst(m);
    g.sai = dconst(m);
    g.sak = dconst(1);
    g.sbk = dconst(n);
    g.sbj = dconst(1);
    g.sci = dconst(n);
    g.scj = dconst(1);
    KL(KC_GEMM, gemm_f64(g, nv, n, 1, 1, ctx->stream));
    KL(KC_OTHER, scale_rows(Vt, n, dconst(n), r_d, S, nv * n, ctx->stream));
  } else {
    // vectors = columns of M (copied vector-major); Vt = Jp; U = (M J) S^-1
    KL(KC_COPY, copy2d(M, s.d_tv, dconst(m), dconst(n), dconst(n), dconst(1), dconst(1), dconst(m), (long long)m * n, 1.0,
              ctx->stream));
    CKS(svd_vm(ctx, s.d_tv, dconst(n), dconst(m), n, m, eps, chic, (int)nv, r_d, Vt, nullptr, nullptr, S));
    GemmArgs g = gemm0();  // W = Jp Mv  (r x m) into jp scratch
    g.A = Vt;
    g.B = s.d_tv;
    g.C = s.d_w1;
    g.M = dptr(r_d);
    g.N = dconst(m);
    g.K = dconst(n);
    g.sai = dconst(n);
    g.sak = dconst(1);
    g.sbk = dconst(m);
    g.sbj = dconst(1);
    g.sci = dconst(m);
    g.scj = dconst(1);
    if ((long long)nv * m > s.w1) return fail(QTT_EINVAL, "matrix larger than the context workspace");
    KL(KC_GEMM, gemm_f64(g, nv, m, 1, 1, ctx->stream));
    KL(KC_OTHER, scale_rows(s.d_w1, m, dconst(m), r_d, S, nv * m, ctx->stream));
    // U[i][j] = W[j][i]
    KL(KC_COPY, copy2d(s.d_w1, U, dptr(r_d), dconst(m), dconst(m), dconst(1), dconst(1), dptr(r_d), nv * m, 1.0,
              ctx->stream));
  }
  CK(cudaMemcpyAsync(rank_out, r_d, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return device_status(ctx);
}

qtt_status qtt_gemm(qtt_ctx* ctx, int kind, int a_trans, int b_trans, int m, int n, int k, const double* A, int lda,
                    const double* B, int ldb, double* C, int ldc, double alpha, double beta, int tile_n) {
  if (!ctx || (!A && k > 0 && m > 0) || (!B && k > 0 && n > 0) || (!C && m > 0 && n > 0))
    return fail(QTT_EINVAL, "null argument");
  if (kind < 0 || kind > 4) return fail(QTT_EINVAL, "kind must be 0..4");
  if (m < 0 || n < 0 || k < 0) return fail(QTT_EINVAL, "negative size");
  if (lda < std::max(1, a_trans ? m : k) || ldb < std::max(1, b_trans ? k : n) || ldc < std::max(1, n))
    return fail(QTT_EINVAL, "leading dimension smaller than the row");
  if (tile_n != 0 && tile_n != 64 && tile_n != 128 && tile_n != 256)
    return fail(QTT_EINVAL, "tile_n must be 0, 64, 128 or 256");
  if (m == 0 || n == 0) return QTT_OK;
  CKS(ensure_ws_basic(ctx));
  GemmArgs g = gemm0();
  g.A = A;
  g.B = B;
  g.C = C;
  g.M = dconst(m);
  g.N = dconst(n);
  g.K = dconst(k);
  g.sai = dconst(a_trans ? 1 : lda);
  g.sak = dconst(a_trans ? lda : 1);
  g.sbk = dconst(b_trans ? 1 : ldb);
  g.sbj = dconst(b_trans ? ldb : 1);
  g.sci = dconst(ldc);
  g.scj = dconst(1);
  g.alpha = alpha;
  g.beta = beta;
  if (kind == 0) {
    KL(KC_GEMM, gemm_f64(g, m, n, 1, 1, ctx->stream));
  } else if (kind == 1) {
    KL(KC_GEMM, gemm_f32(g, m, n, 1, 1, ctx->stream));
  } else {
    const int bn = tile_n ? tile_n : tc_tile_n(ctx, m, n, 1);
    KL(KC_GEMM, gemm_tc(g, m, n, 1, 1, kind - 2, bn, ctx->ws.d_sync, ctx->stream));
  }
  return QTT_OK;
}

qtt_status qtt_fdtd_step(qtt_ctx* ctx, const double* c2, double lambda2, const double* up, const double* uc,
                         double* un, long sx, long sz, double amp) {
  if (!ctx || !c2 || !up || !uc || !un) return fail(QTT_EINVAL, "null argument");
  if (ctx->dims != 2) return fail(QTT_EINVAL, "3D context: use qtt_fdtd_step_3d");
  const long N = 1L << ctx->p.n;
  if (sx >= N || sz < 0 || sz >= N) sx = -1;
  KL(KC_FDTD, fdtd(c2, lambda2, up, uc, un, ctx->p.n, ctx->p.bc, sx, sz, amp, ctx->stream));
  return QTT_OK;
}

qtt_status qtt_fdtd_step_3d(qtt_ctx* ctx, const double* c2, double lambda2, const double* up, const double* uc,
                            double* un, long sx, long sy, long sz, double amp) {
  if (!ctx || !c2 || !up || !uc || !un) return fail(QTT_EINVAL, "null argument");
  if (ctx->dims != 3) return fail(QTT_EINVAL, "2D context: use qtt_fdtd_step");
  const long N = 1L << ctx->p.n;
  if (sx < 0 || sx >= N || sy < 0 || sy >= N || sz < 0 || sz >= N) sx = -1;
  KL(KC_FDTD, fdtd3(c2, lambda2, up, uc, un, ctx->p.n, ctx->p.bc, sx, sy, sz, amp, ctx->stream));
  return QTT_OK;
}

qtt_status qtt_profile_start(qtt_ctx* ctx, int timing, int log_svd) {
  if (!ctx) return fail(QTT_EINVAL, "null context");
  Prof& p = ctx->prof;
  CK(cudaStreamSynchronize(ctx->stream));
  for (int c = 0; c < KC_N; ++c) p.launches[c] = 0;
  p.used = 0;
  p.timing = timing ? 1 : 0;
  p.log_used = 0;
  if (log_svd) {
    if (!p.d_log) {
      p.log_cap = 65536;
      CK(cudaMalloc(&p.d_log, 3 * p.log_cap * sizeof(int)));
    }
    if (!p.d_flops) CK(cudaMalloc(&p.d_flops, KC_N * sizeof(double)));
    CK(cudaMemsetAsync(p.d_flops, 0, KC_N * sizeof(double), ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  } else {
    if (p.d_log) cudaFree(p.d_log);
    if (p.d_flops) cudaFree(p.d_flops);
    p.d_log = nullptr;
    p.d_flops = nullptr;
    p.log_cap = 0;
  }
  return QTT_OK;
}

qtt_status qtt_profile_read(qtt_ctx* ctx, qtt_profile* out) {
  if (!ctx || !out) return fail(QTT_EINVAL, "null argument");
  Prof& p = ctx->prof;
  CK(cudaStreamSynchronize(ctx->stream));
  std::memset(out, 0, sizeof(*out));
  for (int c = 0; c < KC_N && c < QTT_KCLASSES; ++c) out->launches[c] = p.launches[c];
  for (int i = 0; i < p.used; ++i) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, p.ev[i].first, p.ev[i].second));
    out->ms[p.cls[i]] += ms;
  }
  if (p.d_log && p.log_used > 0) {
    std::vector<int> h(3 * p.log_used);
    CK(cudaMemcpy(h.data(), p.d_log, h.size() * sizeof(int), cudaMemcpyDeviceToHost));
    double f = 0.0;
    long sweeps = 0;
    for (int i = 0; i < p.log_used; ++i) {
      double a = h[3 * i], b = h[3 * i + 1];
      double n = std::min(a, b), m = std::max(a, b);
      f += 6.0 * m * n * n + 20.0 * n * n * n;
      sweeps += h[3 * i + 2];
    }
    out->svd_logged = p.log_used;
    out->svd_flops = f;
    out->svd_sweeps = sweeps;
  }
  if (p.d_flops) {
    double h[KC_N];
    CK(cudaMemcpy(h, p.d_flops, sizeof(h), cudaMemcpyDeviceToHost));
    for (int c = 0; c < KC_N && c < QTT_KCLASSES; ++c) out->flops[c] = h[c];
  }
  return device_status(ctx);
}

qtt_status qtt_last_step_discarded(qtt_ctx* ctx, double* out) {
  if (!ctx || !out) return fail(QTT_EINVAL, "null argument");
  if (!ctx->ws_ready) return fail(QTT_EINVAL, "no step has run");
  const int d = ctx->d;
  std::vector<double> h(3 * (d + 1));
  CK(cudaMemcpyAsync(h.data(), ctx->ws.d_disc, h.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  for (int ph = 0; ph < 3; ++ph)
    for (int b = 1; b < d; ++b) out[ph * (d - 1) + b - 1] = h[ph * (d + 1) + b];
  return device_status(ctx);
}

}  // extern "C"
