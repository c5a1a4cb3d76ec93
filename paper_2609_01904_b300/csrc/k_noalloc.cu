// Truncated SVD that allocates no memory.
//
// Some callers cannot call cudaMalloc: code whose device memory is owned
// entirely by another allocator (a framework's caching pool, a fixed arena
// sized at start-up), where a new allocation would fail or fragment that
// pool, and latency-critical loops that cannot afford the device-wide
// synchronisation cudaMalloc and cudaFree may imply.  For them this file
// provides qtt_svd_trunc_noalloc: the same factorisation as qtt_svd_trunc
// (Householder QR, one-sided Jacobi, the keep-sigma >= eps*sigma_1 rule) with
// all of its scratch in one file-scope device array.  The caller passes only
// the input matrix and the output buffers.
//
// Limits: max(m, n) <= kMaxDim and min(m, n) <= kMaxRank; larger sizes are
// rejected with QTT_EINVAL.  The array lives in every GPU that loads the
// library until the process exits.  All calls share it: two calls whose work
// overlaps on the GPU (e.g. on two streams) race and corrupt each other.
#include <cstring>
#include <mutex>
#include <string>

#include "k_mps.cuh"
#include "qtt_internal.cuh"

namespace qtt {
void set_last_error(const std::string& msg);  // qtt_api.cu: text for qtt_last_error()

namespace {

constexpr long long kMaxDim = 512;   // longest side of the matrix
constexpr long long kMaxRank = 128;  // shortest side of the matrix
constexpr long long kBig = kMaxDim * kMaxRank;
constexpr long long kSq = kMaxRank * kMaxRank;
// layout of the scratch array, in doubles
constexpr long long kOffTq = 0, kOffTt = kOffTq + kBig, kOffQt = kOffTt + kBig, kOffTv = kOffQt + kBig,
                    kOffW1 = kOffTv + kBig, kOffRv = kOffW1 + kBig, kOffJv = kOffRv + kSq, kOffJh = kOffJv + kSq,
                    kOffJp = kOffJh + kSq, kOffNorm = kOffJp + kSq, kOffSig = kOffNorm + kMaxDim,
                    kOffTau = kOffSig + kMaxDim, kOffInts = kOffTau + kMaxDim, kOffFlags = kOffInts + 64,
                    kOffSync = kOffFlags + (kMaxDim + 64) / 2,
                    kScratchDoubles = kOffSync + (long long)(sizeof(DevSync) / sizeof(double)) + 8;

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {nullptr};
int g_num_sms[kMaxDevices] = {0};

qtt_status nfail(qtt_status s, const std::string& m) {
  set_last_error(m);
  return s;
}

#define NCK(call)                                                                              \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return nfail(QTT_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

GemmArgs g0() {
  GemmArgs g;
  std::memset(&g, 0, sizeof(g));
  g.nb1 = g.nb2 = dconst(1);
  g.sa1 = g.sa2 = g.sb1 = g.sb2 = g.sc1 = g.sc2 = dconst(0);
  g.alpha = 1.0;
  return g;
}

}  // namespace
}  // namespace qtt

using namespace qtt;

extern "C" qtt_status qtt_svd_trunc_noalloc(const double* M, int m, int n, double eps, int chi, double* U,
                                            double* S, double* Vt, int* rank_out, void* cuda_stream) {
  if (!M || !U || !S || !Vt || !rank_out) return nfail(QTT_EINVAL, "null argument");
  if (m < 1 || n < 1) return nfail(QTT_EINVAL, "empty matrix");
  if (!(eps >= 0.0)) return nfail(QTT_EINVAL, "eps must be >= 0");
  const long long nv = m < n ? m : n, ell = m < n ? n : m;
  if (ell > kMaxDim || nv > kMaxRank)
    return nfail(QTT_EINVAL, "qtt_svd_trunc_noalloc: matrix larger than the static scratch (max(m,n) <= " +
                                 std::to_string(kMaxDim) + ", min(m,n) <= " + std::to_string(kMaxRank) + ")");
  int dev = 0;
  NCK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return nfail(QTT_EINVAL, "device ordinal out of range");
  // once per device, with that device current: the device address of the array
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      NCK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
      NCK(cudaDeviceGetAttribute(&g_num_sms[dev], cudaDevAttrMultiProcessorCount, dev));
      g_scratch_ptr[dev] = (double*)p;
    }
  }
  double* base = g_scratch_ptr[dev];
  cudaStream_t st = (cudaStream_t)cuda_stream;

  // a context on the stack whose workspace points into the array (no allocation)
  qtt_ctx c;
  c.stream = st;
  c.device = dev;
  c.num_sms = g_num_sms[dev];
  c.coop_blocks = g_num_sms[dev];
  c.ws.d_tq = base + kOffTq;
  c.ws.d_tt = base + kOffTt;
  c.ws.d_qt = base + kOffQt;
  c.ws.d_tv = base + kOffTv;
  c.ws.d_w1 = base + kOffW1;
  c.ws.d_rv = base + kOffRv;
  c.ws.d_jv = base + kOffJv;
  c.ws.d_jh = base + kOffJh;
  c.ws.d_jp = base + kOffJp;
  c.ws.d_norm = base + kOffNorm;
  c.ws.d_sig = base + kOffSig;
  c.ws.d_tau = base + kOffTau;
  c.ws.d_ints = (int*)(base + kOffInts);
  c.ws.d_flags = (int*)(base + kOffFlags);
  c.ws.d_sync = (DevSync*)(base + kOffSync);
  Workspace& s = c.ws;
  qtt_ctx* ctx = &c;
  const long long ldv = kMaxRank;
  int* kq = s.d_ints + 0;
  int* r_d = s.d_ints + 4;
  const int chic = chi <= 0 ? (int)nv : chi;

  // the barrier counters and the status word must start at zero
  NCK(cudaMemsetAsync(s.d_sync, 0, sizeof(DevSync), st));

  // vectors: rows of M (m <= n) or columns of M copied vector-major (m > n)
  const double* Tv = M;
  if (m > n) {
    NCK(copy2d(M, s.d_tv, dconst(m), dconst(n), dconst(n), dconst(1), dconst(1), dconst(m), (long long)m * n, 1.0,
               st));
    Tv = s.d_tv;
  }
  double* Jp = (m <= n) ? s.d_jp : Vt;  // m > n: V^T is the kept rotations
  double* Jt = (m <= n) ? U : nullptr;  // m <= n: U is the kept rotations
  const Dim dnv = dconst(nv), dell = dconst(ell);
  if (ell > nv) {
    NCK(qr_f64(ctx, Tv, dell, s.d_tq, ell, dell, dnv, nv, s.d_rv, false, nullptr, kq, ldv, 0));
    NCK(jacobi_f64(ctx, s.d_rv, ldv, dnv, dptr(kq), nv, s.d_jv, ldv, s.d_norm));
    NCK(svd_post(ctx, s.d_norm, dnv, dptr(kq), dnv, s.d_jv, ldv, eps, chic, (int)nv, r_d, S, nullptr, Jp, Jt));
  } else {  // square
    NCK(copy2d(Tv, s.d_tq, dnv, dell, dell, dconst(1), dconst(ell), dconst(1), nv * ell, 1.0, st));
    NCK(jacobi_f64(ctx, s.d_tq, ell, dnv, dell, nv, s.d_jv, ldv, s.d_norm));
    NCK(svd_post(ctx, s.d_norm, dnv, dell, dnv, s.d_jv, ldv, eps, chic, (int)nv, r_d, S, nullptr, Jp, Jt));
  }
  if (m <= n) {  // V^T = S^-1 Jp M
    GemmArgs g = g0();
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
    NCK(gemm_f64(g, nv, n, 1, 1, st));
    NCK(scale_rows(Vt, n, dconst(n), r_d, S, nv * n, st));
  } else {  // U = (M J) S^-1, built as W = Jp Mv then transposed
    GemmArgs g = g0();
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
    NCK(gemm_f64(g, nv, m, 1, 1, st));
    NCK(scale_rows(s.d_w1, m, dconst(m), r_d, S, nv * m, st));
    NCK(copy2d(s.d_w1, U, dptr(r_d), dconst(m), dconst(m), dconst(1), dconst(1), dptr(r_d), nv * m, 1.0, st));
  }
  int status = 0;
  NCK(cudaMemcpyAsync(rank_out, r_d, sizeof(int), cudaMemcpyDeviceToHost, st));
  NCK(cudaMemcpyAsync(&status, &s.d_sync->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  NCK(cudaStreamSynchronize(st));
  if (status != 0) return nfail((qtt_status)status, "device status from the Jacobi SVD");
  return QTT_OK;
}
