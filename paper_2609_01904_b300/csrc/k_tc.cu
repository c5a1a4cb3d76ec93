// Core contractions on the 5th-generation tensor cores (tcgen05, TMEM).
//
// The contractions of a step (zip-up site contractions, the Hadamard
// contraction with the c^2 cores, the absorption of R and U S factors into
// the neighbouring cores; Sec. 4.3) are small GEMMs whose sizes are bond
// ranks held in device memory.  This kernel computes one 128 x BN tile of
// C = alpha A B + beta C per CTA with tcgen05.mma, the accumulator in tensor
// memory:
//   - 128 threads load the FP64 operands (strides evaluated on the device,
//     coalesced along whichever index is contiguous), round them to the
//     operand type and store them into shared memory in the 128-byte
//     swizzled K-major layout the MMA reads (8-row atoms of 128-byte rows,
//     16-byte chunks XOR-ed with the row index);
//   - one thread issues the MMAs of a K chunk (4 instructions of K = 8 TF32
//     or K = 16 BF16) and commits them to the stage's mbarrier, while the
//     other threads fill the second stage;
//   - the epilogue reads the accumulator with tcgen05.ld (warp w owns TMEM
//     lanes 32w..32w+31 = tile rows) and writes alpha * acc + beta * C in FP64.
// Operand forms: TF32 (one pass, FP32 accumulation), 3xTF32 (x = hi + lo
// with both parts TF32, products hi*hi + hi*lo + lo*hi accumulated in FP32:
// about FP32 accuracy on the tensor pipe) and BF16 (one pass, FP32
// accumulation).  Operands are FP64 in memory, so the rounding happens in
// the load path and TMA (which copies bytes, with strides fixed on the host)
// is not used: the strides here are bond ranks known only on the device.
//
// Every wait on an mbarrier is bounded by the context's wait limit; a wait
// that runs out records QTT_ETIMEOUT, waits (bounded) for the MMAs already
// issued, frees the tensor memory and returns.
#include <cuda_bf16.h>

#include <cstdint>

#include "qtt_internal.cuh"

namespace qtt {

namespace {

constexpr int kTcThreads = 128;
constexpr int kTcRows = 128;  // UMMA M
constexpr int kRowBytes = 128;  // one swizzle row: 32 TF32 or 64 BF16 values of K

template <int KIND, int BN>
struct TcCfg {
  static constexpr int kSplit = (KIND == 1) ? 2 : 1;  // hi (and lo) tiles per operand
  static constexpr int kBK = (KIND == 2) ? 64 : 32;   // K elements per chunk (one 128-byte row)
  static constexpr int kABytes = kTcRows * kRowBytes;
  static constexpr int kBBytes = BN * kRowBytes;
  static constexpr int kStage = kSplit * (kABytes + kBBytes);
  static constexpr int kStages = 2;
  static constexpr int kSmem = kStages * kStage + 1024;  // + alignment of the 1024-byte swizzle atoms
};

struct TcArgs {
  GemmArgs a;
  long long nb2max;
  double* flops;
  DevSync* sync;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ uint32_t bf16_bits(float x) {
  const __nv_bfloat16_raw r = __nv_bfloat16_raw(__float2bfloat16_rn(x));
  return (uint32_t)r.x;
}

// byte offset of (row r, byte b of the 128-byte row) in a 128-byte swizzled tile
__device__ __forceinline__ uint32_t swz(int r, int b) {
  return (uint32_t)(r * kRowBytes + ((((b >> 4) ^ (r & 7)) << 4) | (b & 15)));
}

// tcgen05 shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row
// groups 1024 bytes apart
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// instruction descriptor: D = F32, A and B K-major, M = 128, N = BN
template <int KIND>
__device__ __forceinline__ uint32_t idesc(int bn) {
  const uint32_t fmt = (KIND == 2) ? 1u : 2u;  // BF16 : TF32
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(bn >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);
}

template <int KIND>
__device__ __forceinline__ void mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t id, uint32_t acc) {
  if constexpr (KIND == 2) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(id), "r"(acc));
  } else {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(id), "r"(acc));
  }
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
}

// bounded wait for the completion of phase `parity` of an mbarrier
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, DevSync* sync) {
  const unsigned long long t0 = globaltimer_ns(), lim = wait_limit(sync);
  for (int it = 0;; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (globaltimer_ns() - t0 > lim) {
      set_status(sync, QTT_ETIMEOUT);
      return false;
    }
    if (it > 8) __nanosleep(32);
  }
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// One operand tile: rows row0 .. row0+NR-1 of P (row stride s_row, K stride
// s_k), K chunk k0 .. k0+BK-1, zero outside (rows_lim, K); rounded to the
// operand type into the swizzled tile(s) hi (and lo for 3xTF32).
template <int KIND, int NR>
__device__ __forceinline__ void load_tile(uint8_t* hi, uint8_t* lo, const double* P, long long s_row, long long s_k,
                                          long long row0, long long rows_lim, long long k0, long long K) {
  const int tid = threadIdx.x;
  constexpr int kPer = NR * 32 / kTcThreads;  // 32 words of 4 bytes per row
  const bool kfast = (s_k == 1);
#pragma unroll 4
  for (int t = 0; t < kPer; ++t) {
    const int e = tid + kTcThreads * t;
    int r, w;  // row and 4-byte word of the row
    if (kfast) {
      w = e & 31;
      r = e >> 5;
    } else {
      r = e % NR;
      w = e / NR;
    }
    const long long gr = row0 + r;
    const uint32_t off = swz(r, w * 4);
    if constexpr (KIND == 2) {
      const long long gk = k0 + 2 * w;
      double x0 = 0.0, x1 = 0.0;
      if (gr < rows_lim) {
        const double* pr = P + gr * s_row;
        if (gk < K) x0 = pr[gk * s_k];
        if (gk + 1 < K) x1 = pr[(gk + 1) * s_k];
      }
      const uint32_t v = bf16_bits((float)x0) | (bf16_bits((float)x1) << 16);
      *reinterpret_cast<uint32_t*>(hi + off) = v;
    } else {
      const long long gk = k0 + w;
      double x = 0.0;
      if (gr < rows_lim && gk < K) x = P[gr * s_row + gk * s_k];
      const uint32_t h = to_tf32((float)x);
      *reinterpret_cast<uint32_t*>(hi + off) = h;
      if constexpr (KIND == 1) {
        const double rem = x - (double)__uint_as_float(h);
        *reinterpret_cast<uint32_t*>(lo + off) = to_tf32((float)rem);
      }
    }
  }
}

template <int KIND, int BN>
__global__ void __launch_bounds__(kTcThreads, 1) tc_gemm_kernel(TcArgs ta) {
  using Cfg = TcCfg<KIND, BN>;
  extern __shared__ uint8_t tc_smem_raw[];
  __shared__ __align__(8) unsigned long long mbar[2];
  __shared__ uint32_t tmem_slot;
  const GemmArgs& a = ta.a;
  const long long M = dv(a.M), N = dv(a.N), K = dv(a.K);
  const long long bz = blockIdx.z;
  const long long b1 = bz / ta.nb2max, b2 = bz % ta.nb2max;
  const long long i0 = (long long)blockIdx.y * kTcRows, j0 = (long long)blockIdx.x * BN;
  if (ta.flops && bz == 0 && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0)
    atomicAdd(ta.flops, 2.0 * (double)M * (double)N * (double)K * (double)dv(a.nb1) * (double)dv(a.nb2));
  if (i0 >= M || j0 >= N || b1 >= dv(a.nb1) || b2 >= dv(a.nb2)) return;  // uniform over the CTA

  const long long sai = dv(a.sai), sak = dv(a.sak), sbk = dv(a.sbk), sbj = dv(a.sbj);
  const long long sci = dv(a.sci), scj = dv(a.scj);
  const double* A = a.A + b1 * dv(a.sa1) + b2 * dv(a.sa2);
  const double* B = a.B + b1 * dv(a.sb1) + b2 * dv(a.sb2);
  double* C = a.C + b1 * dv(a.sc1) + b2 * dv(a.sc2);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t raw = smem_u32(tc_smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gbase = tc_smem_raw + (base - raw);
  const uint32_t mb0 = smem_u32(&mbar[0]), mb1 = smem_u32(&mbar[1]);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"((uint32_t)BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(mb0);
    mbar_init(mb1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  const long long nk = (K + Cfg::kBK - 1) / Cfg::kBK;
  const uint32_t id = idesc<KIND>(BN);
  bool fail = false;
  long long last = -1;  // last chunk whose MMAs were committed
  for (long long c = 0; c < nk; ++c) {
    const int s = (int)(c & 1);
    const uint32_t mb = s ? mb1 : mb0;
    if (c >= 2 && !mbar_wait(mb, (uint32_t)(((c >> 1) - 1) & 1), ta.sync)) fail = true;
    if (__syncthreads_or(fail)) {
      fail = true;
      break;
    }
    uint8_t* st = gbase + s * Cfg::kStage;
    const long long k0 = c * Cfg::kBK;
    load_tile<KIND, kTcRows>(st, st + Cfg::kABytes, A, sai, sak, i0, M, k0, K);
    load_tile<KIND, BN>(st + Cfg::kSplit * Cfg::kABytes, st + Cfg::kSplit * Cfg::kABytes + Cfg::kBBytes, B, sbj, sbk,
                        j0, N, k0, K);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t sa = base + s * Cfg::kStage;
      const uint32_t sb = sa + Cfg::kSplit * Cfg::kABytes;
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        const uint32_t acc0 = (c > 0 || ks > 0) ? 1u : 0u;
        if constexpr (KIND == 1) {  // lo*hi + hi*lo + hi*hi, small terms first
          mma<KIND>(tmem, sdesc(sa + Cfg::kABytes + 32 * ks), sdesc(sb + 32 * ks), id, acc0);
          mma<KIND>(tmem, sdesc(sa + 32 * ks), sdesc(sb + Cfg::kBBytes + 32 * ks), id, 1u);
          mma<KIND>(tmem, sdesc(sa + 32 * ks), sdesc(sb + 32 * ks), id, 1u);
        } else {
          mma<KIND>(tmem, sdesc(sa + 32 * ks), sdesc(sb + 32 * ks), id, acc0);
        }
      }
      mma_commit(mb);
    }
    last = c;
  }
  if (!fail && last >= 0 && !mbar_wait((last & 1) ? mb1 : mb0, (uint32_t)((last >> 1) & 1), ta.sync)) fail = true;
  fail = __syncthreads_or(fail);
  tc_fence_after();
  if (!fail) {
    const long long row = i0 + warp * 32 + lane;
    const double al = a.alpha, be = a.beta;
#pragma unroll 1
    for (int cb = 0; cb < BN; cb += 32) {
      if (j0 + cb >= N) break;  // uniform over the warp
      uint32_t v[32];
      if (nk > 0) {
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb, v);
      } else {
#pragma unroll
        for (int t = 0; t < 32; ++t) v[t] = 0u;
      }
      if (row < M) {
        double* cr = C + row * sci;
#pragma unroll
        for (int t = 0; t < 32; ++t) {
          const long long j = j0 + cb + t;
          if (j < N) {
            double* cp = cr + j * scj;
            double o = al * (double)__uint_as_float(v[t]);
            if (be != 0.0) o += be * (*cp);
            *cp = o;
          }
        }
      }
    }
  } else if (last >= 0) {
    // gave up: let the MMAs already issued finish before the memory goes
    mbar_wait((last & 1) ? mb1 : mb0, (uint32_t)((last >> 1) & 1), ta.sync);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)BN) : "memory");
}

template <int KIND, int BN>
cudaError_t tc_launch(const TcArgs& ta, long long Mmax, long long Nmax, long long gz, cudaStream_t st) {
  const long long gx = (Nmax + BN - 1) / BN, gy = (Mmax + kTcRows - 1) / kTcRows;
  if (gx > 2147483647LL || gy > 65535 || gz > 65535) return cudaErrorInvalidConfiguration;
  tc_gemm_kernel<KIND, BN><<<dim3((unsigned)gx, (unsigned)gy, (unsigned)gz), kTcThreads, TcCfg<KIND, BN>::kSmem, st>>>(
      ta);
  return cudaGetLastError();
}

template <int KIND, int BN>
cudaError_t tc_attr() {
  return cudaFuncSetAttribute((const void*)tc_gemm_kernel<KIND, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              TcCfg<KIND, BN>::kSmem);
}

}  // namespace

cudaError_t gemm_tc(const GemmArgs& a, long long Mmax, long long Nmax, long long nb1max, long long nb2max, int kind,
                    int bn, DevSync* sync, cudaStream_t st) {
  if (Mmax <= 0 || Nmax <= 0 || nb1max <= 0 || nb2max <= 0) return cudaSuccess;
  if (!sync) return cudaErrorInvalidValue;
  TcArgs ta{a, nb2max, g_flop_ctr, sync};
  const long long gz = nb1max * nb2max;
#define TC_CASE(K_, BN_) \
  if (kind == K_ && bn == BN_) return tc_launch<K_, BN_>(ta, Mmax, Nmax, gz, st);
  TC_CASE(0, 64) TC_CASE(0, 128) TC_CASE(0, 256)
  TC_CASE(1, 64) TC_CASE(1, 128) TC_CASE(1, 256)
  TC_CASE(2, 64) TC_CASE(2, 128) TC_CASE(2, 256)
#undef TC_CASE
  return cudaErrorInvalidValue;
}

cudaError_t tc_init() {
  cudaError_t (*fs[])() = {tc_attr<0, 64>, tc_attr<0, 128>, tc_attr<0, 256>, tc_attr<1, 64>, tc_attr<1, 128>,
                           tc_attr<1, 256>, tc_attr<2, 64>, tc_attr<2, 128>, tc_attr<2, 256>};
  for (auto f : fs) {
    const cudaError_t e = f();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace qtt
