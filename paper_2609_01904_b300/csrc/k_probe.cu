// ALU throughput probe: the FP32 and FP64 fused multiply-add rates of the
// device, measured rather than derived from unit counts and clocks.  The
// SIMT kernels of the step (the FP32 cluster Jacobi, the FP64 refinement
// GEMMs, the FP64 Jacobi of the plain form) are bound by these pipes, so
// their roofline fractions are taken against the numbers this returns.
#include <algorithm>

#include "qtt_internal.cuh"

namespace qtt {
void set_last_error(const std::string& msg);
}

namespace {

constexpr int kChains = 8;   // independent FMA chains per thread (covers the pipe latency)
constexpr int kUnroll = 16;  // FMAs per chain per loop iteration

template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(T* out, long long iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = T(threadIdx.x + i) * T(1e-3);
  for (long long it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < kUnroll; ++r)
#pragma unroll
      for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  // a store the compiler cannot prove dead keeps every chain
  if (s == T(-1.25)) out[blockIdx.x] = s;
}

template <typename T>
cudaError_t probe_run(T* out, long long iters, int grid, cudaStream_t st, float* ms) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  cudaEventRecord(e0, st);
  fma_probe_kernel<T><<<grid, 256, 0, st>>>(out, iters, T(0.9999), T(1e-4));
  e = cudaGetLastError();
  cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e;
}

template <typename T>
cudaError_t probe(long long iters0, cudaStream_t st, double* tflops) {
  const int grid = qtt::device_sms() * 4;  // 32 warps per SM
  T* out = nullptr;
  cudaError_t e = cudaMalloc(&out, grid * sizeof(T));
  if (e != cudaSuccess) return e;
  float ms = 0.f;
  long long iters = iters0;
  e = probe_run<T>(out, iters, grid, st, &ms);  // warm-up and calibration
  if (e == cudaSuccess && ms > 0.f) {
    iters = std::max<long long>(1, (long long)((double)iters * 60.0 / ms));  // ~60 ms
    e = probe_run<T>(out, iters, grid, st, &ms);
  }
  if (e == cudaSuccess) {
    const double flop = 2.0 * (double)grid * 256.0 * (double)iters * kUnroll * kChains;
    *tflops = flop / (ms * 1e-3) / 1e12;
  }
  cudaFree(out);
  return e;
}

}  // namespace

extern "C" {

qtt_status qtt_peak_probe(int kind, double* tflops, void* cuda_stream) {
  if (!tflops || (kind != 0 && kind != 1)) {
    qtt::set_last_error("qtt_peak_probe: kind must be 0 (FP32) or 1 (FP64), tflops not null");
    return QTT_EINVAL;
  }
  *tflops = 0.0;
  const cudaStream_t st = (cudaStream_t)cuda_stream;
  const cudaError_t e = kind == 0 ? probe<float>(2000, st, tflops) : probe<double>(50, st, tflops);
  if (e != cudaSuccess) {
    qtt::set_last_error(std::string("qtt_peak_probe: ") + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? QTT_ENOMEM : QTT_ECUDA;
  }
  return QTT_OK;
}

}  // extern "C"
