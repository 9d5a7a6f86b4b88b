// Arithmetic-throughput probe: the FP32 and FP64 fused multiply-add rates of
// the device, measured with CUDA events.  These are the denominators of the
// ALU roofline of the energy/force kernels (FP32 on the mixed path, FP64 on
// the FP64 path).  The probe changes no device setting.
//
// Each thread runs kChains independent multiply-add chains (enough to cover
// the FMA latency with a few resident warps per scheduler) for `iters`
// iterations; multiplier and addend come from kernel arguments so nothing
// folds at compile time, and the chains' sum is stored so nothing is removed.
// The grid is a whole number of blocks per SM.
#include <cuda_runtime.h>

#include "mtp_internal.cuh"

namespace mtp {
namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;

template <class T>
__global__ void __launch_bounds__(kProbeThreads) fma_probe_kernel(T b, T c, int64_t iters, T* out) {
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = T(threadIdx.x + k);
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll 16
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
    }
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Packed FP32 pairs (fma.rn.f32x2, one instruction for two lanes' worth of
// FP32 multiply-adds per thread).
__global__ void __launch_bounds__(kProbeThreads) ffma2_probe_kernel(float b, float c, int64_t iters, float* out) {
  unsigned long long a[kChains / 2];
  unsigned long long bb, cc;
  asm("mov.b64 %0, {%1, %1};" : "=l"(bb) : "f"(b));
  asm("mov.b64 %0, {%1, %1};" : "=l"(cc) : "f"(c));
#pragma unroll
  for (int k = 0; k < kChains / 2; ++k) {
    const float lo = (float)(threadIdx.x + 2 * k), hi = (float)(threadIdx.x + 2 * k + 1);
    asm("mov.b64 %0, {%1, %2};" : "=l"(a[k]) : "f"(lo), "f"(hi));
  }
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll 16
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int k = 0; k < kChains / 2; ++k) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[k]) : "l"(bb), "l"(cc));
    }
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains / 2; ++k) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a[k]));
    s += lo + hi;
  }
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace mtp

extern "C" int mtp_probe_fma(int32_t kind, int64_t iters, int32_t blocks_per_sm, double* flops_per_s, double* ms) {
  using namespace mtp;
  if (kind < 0 || kind > 2 || iters <= 0 || blocks_per_sm <= 0 || blocks_per_sm > 32 || !flops_per_s || !ms) {
    set_error("mtp_probe_fma: kind must be 0 (FP32), 1 (FP64) or 2 (packed FP32), iters > 0, 1..32 blocks per SM");
    return MTP_ERR_ARG;
  }
  int dev = 0, sms = 0;
  MTP_TRY_CUDA(cudaGetDevice(&dev));
  MTP_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const unsigned grid = (unsigned)(sms * blocks_per_sm);
  const size_t n = (size_t)grid * kProbeThreads;
  void* out = nullptr;
  MTP_TRY_CUDA(cudaMalloc(&out, n * sizeof(double)));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = MTP_OK;
  float t = 0.f;
  auto launch = [&]() {
    if (kind == 0) fma_probe_kernel<float><<<grid, kProbeThreads>>>(0.9999999f, 1e-7f, iters, (float*)out);
    else if (kind == 1) fma_probe_kernel<double><<<grid, kProbeThreads>>>(0.9999999, 1e-7, iters, (double*)out);
    else ffma2_probe_kernel<<<grid, kProbeThreads>>>(0.9999999f, 1e-7f, iters, (float*)out);
  };
  do {
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) { rc = MTP_ERR_CUDA; break; }
    launch();   // warm-up (clocks ramp, code loaded)
    if (cudaEventRecord(e0) != cudaSuccess) { rc = MTP_ERR_CUDA; break; }
    launch();
    if (cudaEventRecord(e1) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) { rc = MTP_ERR_CUDA; break; }
    if (cudaGetLastError() != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) { rc = MTP_ERR_CUDA; break; }
  } while (0);
  if (rc != MTP_OK) set_error("mtp_probe_fma: %s", cudaGetErrorString(cudaGetLastError()));
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (rc != MTP_OK) return rc;
  const double fma_per_thread = (double)iters * 16.0 * kChains;
  *ms = t;
  *flops_per_s = 2.0 * fma_per_thread * (double)n / (t * 1e-3);
  return MTP_OK;
}
