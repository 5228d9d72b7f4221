// Measured issue rates of the ALU work the force kernel does, for its
// roofline: register-only loops timed with CUDA events on the caller's
// stream.
//   FP32: fused multiply-adds, eight independent chains per thread.
//   pair noise: Philox-4x32-R words (the generator of the pair noise, Sec.
//     2.1, with its 32 x 32 -> 64-bit products), four independent counters
//     per thread, the same device function the force kernels call.
#include <cuda_runtime.h>

#include <cstdint>

#include "dpd.h"
#include "dpd_device.cuh"
#include "engine.h"

namespace dpd {
namespace {

constexpr int kPeakThreads = 256;

__global__ void __launch_bounds__(kPeakThreads) k_peak_fma(float *out, int iters, float a,
                                                           float b) {
  float x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = threadIdx.x * 1e-3f + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fmaf(x[k], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == 1234.5f) out[threadIdx.x] = s;  // keeps the chains live
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_philox(uint32_t *out, int iters,
                                                              uint32_t k0, uint32_t k1) {
  const uint32_t t = blockIdx.x * kPeakThreads + threadIdx.x;
  uint32_t acc = 0u;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      acc ^= philox_word0(t, (uint32_t)(4 * i + k), (uint32_t)i, 0u, k0, k1);
  }
  if (acc == 0x12345678u) out[threadIdx.x] = acc;
}

}  // namespace
}  // namespace dpd

extern "C" int dpd_issue_rates(double rates[2], void *stream) {
  using namespace dpd;
  clear_error();
  if (!rates) return set_error(DPD_ERR_ARG, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  DPD_CUDA_TRY(cudaGetDevice(&dev));
  DPD_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8;  // eight resident blocks of 256 threads per SM
  void *buf = nullptr;
  DPD_CUDA_TRY(cudaMalloc(&buf, kPeakThreads * sizeof(float)));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float ms_fma = 0.f, ms_phx = 0.f;
  const int it_fma = 8192, it_phx = 256;
  for (int rep = 0; e == cudaSuccess && rep < 2; ++rep) {  // the first pass warms up
    k_peak_fma<<<blocks, kPeakThreads, 0, s>>>((float *)buf, it_fma, 1.0001f, 0.5f);
    if ((e = cudaEventRecord(e0, s)) != cudaSuccess) break;
    k_peak_fma<<<blocks, kPeakThreads, 0, s>>>((float *)buf, it_fma, 1.0001f, 0.5f);
    if ((e = cudaEventRecord(e1, s)) != cudaSuccess) break;
    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
    if ((e = cudaEventElapsedTime(&ms_fma, e0, e1)) != cudaSuccess) break;
    k_peak_philox<<<blocks, kPeakThreads, 0, s>>>((uint32_t *)buf, it_phx, 7u, 9u);
    if ((e = cudaEventRecord(e0, s)) != cudaSuccess) break;
    k_peak_philox<<<blocks, kPeakThreads, 0, s>>>((uint32_t *)buf, it_phx, 7u, 9u);
    if ((e = cudaEventRecord(e1, s)) != cudaSuccess) break;
    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
    e = cudaEventElapsedTime(&ms_phx, e0, e1);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(buf);
  if (e != cudaSuccess) return set_error(DPD_ERR_CUDA, "issue rates: %s", cudaGetErrorString(e));
  const double threads = (double)blocks * kPeakThreads;
  rates[0] = threads * 8.0 * it_fma / (ms_fma * 1e-3);  // FP32 FMA lane-ops/s
  rates[1] = threads * 4.0 * it_phx / (ms_phx * 1e-3);  // Philox words/s
  return DPD_OK;
}
