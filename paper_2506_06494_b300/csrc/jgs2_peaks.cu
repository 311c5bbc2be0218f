// Measured arithmetic peak of the CUDA cores, for the roofline of the ALU-bound kernels.
//
// Every thread runs eight independent fused multiply-add chains (no memory traffic inside
// the timed loop); the grid is four 256-thread blocks per SM, enough resident warps to keep
// the FMA pipes busy. FLOPs = 2 per FMA. The result buffer is written only when a thread's
// sum equals a value no chain reaches, so the chains stay live without any stores.
#include <cuda_runtime.h>

#include <string>

#include "../../include/jgs2.h"
#include "jgs2_host.h"

namespace jgs2 {
namespace {

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return fail(e_ == cudaErrorMemoryAllocation ? JGS2_ENOMEM : JGS2_ECUDA,         \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                \
  } while (0)

template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T* out, T b, T c, int iters) {
  T a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = T(1) + T(threadIdx.x * 8 + j) * T(1e-6);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int j = 0; j < 8; ++j) a[j] = fma(a[j], b, c);
  }
  T s = T(0);
#pragma unroll
  for (int j = 0; j < 8; ++j) s += a[j];
  if (s == T(-1)) out[blockIdx.x] = s;
}

template <typename T>
jgs2_status peak(double* gflops, cudaStream_t s, int iters) {
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = 4 * sms;
  T* out = nullptr;
  CK(cudaMalloc(&out, sizeof(T) * blocks));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  // b < 1 with c = (1 - b): every chain stays near 1 (no overflow, no denormals)
  const T b = T(0.9999999), c = T(1) - b;
  k_fma_peak<T><<<blocks, 256, 0, s>>>(out, b, c, iters / 8);  // warm-up
  float best = 1e30f;
  for (int rep = 0; rep < 5; ++rep) {
    CK(cudaEventRecord(e0, s));
    k_fma_peak<T><<<blocks, 256, 0, s>>>(out, b, c, iters);
    CK(cudaEventRecord(e1, s));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    best = ms < best ? ms : best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  CK(cudaGetLastError());
  const double flops = 2.0 * 8.0 * 4.0 * double(iters) * double(blocks) * 256.0;
  *gflops = flops / (double(best) * 1e-3) / 1e9;
  return JGS2_OK;
}

}  // namespace
}  // namespace jgs2

extern "C" jgs2_status jgs2_alu_peak(int32_t precision, double* gflops, void* stream) {
  using namespace jgs2;
  if (!gflops) return fail(JGS2_EINVAL, "null argument");
  if (precision == JGS2_FP32) return peak<float>(gflops, (cudaStream_t)stream, 1 << 14);
  if (precision == JGS2_FP64) return peak<double>(gflops, (cudaStream_t)stream, 1 << 10);
  return fail(JGS2_EINVAL, "bad precision");
}
