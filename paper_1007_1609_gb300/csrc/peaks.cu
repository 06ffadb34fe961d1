// peaks.cu -- arithmetic peaks of this GPU, measured by the library's own
// microbenchmarks: the roofline denominators of the arithmetic-bound kernels
// (the FP64 recursion and contractions, the 3xTF32 LDOS contraction).  Not
// part of the method; the caller times one launch with CUDA events.
//
//   FP64 / FP32 FMA: every thread runs independent fused multiply-add chains
//     x <- x * a + b (a, b run-time values, so nothing folds) for `work`
//     iterations; 8 CTAs of 256 threads per SM (full occupancy), 2 flops per
//     FMA.  FP64: 8 chains whose coefficients alternate between two (a, b)
//     register pairs (when every FMA reads the same two registers the FP64
//     pipe runs at 84% of its rate); FP32: 16 chains (8 reach 93% of 16's).
//   TF32 MMA: tcgen05.mma kind::tf32 at the contraction's instruction shape,
//     one CTA per SM (contract.cu, tf32_peak_kernel), 2 M N K flops per MMA.
#include <cuda_runtime.h>

#include "../../include/cbdg.h"
#include "internal.h"

using namespace cbdg;

namespace {

constexpr int kFmaThreads = 256;
constexpr int kFmaCtasPerSm = 8;
template <typename T>
constexpr int chains() { return sizeof(T) == 8 ? 8 : 16; }

template <typename T>
__device__ T g_peak_sink;

template <typename T>
__global__ void __launch_bounds__(kFmaThreads) fma_peak_kernel(long long iters, T a, T b) {
  constexpr int C = chains<T>();
  T x[C];
#pragma unroll
  for (int j = 0; j < C; ++j) x[j] = static_cast<T>(threadIdx.x + j) * static_cast<T>(1e-3);
  const T a2 = a * static_cast<T>(0.5), b2 = b * static_cast<T>(2);
#pragma unroll 4
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < C; ++j) {
      if constexpr (sizeof(T) == 8)
        x[j] = fma(x[j], (j & 1) ? a : a2, (j & 2) ? b : b2);
      else
        x[j] = fma(x[j], a, b);
    }
  }
  T s = x[0];
#pragma unroll
  for (int j = 1; j < C; ++j) s += x[j];
  // a store the compiler cannot rule out keeps every chain alive
  if (s == a) g_peak_sink<T> = s;
}

// error word of the probes
__device__ unsigned g_peak_flag;

cbdg_status pfail(cbdg_status st, const char *msg) {
  cbdg_internal_set_error(msg);
  return st;
}

}  // namespace

extern "C" cbdg_status cbdg_measure_peak(int32_t kind, int64_t work, cbdg_stream stream, double *flops) {
  if (!flops) return pfail(CBDG_ERR_INVALID_ARG, "flops is NULL");
  if (work < 1 || work > (1LL << 40)) return pfail(CBDG_ERR_INVALID_ARG, "work must be in [1, 2^40]");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return pfail(CBDG_ERR_CUDA, "no CUDA device");
  cudaError_t e = cudaSuccess;
  if (kind == CBDG_PEAK_FP64_FMA || kind == CBDG_PEAK_FP32_FMA) {
    const int ctas = sms * kFmaCtasPerSm;
    int C;
    if (kind == CBDG_PEAK_FP64_FMA) {
      fma_peak_kernel<double><<<ctas, kFmaThreads, 0, s>>>(work, 0.999999, 1e-7);
      C = chains<double>();
    } else {
      fma_peak_kernel<float><<<ctas, kFmaThreads, 0, s>>>(work, 0.999999f, 1e-7f);
      C = chains<float>();
    }
    e = cudaGetLastError();
    *flops = 2.0 * C * static_cast<double>(work) * ctas * kFmaThreads;
  } else if (kind == CBDG_PEAK_TF32_MMA) {
    unsigned *flag = nullptr;
    e = cudaGetSymbolAddress(reinterpret_cast<void **>(&flag), g_peak_flag);
    if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) e = launch_tf32_peak(sms, work, flag, s);
    *flops = tf32_peak_flops_per_mma() * static_cast<double>(work) * sms;
  } else {
    return pfail(CBDG_ERR_INVALID_ARG, "unknown peak kind");
  }
  if (e != cudaSuccess) return pfail(CBDG_ERR_CUDA, cudaGetErrorString(e));
  return CBDG_OK;
}

extern "C" cbdg_status cbdg_peak_status(cbdg_stream stream) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  unsigned h = 0;
  unsigned *flag = nullptr;
  cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void **>(&flag), g_peak_flag);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return pfail(CBDG_ERR_CUDA, cudaGetErrorString(e));
  if (h & kFlagTimeout) return pfail(CBDG_ERR_CUDA, "the tensor-core probe gave up waiting for its MMAs");
  return CBDG_OK;
}
