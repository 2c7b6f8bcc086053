// Arithmetic peak probe: FP32 / FP64 fused multiply-add throughput of the current device,
// measured with CUDA events on independent FMA chains (the denominators of the roofline of
// the ALU-bound kernels: pair-arithmetic (de)gridding and the double-float FFT run on the FP32
// pipes, the FP64-arithmetic kernels on the FP64 pipe).
#include <cuda_runtime.h>

#include "wgrid_internal.h"

namespace wg {

constexpr int kProbeChains = 8;

// Each thread advances kProbeChains independent recurrences x <- x * b + c for `iters` steps
// (b slightly below 1 and c small keep the values bounded); the sum is stored so that the
// compiler keeps the work.
template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(int iters, T b, T c, T* __restrict__ out) {
  T x[kProbeChains];
#pragma unroll
  for (int i = 0; i < kProbeChains; ++i) x[i] = (T)(threadIdx.x + i) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kProbeChains; ++i) x[i] = fma(x[i], b, c);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < kProbeChains; ++i) s += x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace wg

extern "C" int wg_fma_peak(int precision, double* flops_per_s) {
  using namespace wg;
  if (flops_per_s == nullptr || (precision != WG_F32 && precision != WG_F64))
    return report_error(WG_ERR_ARG, "wg_fma_peak: bad arguments");
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return report_error(WG_ERR_CUDA, "wg_fma_peak: no current device");
  const int threads = 256, blocks = sms * 8;
  const int iters = precision == WG_F32 ? 16384 : 256;
  void* out = nullptr;
  if (cudaMalloc(&out, (size_t)blocks * threads * 8) != cudaSuccess)
    return report_error(WG_ERR_OOM, "wg_fma_peak: cudaMalloc failed");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int rc = WG_OK;
  for (int rep = 0; rep < 6 && rc == WG_OK; ++rep) {
    cudaEventRecord(e0, 0);
    if (precision == WG_F32)
      k_fma_chains<float><<<blocks, threads>>>(iters, 0.999999f, 1e-7f, (float*)out);
    else
      k_fma_chains<double><<<blocks, threads>>>(iters, 0.999999, 1e-7, (double*)out);
    cudaEventRecord(e1, 0);
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      rc = WG_ERR_CUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;   // the first launch is a warm-up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (rc != WG_OK) return report_error(rc, "wg_fma_peak: launch or synchronisation failed");
  const double flops = 2.0 * kProbeChains * (double)iters * threads * blocks;
  *flops_per_s = flops / (best * 1e-3);
  return WG_OK;
}
