// Device measurement utility: the double-precision FMA rate of this GPU, the
// ceiling of the FP64-bound hydro kernels. Each thread runs 8 independent FMA
// chains (enough to cover the pipe latency) on a grid of 8 blocks per SM.
#include "hpac_internal.cuh"

namespace hpac {
namespace {

__global__ void __launch_bounds__(256) fp64_fma_chains(double *out, int iters) {
  double a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = 1.0 + 1e-9 * (threadIdx.x + 7 * j);
  const double b = 0.9999999999, c = 1e-12;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = fma(a[j], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += a[j];
  if (s == 12345.678) out[0] = s;  // never true; keeps the chains live
}

}  // namespace
}  // namespace hpac

using namespace hpac;

extern "C" hpac_status hpac_device_fp64_rate(double *h_tflops, void *cuda_stream) {
  if (!h_tflops) return set_error(HPAC_EINVAL, "h_tflops is NULL");
  int dev = 0, sms = 0;
  HPAC_CUDA_TRY(cudaGetDevice(&dev));
  HPAC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  double *out = nullptr;
  HPAC_CUDA_TRY(cudaMalloc(&out, sizeof(double)));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = sms * 8, threads = 256, iters = 8192;
  fp64_fma_chains<<<blocks, threads, 0, st>>>(out, 256);  // warm-up
  cudaEventRecord(e0, st);
  fp64_fma_chains<<<blocks, threads, 0, st>>>(out, iters);
  cudaEventRecord(e1, st);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess) return cuda_error(err, "hpac_device_fp64_rate");
  const double fmas = (double)blocks * threads * 8.0 * iters;
  *h_tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
  return HPAC_OK;
}
