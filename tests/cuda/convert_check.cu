// Bit-exactness of the integer-pipe precision conversions (convert.cuh, both
// double-to-single variants) against the hardware conversions: every single-precision input, and 2^30
// doubles of each of five kinds over the whole range. Prints one line per
// case and exits non-zero on any mismatch.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>
#include "convert.cuh"
using namespace hpac;
__device__ __forceinline__ uint64_t mix(uint64_t x) {
  x ^= x >> 33; x *= 0xff51afd7ed558ccdull; x ^= x >> 33; x *= 0xc4ceb9fe1a85ec53ull; x ^= x >> 33; return x;
}
__global__ void f2d(unsigned long long *bad, unsigned long long *first) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < (1ull << 32); i += (uint64_t)gridDim.x * blockDim.x) {
    const float f = __uint_as_float((uint32_t)i);
    const double a = float_to_double(f), b = (double)f;
    if (__double_as_longlong(a) != __double_as_longlong(b)) {
      if (atomicAdd(bad, 1ull) == 0) { first[0] = i; first[1] = __double_as_longlong(a); first[2] = __double_as_longlong(b); }
    }
  }
}
__global__ void d2f(int kind, unsigned long long *bad, unsigned long long *first) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < (1ull << 30); i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t r = mix(i + ((uint64_t)kind << 40));
    uint64_t u;
    if (kind == 0) u = r;                                                               // any bits
    else if (kind == 1) u = (r & 0x800fffffffffffffull) | ((uint64_t)(1023 - 160 + (r >> 52) % 320) << 52);  // around the single range
    else if (kind == 2) u = (r & 0x800fffffe0000000ull) | ((uint64_t)(1023 + (int)((r >> 56) % 200) - 100) << 52) | (((r >> 8) & 1) << 28);  // ties
    else if (kind == 3) u = (r & 0x8000000000000000ull) | ((uint64_t)(1023 - 127 - (r >> 52) % 30) << 52) | (r & 0xfffffffffffffull);  // single subnormal range
    else { const uint64_t e = 1023 - 127 - (r >> 52) % 30; u = (r & 0x8000000000000000ull) | (e << 52) | (r & 0xfffffe0000000ull) | ((r & 1) << 28); }  // subnormal ties
    const double x = __longlong_as_double((long long)u);
    const float a = double_to_float_rn(x), b = __double2float_rn(x), c = double_to_float_rn_novote(x);
    if (__float_as_uint(a) != __float_as_uint(b) || __float_as_uint(c) != __float_as_uint(b)) {
      if (atomicAdd(bad, 1ull) == 0) { first[0] = u; first[1] = __float_as_uint(a); first[2] = __float_as_uint(b); }
    }
  }
}
int main() {
  int sms; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  unsigned long long *bad, *first, hb, f[3], total = 0;
  cudaMalloc(&bad, 8); cudaMalloc(&first, 24);
  cudaMemset(bad, 0, 8); cudaMemset(first, 0, 24);
  f2d<<<sms * 8, 256>>>(bad, first);
  cudaMemcpy(&hb, bad, 8, cudaMemcpyDeviceToHost); cudaMemcpy(f, first, 24, cudaMemcpyDeviceToHost);
  total += hb;
  printf("float->double, all 2^32 inputs: mismatches %llu", hb);
  if (hb) printf(" first %08llx emul %016llx hw %016llx", f[0], f[1], f[2]);
  printf("\n");
  for (int k = 0; k < 5; ++k) {
    cudaMemset(bad, 0, 8); cudaMemset(first, 0, 24);
    d2f<<<sms * 8, 256>>>(k, bad, first);
    cudaMemcpy(&hb, bad, 8, cudaMemcpyDeviceToHost); cudaMemcpy(f, first, 24, cudaMemcpyDeviceToHost);
    total += hb;
    printf("double->float kind %d, 2^30 inputs: mismatches %llu", k, hb);
    if (hb) printf(" first %016llx emul %08llx hw %08llx", f[0], f[1], f[2]);
    printf("\n");
  }
  const cudaError_t err = cudaGetLastError();
  printf("status %s\n", cudaGetErrorString(err));
  return (err != cudaSuccess || total) ? 1 : 0;
}
