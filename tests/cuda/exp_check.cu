// Accuracy of the table-driven exponential (fast_exp.cuh) against CUDA's exp
// over [-700, 700] (2^28 points of a uniform grid: the largest difference in
// units in the last place) and against the host's long-double expl on 2^20
// random points (the largest relative error), plus its exact cases and the
// range test. Prints one line per check; exits non-zero on a failure.
#include <cstdio>
#include <cstdint>
#include <cmath>
#include <vector>
#include <random>
#include <cuda_runtime.h>
#include "fast_exp.cuh"
using namespace hpac;

__constant__ ExpTang c_ex;

__global__ void grid_ulp(unsigned long long n, unsigned long long *worst) {
  __shared__ double tab[64];
  for (int t = threadIdx.x; t < 64; t += blockDim.x) tab[t] = c_ex.t[t];
  __syncthreads();
  unsigned long long w = 0;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const double x = -700.0 + 1400.0 * ((double)i + 0.5) / (double)n;
    const long long a = __double_as_longlong(exp_tang(x, tab, c_ex.inv_l, c_ex.l1, c_ex.l2));
    const long long b = __double_as_longlong(exp(x));
    const unsigned long long d = (unsigned long long)(a > b ? a - b : b - a);
    w = d > w ? d : w;
  }
  atomicMax(worst, w);
}

__global__ void values(const double *x, double *y, int n) {
  __shared__ double tab[64];
  for (int t = threadIdx.x; t < 64; t += blockDim.x) tab[t] = c_ex.t[t];
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = exp_tang(x[i], tab, c_ex.inv_l, c_ex.l1, c_ex.l2);
}

__global__ void ranges(const double *x, int *ok, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) ok[i] = exp_tang_in_range(x[i]) ? 1 : 0;
}

int main() {
  const ExpTang ex = exp_tang_constants();
  cudaMemcpyToSymbol(c_ex, &ex, sizeof ex);
  int fails = 0;
  // 1. against CUDA's exp on a grid
  unsigned long long *dw, hw = 0;
  cudaMalloc(&dw, sizeof *dw);
  cudaMemset(dw, 0, sizeof *dw);
  grid_ulp<<<1216, 256>>>(1ull << 28, dw);
  cudaMemcpy(&hw, dw, sizeof hw, cudaMemcpyDeviceToHost);
  printf("grid max ulp vs CUDA exp %llu\n", hw);
  fails += hw > 2;
  // 2. against expl on random points, and the exact cases
  const int n = 1 << 20, ns = 6;
  std::vector<double> hx(n + ns), hy(n + ns);
  std::mt19937_64 g(2308);
  std::uniform_real_distribution<double> u(-700.0, 700.0);
  for (int i = 0; i < n; ++i) hx[i] = u(g);
  const double special[ns] = {0.0, -0.0, 1e-300, -1e-300, 700.0, -700.0};
  for (int i = 0; i < ns; ++i) hx[n + i] = special[i];
  double *dx, *dy;
  cudaMalloc(&dx, (n + ns) * sizeof(double));
  cudaMalloc(&dy, (n + ns) * sizeof(double));
  cudaMemcpy(dx, hx.data(), (n + ns) * sizeof(double), cudaMemcpyHostToDevice);
  values<<<(n + ns + 255) / 256, 256>>>(dx, dy, n + ns);
  cudaMemcpy(hy.data(), dy, (n + ns) * sizeof(double), cudaMemcpyDeviceToHost);
  double worst = 0.0;
  for (int i = 0; i < n + ns; ++i) {
    const long double r = expl((long double)hx[i]);
    const double e = (double)fabsl(((long double)hy[i] - r) / r);
    worst = e > worst ? e : worst;
  }
  printf("max relative error vs expl %.3e\n", worst);
  fails += !(worst <= 4e-16);
  const bool ones = hy[n] == 1.0 && hy[n + 1] == 1.0 && hy[n + 2] == 1.0 && hy[n + 3] == 1.0;
  printf("exp of zero and of +-1e-300 is one %s\n", ones ? "yes" : "no");
  fails += !ones;
  // 3. the range test
  const double rx[6] = {700.0, -700.0, std::nextafter(700.0, 1e300), -std::nextafter(700.0, 1e300), NAN, INFINITY};
  const int expect[6] = {1, 1, 0, 0, 0, 0};
  int *dok, hok[6];
  cudaMemcpy(dx, rx, sizeof rx, cudaMemcpyHostToDevice);
  cudaMalloc(&dok, sizeof hok);
  ranges<<<1, 32>>>(dx, dok, 6);
  cudaMemcpy(hok, dok, sizeof hok, cudaMemcpyDeviceToHost);
  int rbad = 0;
  for (int i = 0; i < 6; ++i) rbad += hok[i] != expect[i];
  printf("range test mismatches %d\n", rbad);
  fails += rbad != 0;
  const cudaError_t e = cudaDeviceSynchronize();
  printf("cuda %s\n", cudaGetErrorString(e));
  return fails || e != cudaSuccess ? 1 : 0;
}
