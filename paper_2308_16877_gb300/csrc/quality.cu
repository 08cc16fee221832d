// Quality loss against an exact reference (Section 4): MAPE (Eq. 1), RMSE and
// the misclassification rate MCR (Eq. 2), accumulated in double precision.
//
// Two deterministic passes: a grid of blocks reduces grid-stride slices to
// per-block partials (a tree inside each block), then one block reduces the
// partials in index order. Two entry points differ only in where the partials
// live:
//  - hpac_quality: a device buffer of kBlocks + 1 partials, allocated with
//    cudaMalloc on a device's first call and kept for the life of the process;
//    a host mutex serializes calls, which wait for their result.
//  - hpac_quality_noalloc: a fixed static __device__ array of kStaticPartials
//    + 1 partials compiled into the library, addressed through a per-device
//    cache of its device address; no lock (callers serialize overlapping
//    calls themselves, see hpac.h).
// Both per-device caches hold device addresses of the primary context: they
// assume that context is not reset (cudaDeviceReset) while the process uses
// the library.
#include <math.h>
#include <mutex>

#include "hpac_internal.cuh"
#include "convert.cuh"

namespace hpac {
namespace {

constexpr int kBlocks = 1216;  // 8 x 152 SMs
constexpr int kThreads = 256;

struct Partial {
  double sum;
  double zmax;
  unsigned long long used;
  unsigned long long zeros;
  unsigned long long zbad;
};

template <typename B, int METRIC>
__global__ void __launch_bounds__(kThreads) quality_partial(const double *__restrict__ a,
                                                            const void *__restrict__ bv_, int64_t n,
                                                            Partial *__restrict__ part) {
  const B *__restrict__ b = static_cast<const B *>(bv_);
  constexpr int metric = METRIC;
  __shared__ double s_sum[kThreads];
  __shared__ double s_zmax[kThreads];
  __shared__ unsigned long long s_used[kThreads], s_zeros[kThreads], s_zbad[kThreads];
  double sum = 0.0;
  unsigned long long zmax = 0;  // bits of the largest |b| where a == 0 (NaN skipped, as fmax does)
  unsigned long long used = 0, zeros = 0, zbad = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // GB300 issues one double-precision warp instruction per 16 cycles per SM, so
  // the per-element work keeps a single FP64 operation (the difference a - b,
  // exact for the single-precision approximations; for MCR the comparison).
  // The conversions between the precisions and the range tests of the exact
  // value run on the integer pipes (the same bits as the hardware conversions
  // and comparisons), the ratio or square is formed in single precision, and the
  // terms are summed in groups of 16 before entering the double-precision
  // accumulator. For MAPE the exact value and the difference are first scaled
  // by the same power of two (an exact change of their exponent fields), so
  // the single-precision ratio covers every finite exact value; only ratios
  // above 2^126 and subnormal operands take the double-precision division.
  // Each thread walks its grid-stride sequence four elements at a
  // time, the four loads issued before the first is used (the same elements
  // in the same order as one at a time, so the same sums).
  float chunk = 0.0f;
  int in_chunk = 0;
  auto element = [&](double ai, B braw) {
    double bi;
    if (sizeof(B) == 4)
      bi = float_to_double((float)braw);
    else
      bi = (double)braw;
    const uint64_t aabs = (uint64_t)__double_as_longlong(ai) & 0x7fffffffffffffffull;
    float term;
    if (metric == HPAC_METRIC_MAPE) {
      if (aabs == 0ull) {
        const uint64_t babs = (uint64_t)__double_as_longlong(bi) & 0x7fffffffffffffffull;
        ++zeros;
        if (babs != 0ull) ++zbad;
        if (babs <= 0x7ff0000000000000ull && babs > zmax) zmax = babs;
        return;
      }
      // |d| / |a| with both scaled by the power of two that puts |a| in
      // [1, 2) (exact, on the exponent fields), then rounded to single
      // precision and divided there; a ratio below 2^-1021 rounds to zero
      // the one FP64 operation; the opaque move keeps the compiler from
      // recomputing it where d is used again
      uint64_t dbits;
      asm volatile("mov.b64 %0, %1;" : "=l"(dbits) : "d"(ai - bi));
      const double d = __longlong_as_double((long long)dbits);
      const uint64_t dabs = dbits & 0x7fffffffffffffffull;
      const int ea = (int)(aabs >> 52), ed = (int)(dabs >> 52), rel = ed - ea;
      if (ea != 0 && ea != 0x7ff && ed != 0x7ff && (ed != 0 || dabs == 0ull) && rel <= 126) {
        float fd = 0.0f;
        if (dabs != 0ull && rel >= -1022)
          fd = double_to_float_rn(__longlong_as_double(
              (long long)((dabs & 0xfffffffffffffull) | ((uint64_t)(rel + 1023) << 52))));
        const uint32_t fa_frac = (uint32_t)((aabs >> 29) & 0x7fffffu), fa_rem = (uint32_t)(aabs & 0x1fffffffu);
        const float fa = __uint_as_float((127u << 23) + fa_frac +
                                         ((fa_rem > 0x10000000u) | ((fa_rem == 0x10000000u) & (fa_frac & 1u))));
        term = __fdiv_rn(fd, fa);
      } else {
        sum += fabs(d) / fabs(ai);
        ++used;
        return;
      }
    } else if (metric == HPAC_METRIC_RMSE) {
      uint64_t dbits;
      asm volatile("mov.b64 %0, %1;" : "=l"(dbits) : "d"(ai - bi));
      const float d = double_to_float_rn(__longlong_as_double((long long)dbits));
      term = d * d;
    } else {
      term = (ai != bi) ? 1.0f : 0.0f;
    }
    chunk += term;
    ++used;
    if (++in_chunk == 16) {
      sum += float_to_double(chunk);
      chunk = 0.0f;
      in_chunk = 0;
    }
  };
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += 4 * stride) {
    double av[4];
    B bv[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t i = i0 + k * stride;
      if (i < n) {
        av[k] = __ldcs(a + i);
        bv[k] = __ldcs(b + i);
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (i0 + k * stride < n) element(av[k], bv[k]);
  }
  sum += float_to_double(chunk);
  s_sum[threadIdx.x] = sum;
  s_zmax[threadIdx.x] = __longlong_as_double((long long)zmax);
  s_used[threadIdx.x] = used;
  s_zeros[threadIdx.x] = zeros;
  s_zbad[threadIdx.x] = zbad;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      s_sum[threadIdx.x] += s_sum[threadIdx.x + w];
      s_zmax[threadIdx.x] = fmax(s_zmax[threadIdx.x], s_zmax[threadIdx.x + w]);
      s_used[threadIdx.x] += s_used[threadIdx.x + w];
      s_zeros[threadIdx.x] += s_zeros[threadIdx.x + w];
      s_zbad[threadIdx.x] += s_zbad[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[blockIdx.x] = Partial{s_sum[0], s_zmax[0], s_used[0], s_zeros[0], s_zbad[0]};
  }
}

// The partial-sum kernel for an approximation type and a metric (one
// instantiation each, so a metric's unused paths are not compiled in).
using PartialKernel = void (*)(const double *, const void *, int64_t, Partial *);
PartialKernel partial_kernel(int32_t approx_dtype, int32_t metric) {
  if (approx_dtype == HPAC_F32) {
    if (metric == HPAC_METRIC_MAPE) return quality_partial<float, HPAC_METRIC_MAPE>;
    if (metric == HPAC_METRIC_RMSE) return quality_partial<float, HPAC_METRIC_RMSE>;
    return quality_partial<float, HPAC_METRIC_MCR>;
  }
  if (metric == HPAC_METRIC_MAPE) return quality_partial<double, HPAC_METRIC_MAPE>;
  if (metric == HPAC_METRIC_RMSE) return quality_partial<double, HPAC_METRIC_RMSE>;
  return quality_partial<double, HPAC_METRIC_MCR>;
}

__global__ void __launch_bounds__(kThreads) quality_final(const Partial *__restrict__ part, int np,
                                                          Partial *__restrict__ res) {
  __shared__ Partial s[kThreads];
  Partial acc{0.0, 0.0, 0, 0, 0};
  for (int j = threadIdx.x; j < np; j += blockDim.x) {
    const Partial p = part[j];
    acc.sum += p.sum;
    acc.zmax = fmax(acc.zmax, p.zmax);
    acc.used += p.used;
    acc.zeros += p.zeros;
    acc.zbad += p.zbad;
  }
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      s[threadIdx.x].sum += s[threadIdx.x + w].sum;
      s[threadIdx.x].zmax = fmax(s[threadIdx.x].zmax, s[threadIdx.x + w].zmax);
      s[threadIdx.x].used += s[threadIdx.x + w].used;
      s[threadIdx.x].zeros += s[threadIdx.x + w].zeros;
      s[threadIdx.x].zbad += s[threadIdx.x + w].zbad;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *res = s[0];
}

// Per-device scratch: kBlocks partials + 1 result.
Partial *g_scratch[64] = {nullptr};
std::mutex g_mu;

// Callers hold g_mu for the whole call: the scratch is shared by every call
// on the device and the call waits for its result before releasing it.
hpac_status scratch_for(int dev, Partial **out) {
  if (dev < 0 || dev >= 64) return set_error(HPAC_EUNSUPPORTED, "device ordinal %d", dev);
  if (!g_scratch[dev]) {
    Partial *p = nullptr;
    cudaError_t e = cudaMalloc(&p, (kBlocks + 1) * sizeof(Partial));
    if (e != cudaSuccess) return cuda_error(e, "hpac_quality scratch");
    g_scratch[dev] = p;
  }
  *out = g_scratch[dev];
  return HPAC_OK;
}

}  // namespace
}  // namespace hpac

using namespace hpac;

extern "C" hpac_status hpac_quality(int32_t approx_dtype, int64_t n, const double *d_exact,
                                    const void *d_approx, int32_t metric,
                                    hpac_quality_result *h_result, void *cuda_stream) {
  TraceRange trace_("hpac_quality");
  if (!h_result) return set_error(HPAC_EINVAL, "h_result is NULL");
  if (n < 0) return set_error(HPAC_EINVAL, "n < 0");
  if (metric < HPAC_METRIC_MAPE || metric > HPAC_METRIC_MCR)
    return set_error(HPAC_EINVAL, "metric %d", metric);
  if (approx_dtype != HPAC_F32 && approx_dtype != HPAC_F64)
    return set_error(HPAC_EINVAL, "dtype %d", approx_dtype);
  if (n > 0 && (!d_exact || !d_approx)) return set_error(HPAC_EINVAL, "NULL data pointer");
  *h_result = hpac_quality_result{0.0, 0.0, 0, 0, 0};
  if (n == 0) return HPAC_OK;
  int dev = 0;
  HPAC_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_mu);
  Partial *scr = nullptr;
  hpac_status s = scratch_for(dev, &scr);
  if (s != HPAC_OK) return s;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // one wave of resident blocks (at most kBlocks): every thread's sequence
  // runs to the end without a second, partly filled wave
  const PartialKernel fn = partial_kernel(approx_dtype, metric);
  int per_sm = 0, sms = 0;
  HPAC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, 0));
  HPAC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t wave = (int64_t)(per_sm > 0 ? per_sm : 1) * sms;
  int64_t blocks = (n + kThreads - 1) / kThreads;
  if (blocks > wave) blocks = wave;
  if (blocks > kBlocks) blocks = kBlocks;
  fn<<<(unsigned)blocks, kThreads, 0, st>>>(d_exact, d_approx, n, scr);
  HPAC_CUDA_TRY(cudaGetLastError());
  quality_final<<<1, kThreads, 0, st>>>(scr, (int)blocks, scr + kBlocks);
  HPAC_CUDA_TRY(cudaGetLastError());
  Partial res;
  HPAC_CUDA_TRY(cudaMemcpyAsync(&res, scr + kBlocks, sizeof(Partial), cudaMemcpyDeviceToHost, st));
  HPAC_CUDA_TRY(cudaStreamSynchronize(st));
  double v = res.used ? res.sum / (double)res.used : 0.0;
  if (metric == HPAC_METRIC_RMSE) v = sqrt(v);
  h_result->value = v;
  h_result->zero_max_abs = res.zmax;
  h_result->used = (int64_t)res.used;
  h_result->zeros = (int64_t)res.zeros;
  h_result->zeros_mismatch = (int64_t)res.zbad;
  return HPAC_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of hpac_quality.
//
// Its scratch is a fixed array compiled into the library instead of a buffer
// obtained from cudaMalloc: every GPU that loads the library holds these
// 16,385 partials (about 656 KB) until the process exits. The reduction runs
// ceil(n / 8192) blocks of the same partial kernel (each thread reduces at most
// 32 elements) followed by the same final kernel, so n may not exceed
// 16,384 * 8,192 = 134,217,728 elements.
// ---------------------------------------------------------------------------
namespace hpac {
namespace {

constexpr int64_t kStaticTile = (int64_t)kThreads * 32;          // elements per block
constexpr int kStaticPartials = 16384;                            // blocks at most
constexpr int64_t kStaticMaxN = kStaticTile * kStaticPartials;    // 134,217,728

static __device__ __align__(256) Partial g_static_scratch[kStaticPartials + 1];

// Device address of g_static_scratch per device ordinal, looked up once with
// that device current (host code may not use the symbol itself as a pointer).
Partial *g_static_addr[64] = {nullptr};
std::mutex g_static_mu;

hpac_status static_scratch(int dev, Partial **out) {
  if (dev < 0 || dev >= 64) return set_error(HPAC_EUNSUPPORTED, "device ordinal %d", dev);
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(g_static_scratch)");
    g_static_addr[dev] = static_cast<Partial *>(p);
  }
  *out = g_static_addr[dev];
  return HPAC_OK;
}

}  // namespace
}  // namespace hpac

extern "C" hpac_status hpac_quality_noalloc(int32_t approx_dtype, int64_t n, const double *d_exact,
                                            const void *d_approx, int32_t metric,
                                            hpac_quality_result *h_result, void *cuda_stream) {
  TraceRange trace_("hpac_quality_noalloc");
  if (!h_result) return set_error(HPAC_EINVAL, "h_result is NULL");
  if (n < 0) return set_error(HPAC_EINVAL, "n < 0");
  if (n > kStaticMaxN)
    return set_error(HPAC_EINVAL,
                     "hpac_quality_noalloc: n = %lld exceeds the %lld-element limit of its fixed "
                     "scratch; use hpac_quality for larger inputs",
                     (long long)n, (long long)kStaticMaxN);
  if (metric < HPAC_METRIC_MAPE || metric > HPAC_METRIC_MCR)
    return set_error(HPAC_EINVAL, "metric %d", metric);
  if (approx_dtype != HPAC_F32 && approx_dtype != HPAC_F64)
    return set_error(HPAC_EINVAL, "dtype %d", approx_dtype);
  if (n > 0 && (!d_exact || !d_approx)) return set_error(HPAC_EINVAL, "NULL data pointer");
  *h_result = hpac_quality_result{0.0, 0.0, 0, 0, 0};
  int dev = 0;
  HPAC_CUDA_TRY(cudaGetDevice(&dev));
  Partial *scr = nullptr;
  hpac_status s = static_scratch(dev, &scr);
  if (s != HPAC_OK) return s;
  if (n == 0) {
    // The warm-up call: besides the address lookup above, make the runtime
    // load the kernels now (with lazy module loading they would load, and
    // allocate device memory for their code, at their first launch).
    cudaFuncAttributes fa;
    for (int32_t dt : {HPAC_F32, HPAC_F64})
      for (int32_t m : {HPAC_METRIC_MAPE, HPAC_METRIC_RMSE, HPAC_METRIC_MCR})
        HPAC_CUDA_TRY(cudaFuncGetAttributes(&fa, partial_kernel(dt, m)));
    HPAC_CUDA_TRY(cudaFuncGetAttributes(&fa, quality_final));
    return HPAC_OK;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // Every partial slot the final kernel reads is written earlier in this call,
  // so nothing left in the shared array by a previous call is used.
  const int64_t blocks = (n + kStaticTile - 1) / kStaticTile;
  partial_kernel(approx_dtype, metric)<<<(unsigned)blocks, kThreads, 0, st>>>(d_exact, d_approx, n, scr);
  HPAC_CUDA_TRY(cudaGetLastError());
  quality_final<<<1, kThreads, 0, st>>>(scr, (int)blocks, scr + kStaticPartials);
  HPAC_CUDA_TRY(cudaGetLastError());
  Partial res;
  HPAC_CUDA_TRY(
      cudaMemcpyAsync(&res, scr + kStaticPartials, sizeof(Partial), cudaMemcpyDeviceToHost, st));
  HPAC_CUDA_TRY(cudaStreamSynchronize(st));
  double v = res.used ? res.sum / (double)res.used : 0.0;
  if (metric == HPAC_METRIC_RMSE) v = sqrt(v);
  h_result->value = v;
  h_result->zero_max_abs = res.zmax;
  h_result->used = (int64_t)res.used;
  h_result->zeros = (int64_t)res.zeros;
  h_result->zeros_mismatch = (int64_t)res.zbad;
  return HPAC_OK;
}
