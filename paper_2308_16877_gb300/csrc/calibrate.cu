// Calibrated fallback bound of a learned surrogate: the exact region judges the
// surrogate's error on held-out invocations, and the bound decides where the
// surrogate's prediction is trusted (prediction >= floor) and where the exact
// region runs instead.
//
// Rule: with bad_i = |pred_i - exact_i| > target |exact_i| (the relative error
// above the target, without a division), the floor is the smallest prediction
// value v such that, among the k predictions >= v, at most
// k - ceil(quantile k) are bad (the nearest-rank quantile of the relative
// error over that set is within the target). NaN predictions are never at or
// above a floor. No such v: the floor is +inf (the exact region everywhere).
//
// Steps, all on the device:
//   keys      32-bit order key of the prediction, descending, with the bad
//             flag as the lowest bit (-0 folded into +0, NaN last);
//   sort      bitonic network on the keys padded to a power of two: the
//             stages whose pairs lie within 2048 keys run in shared memory,
//             the wider ones as one global pass each;
//   prefix    bad counts in sorted order (block scans, then the block sums);
//   select    at every boundary between distinct predictions, the rule's
//             test on (k, bad count); the largest passing k by atomic max;
//   finish    the floor is the prediction at position k - 1.
#include <math.h>

#include "hpac_internal.cuh"

namespace hpac {
namespace {

constexpr int kChunk = 2048;      // keys per shared-memory sorting block
constexpr int kScanBlock = 1024;  // keys per prefix-scan block (256 threads x 4)

__device__ __forceinline__ unsigned desc_key(float y) {
  const unsigned b = __float_as_uint(y);
  const unsigned asc = (b & 0x80000000u) ? ~b : (b | 0x80000000u);  // ascending in y
  return ~asc;                                                       // descending in y
}

__device__ __forceinline__ float key_value(unsigned long long key) {
  const unsigned asc = ~(unsigned)(key >> 1);
  const unsigned b = (asc & 0x80000000u) ? (asc & 0x7fffffffu) : ~asc;
  return __uint_as_float(b);
}

__global__ void __launch_bounds__(256) keys_kernel(const float *__restrict__ pred,
                                                   const double *__restrict__ exact, int64_t n,
                                                   int64_t n_pad, double target,
                                                   unsigned long long *__restrict__ key,
                                                   unsigned long long *__restrict__ n_nan) {
  unsigned long long nan_here = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_pad;
       i += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long k = ~0ull;
    if (i < n) {
      const float y = pred[i] + 0.0f;  // -0 becomes +0: one key per value
      if (isnan(y)) {
        ++nan_here;
      } else {
        const double a = exact[i];
        const bool bad = fabs((double)y - a) > target * fabs(a);
        k = ((unsigned long long)desc_key(y) << 1) | (bad ? 1ull : 0ull);
      }
    }
    key[i] = k;
  }
  for (int off = 16; off > 0; off >>= 1) nan_here += __shfl_down_sync(0xffffffffu, nan_here, off);
  if ((threadIdx.x & 31) == 0 && nan_here) atomicAdd(n_nan, nan_here);
}

// Bitonic stages k = kfirst, 2 kfirst, ..., klast, each with its pair
// distances j = min(k / 2, 1024) .. 1, on one chunk of 2048 keys in shared
// memory (pairs at distance < 2048 stay inside an aligned chunk).
__global__ void __launch_bounds__(1024) bitonic_chunk(unsigned long long *__restrict__ key,
                                                      int64_t kfirst, int64_t klast) {
  __shared__ unsigned long long s[kChunk];
  const int64_t base = (int64_t)blockIdx.x * kChunk;
  const int t = threadIdx.x;
  s[t] = key[base + t];
  s[t + 1024] = key[base + t + 1024];
  __syncthreads();
  for (int64_t k = kfirst; k <= klast; k <<= 1) {
    for (int j = (int)(k / 2 < 1024 ? k / 2 : 1024); j > 0; j >>= 1) {
      const int i = 2 * j * (t / j) + (t % j);  // the pair's lower index (bit j clear)
      const bool asc = ((base + i) & k) == 0;
      const unsigned long long a = s[i], b = s[i + j];
      if ((a > b) == asc) {
        s[i] = b;
        s[i + j] = a;
      }
      __syncthreads();
    }
  }
  key[base + t] = s[t];
  key[base + t + 1024] = s[t + 1024];
}

// One bitonic pass at pair distance j = 2^lj >= 2048 of stage k.
__global__ void __launch_bounds__(256) bitonic_pass(unsigned long long *__restrict__ key,
                                                    int64_t n_pad, int lj, int64_t k) {
  const int64_t pairs = n_pad >> 1, j = 1ll << lj;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < pairs;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = ((t >> lj) << (lj + 1)) | (t & (j - 1));
    const bool asc = (i & k) == 0;
    const unsigned long long a = key[i], b = key[i + j];
    if ((a > b) == asc) {
      key[i] = b;
      key[i + j] = a;
    }
  }
}

// Inclusive bad counts within each block of 1024 sorted keys, and the
// block totals.
__global__ void __launch_bounds__(256) scan_blocks(const unsigned long long *__restrict__ key,
                                                   int64_t n_valid, unsigned *__restrict__ pre,
                                                   unsigned long long *__restrict__ bsum) {
  __shared__ unsigned warp_tot[8];
  const int64_t j0 = (int64_t)blockIdx.x * kScanBlock + 4 * threadIdx.x;
  unsigned v[4];
  unsigned run = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int64_t j = j0 + q;
    run += (j < n_valid) ? (unsigned)(key[j] & 1ull) : 0u;
    v[q] = run;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned x = run;  // inclusive scan of the per-thread totals within the warp
  for (int off = 1; off < 32; off <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  unsigned before = x - run;
  for (int u = 0; u < w; ++u) before += warp_tot[u];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int64_t j = j0 + q;
    if (j < n_valid) pre[j] = before + v[q];
  }
  if (threadIdx.x == 255) bsum[blockIdx.x] = before + run;
}

// Exclusive offsets of the block totals (one block, chunks of 1024 with a
// carried total), in place.
__global__ void __launch_bounds__(1024) scan_sums(unsigned long long *__restrict__ bsum, int64_t nb) {
  __shared__ unsigned long long warp_tot[32];
  __shared__ unsigned long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int64_t c = 0; c < nb; c += 1024) {
    const int64_t b = c + threadIdx.x;
    const unsigned long long mine = b < nb ? bsum[b] : 0ull;
    unsigned long long x = mine;
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, x, off);
      if (lane >= off) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    unsigned long long before = carry + x - mine;
    for (int u = 0; u < w; ++u) before += warp_tot[u];
    __syncthreads();
    if (b < nb) bsum[b] = before;
    if (threadIdx.x == 1023) carry = before + mine;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) select_kernel(const unsigned long long *__restrict__ key,
                                                     const unsigned *__restrict__ pre,
                                                     const unsigned long long *__restrict__ off,
                                                     int64_t n_valid, double quantile,
                                                     unsigned long long *__restrict__ best) {
  unsigned long long mine = 0;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_valid;
       j += (int64_t)gridDim.x * blockDim.x) {
    const bool boundary = (j + 1 == n_valid) || ((key[j] >> 1) != (key[j + 1] >> 1));
    if (!boundary) continue;
    const int64_t k = j + 1;
    const int64_t bad = (int64_t)(off[j / kScanBlock] + pre[j]);
    const int64_t allowed = k - (int64_t)ceil(quantile * (double)k);
    if (bad <= allowed && (unsigned long long)k > mine) mine = (unsigned long long)k;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_down_sync(0xffffffffu, mine, o);
    mine = y > mine ? y : mine;
  }
  if ((threadIdx.x & 31) == 0 && mine) atomicMax(best, mine);
}

__global__ void finish_kernel(const unsigned long long *__restrict__ key,
                              const unsigned long long *__restrict__ best, float *__restrict__ floor_out) {
  const unsigned long long k = *best;
  *floor_out = k ? key_value(key[k - 1]) : __int_as_float(0x7f800000);  // +inf: nothing passes
}

}  // namespace
}  // namespace hpac

using namespace hpac;

extern "C" hpac_status hpac_calibrate_floor(int64_t n, const float *d_pred, const double *d_exact,
                                            double target, double quantile, float *h_floor,
                                            int64_t *h_kept, void *cuda_stream) {
  TraceRange trace_("hpac_calibrate_floor");
  if (!h_floor) return set_error(HPAC_EINVAL, "h_floor is NULL");
  if (n < 0 || n > (1ll << 31)) return set_error(HPAC_EINVAL, "n = %lld not in 0..2^31", (long long)n);
  if (n > 0 && (!d_pred || !d_exact)) return set_error(HPAC_EINVAL, "NULL data pointer");
  if (!(target >= 0.0) || !isfinite(target)) return set_error(HPAC_EINVAL, "target must be finite and >= 0");
  if (!(quantile > 0.0 && quantile <= 1.0)) return set_error(HPAC_EINVAL, "quantile must be in (0, 1]");
  *h_floor = INFINITY;
  if (h_kept) *h_kept = 0;
  if (n == 0) return HPAC_OK;
  int dev = 0;
  HPAC_CUDA_TRY(cudaGetDevice(&dev));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int64_t n_pad = kChunk;
  while (n_pad < n) n_pad <<= 1;
  const int64_t nb = (n_pad + kScanBlock - 1) / kScanBlock;
  // workspace: keys, per-key prefix, block sums, and three words
  const size_t b_key = align256(sizeof(unsigned long long) * n_pad);
  const size_t b_pre = align256(sizeof(unsigned) * n_pad);
  const size_t b_sum = align256(sizeof(unsigned long long) * nb);
  char *w = nullptr;
  HPAC_CUDA_TRY(cudaMalloc(&w, b_key + b_pre + b_sum + 256));
  unsigned long long *key = (unsigned long long *)w;
  unsigned *pre = (unsigned *)(w + b_key);
  unsigned long long *bsum = (unsigned long long *)(w + b_key + b_pre);
  unsigned long long *words = (unsigned long long *)(w + b_key + b_pre + b_sum);  // n_nan, best
  float *floor_dev = (float *)(words + 2);
  hpac_status status = HPAC_OK;
  auto fail = [&](cudaError_t e, const char *what) {
    if (status == HPAC_OK && e != cudaSuccess) status = cuda_error(e, what);
  };
  fail(cudaMemsetAsync(words, 0, 3 * sizeof(unsigned long long), st), "cudaMemsetAsync");
  const int sms = sm_count(dev);
  const int64_t want = (n_pad + 255) / 256;
  const unsigned grid = (unsigned)(want < (int64_t)sms * 16 ? want : (int64_t)sms * 16);
  keys_kernel<<<grid, 256, 0, st>>>(d_pred, d_exact, n, n_pad, target, key, words);
  fail(cudaGetLastError(), "keys_kernel");
  const unsigned chunks = (unsigned)(n_pad / kChunk);
  bitonic_chunk<<<chunks, 1024, 0, st>>>(key, 2, kChunk);
  fail(cudaGetLastError(), "bitonic_chunk");
  const int64_t pairs = n_pad / 2;
  const unsigned pgrid = (unsigned)((pairs + 255) / 256 < (int64_t)sms * 16 ? (pairs + 255) / 256
                                                                             : (int64_t)sms * 16);
  for (int64_t k = 2 * kChunk; k <= n_pad; k <<= 1) {
    int lj = 0;
    while ((1ll << lj) < k / 2) ++lj;
    for (; (1ll << lj) >= kChunk; --lj) {
      bitonic_pass<<<pgrid, 256, 0, st>>>(key, n_pad, lj, k);
      fail(cudaGetLastError(), "bitonic_pass");
    }
    bitonic_chunk<<<chunks, 1024, 0, st>>>(key, k, k);
    fail(cudaGetLastError(), "bitonic_chunk");
  }
  unsigned long long n_nan = 0;
  fail(cudaMemcpyAsync(&n_nan, words, sizeof(n_nan), cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync");
  fail(cudaStreamSynchronize(st), "cudaStreamSynchronize");
  const int64_t n_valid = n - (int64_t)n_nan;
  if (status == HPAC_OK && n_valid > 0) {
    const int64_t nbv = (n_valid + kScanBlock - 1) / kScanBlock;
    scan_blocks<<<(unsigned)nbv, 256, 0, st>>>(key, n_valid, pre, bsum);
    fail(cudaGetLastError(), "scan_blocks");
    scan_sums<<<1, 1024, 0, st>>>(bsum, nbv);
    fail(cudaGetLastError(), "scan_sums");
    const unsigned sgrid = (unsigned)((n_valid + 255) / 256 < (int64_t)sms * 16 ? (n_valid + 255) / 256
                                                                                 : (int64_t)sms * 16);
    select_kernel<<<sgrid, 256, 0, st>>>(key, pre, bsum, n_valid, quantile, words + 1);
    fail(cudaGetLastError(), "select_kernel");
    finish_kernel<<<1, 1, 0, st>>>(key, words + 1, floor_dev);
    fail(cudaGetLastError(), "finish_kernel");
    unsigned long long best = 0;
    float fl = INFINITY;
    fail(cudaMemcpyAsync(&best, words + 1, sizeof(best), cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync");
    fail(cudaMemcpyAsync(&fl, floor_dev, sizeof(fl), cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync");
    fail(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    if (status == HPAC_OK) {
      *h_floor = fl;
      if (h_kept) *h_kept = (int64_t)best;
    }
  }
  const cudaError_t fe = cudaFree(w);
  if (status == HPAC_OK && fe != cudaSuccess) status = cuda_error(fe, "cudaFree");
  return status;
}
