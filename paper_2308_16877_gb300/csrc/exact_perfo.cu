// Accurate execution path and loop perforation (Sections 2.3, 3.1.5, 3.3).
//
// Both are maps over invocations, so the physical launch ignores the logical
// thread layout except where perforation decides on it: the drop rule of a
// herded pattern depends on the step k = i / T of the invocation, which is the
// same for every invocation of a step, so whole vector groups (and, for
// T a multiple of the vector width, whole steps) are dropped without reading
// their inputs.
//
// Memory: structure-of-arrays inputs are read with 16-byte vector loads
// (4 floats / 2 doubles per input row per thread), outputs written with
// 16-byte vector stores; grid-stride loops over a grid of at most 2048 threads
// per SM, in blocks small enough that every SM gets about eight
// (balanced_block).
#include <stdio.h>

#include "hpac_internal.cuh"
#include "perfo_rule.cuh"
#include "regions.cuh"

namespace hpac {
namespace {

template <typename T, int V>
struct VecT;
template <>
struct VecT<float, 4> { using type = float4; };
template <>
struct VecT<double, 2> { using type = double2; };
template <>
struct VecT<float, 1> { using type = float; };
template <>
struct VecT<double, 1> { using type = double; };

template <typename T, int V>
__device__ __forceinline__ void load_vec(const T *p, T (&v)[V]) {
  using VT = typename VecT<T, V>::type;
  const VT x = __ldcs(reinterpret_cast<const VT *>(p));
  const T *e = reinterpret_cast<const T *>(&x);
#pragma unroll
  for (int j = 0; j < V; ++j) v[j] = e[j];
}

template <typename T, int V>
__device__ __forceinline__ void store_vec(T *p, const T (&v)[V]) {
  using VT = typename VecT<T, V>::type;
  VT x;
  T *e = reinterpret_cast<T *>(&x);
#pragma unroll
  for (int j = 0; j < V; ++j) e[j] = v[j];
  __stcs(reinterpret_cast<VT *>(p), x);
}

// Perforation over invocations [0, n) in groups of V; group g covers
// [g*V, g*V + V). UNIFORM: every group is kept or dropped as a whole
// (DropWalk::uniform), so a group costs one decision and no per-invocation
// selects.
template <class R, int V, bool UNIFORM>
__device__ __forceinline__ void perfo_body(R reg, const typename R::T *__restrict__ in, int64_t stride,
                                         typename R::T *__restrict__ out,
                                         uint8_t *__restrict__ mask, int64_t n, DropRule rule,
                                         unsigned long long *__restrict__ counters) {
  using T = typename R::T;
  __shared__ unsigned long long s_cnt[2];
  if (threadIdx.x < 2) s_cnt[threadIdx.x] = 0;
  __syncthreads();
  unsigned long long n_drop = 0;
  const int64_t groups = n / V;
  const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
  const int64_t g0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  DropWalk<V> walk;
  walk.init(rule, g0 * V, gstride * V);
  if (UNIFORM) {
    // (two groups per iteration, as in the accurate map, took 74 registers
    // here and ran slower: 62.9 against 55.0 us for 2^24 options)
    for (int64_t g = g0; g < groups; g += gstride) {
      const int64_t i0 = g * V;
      const bool dd = walk.uniform(rule, i0);
      walk.advance(rule);
      if (mask) {
        const uint8_t mv = dd ? HPAC_MASK_SKIPPED : HPAC_MASK_EXACT;
        if (V == 4) {
          *reinterpret_cast<uchar4 *>(mask + i0) = make_uchar4(mv, mv, mv, mv);
        } else {
#pragma unroll
          for (int j = 0; j < V; ++j) mask[i0 + j] = mv;
        }
      }
      if (dd) {
        n_drop += V;
        continue;
      }
      T x[R::kReads][V];
#pragma unroll
      for (int d = 0; d < R::kReads; ++d) load_vec<T, V>(in + d * stride + i0, x[d]);
      T y[V];
      eval_group<R, V>(reg, x, y);
      store_vec<T, V>(out + i0, y);
    }
  }
  for (int64_t g = g0; g < groups && !UNIFORM; g += gstride) {
    const int64_t i0 = g * V;
    bool drop[V];
    walk.drops(rule, i0, drop);
    walk.advance(rule);
    bool all_drop = true, none_drop = true;
#pragma unroll
    for (int j = 0; j < V; ++j) {
      all_drop &= drop[j];
      none_drop &= !drop[j];
    }
    if (mask) {
      if (V == 4) {
        uchar4 mv;
        mv.x = drop[0] ? HPAC_MASK_SKIPPED : HPAC_MASK_EXACT;
        mv.y = drop[V > 1 ? 1 : 0] ? HPAC_MASK_SKIPPED : HPAC_MASK_EXACT;
        mv.z = drop[V > 2 ? 2 : 0] ? HPAC_MASK_SKIPPED : HPAC_MASK_EXACT;
        mv.w = drop[V > 3 ? 3 : 0] ? HPAC_MASK_SKIPPED : HPAC_MASK_EXACT;
        *reinterpret_cast<uchar4 *>(mask + i0) = mv;
      } else {
#pragma unroll
        for (int j = 0; j < V; ++j) mask[i0 + j] = drop[j] ? HPAC_MASK_SKIPPED : HPAC_MASK_EXACT;
      }
    }
    if (counters) {
#pragma unroll
      for (int j = 0; j < V; ++j) n_drop += drop[j] ? 1 : 0;
    }
    if (all_drop) continue;
    T x[R::kReads][V];
#pragma unroll
    for (int d = 0; d < R::kReads; ++d) load_vec<T, V>(in + d * stride + i0, x[d]);
    T y[V];
#pragma unroll
    for (int j = 0; j < V; ++j) {
      T xi[R::kReads];
#pragma unroll
      for (int d = 0; d < R::kReads; ++d) xi[d] = x[d][j];
      y[j] = reg(xi);
    }
    if (none_drop) {
      store_vec<T, V>(out + i0, y);
    } else {
#pragma unroll
      for (int j = 0; j < V; ++j)
        if (!drop[j]) out[i0 + j] = y[j];
    }
  }
  // tail [groups*V, n): one invocation per thread of block 0
  if (blockIdx.x == 0) {
    const int64_t i = groups * V + threadIdx.x;
    if (threadIdx.x < V && i < n) {
      bool drop[1] = {false};
      rule.drops<1>(i, drop);
      if (mask) mask[i] = drop[0] ? HPAC_MASK_SKIPPED : HPAC_MASK_EXACT;
      n_drop += drop[0] ? 1 : 0;
      if (!drop[0]) {
        T xi[R::kReads];
#pragma unroll
        for (int d = 0; d < R::kReads; ++d) xi[d] = in[d * stride + i];
        out[i] = reg(xi);
      }
    }
  }
  if (counters) {
    warp_count(s_cnt, n_drop, 0);
    __syncthreads();
    if (threadIdx.x == 0 && s_cnt[0]) atomicAdd(&counters[0], s_cnt[0]);
  }
}

// The accurate map, and perforation: the same body with the drop rule. (Capping
// the perforation kernel's registers at five 256-thread blocks per SM, the
// accurate map's occupancy, made the Black-Scholes stream slower: 59.4 against
// 57.6 us for 2^24 options at small:4.)
// The accurate map takes U groups per iteration (two for single-precision
// regions of up to four inputs), so that all their loads are in flight before
// any of them computes.
template <class R, int V>
__global__ void __launch_bounds__(256) map_kernel(R reg, const typename R::T *__restrict__ in,
                                                  int64_t stride, typename R::T *__restrict__ out,
                                                  int64_t n) {
  using T = typename R::T;
  constexpr int U = sizeof(T) == 4 && R::kReads <= 4 ? 2 : 1;
  const int64_t groups = n / V;
  const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; g + (U - 1) * gstride < groups; g += U * gstride) {
    T x[U][R::kReads][V];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int d = 0; d < R::kReads; ++d) load_vec<T, V>(in + d * stride + (g + u * gstride) * V, x[u][d]);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      T y[V];
      eval_group<R, V>(reg, x[u], y);
      store_vec<T, V>(out + (g + u * gstride) * V, y);
    }
  }
  for (; g < groups; g += gstride) {  // at most U - 1 groups left
    T x[R::kReads][V];
#pragma unroll
    for (int d = 0; d < R::kReads; ++d) load_vec<T, V>(in + d * stride + g * V, x[d]);
    T y[V];
    eval_group<R, V>(reg, x, y);
    store_vec<T, V>(out + g * V, y);
  }
  // tail [groups*V, n): one invocation per thread of block 0
  if (blockIdx.x == 0) {
    const int64_t i = groups * V + threadIdx.x;
    if (threadIdx.x < V && i < n) {
      T xi[R::kReads];
#pragma unroll
      for (int d = 0; d < R::kReads; ++d) xi[d] = in[d * stride + i];
      out[i] = reg(xi);
    }
  }
}

template <class R, int V, bool UNIFORM>
__global__ void __launch_bounds__(256) perfo_kernel(R reg, const typename R::T *__restrict__ in,
                                                    int64_t stride, typename R::T *__restrict__ out,
                                                    uint8_t *__restrict__ mask, int64_t n,
                                                    DropRule rule,
                                                    unsigned long long *__restrict__ counters) {
  perfo_body<R, V, UNIFORM>(reg, in, stride, out, mask, n, rule, counters);
}

template <class R>
hpac_status launch_map(const hpac_region *r, R reg, const void *in_, void *out_, uint8_t *mask,
                       const DropRule &rule, unsigned long long *counters) {
  using T = typename R::T;
  const int64_t n = r->d.n;
  if (n == 0) return HPAC_OK;
  const T *in = static_cast<const T *>(in_);
  T *out = static_cast<T *>(out_);
  constexpr int VW = 16 / sizeof(T);
  const bool vec_ok = (r->d.in_stride % VW == 0) && ((uintptr_t)in % 16 == 0) &&
                      ((uintptr_t)out % 16 == 0) && (mask == nullptr || (uintptr_t)mask % 4 == 0);
  const bool perfo = rule.kind >= 0;
  const int vw = vec_ok ? VW : 1;
  const int threads = balanced_block(n / vw, 256, r->device);
  const int64_t per_block_max = (int64_t)sm_count(r->device) * 2048 / threads;
  int64_t blocks = (n / vw + threads - 1) / threads;
  blocks = blocks < 1 ? 1 : (blocks > per_block_max ? per_block_max : blocks);
  if (!perfo) {
    auto kern = vec_ok ? map_kernel<R, VW> : map_kernel<R, 1>;
    kern<<<(unsigned)blocks, threads, 0, r->stream>>>(reg, in, r->d.in_stride, out, n);
  } else {
    const bool range = rule.kind == HPAC_PERFO_INI || rule.kind == HPAC_PERFO_FINI;
    // (groups cover [0, n - n % VW); the tail runs per invocation, so hi = n splits none)
    const bool uniform = vec_ok && (range ? (rule.lo % VW == 0 && (rule.hi % VW == 0 || rule.hi == n))
                                          : (rule.herded && rule.T % VW == 0));
    auto kern = uniform ? perfo_kernel<R, VW, true>
                        : (vec_ok ? perfo_kernel<R, VW, false> : perfo_kernel<R, 1, false>);
    kern<<<(unsigned)blocks, threads, 0, r->stream>>>(reg, in, r->d.in_stride, out, mask, n, rule,
                                                       counters);
  }
  HPAC_CUDA_TRY(cudaGetLastError());
  return HPAC_OK;
}

hpac_status dispatch_map(const hpac_region *r, const void *in, void *out, uint8_t *mask,
                         const DropRule &rule, unsigned long long *counters) {
  const hpac_region_desc &d = r->d;
  switch (d.kind) {
    case HPAC_REGION_BLACKSCHOLES:
      if (d.dtype == HPAC_F32) return launch_map(r, BlackScholes32{(float)d.param}, in, out, mask, rule, counters);
      return launch_map(r, BlackScholes64{d.param}, in, out, mask, rule, counters);
    case HPAC_REGION_EOS:
      return launch_map(r, Eos64{d.param}, in, out, mask, rule, counters);
    case HPAC_REGION_IDENTITY:
      if (d.dtype == HPAC_F32) return launch_map(r, Identity<float>{}, in, out, mask, rule, counters);
      return launch_map(r, Identity<double>{}, in, out, mask, rule, counters);
    case HPAC_REGION_KMEANS:
      return launch_map(r, KMeans32{static_cast<const float *>(r->aux), d.arg}, in, out, mask, rule,
                        counters);
  }
  return set_error(HPAC_EUNSUPPORTED, "region kind %d", d.kind);
}

}  // namespace

hpac_status launch_exact(const hpac_region *r, const void *in, void *out) {
  DropRule rule{};
  rule.kind = -1;
  rule.T = logical_threads(r->d);
  return dispatch_map(r, in, out, nullptr, rule, nullptr);
}

hpac_status launch_perfo(const hpac_region *r, const hpac_perfo_knobs *k, const void *in, void *out,
                         uint8_t *mask, unsigned long long *counters) {
  DropRule rule{};
  rule.kind = k->kind;
  rule.herded = k->herded ? 1 : 0;
  rule.m = k->m_or_percent;
  rule.seed = k->seed;
  rule.cut = (uint32_t)floor(k->rate * 16777216.0);
  rule.T = logical_threads(r->d);
  const int64_t n = r->d.n;
  const int64_t cutn = (n * (int64_t)k->m_or_percent) / 100;
  rule.lo = 0;
  rule.hi = n;
  if (k->kind == HPAC_PERFO_INI) rule.lo = cutn;
  if (k->kind == HPAC_PERFO_FINI) rule.hi = n - cutn;
  return dispatch_map(r, in, out, mask, rule, counters);
}

}  // namespace hpac
