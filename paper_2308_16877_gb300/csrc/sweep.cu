// Batched knob sweep: many approximation configurations over many
// Black-Scholes regions of uneven sizes in one persistent, graph-captured
// launch (the paper's design-space exploration of Section 2.4 / Section 4,
// Table 2, which builds and runs every configuration separately).
//
// Work is the cross product (region tile, configuration). A tile is
// `tile_blocks` x blockDim.x consecutive logical threads of one region, each
// walking its grid-stride invocations i = t + k T_r (Section 3.1.3). Items are
// ordered region-tile major, configuration minor, so the configurations of one
// tile run close together in time and reuse its inputs from L2. A persistent
// grid takes items from one atomic counter (no waits between blocks). For every
// invocation the kernel computes the region's output under the item's
// configuration - TAF at thread level or a perforation pattern - and folds its
// error against the double-precision exact price into per-(configuration,
// region) sums; no per-configuration output array exists.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "hpac_internal.cuh"
#include "perfo_rule.cuh"
#include "regions.cuh"

struct hpac_sweep {
  int device;
  cudaStream_t user_stream;
  cudaStream_t cap_stream;
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  int n_cfg, n_reg;
  void *d_cfg, *d_reg, *d_tile_prefix;
  float4 *d_x4;    // the inputs packed per option: S, K, T, sigma
  float4 *d_ref4;  // the exact prices split: hi, lo, 1/|a|, 0
  float4 *d_tiny;
  hpac_sweep_stats *d_stats;
  unsigned long long *d_counter;
};

namespace hpac {
namespace {

struct SweepCfg {
  int tech;      // HPAC_SWEEP_TAF or HPAC_SWEEP_PERFO
  int hsize, psize;
  int thr_inf;
  float thr_f;
  double thr_d;
  DropRule rule;  // lo/hi/T are filled per region on the device
  int m_or_percent;
};

struct SweepReg {
  int64_t n, off, T;
  int64_t tiles;
};

// The exact price a is held as two floats, hi = fl(a) and lo = fl(a - hi), so
// that the error a - y of a single-precision output comes out in single
// precision as (hi - y) + lo. Prices with |fl(a)| < 1e-30 (deep out-of-the-money
// options) are "tiny": their relative error needs an exponent range single
// precision lacks, so lo instead holds (as integer bits) an index into a
// compact table of {m_hi, m_lo, k} with a = (m_hi + m_lo) 2^k, m_hi in [1, 2)
// (index -1 where a = 0, which carries no relative term). The squared error of
// a tiny price uses d = hi - y, whose square differs from (a - y)^2 only below
// the single-precision range.
__device__ __forceinline__ bool is_tiny(float hi) { return !(fabsf(hi) >= 1e-30f); }

__global__ void count_tiny(const double *__restrict__ ref, int64_t n, unsigned long long *count) {
  unsigned c = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double a = ref[i];
    if (is_tiny((float)a) && a != 0.0) ++c;
  }
  c = __reduce_add_sync(0xffffffffu, c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, (unsigned long long)c);
}

__global__ void split_ref(const double *__restrict__ ref, float4 *__restrict__ ref4,
                          float4 *__restrict__ tiny, unsigned long long *__restrict__ slot,
                          int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double a = ref[i];
    const float h = (float)a;
    const float inv = (float)(1.0 / fabs(a));  // 1/|a| rounded once: the relative term is one multiply
    if (!is_tiny(h)) {
      ref4[i] = make_float4(h, (float)(a - (double)h), inv, 0.0f);
    } else if (a == 0.0) {
      ref4[i] = make_float4(h, __int_as_float(-1), inv, 0.0f);
    } else {
      const unsigned long long j = atomicAdd(slot, 1ull);
      // NaN keeps k = -100 so that its term stays NaN, as in double precision
      const int k = isnan(a) ? -100 : ilogb(a);
      const double m = isnan(a) ? a : ldexp(a, -k);
      const float mh = (float)m;
      tiny[j] = make_float4(mh, (float)(m - (double)mh), __int_as_float(k), 0.0f);
      ref4[i] = make_float4(h, __int_as_float((int)j), inv, 0.0f);
    }
  }
}

// Packs the four input rows into one 16-byte vector per option, so that an
// invocation issues one load for its inputs.
__global__ void pack_inputs(const float *__restrict__ in, int64_t stride, float4 *__restrict__ x4,
                            int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x4[i] = make_float4(in[i], in[stride + i], in[2 * stride + i], in[3 * stride + i]);
}

// y 2^s for s >= 0, exact whenever representable; +-inf past the float range.
// Integer exponent arithmetic (subnormal y normalised first), no rounding.
__device__ __forceinline__ float scale_up_pow2(float y, int s) {
  unsigned b = __float_as_uint(y);
  const unsigned sign = b & 0x80000000u;
  b &= 0x7fffffffu;
  if (b == 0u || b >= 0x7f800000u) return y;  // zero, inf, NaN
  int e = (int)(b >> 23);
  unsigned m = b & 0x7fffffu;
  if (e == 0) {
    const int lz = __clz((int)m) - 8;  // bring the leading one to bit 23
    m = (m << lz) & 0x7fffffu;
    e = 1 - lz;
  }
  e += s;
  if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
  return __uint_as_float(sign | ((unsigned)e << 23) | m);
}

// (hi, lo) += x with an error-free two-sum: the float pair keeps about 48 bits.
__device__ __forceinline__ void ff_add(float &hi, float &lo, float x) {
  const float s = __fadd_rn(hi, x);
  const float bp = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
  hi = s;
  lo = __fadd_rn(lo, e);
}

__device__ __forceinline__ void ff_warp_sum(float &hi, float &lo) {
  for (int off = 16; off > 0; off >>= 1) {
    const float oh = __shfl_down_sync(0xffffffffu, hi, off);
    const float ol = __shfl_down_sync(0xffffffffu, lo, off);
    lo = __fadd_rn(lo, ol);
    ff_add(hi, lo, oh);
  }
}

struct ItemSums {
  float rel_hi, rel_lo, sq_hi, sq_lo;
  double rel_wide;  // terms beyond the single-precision range
  unsigned n_inv, n_alt, n_used;
};

// The decision RSD(window) < thr of the TAF kernel on a window stored twice
// over (slot s and s + h hold the same value), so that the h values oldest ..
// newest are the contiguous slots p[0], p[BT], ..., p[(h-1) BT]: the same IEEE
// two-pass moments in the same order, the same guard-banded fast test, and
// the correctly rounded statistic from those moments inside the band.
template <int BT>
__device__ __forceinline__ bool rsd_below_contig(const float *p, int h, float thr, float inv_h) {
  float sum = 0.f;
#pragma unroll 4
  for (int j = 0; j < h; ++j) sum = __fadd_rn(sum, p[j * BT]);
  const float mu = div_count(sum, h, inv_h);
  float acc = 0.f;
#pragma unroll 4
  for (int j = 0; j < h; ++j) {
    const float d = __fsub_rn(p[j * BT], mu);
    acc = __fadd_rn(acc, __fmul_rn(d, d));
  }
  return rsd_below_moments(mu, acc, h, thr, inv_h);
}

// One work item: `tile_blocks` x BT logical threads of region R under
// configuration C. Idx is the index type (32-bit when every offset fits).
template <int BT, typename Idx>
__device__ __forceinline__ void sweep_item(const BlackScholes32 &reg, const SweepCfg &C,
                                           const SweepReg &R, int64_t tile, int tile_blocks,
                                           const float4 *__restrict__ x4,
                                           const float4 *__restrict__ ref4,
                                           const float4 *__restrict__ tiny,
                                           const double *__restrict__ ref64, float *win,
                                           ItemSums &acc) {
  const Idx n = (Idx)R.n, T = (Idx)R.T;
  const float4 *xr = x4 + R.off, *rr = ref4 + R.off;
  const double *r64 = ref64 + R.off;
  const int h = C.hsize;
  const float inv_h = 1.0f / (float)h;
  // perforation: kept range for ini/fini, residues of the key modulo M for
  // small/large advanced incrementally (key k with step 1 when herded, i with step T otherwise)
  Idx keep_lo = 0, keep_hi = n;
  if (C.tech == HPAC_SWEEP_PERFO) {
    const int64_t cut = (R.n * (int64_t)C.m_or_percent) / 100;
    if (C.rule.kind == HPAC_PERFO_INI) keep_lo = (Idx)cut;
    if (C.rule.kind == HPAC_PERFO_FINI) keep_hi = (Idx)(R.n - cut);
  }
  const int kind = C.rule.kind;
  const bool herded = C.rule.herded != 0;
  const unsigned m = (unsigned)C.rule.m;
  float rel_chunk = 0.f, sq_chunk = 0.f;
  int in_chunk = 0;
  for (int lb = 0; lb < tile_blocks; ++lb) {
    const int64_t t64 = (tile * tile_blocks + lb) * (int64_t)BT + threadIdx.x;
    if (t64 >= R.T) break;  // later logical blocks of this tile are past T too
    const Idx t = (Idx)t64;
    int pos = 0, cnt = 0, pred = 0;
    unsigned res = 0, res_inc = 0;
    if (kind == HPAC_PERFO_SMALL || kind == HPAC_PERFO_LARGE) {
      res = herded ? 0u : (unsigned)(t64 % (int64_t)m);
      res_inc = herded ? 1u % m : (unsigned)(R.T % (int64_t)m);
    }
    Idx k = 0;
    for (Idx i = t; i < n; i += T, ++k) {
      float y;
      if (C.tech == HPAC_SWEEP_TAF) {
        if (pred > 0) {
          y = win[(pos + h - 1) * BT + threadIdx.x];  // newest window value
          --pred;
          ++acc.n_alt;
        } else {
          const float4 v = xr[i];
          const float x[4] = {v.x, v.y, v.z, v.w};
          y = reg(x);
          win[pos * BT + threadIdx.x] = y;
          win[(pos + h) * BT + threadIdx.x] = y;
          pos = (pos + 1 == h) ? 0 : pos + 1;
          cnt = cnt < h ? cnt + 1 : h;
          if (cnt == h &&
              (C.thr_inf || rsd_below_contig<BT>(win + pos * BT + threadIdx.x, h, C.thr_f, inv_h)))
            pred = C.psize;
        }
      } else {
        bool drop;
        if (kind == HPAC_PERFO_INI || kind == HPAC_PERFO_FINI) {
          drop = (i < keep_lo) || (i >= keep_hi);
        } else if (kind == HPAC_PERFO_RANDOM) {
          drop = C.rule.drop_key(herded ? (int64_t)k : (int64_t)i);
        } else {
          drop = kind == HPAC_PERFO_SMALL ? res == m - 1u : res != 0u;
          res += res_inc;
          res = res >= m ? res - m : res;
        }
        if (drop) {
          y = 0.0f;  // a dropped output keeps the (zero) prefill
          ++acc.n_alt;
        } else {
          const float4 v = xr[i];
          const float x[4] = {v.x, v.y, v.z, v.w};
          y = reg(x);
        }
      }
      ++acc.n_inv;
      const float4 rf = rr[i];
      const float hi = rf.x, lo = rf.y;
      if (!is_tiny(hi)) {
        const float d = (hi - y) + lo;
        sq_chunk = fmaf(d, d, sq_chunk);
        rel_chunk = fmaf(fabsf(d), rf.z, rel_chunk);
        ++acc.n_used;
      } else {
        const float d = hi - y;
        sq_chunk = fmaf(d, d, sq_chunk);
        const int j = __float_as_int(lo);
        if (j >= 0) {
          // |a - y| / |a| = |(m_hi - y 2^-k) + m_lo| / |m_hi| to float precision
          const float4 e = tiny[j];
          const float ys = scale_up_pow2(y, -__float_as_int(e.z));
          if (fabsf(ys) < 1e30f || isnan(ys)) {
            rel_chunk += __fdiv_rn(fabsf((e.x - ys) + e.y), fabsf(e.x));
          } else {
            const double a = r64[i];  // a ratio past 1e30: double precision
            acc.rel_wide += fabs(a - (double)y) / fabs(a);
          }
          ++acc.n_used;
        }
      }
      if (++in_chunk == 16) {
        ff_add(acc.rel_hi, acc.rel_lo, rel_chunk);
        ff_add(acc.sq_hi, acc.sq_lo, sq_chunk);
        rel_chunk = sq_chunk = 0.f;
        in_chunk = 0;
      }
    }
  }
  ff_add(acc.rel_hi, acc.rel_lo, rel_chunk);
  ff_add(acc.sq_hi, acc.sq_lo, sq_chunk);
}

template <int BT, typename Idx>
__global__ void __launch_bounds__(BT, 1024 / BT) sweep_kernel(
    const SweepCfg *__restrict__ cfgs, int n_cfg, const SweepReg *__restrict__ regs, int n_reg,
    const int64_t *__restrict__ tile_prefix, int64_t n_items, int tile_blocks,
    const float4 *__restrict__ x4, const float4 *__restrict__ ref4,
    const float4 *__restrict__ tiny, const double *__restrict__ ref64, float rate,
    hpac_sweep_stats *__restrict__ stats, unsigned long long *__restrict__ counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float *win = reinterpret_cast<float *>(smem_raw);
  __shared__ long long s_item;
  __shared__ int s_reg;
  __shared__ ItemSums s_warp[BT / 32];
  const BlackScholes32 reg{rate};
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (;;) {
    __syncthreads();  // everyone has read the previous item and its sums
    if (threadIdx.x == 0) {
      const long long item = (long long)atomicAdd(counter, 1ull);
      int r = 0;
      if (item < n_items) {
        const int64_t g = item / n_cfg;
        int lo = 0, hi = n_reg - 1;  // last r with tile_prefix[r] <= g
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (tile_prefix[mid] <= g) lo = mid; else hi = mid - 1;
        }
        r = lo;
      }
      s_item = item;
      s_reg = r;
    }
    __syncthreads();
    const long long item = s_item;
    if (item >= n_items) break;
    const int c = (int)(item % n_cfg);
    const int r = s_reg;
    const int64_t tile = item / n_cfg - tile_prefix[r];
    const SweepReg R = regs[r];
    const SweepCfg C = cfgs[c];
    ItemSums acc{0.f, 0.f, 0.f, 0.f, 0.0, 0u, 0u, 0u};
    sweep_item<BT, Idx>(reg, C, R, tile, tile_blocks, x4, ref4, tiny,
                        ref64, win, acc);
    // warp then block reductions, then one atomic set per item
    ff_warp_sum(acc.rel_hi, acc.rel_lo);
    ff_warp_sum(acc.sq_hi, acc.sq_lo);
    acc.n_inv = __reduce_add_sync(0xffffffffu, acc.n_inv);
    acc.n_alt = __reduce_add_sync(0xffffffffu, acc.n_alt);
    acc.n_used = __reduce_add_sync(0xffffffffu, acc.n_used);
    if (__any_sync(0xffffffffu, acc.rel_wide != 0.0))
      for (int off = 16; off > 0; off >>= 1) acc.rel_wide += __shfl_down_sync(0xffffffffu, acc.rel_wide, off);
    if (lane == 0) s_warp[wid] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      ItemSums a = s_warp[0];
      for (int w = 1; w < BT / 32; ++w) {
        const ItemSums &b = s_warp[w];
        a.rel_lo = __fadd_rn(a.rel_lo, b.rel_lo);
        ff_add(a.rel_hi, a.rel_lo, b.rel_hi);
        a.sq_lo = __fadd_rn(a.sq_lo, b.sq_lo);
        ff_add(a.sq_hi, a.sq_lo, b.sq_hi);
        a.rel_wide += b.rel_wide;  // zero unless some term needed double range
        a.n_inv += b.n_inv;
        a.n_alt += b.n_alt;
        a.n_used += b.n_used;
      }
      hpac_sweep_stats *o = stats + (size_t)c * n_reg + r;
      atomicAdd(&o->sum_abs_rel, ((double)a.rel_hi + (double)a.rel_lo) + a.rel_wide);
      atomicAdd(&o->sum_sq, (double)a.sq_hi + (double)a.sq_lo);
      atomicAdd((unsigned long long *)&o->invocations, (unsigned long long)a.n_inv);
      atomicAdd((unsigned long long *)(C.tech == HPAC_SWEEP_TAF ? &o->approximated : &o->skipped),
                (unsigned long long)a.n_alt);
      atomicAdd((unsigned long long *)&o->mape_terms, (unsigned long long)a.n_used);
    }
  }
}

// set_only: raise the kernel's dynamic shared memory limit (outside capture);
// otherwise launch it on the capture stream.
template <int BT, typename Idx>
cudaError_t launch_sweep(bool set_only, hpac_sweep *p, unsigned grid, size_t smem, int64_t n_items,
                         int tile_blocks, const double *d_ref,
                         float rate) {
  if (set_only)
    return cudaFuncSetAttribute(sweep_kernel<BT, Idx>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
  sweep_kernel<BT, Idx><<<grid, BT, smem, p->cap_stream>>>(
      (const SweepCfg *)p->d_cfg, p->n_cfg, (const SweepReg *)p->d_reg, p->n_reg,
      (const int64_t *)p->d_tile_prefix, n_items, tile_blocks, p->d_x4, p->d_ref4, p->d_tiny, d_ref,
      rate, p->d_stats, p->d_counter);
  return cudaGetLastError();
}

void free_plan(hpac_sweep *p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  cudaFree(p->d_cfg);
  cudaFree(p->d_reg);
  cudaFree(p->d_tile_prefix);
  cudaFree(p->d_x4);
  cudaFree(p->d_ref4);
  cudaFree(p->d_tiny);
  cudaFree(p->d_stats);
  cudaFree(p->d_counter);
  free(p);
}

}  // namespace
}  // namespace hpac

using namespace hpac;

extern "C" hpac_status hpac_sweep_create(int32_t n_configs, const hpac_sweep_config *h_configs,
                                         int32_t n_regions, const hpac_sweep_region *h_regions,
                                         const float *d_in, int64_t in_stride,
                                         const double *d_ref, double rate, int32_t block_threads,
                                         int32_t blocks_per_sm, int32_t tile_blocks,
                                         void *cuda_stream, hpac_sweep **out) {
  if (!out) return set_error(HPAC_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_configs < 1 || n_regions < 1 || !h_configs || !h_regions || !d_in || !d_ref)
    return set_error(HPAC_EINVAL, "empty sweep or NULL pointer");
  if (block_threads != 64 && block_threads != 128 && block_threads != 256)
    return set_error(HPAC_EINVAL, "block_threads must be 64, 128 or 256");
  if (blocks_per_sm < 1 || blocks_per_sm > 32 || tile_blocks < 1 || tile_blocks > 64)
    return set_error(HPAC_EINVAL, "blocks_per_sm in 1..32, tile_blocks in 1..64");
  if (!isfinite(rate)) return set_error(HPAC_EINVAL, "rate is not finite");
  std::vector<SweepCfg> cfg(n_configs);
  int hmax = 1;
  for (int c = 0; c < n_configs; ++c) {
    const hpac_sweep_config &k = h_configs[c];
    SweepCfg &s = cfg[c];
    memset(&s, 0, sizeof(s));
    s.tech = k.technique;
    if (k.technique == HPAC_SWEEP_TAF) {
      if (k.hsize < 1 || k.hsize > kMaxHsize || k.psize < 0 || !(k.thresh >= 0.0))
        return set_error(HPAC_EINVAL, "config %d: bad TAF knobs", c);
      if (k.level != HPAC_LEVEL_THREAD)
        return set_error(HPAC_EUNSUPPORTED, "config %d: the sweep runs TAF at thread level", c);
      s.hsize = k.hsize;
      s.psize = k.psize;
      s.thr_f = (float)k.thresh;
      s.thr_d = k.thresh;
      s.thr_inf = isinf(k.thresh) ? 1 : 0;
      hmax = k.hsize > hmax ? k.hsize : hmax;
    } else if (k.technique == HPAC_SWEEP_PERFO) {
      const int pk = k.perfo_kind;
      if (pk < HPAC_PERFO_SMALL || pk > HPAC_PERFO_RANDOM)
        return set_error(HPAC_EINVAL, "config %d: perforation kind %d", c, pk);
      if ((pk == HPAC_PERFO_SMALL || pk == HPAC_PERFO_LARGE) && k.m_or_percent < 1)
        return set_error(HPAC_EINVAL, "config %d: M < 1", c);
      if ((pk == HPAC_PERFO_INI || pk == HPAC_PERFO_FINI) &&
          (k.m_or_percent < 0 || k.m_or_percent > 100))
        return set_error(HPAC_EINVAL, "config %d: percent not in 0..100", c);
      if (pk == HPAC_PERFO_RANDOM && !(k.rate >= 0.0 && k.rate <= 1.0))
        return set_error(HPAC_EINVAL, "config %d: rate not in [0,1]", c);
      s.rule.kind = pk;
      s.rule.herded = k.herded ? 1 : 0;
      s.rule.m = k.m_or_percent;
      s.rule.seed = k.seed;
      s.rule.cut = (uint32_t)floor(k.rate * 16777216.0);
      s.m_or_percent = k.m_or_percent;
    } else {
      return set_error(HPAC_EINVAL, "config %d: technique %d", c, k.technique);
    }
  }
  std::vector<SweepReg> reg(n_regions);
  std::vector<int64_t> prefix(n_regions + 1, 0);
  int64_t total = 0;
  const int64_t lt = (int64_t)block_threads * tile_blocks;
  for (int r = 0; r < n_regions; ++r) {
    const hpac_sweep_region &g = h_regions[r];
    if (g.n < 1 || g.offset < 0 || g.offset + g.n > in_stride || g.logical_threads < 0)
      return set_error(HPAC_EINVAL, "region %d: bad size, offset or logical threads", r);
    reg[r].n = g.n;
    reg[r].off = g.offset;
    reg[r].T = g.logical_threads > 0 ? g.logical_threads : g.n;
    reg[r].tiles = (reg[r].T + lt - 1) / lt;
    // per-item counts are 32-bit: a work item covers fewer than 2^32 invocations
    if ((double)lt * (double)((g.n + reg[r].T - 1) / reg[r].T) >= 4294967295.0)
      return set_error(HPAC_EUNSUPPORTED, "region %d: a work item would exceed 2^32 invocations", r);
    prefix[r + 1] = prefix[r] + reg[r].tiles;
    total = total > g.offset + g.n ? total : g.offset + g.n;
  }
  const int64_t n_items = prefix[n_regions] * n_configs;
  hpac_sweep *p = (hpac_sweep *)calloc(1, sizeof(hpac_sweep));
  if (!p) return set_error(HPAC_ENOMEM, "host allocation failed");
  p->n_cfg = n_configs;
  p->n_reg = n_regions;
  p->user_stream = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaGetDevice(&p->device);
#define SW_TRY(call)                          \
  do {                                        \
    e = (call);                               \
    if (e != cudaSuccess) {                   \
      free_plan(p);                           \
      return cuda_error(e, #call);            \
    }                                         \
  } while (0)
  SW_TRY(e);
  SW_TRY(cudaMalloc(&p->d_cfg, sizeof(SweepCfg) * n_configs));
  SW_TRY(cudaMalloc(&p->d_reg, sizeof(SweepReg) * n_regions));
  SW_TRY(cudaMalloc(&p->d_tile_prefix, sizeof(int64_t) * (n_regions + 1)));
  SW_TRY(cudaMalloc(&p->d_x4, sizeof(float4) * total));
  SW_TRY(cudaMalloc(&p->d_ref4, sizeof(float4) * total));
  SW_TRY(cudaMalloc(&p->d_stats, sizeof(hpac_sweep_stats) * n_configs * n_regions));
  SW_TRY(cudaMalloc(&p->d_counter, sizeof(unsigned long long)));
  SW_TRY(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
  SW_TRY(cudaMemcpyAsync(p->d_cfg, cfg.data(), sizeof(SweepCfg) * n_configs, cudaMemcpyHostToDevice,
                         p->cap_stream));
  SW_TRY(cudaMemcpyAsync(p->d_reg, reg.data(), sizeof(SweepReg) * n_regions, cudaMemcpyHostToDevice,
                         p->cap_stream));
  SW_TRY(cudaMemcpyAsync(p->d_tile_prefix, prefix.data(), sizeof(int64_t) * (n_regions + 1),
                         cudaMemcpyHostToDevice, p->cap_stream));
  // the inputs and reference come from the caller's stream
  cudaEvent_t ready;
  SW_TRY(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
  SW_TRY(cudaEventRecord(ready, p->user_stream));
  SW_TRY(cudaStreamWaitEvent(p->cap_stream, ready, 0));
  cudaEventDestroy(ready);
  // the tiny-price table: count, size it, then split (slots in any order)
  SW_TRY(cudaMemsetAsync(p->d_counter, 0, sizeof(unsigned long long), p->cap_stream));
  count_tiny<<<1024, 256, 0, p->cap_stream>>>(d_ref, total, p->d_counter);
  SW_TRY(cudaGetLastError());
  unsigned long long n_tiny = 0;
  SW_TRY(cudaMemcpyAsync(&n_tiny, p->d_counter, sizeof(n_tiny), cudaMemcpyDeviceToHost, p->cap_stream));
  SW_TRY(cudaStreamSynchronize(p->cap_stream));
  if (n_tiny >= (1ull << 31)) {
    free_plan(p);
    return set_error(HPAC_EUNSUPPORTED, "more than 2^31 exact prices below 1e-30");
  }
  SW_TRY(cudaMalloc(&p->d_tiny, sizeof(float4) * (n_tiny ? n_tiny : 1)));
  SW_TRY(cudaMemsetAsync(p->d_counter, 0, sizeof(unsigned long long), p->cap_stream));
  split_ref<<<1024, 256, 0, p->cap_stream>>>(d_ref, p->d_ref4, p->d_tiny, p->d_counter, total);
  SW_TRY(cudaGetLastError());
  pack_inputs<<<1024, 256, 0, p->cap_stream>>>(d_in, in_stride, p->d_x4, total);
  SW_TRY(cudaGetLastError());
  SW_TRY(cudaStreamSynchronize(p->cap_stream));
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
  // the TAF window is stored twice over (2 hsize slots per lane)
  const size_t smem = (size_t)2 * hmax * block_threads * sizeof(float);
  const bool idx32 = 2 * total < (int64_t)INT32_MAX;  // i + T stays below 2 total
  const unsigned grid = (unsigned)(sms * blocks_per_sm);
  auto launch = [&](bool set_only) -> cudaError_t {
    const float fr = (float)rate;
    if (block_threads == 64)
      return idx32 ? launch_sweep<64, int>(set_only, p, grid, smem, n_items, tile_blocks, d_ref, fr)
                   : launch_sweep<64, int64_t>(set_only, p, grid, smem, n_items, tile_blocks, d_ref, fr);
    if (block_threads == 128)
      return idx32 ? launch_sweep<128, int>(set_only, p, grid, smem, n_items, tile_blocks, d_ref, fr)
                   : launch_sweep<128, int64_t>(set_only, p, grid, smem, n_items, tile_blocks, d_ref, fr);
    return idx32 ? launch_sweep<256, int>(set_only, p, grid, smem, n_items, tile_blocks, d_ref, fr)
                 : launch_sweep<256, int64_t>(set_only, p, grid, smem, n_items, tile_blocks, d_ref, fr);
  };
  SW_TRY(launch(true));
  // capture: clear the counter and the sums, then the persistent kernel
  SW_TRY(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
  cudaMemsetAsync(p->d_counter, 0, sizeof(unsigned long long), p->cap_stream);
  cudaMemsetAsync(p->d_stats, 0, sizeof(hpac_sweep_stats) * n_configs * n_regions, p->cap_stream);
  const cudaError_t launch_err = launch(false);
  e = cudaStreamEndCapture(p->cap_stream, &p->graph);
  if (launch_err != cudaSuccess) e = launch_err;
  SW_TRY(e);
  SW_TRY(cudaGraphInstantiate(&p->exec, p->graph, 0));
#undef SW_TRY
  *out = p;
  return HPAC_OK;
}

extern "C" hpac_status hpac_sweep_run(hpac_sweep *p) {
  TraceRange trace_("hpac_sweep_run");
  if (!p) return set_error(HPAC_EINVAL, "sweep is NULL");
  HPAC_CUDA_TRY(cudaGraphLaunch(p->exec, p->user_stream));
  return HPAC_OK;
}

extern "C" hpac_status hpac_sweep_results(hpac_sweep *p, hpac_sweep_stats *h_stats) {
  if (!p || !h_stats) return set_error(HPAC_EINVAL, "NULL argument");
  HPAC_CUDA_TRY(cudaMemcpyAsync(h_stats, p->d_stats,
                                sizeof(hpac_sweep_stats) * p->n_cfg * p->n_reg,
                                cudaMemcpyDeviceToHost, p->user_stream));
  HPAC_CUDA_TRY(cudaStreamSynchronize(p->user_stream));
  return HPAC_OK;
}

extern "C" hpac_status hpac_sweep_destroy(hpac_sweep *p) {
  if (!p) return HPAC_OK;
  cudaStreamSynchronize(p->user_stream);
  free_plan(p);
  return HPAC_OK;
}
