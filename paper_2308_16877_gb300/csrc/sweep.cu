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
  float *d_ref_hi, *d_ref_lo;
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

__global__ void split_ref(const double *__restrict__ ref, float *__restrict__ hi,
                          float *__restrict__ lo, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double a = ref[i];
    const float h = (float)a;
    hi[i] = h;
    lo[i] = (float)(a - (double)h);
  }
}

__device__ __forceinline__ double block_sum(double v, double *red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int j = 0; j < (int)(blockDim.x >> 5); ++j) s += red[j];
  return s;  // valid in thread 0
}

__global__ void __launch_bounds__(256) sweep_kernel(
    const SweepCfg *__restrict__ cfgs, int n_cfg, const SweepReg *__restrict__ regs, int n_reg,
    const int64_t *__restrict__ tile_prefix, int64_t n_items, int tile_blocks,
    const float *__restrict__ in, int64_t stride, const float *__restrict__ ref_hi,
    const float *__restrict__ ref_lo, const double *__restrict__ ref64, float rate,
    hpac_sweep_stats *__restrict__ stats, unsigned long long *__restrict__ counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float *win = reinterpret_cast<float *>(smem_raw);
  __shared__ long long s_item;
  __shared__ double s_red[32];
  const BlackScholes32 reg{rate};
  const int ld = blockDim.x;
  for (;;) {
    __syncthreads();  // everyone has read the previous item
    if (threadIdx.x == 0) s_item = (long long)atomicAdd(counter, 1ull);
    __syncthreads();
    const long long item = s_item;
    if (item >= n_items) break;
    const int c = (int)(item % n_cfg);
    const int64_t g = item / n_cfg;  // global tile index
    int r = 0;
    while (r + 1 < n_reg && tile_prefix[r + 1] <= g) ++r;
    const int64_t tile = g - tile_prefix[r];
    const SweepReg R = regs[r];
    const SweepCfg C = cfgs[c];
    DropRule rule = C.rule;
    rule.T = R.T;
    rule.lo = 0;
    rule.hi = R.n;
    if (C.tech == HPAC_SWEEP_PERFO) {
      const int64_t cut = (R.n * (int64_t)C.m_or_percent) / 100;
      if (rule.kind == HPAC_PERFO_INI) rule.lo = cut;
      if (rule.kind == HPAC_PERFO_FINI) rule.hi = R.n - cut;
    }
    float rel_chunk = 0.f, sq_chunk = 0.f;
    double rel_sum = 0.0, sq_sum = 0.0;
    unsigned long long n_inv = 0, n_apx = 0, n_skip = 0, n_used = 0;
    int in_chunk = 0;
    for (int lb = 0; lb < tile_blocks; ++lb) {
      const int64_t t = (tile * tile_blocks + lb) * (int64_t)blockDim.x + threadIdx.x;
      if (t >= R.T) continue;
      int pos = 0, cnt = 0, pred = 0;
      int64_t k = 0;
      for (int64_t i = t; i < R.n; i += R.T, ++k) {
        const int64_t gi = R.off + i;
        float y;
        if (C.tech == HPAC_SWEEP_TAF) {
          if (pred > 0) {
            y = win[(pos == 0 ? C.hsize - 1 : pos - 1) * ld + threadIdx.x];
            --pred;
            ++n_apx;
          } else {
            float x[4];
#pragma unroll
            for (int d = 0; d < 4; ++d) x[d] = in[d * stride + gi];
            y = reg(x);
            win[pos * ld + threadIdx.x] = y;
            pos = (pos + 1 == C.hsize) ? 0 : pos + 1;
            cnt = cnt < C.hsize ? cnt + 1 : C.hsize;
            if (cnt == C.hsize) {
              const float s = window_rsd<float>(win + threadIdx.x, ld, pos, C.hsize);
              if (C.thr_inf || s < C.thr_f) pred = C.psize;
            }
          }
        } else {
          bool drop[1];
          // the step index of invocation i is k = i / T (herded key)
          if (rule.kind == HPAC_PERFO_INI || rule.kind == HPAC_PERFO_FINI)
            drop[0] = (i < rule.lo) || (i >= rule.hi);
          else
            drop[0] = rule.drop_key(rule.herded ? k : i);
          if (drop[0]) {
            y = 0.0f;  // a dropped output keeps the (zero) prefill
            ++n_skip;
          } else {
            float x[4];
#pragma unroll
            for (int d = 0; d < 4; ++d) x[d] = in[d * stride + gi];
            y = reg(x);
          }
        }
        ++n_inv;
        // error against the exact price a = hi + lo (two floats); prices
        // below 1e-30 (about 3% of these options) take the double path so that
        // the MAPE terms are exactly those of hpac_quality (a != 0)
        const float hi = ref_hi[gi], lo = ref_lo[gi];
        const float d = (hi - y) + lo;
        sq_chunk = fmaf(d, d, sq_chunk);
        if (fabsf(hi) >= 1e-30f) {
          rel_chunk += __fdiv_rn(fabsf(d), fabsf(hi));
          ++n_used;
        } else {
          const double a = ref64[gi];
          if (a != 0.0) {
            rel_sum += fabs(a - (double)y) / fabs(a);
            ++n_used;
          }
        }
        if (++in_chunk == 16) {
          rel_sum += (double)rel_chunk;
          sq_sum += (double)sq_chunk;
          rel_chunk = sq_chunk = 0.f;
          in_chunk = 0;
        }
      }
    }
    rel_sum += (double)rel_chunk;
    sq_sum += (double)sq_chunk;
    // block reductions, then one atomic set per item
    const double rs = block_sum(rel_sum, s_red);
    const double ss = block_sum(sq_sum, s_red);
    const double ni = block_sum((double)n_inv, s_red);
    const double na = block_sum((double)n_apx, s_red);
    const double nk = block_sum((double)n_skip, s_red);
    const double nu = block_sum((double)n_used, s_red);
    if (threadIdx.x == 0) {
      hpac_sweep_stats *o = stats + (size_t)c * n_reg + r;
      atomicAdd(&o->sum_abs_rel, rs);
      atomicAdd(&o->sum_sq, ss);
      atomicAdd((unsigned long long *)&o->invocations, (unsigned long long)ni);
      atomicAdd((unsigned long long *)&o->approximated, (unsigned long long)na);
      atomicAdd((unsigned long long *)&o->skipped, (unsigned long long)nk);
      atomicAdd((unsigned long long *)&o->mape_terms, (unsigned long long)nu);
    }
  }
}

void free_plan(hpac_sweep *p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  cudaFree(p->d_cfg);
  cudaFree(p->d_reg);
  cudaFree(p->d_tile_prefix);
  cudaFree(p->d_ref_hi);
  cudaFree(p->d_ref_lo);
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
  SW_TRY(cudaMalloc(&p->d_ref_hi, sizeof(float) * total));
  SW_TRY(cudaMalloc(&p->d_ref_lo, sizeof(float) * total));
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
  split_ref<<<1024, 256, 0, p->cap_stream>>>(d_ref, p->d_ref_hi, p->d_ref_lo, total);
  SW_TRY(cudaGetLastError());
  SW_TRY(cudaStreamSynchronize(p->cap_stream));
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
  const size_t smem = (size_t)hmax * block_threads * sizeof(float);
  SW_TRY(cudaFuncSetAttribute(sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // capture: clear the counter and the sums, then the persistent kernel
  SW_TRY(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
  cudaMemsetAsync(p->d_counter, 0, sizeof(unsigned long long), p->cap_stream);
  cudaMemsetAsync(p->d_stats, 0, sizeof(hpac_sweep_stats) * n_configs * n_regions, p->cap_stream);
  sweep_kernel<<<(unsigned)(sms * blocks_per_sm), block_threads, smem, p->cap_stream>>>(
      (const SweepCfg *)p->d_cfg, n_configs, (const SweepReg *)p->d_reg, n_regions,
      (const int64_t *)p->d_tile_prefix, n_items, tile_blocks, d_in, in_stride, p->d_ref_hi,
      p->d_ref_lo, d_ref, (float)rate, p->d_stats, p->d_counter);
  cudaError_t launch_err = cudaGetLastError();
  e = cudaStreamEndCapture(p->cap_stream, &p->graph);
  if (launch_err != cudaSuccess) e = launch_err;
  SW_TRY(e);
  SW_TRY(cudaGraphInstantiate(&p->exec, p->graph, 0));
#undef SW_TRY
  *out = p;
  return HPAC_OK;
}

extern "C" hpac_status hpac_sweep_run(hpac_sweep *p) {
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
