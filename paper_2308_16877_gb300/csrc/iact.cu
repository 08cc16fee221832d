// iACT: approximate input memoization with tables shared within a warp
// (Sections 2.3 and 3.1.4; read/write phases, farthest-lane writer and
// round-robin replacement, Section 3.3).
//
// Each warp owns tperwarp tables in shared memory; lanes [j*L, (j+1)*L),
// L = 32/tperwarp, share table j. Layout puts the table index innermost,
//   z[slot][d][table] (float, scaled inputs), y[slot][table] (region type),
// so at a given (slot, d) the lanes of a warp read consecutive words, and the
// lanes that share a table read one word (a broadcast): no bank conflicts.
// Valid slots always form a prefix [0, filled) because replacement is
// round-robin from slot 0.
//
// A step is: read phase (every active lane scans its table), decision
// (per lane, or ballot/popcount majority per warp, or a shared tally per
// block), execution (table value or exact region), __syncwarp, write phase
// (segmented arg-max of the distance over each table's exactly computing
// lanes with shuffles; the winner writes its slot), __syncwarp.
#include "hpac_internal.cuh"
#include "convert.cuh"
#include "regions.cuh"

namespace hpac {
namespace {

struct IactParams {
  float scale_f[kMaxIn];   // per-dimension scale, single precision
  double scale_d[kMaxIn];  // per-dimension scale, double precision
  int D;
  int tsize;
  int g;                   // tables per warp
  int L;                   // lanes per table
  float thr;
  double thr_d;
};


template <typename V>
struct WarpTables {
  float *z;     // [tsize][D][g]
  V *y;         // [tsize][g]
  int *filled;  // [g]
  int *rr;      // [g]
};

// Bytes of one warp's tables, a multiple of 16 so that every warp's image
// starts on a 16-byte boundary (the kept-state kernel copies images in
// 16-byte pieces).
template <typename V>
__host__ __device__ inline size_t warp_table_bytes(int tsize, int D, int g) {
  size_t zb = (size_t)tsize * D * g * sizeof(float);
  zb = (zb + 7) & ~(size_t)7;
  const size_t b = zb + (size_t)tsize * g * sizeof(V) + 2 * (size_t)g * sizeof(int);
  return (b + 15) & ~(size_t)15;
}

// One invocation of a logical thread: read phase (scaled inputs and the
// nearest valid slot of the lane's table), decision at the level, execution
// (the slot's output or the exact region), and the write phase (per table
// the farthest exactly computing lane writes the round-robin slot). Shared by
// the launch-scoped kernel and the pipelined kept-state kernel.
template <class R, int LEVEL, int DC, bool COUNT>
__device__ __forceinline__ void iact_step(const R &reg, const WarpTables<typename R::T> &W,
                                          const IactParams &P, int D, int g, int L, int tab, int lane,
                                          bool act, int64_t i,
                                          const typename R::T (&x)[DC > 0 ? DC : kMaxIn],
                                          typename R::T *__restrict__ out, uint8_t *__restrict__ mask,
                                          typename R::T *__restrict__ stat, int *s_tally, int &k3,
                                          unsigned long long &n_apx, unsigned long long &n_border) {
  using V = typename R::T;
  constexpr int KD = DC > 0 ? DC : kMaxIn;
  const int tsize = P.tsize;
  float z[KD];
  bool has = false;
  float best = INFINITY;
  int near = 0;
  if (act) {
#pragma unroll
    for (int d = 0; d < KD; ++d) {
      if (d < D) {
        if (sizeof(V) == 4)
          z[d] = __fmul_rn(P.scale_f[d], (float)x[d]);
        else
          z[d] = double_to_float_rn_novote(__dmul_rn(P.scale_d[d], (double)x[d]));
      }
    }
    const int filled = W.filled[tab];
    for (int j = 0; j < filled; ++j) {
      float acc = 0.0f;
      const float *zs = W.z + (size_t)j * D * g + tab;
#pragma unroll
      for (int d = 0; d < KD; ++d) {
        if (d < D) {
          const float df = __fsub_rn(z[d], zs[d * g]);
          acc = __fadd_rn(acc, __fmul_rn(df, df));
        }
      }
      if (!has || acc < best) {
        best = acc;
        near = j;
      }
      has = true;
    }
  }
  const float dmin = has ? __fsqrt_rn(best) : INFINITY;
  const bool wants = act && has && dmin < P.thr;
  // ---- decision
  bool apx;
  if (LEVEL == HPAC_LEVEL_THREAD) {
    apx = wants;
  } else if (LEVEL == HPAC_LEVEL_WARP) {
    const unsigned na = __ballot_sync(0xffffffffu, act);
    const unsigned nw = __ballot_sync(0xffffffffu, wants);
    apx = (2 * __popc(nw) > __popc(na)) && act && has;
  } else {
    const unsigned na = __ballot_sync(0xffffffffu, act);
    const unsigned nw = __ballot_sync(0xffffffffu, wants);
    if (threadIdx.x == 0) s_tally[k3 == 2 ? 0 : k3 + 1] = 0;
    if (lane == 0) atomicAdd(&s_tally[k3], (__popc(nw) << 16) | __popc(na));
    __syncthreads();
    const int tally = s_tally[k3];
    apx = (2 * (tally >> 16) > (tally & 0xffff)) && act && has;
    k3 = k3 == 2 ? 0 : k3 + 1;
  }
  // ---- execute
  V y = (V)0;
  if (act) {
    if (apx) {
      y = W.y[(size_t)near * g + tab];
      if (mask) mask[i] = HPAC_MASK_APPROX;
      ++n_apx;
    } else {
      y = reg(x);
      if (mask) mask[i] = HPAC_MASK_EXACT;
    }
    out[i] = y;
    if (stat) stat[i] = (V)dmin;
    // diagnostic, compiled only into the counting variant: its double-precision
    // test would otherwise be evaluated (and discarded) for every invocation
    if (COUNT && has && borderline((double)dmin, P.thr_d)) ++n_border;
  }
  __syncwarp();
  // ---- write phase: per table, the farthest exactly computing lane
  float key = (act && !apx) ? dmin : -1.0f;
  int who = lane;
  for (int off = 1; off < L; off <<= 1) {
    const float ok = __shfl_xor_sync(0xffffffffu, key, off);
    const int ow = __shfl_xor_sync(0xffffffffu, who, off);
    if (ok > key || (ok == key && ow < who)) {
      key = ok;
      who = ow;
    }
  }
  if (who == lane && key >= 0.0f) {
    const int slot = W.rr[tab];
#pragma unroll
    for (int d = 0; d < KD; ++d)
      if (d < D) W.z[((size_t)slot * D + d) * g + tab] = z[d];
    W.y[(size_t)slot * g + tab] = y;
    W.rr[tab] = slot + 1 == tsize ? 0 : slot + 1;
    if (W.filled[tab] < tsize) W.filled[tab] += 1;
  }
  __syncwarp();
}

// DC: the number of inputs when fixed by the region (4 for Black-Scholes and
// the EOS), so that the distance loops are fully unrolled; 0 reads P.D.
// COUNT: the caller asked for counters.
// PERSIST: the warp's tables are loaded from and saved to st (persistent
// state), in a separate instantiation so the plain kernels carry none of it.
template <class R, int LEVEL, int DC, bool COUNT, bool PERSIST = false>
__global__ void __launch_bounds__(1024) iact_kernel(R reg, const typename R::T *__restrict__ in,
                                                    int64_t stride, typename R::T *__restrict__ out,
                                                    uint8_t *__restrict__ mask,
                                                    typename R::T *__restrict__ stat, int64_t n,
                                                    int64_t T, IactParams P,
                                                    unsigned long long *__restrict__ counters,
                                                    uint32_t *__restrict__ st) {
  using V = typename R::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ unsigned long long s_cnt[2];
  __shared__ int s_tally[3];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  constexpr int KD = DC > 0 ? DC : kMaxIn;
  const int D = DC > 0 ? DC : P.D, tsize = P.tsize, g = P.g, L = P.L;
  const int tab = lane / L;
  const size_t wbytes = warp_table_bytes<V>(tsize, D, g);
  unsigned char *base = smem_raw + (size_t)warp * wbytes;
  WarpTables<V> W;
  W.z = reinterpret_cast<float *>(base);
  size_t zb = ((size_t)tsize * D * g * sizeof(float) + 7) & ~(size_t)7;
  W.y = reinterpret_cast<V *>(base + zb);
  W.filled = reinterpret_cast<int *>(base + zb + (size_t)tsize * g * sizeof(V));
  W.rr = W.filled + g;
  // logical warp of this physical warp; with persistent state (st, one table
  // image of wbytes per logical warp) its tables resume from the last call
  const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x) / 32 + warp;
  const bool has_state = PERSIST && gwarp * 32 < T;
  uint32_t *wst = has_state ? st + (size_t)gwarp * (wbytes / 4) : nullptr;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t t_lead = LEVEL == HPAC_LEVEL_BLOCK ? (int64_t)blockIdx.x * blockDim.x : t - lane;
  // The first invocation's inputs are requested before the tables are read
  // in, so that the two loads' latencies overlap; every invocation reads its
  // inputs, and the next one's are loaded while this one scans its table and
  // computes (one invocation ahead).
  V xn[KD];
  if (t_lead < T && t < T && t < n) {
#pragma unroll
    for (int d = 0; d < KD; ++d)
      if (d < D) xn[d] = in[d * stride + t];
  }
  if (has_state) {
    uint32_t *dst = reinterpret_cast<uint32_t *>(base);
    for (size_t q = lane; q < wbytes / 4; q += 32) dst[q] = wst[q];
  } else if (lane < g) {
    W.filled[lane] = 0;
    W.rr[lane] = 0;
  }
  if (threadIdx.x < 2) s_cnt[threadIdx.x] = 0;
  if (LEVEL == HPAC_LEVEL_BLOCK && threadIdx.x == 0) s_tally[0] = s_tally[1] = s_tally[2] = 0;
  __syncthreads();

  unsigned long long n_apx = 0, n_border = 0;

  if (t_lead < T) {
    int k3 = 0;
    for (int64_t i = t; t_lead + (i - t) < n; i += T) {
      const bool act = (t < T) && (i < n);
      V x[KD];
      if (act) {
#pragma unroll
        for (int d = 0; d < KD; ++d) x[d] = xn[d];
        if (i + T < n) {
#pragma unroll
          for (int d = 0; d < KD; ++d)
            if (d < D) xn[d] = in[d * stride + i + T];
        }
      }
      iact_step<R, LEVEL, DC, COUNT>(reg, W, P, D, g, L, tab, lane, act, i, x, out, mask, stat, s_tally,
                                     k3, n_apx, n_border);
    }
  }
  if (has_state) {  // save this warp's tables for the next call
    __syncwarp();
    const uint32_t *src = reinterpret_cast<const uint32_t *>(base);
    for (size_t q = lane; q < wbytes / 4; q += 32) wst[q] = src[q];
  }
  warp_count(s_cnt, n_apx, n_border);
  __syncthreads();
  if (counters && threadIdx.x == 0) {
    if (s_cnt[0]) atomicAdd(&counters[0], s_cnt[0]);
    if (s_cnt[1]) atomicAdd(&counters[1], s_cnt[1]);
  }
}

// Kept-state iACT at thread and warp level, the call's logical warps
// pipelined over persistent physical warps. Each physical warp works through
// logical warps lw = first, first + stride, ... with two table buffers in
// shared memory: while the invocations of one logical warp run on one
// buffer, the next logical warp's table image is copied into the other by
// cp.async (16-byte copies that hold no registers) and its first inputs are
// loaded into registers. The decisions, outputs and saved images are those
// of iact_kernel with one physical warp per logical warp.
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
               "l"(gmem_src)
               : "memory");
}

template <class R, int LEVEL, int DC, bool COUNT>
__global__ void __launch_bounds__(256) iact_kept_kernel(R reg, const typename R::T *__restrict__ in,
                                                        int64_t stride, typename R::T *__restrict__ out,
                                                        uint8_t *__restrict__ mask,
                                                        typename R::T *__restrict__ stat, int64_t n,
                                                        int64_t T, IactParams P,
                                                        unsigned long long *__restrict__ counters,
                                                        uint32_t *__restrict__ st) {
  using V = typename R::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ unsigned long long s_cnt[2];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  constexpr int KD = DC > 0 ? DC : kMaxIn;
  const int D = DC > 0 ? DC : P.D, tsize = P.tsize, g = P.g, L = P.L;
  const int tab = lane / L;
  const size_t wbytes = warp_table_bytes<V>(tsize, D, g);
  const size_t zb = ((size_t)tsize * D * g * sizeof(float) + 7) & ~(size_t)7;
  unsigned char *const buf0 = smem_raw + (size_t)warp * 2 * wbytes;  // buffers buf0 and buf0 + wbytes
  const int64_t nlw = (T + 31) / 32;
  const int64_t wstride = (int64_t)gridDim.x * (blockDim.x / 32);
  const int64_t first = (int64_t)blockIdx.x * (blockDim.x / 32) + warp;
  const int chunks = (int)(wbytes / 16);
  const unsigned char *img = reinterpret_cast<const unsigned char *>(st);
  if (threadIdx.x < 2) s_cnt[threadIdx.x] = 0;
  __syncthreads();

  V xn[KD];
  auto fetch = [&](int64_t lw, unsigned char *dst) {
    const unsigned char *src = img + (size_t)lw * wbytes;
    for (int q = lane; q < chunks; q += 32) cp_async16(dst + 16 * q, src + 16 * q);
    asm volatile("cp.async.commit_group;" ::: "memory");
    const int64_t t = lw * 32 + lane;
    if (t < T && t < n) {
#pragma unroll
      for (int d = 0; d < KD; ++d)
        if (d < D) xn[d] = in[d * stride + t];
    }
  };
  if (first < nlw) fetch(first, buf0);

  unsigned long long n_apx = 0, n_border = 0;
  int cur = 0, k3 = 0;
  for (int64_t lw = first; lw < nlw; lw += wstride) {
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncwarp();
    V xc[KD];
#pragma unroll
    for (int d = 0; d < KD; ++d) xc[d] = xn[d];
    if (lw + wstride < nlw) fetch(lw + wstride, buf0 + (cur ^ 1) * wbytes);
    unsigned char *base = buf0 + cur * wbytes;
    WarpTables<V> W;
    W.z = reinterpret_cast<float *>(base);
    W.y = reinterpret_cast<V *>(base + zb);
    W.filled = reinterpret_cast<int *>(base + zb + (size_t)tsize * g * sizeof(V));
    W.rr = W.filled + g;
    const int64_t t = lw * 32 + lane, t_lead = lw * 32;
    for (int64_t i = t; t_lead + (i - t) < n; i += T) {
      const bool act = (t < T) && (i < n);
      V x[KD];
      if (act) {
#pragma unroll
        for (int d = 0; d < KD; ++d) x[d] = xc[d];
        if (i + T < n) {
#pragma unroll
          for (int d = 0; d < KD; ++d)
            if (d < D) xc[d] = in[d * stride + i + T];
        }
      }
      iact_step<R, LEVEL, DC, COUNT>(reg, W, P, D, g, L, tab, lane, act, i, x, out, mask, stat, nullptr,
                                     k3, n_apx, n_border);
    }
    // save this logical warp's tables for the next call; the buffer is
    // refilled two logical warps later, after the __syncwarp below
    uint4 *dst = reinterpret_cast<uint4 *>(st + (size_t)lw * (wbytes / 4));
    const uint4 *src = reinterpret_cast<const uint4 *>(base);
    for (int q = lane; q < chunks; q += 32) dst[q] = src[q];
    __syncwarp();
    cur ^= 1;
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  warp_count(s_cnt, n_apx, n_border);
  __syncthreads();
  if (counters && threadIdx.x == 0) {
    if (s_cnt[0]) atomicAdd(&counters[0], s_cnt[0]);
    if (s_cnt[1]) atomicAdd(&counters[1], s_cnt[1]);
  }
}

template <class R>
hpac_status launch(hpac_region *r, R reg, const hpac_iact_knobs *k, const void *in, void *out,
                   uint8_t *mask, void *stat, unsigned long long *counters) {
  using V = typename R::T;
  const hpac_region_desc &d = r->d;
  if (d.n == 0) return HPAC_OK;
  IactParams P{};
  P.D = d.n_in;
  P.tsize = k->tsize;
  P.g = k->tperwarp;
  P.L = 32 / k->tperwarp;
  P.thr = (float)k->thresh;
  P.thr_d = k->thresh;
  for (int j = 0; j < kMaxIn; ++j) {
    const double s = (k->in_scale && j < d.n_in) ? k->in_scale[j] : 1.0;
    P.scale_d[j] = s;
    P.scale_f[j] = (float)s;
  }
  const int64_t T = logical_threads(d);
  const size_t wbytes = warp_table_bytes<V>(P.tsize, P.D, P.g);
  const int limit = max_dyn_smem(r->device);
  // At thread and warp level only the warp is semantic, so the physical block
  // may shrink, to spread the warps over all SMs and to fit the tables; at
  // block level B is part of the semantics.
  int B = d.block_threads;
  if (k->level != HPAC_LEVEL_BLOCK) {
    B = balanced_block(T, B, r->device);
    while (B > 32 && (size_t)(B / 32) * wbytes > (size_t)limit) B -= 32;
  }
  const size_t smem = (size_t)(B / 32) * wbytes;
  if (smem > (size_t)limit)
    return set_error(HPAC_EUNSUPPORTED, "iACT tables of %zu bytes per block exceed %d", smem, limit);
  // persistent state: one image of a warp's tables per logical warp
  const int64_t key[6] = {2, P.tsize, P.g, P.D, T, (int64_t)sizeof(V)};
  void *stv = nullptr;
  hpac_status ss = region_state(r, key, (size_t)((T + 31) / 32) * wbytes, &stv);
  if (ss != HPAC_OK) return ss;
  uint32_t *st_words = static_cast<uint32_t *>(stv);
  const int64_t blocks = (T + B - 1) / B;
  if (blocks > 0x7fffffffLL) return set_error(HPAC_EINVAL, "too many logical threads");
  V *o = static_cast<V *>(out);
  V *st = static_cast<V *>(stat);
  const V *x = static_cast<const V *>(in);
  constexpr int kDC = R::kReads == 4 ? 4 : 0;
  if (st_words && k->level != HPAC_LEVEL_BLOCK) {
    // kept state at thread or warp level: persistent warps, two buffers each
    int Bk = 256;
    while (Bk > 32 && (size_t)(Bk / 32) * 2 * wbytes > (size_t)limit) Bk -= 32;
    const size_t smem_k = (size_t)(Bk / 32) * 2 * wbytes;
    if (smem_k > (size_t)limit)
      return set_error(HPAC_EUNSUPPORTED, "iACT tables of %zu bytes per block exceed %d", smem_k, limit);
    auto fn = k->level == HPAC_LEVEL_THREAD
                  ? (counters ? iact_kept_kernel<R, HPAC_LEVEL_THREAD, kDC, true>
                              : iact_kept_kernel<R, HPAC_LEVEL_THREAD, kDC, false>)
                  : (counters ? iact_kept_kernel<R, HPAC_LEVEL_WARP, kDC, true>
                              : iact_kept_kernel<R, HPAC_LEVEL_WARP, kDC, false>);
    HPAC_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_k));
    int per_sm = 0;
    HPAC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, Bk, smem_k));
    if (per_sm < 1) per_sm = 1;
    const int64_t nlw = (T + 31) / 32;
    int64_t kb = (int64_t)sm_count(r->device) * per_sm;
    const int64_t need = (nlw + Bk / 32 - 1) / (Bk / 32);
    if (kb > need) kb = need;
    fn<<<(unsigned)kb, Bk, smem_k, r->stream>>>(reg, x, d.in_stride, o, mask, st, d.n, T, P, counters,
                                               st_words);
    HPAC_CUDA_TRY(cudaGetLastError());
    return HPAC_OK;
  }
  switch (k->level) {
    case HPAC_LEVEL_THREAD: {
      auto fn = st_words ? (counters ? iact_kernel<R, HPAC_LEVEL_THREAD, kDC, true, true>
                                     : iact_kernel<R, HPAC_LEVEL_THREAD, kDC, false, true>)
                         : (counters ? iact_kernel<R, HPAC_LEVEL_THREAD, kDC, true> : iact_kernel<R, HPAC_LEVEL_THREAD, kDC, false>);
      HPAC_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      fn<<<(unsigned)blocks, B, smem, r->stream>>>(reg, x, d.in_stride, o, mask, st, d.n, T, P, counters,
                                                   st_words);
      break;
    }
    case HPAC_LEVEL_WARP: {
      auto fn = st_words ? (counters ? iact_kernel<R, HPAC_LEVEL_WARP, kDC, true, true>
                                     : iact_kernel<R, HPAC_LEVEL_WARP, kDC, false, true>)
                         : (counters ? iact_kernel<R, HPAC_LEVEL_WARP, kDC, true> : iact_kernel<R, HPAC_LEVEL_WARP, kDC, false>);
      HPAC_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      fn<<<(unsigned)blocks, B, smem, r->stream>>>(reg, x, d.in_stride, o, mask, st, d.n, T, P, counters,
                                                   st_words);
      break;
    }
    default: {
      auto fn = st_words ? (counters ? iact_kernel<R, HPAC_LEVEL_BLOCK, kDC, true, true>
                                     : iact_kernel<R, HPAC_LEVEL_BLOCK, kDC, false, true>)
                         : (counters ? iact_kernel<R, HPAC_LEVEL_BLOCK, kDC, true> : iact_kernel<R, HPAC_LEVEL_BLOCK, kDC, false>);
      HPAC_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      fn<<<(unsigned)blocks, B, smem, r->stream>>>(reg, x, d.in_stride, o, mask, st, d.n, T, P, counters,
                                                   st_words);
      break;
    }
  }
  HPAC_CUDA_TRY(cudaGetLastError());
  return HPAC_OK;
}

// Identity reads only its first input for the exact value, but iACT needs all
// D inputs for the distance; the kernel loads them regardless of kReads.
}  // namespace

hpac_status launch_iact(hpac_region *r, const hpac_iact_knobs *k, const void *in, void *out,
                        uint8_t *mask, void *stat, unsigned long long *counters) {
  const hpac_region_desc &d = r->d;
  switch (d.kind) {
    case HPAC_REGION_BLACKSCHOLES:
      if (d.dtype == HPAC_F32)
        return launch(r, BlackScholes32{(float)d.param}, k, in, out, mask, stat, counters);
      return launch(r, BlackScholes64{d.param}, k, in, out, mask, stat, counters);
    case HPAC_REGION_EOS:
      return launch(r, Eos64{d.param}, k, in, out, mask, stat, counters);
    case HPAC_REGION_IDENTITY:
      if (d.dtype == HPAC_F32) return launch(r, Identity<float>{}, k, in, out, mask, stat, counters);
      return launch(r, Identity<double>{}, k, in, out, mask, stat, counters);
    case HPAC_REGION_KMEANS:
      return launch(r, KMeans32{static_cast<const float *>(r->aux), d.arg}, k, in, out, mask, stat,
                    counters);
  }
  return set_error(HPAC_EUNSUPPORTED, "region kind %d", d.kind);
}

}  // namespace hpac
