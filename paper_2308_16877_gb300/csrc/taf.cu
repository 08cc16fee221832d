// TAF: temporal approximate function memoization, HPAC-Offload GPU algorithm
// (Section 3.1.3, Figure 3(d); runtime Section 3.3; majority rules Section 3.3).
//
// One physical thread per logical thread t, walking its grid-stride sequence
// i = t + k*T. Its window of the last hsize accurate outputs lives in
// registers for hsize 2, 4 and 8, otherwise in shared memory (Section 3.1.1),
// column-major so that the lanes of a warp touch consecutive words:
// win[slot * blockDim.x + threadIdx.x]. A predicting
// thread stores the newest window value and issues no input load, so
// prediction removes the region's input bytes and arithmetic. At warp level the
// decision is a ballot + popcount over the lanes that computed this step; at
// block level each warp's count goes to a shared tally read after a barrier.
// Every lane of a group keeps looping until the group's first lane is done, so
// barriers and ballots are always reached by the whole group.
#include "hpac_internal.cuh"
#include "regions.cuh"

namespace hpac {
namespace {

// KH > 0: the history size is KH, known at compile time, and the window lives
// in registers (shifted on insertion, oldest first), so the statistic is two
// unrolled passes over registers. KH = 0: the window is in shared memory and h
// is a run-time argument.
// PERSIST: the window and owed predictions are read from and written back to
// st_* (persistent state); a separate instantiation so that the plain kernels
// carry none of its registers. Persistent runs use the shared-memory window.
template <class R, int LEVEL, int KH, bool PERSIST = false>
__global__ void __launch_bounds__(1024) taf_kernel(R reg, const typename R::T *__restrict__ in,
                                                   int64_t stride, typename R::T *__restrict__ out,
                                                   uint8_t *__restrict__ mask,
                                                   typename R::T *__restrict__ stat, int64_t n,
                                                   int64_t T, int h, int p,
                                                   typename R::T thr, int thr_inf, double thr_d,
                                                   int reset_on_exit,
                                                   unsigned long long *__restrict__ counters,
                                                   typename R::T *__restrict__ st_vals,
                                                   int *__restrict__ st_cnt,
                                                   int *__restrict__ st_pred) {
  using V = typename R::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ unsigned long long s_cnt[2];
  __shared__ int s_tally[3];
  V *win = reinterpret_cast<V *>(smem_raw);
  V w[KH > 0 ? KH : 1];  // register window (KH > 0), defined from the start
#pragma unroll
  for (int j = 0; j < (KH > 0 ? KH : 1); ++j) w[j] = (V)0;
  // double-precision register windows of 2 or 4 values also keep a
  // single-precision copy for the single-precision decision test
  // (rsd_below_f32); windows of 8 stay within the 64 registers of
  // 1024-thread blocks without it
  constexpr bool F32T = KH > 0 && KH <= 4 && sizeof(V) == 8;
  float wf[F32T ? KH : 1];
#pragma unroll
  for (int j = 0; j < (F32T ? KH : 1); ++j) wf[j] = 0.0f;
  const float thr_f = (float)thr;
  const bool thr_ok = F32T && !thr_inf && (double)thr >= 1e-7 && (double)thr <= 1e12;
  if (KH > 0) h = KH;
  const V inv_h = (V)1 / (V)h;
  const int ld = blockDim.x;
  const int lane = threadIdx.x & 31;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // first logical thread whose activity bounds this thread's loop
  const int64_t t_lead = LEVEL == HPAC_LEVEL_THREAD ? t
                         : LEVEL == HPAC_LEVEL_WARP ? t - lane
                                                    : (int64_t)blockIdx.x * blockDim.x;
  if (threadIdx.x < 2) s_cnt[threadIdx.x] = 0;
  if (LEVEL == HPAC_LEVEL_BLOCK && threadIdx.x == 0) s_tally[0] = s_tally[1] = s_tally[2] = 0;
  __syncthreads();

  int pos = 0;   // next slot to write
  int cnt = 0;   // filled slots
  int pred = 0;  // predictions still owed
  unsigned long long n_apx = 0, n_border = 0;
  // persistent state (st_vals[j * T + t], oldest first, j < cnt): resume
  if (PERSIST && t < T) {
    cnt = st_cnt[t];
    pred = st_pred[t];
    if (KH > 0) {
#pragma unroll
      for (int j = 0; j < (KH > 0 ? KH : 1); ++j)
        if (j >= KH - cnt) w[j] = st_vals[(int64_t)(j - (KH - cnt)) * T + t];
    } else {
      for (int j = 0; j < cnt; ++j) win[j * ld + threadIdx.x] = st_vals[(int64_t)j * T + t];
      pos = cnt == h ? 0 : cnt;
    }
  }

  if (t_lead < T) {
    int k3 = 0;  // step index mod 3 (block-level tally buffer)
    for (int64_t i = t; t_lead + (i - t) < n; i += T) {
      const bool act = (t < T) && (i < n);
      bool decided = false, wants = false;
      if (act) {
        if (pred > 0) {
          const int newest = pos == 0 ? h - 1 : pos - 1;
          out[i] = KH > 0 ? w[KH > 0 ? KH - 1 : 0] : win[newest * ld + threadIdx.x];
          if (mask) mask[i] = HPAC_MASK_APPROX;
          if (stat) stat[i] = nan_v<V>();
          --pred;
          ++n_apx;
          if (reset_on_exit && pred == 0) cnt = 0;  // the run ends: refill the window
        } else {
          V x[R::kReads];
#pragma unroll
          for (int d = 0; d < R::kReads; ++d) x[d] = in[d * stride + i];
          const V y = reg(x);
          out[i] = y;
          if (mask) mask[i] = HPAC_MASK_EXACT;
          if (KH > 0) {
#pragma unroll
            for (int j = 0; j + 1 < KH; ++j) w[j] = w[j + 1];
            w[KH > 0 ? KH - 1 : 0] = y;
            if (F32T) {
#pragma unroll
              for (int j = 0; j + 1 < (F32T ? KH : 1); ++j) wf[j] = wf[j + 1];
              wf[F32T ? KH - 1 : 0] = (float)y;
            }
          } else {
            win[pos * ld + threadIdx.x] = y;
            pos = (pos + 1 == h) ? 0 : pos + 1;
          }
          cnt = cnt < h ? cnt + 1 : h;
          decided = true;
          if (cnt == h) {
            V mu = (V)0, acc = (V)0;
            if (stat == nullptr && counters == nullptr && !thr_inf) {
              int f = -1;
              if constexpr (F32T) f = rsd_below_f32<KH>(wf, w, thr_f, thr_ok);
              if (f >= 0) {
                wants = f == 1;
              } else if (KH > 0) {
                reg_window_moments(w, inv_h, mu, acc);
                wants = rsd_below_moments(mu, acc, h, thr, inv_h);
              } else {
                wants = rsd_below_fast<V>(win + threadIdx.x, ld, pos, h, thr, inv_h);
              }
            } else {
              if (KH > 0) reg_window_moments(w, inv_h, mu, acc);
              const V s = KH > 0 ? rsd_from_moments(mu, acc, h, inv_h)
                                 : window_rsd<V>(win + threadIdx.x, ld, pos, h, inv_h);
              if (stat) stat[i] = s;
              if (counters) n_border += borderline((double)s, thr_d) ? 1 : 0;
              wants = thr_inf || s < thr;
            }
          } else if (stat) {
            stat[i] = nan_v<V>();
          }
        }
      }
      if (LEVEL == HPAC_LEVEL_THREAD) {
        if (decided && wants) pred = p;
      } else if (LEVEL == HPAC_LEVEL_WARP) {
        const unsigned dec = __ballot_sync(0xffffffffu, decided);
        const unsigned wan = __ballot_sync(0xffffffffu, decided && wants);
        if (2 * __popc(wan) > __popc(dec) && decided && cnt == h) pred = p;
      } else {
        const unsigned dec = __ballot_sync(0xffffffffu, decided);
        const unsigned wan = __ballot_sync(0xffffffffu, decided && wants);
        // Three tally buffers: step k adds into buffer k%3 and thread 0 clears
        // buffer (k+1)%3 before the barrier; that buffer was last read at step
        // k-2, before the barrier of step k-1, and is next written at step k+1,
        // after the barrier of step k.
        if (threadIdx.x == 0) s_tally[k3 == 2 ? 0 : k3 + 1] = 0;
        if (lane == 0) atomicAdd(&s_tally[k3], (__popc(wan) << 16) | __popc(dec));
        __syncthreads();
        const int tally = s_tally[k3];
        const int nw = tally >> 16, nd = tally & 0xffff;
        if (2 * nw > nd && decided && cnt == h) pred = p;
        k3 = k3 == 2 ? 0 : k3 + 1;
      }
    }
  }
  if (PERSIST && t < T) {  // persistent state: save where this thread stopped
    st_cnt[t] = cnt;
    st_pred[t] = pred;
    if (KH > 0) {
#pragma unroll
      for (int j = 0; j < (KH > 0 ? KH : 1); ++j)
        if (j >= KH - cnt) st_vals[(int64_t)(j - (KH - cnt)) * T + t] = w[j];
    } else {
      const int oldest = pos - cnt < 0 ? pos - cnt + h : pos - cnt;
      for (int j = 0; j < cnt; ++j) {
        const int slot = oldest + j >= h ? oldest + j - h : oldest + j;
        st_vals[(int64_t)j * T + t] = win[slot * ld + threadIdx.x];
      }
    }
  }
  warp_count(s_cnt, n_apx, n_border);
  __syncthreads();
  if (counters && threadIdx.x == 0) {
    if (s_cnt[0]) atomicAdd(&counters[0], s_cnt[0]);
    if (s_cnt[1]) atomicAdd(&counters[1], s_cnt[1]);
  }
}

template <class R>
hpac_status launch(hpac_region *r, R reg, const hpac_taf_knobs *k, const void *in, void *out,
                   uint8_t *mask, void *stat, unsigned long long *counters) {
  using V = typename R::T;
  const hpac_region_desc &d = r->d;
  if (d.n == 0) return HPAC_OK;
  const int64_t T = logical_threads(d);
  // persistent state: window values [h][T], then counts [T] and owed predictions [T]
  const size_t b_vals = align256((size_t)k->hsize * T * sizeof(V)), b_int = align256((size_t)T * 4);
  const int64_t key[6] = {1, k->hsize, T, (int64_t)sizeof(V), 0, 0};
  void *sbuf = nullptr;
  hpac_status ss = region_state(r, key, b_vals + 2 * b_int, &sbuf);
  if (ss != HPAC_OK) return ss;
  char *sb = static_cast<char *>(sbuf);
  V *st_vals = reinterpret_cast<V *>(sb);
  int *st_cnt = sb ? reinterpret_cast<int *>(sb + b_vals) : nullptr;
  int *st_pred = sb ? reinterpret_cast<int *>(sb + b_vals + b_int) : nullptr;
  // the block is part of the semantics at block level only
  const int B = k->level == HPAC_LEVEL_BLOCK ? d.block_threads
                                             : balanced_block(T, d.block_threads, r->device);
  const int h = k->hsize;
  // register-window sizes; persistent state runs the shared-memory window
  const int kh = !sb && (h == 2 || h == 4 || h == 8) ? h : 0;
  const size_t smem = kh ? 0 : (size_t)h * B * sizeof(V);
  const int limit = max_dyn_smem(r->device);
  if ((int64_t)smem > limit)
    return set_error(HPAC_EUNSUPPORTED, "TAF window of %zu bytes per block exceeds %d", smem, limit);
  const int64_t blocks = (T + B - 1) / B;
  if (blocks > 0x7fffffffLL) return set_error(HPAC_EINVAL, "too many logical threads");
  const V thr = (V)k->thresh;
  const int thr_inf = isinf(k->thresh) ? 1 : 0;
  V *o = static_cast<V *>(out);
  V *st = static_cast<V *>(stat);
  const V *x = static_cast<const V *>(in);
  const int lvl = k->level == HPAC_LEVEL_THREAD ? 0 : k->level == HPAC_LEVEL_WARP ? 1 : 2;
  using Fn = decltype(&taf_kernel<R, HPAC_LEVEL_THREAD, 0>);
  static const Fn table[3][4] = {
      {taf_kernel<R, HPAC_LEVEL_THREAD, 0>, taf_kernel<R, HPAC_LEVEL_THREAD, 2>,
       taf_kernel<R, HPAC_LEVEL_THREAD, 4>, taf_kernel<R, HPAC_LEVEL_THREAD, 8>},
      {taf_kernel<R, HPAC_LEVEL_WARP, 0>, taf_kernel<R, HPAC_LEVEL_WARP, 2>,
       taf_kernel<R, HPAC_LEVEL_WARP, 4>, taf_kernel<R, HPAC_LEVEL_WARP, 8>},
      {taf_kernel<R, HPAC_LEVEL_BLOCK, 0>, taf_kernel<R, HPAC_LEVEL_BLOCK, 2>,
       taf_kernel<R, HPAC_LEVEL_BLOCK, 4>, taf_kernel<R, HPAC_LEVEL_BLOCK, 8>}};
  static const Fn persistent[3] = {taf_kernel<R, HPAC_LEVEL_THREAD, 0, true>,
                                   taf_kernel<R, HPAC_LEVEL_WARP, 0, true>,
                                   taf_kernel<R, HPAC_LEVEL_BLOCK, 0, true>};
  const Fn fn = sb ? persistent[lvl] : table[lvl][kh == 0 ? 0 : kh == 2 ? 1 : kh == 4 ? 2 : 3];
  if (smem > 0)
    HPAC_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  fn<<<(unsigned)blocks, B, smem, r->stream>>>(reg, x, d.in_stride, o, mask, st, d.n, T, h, k->psize,
                                               thr, thr_inf, k->thresh, k->reset_on_exit, counters,
                                               st_vals, st_cnt, st_pred);
  HPAC_CUDA_TRY(cudaGetLastError());
  return HPAC_OK;
}

}  // namespace

hpac_status launch_taf(hpac_region *r, const hpac_taf_knobs *k, const void *in, void *out,
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
