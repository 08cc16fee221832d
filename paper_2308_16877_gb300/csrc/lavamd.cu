// LavaMD-style neighbour-box forces (Table 1, LavaMD: particle potential and
// forces from the particles of the neighbouring boxes). Section 5 approximates
// the force calculation for a neighbouring box with TAF and iACT and compares
// thread- and warp-level decisions (Figure 9).
//
// One block per home box, one thread per particle of the box (NP of
// ceil(NP / 32) * 32 threads). The block walks the box's neighbour sequence
// (the home box, then the touching boxes in the order dz, dy, dx); at each
// step the neighbour's NP particles are staged in shared memory once for the
// whole block. Each warp then sums the pair terms of its computing lanes'
// particles, four lanes to a particle (box_force), so its cost follows the
// number of particles it computes rather than the slowest lane. A step in
// which no thread of the block computes stages nothing, so decisions taken
// per block drop the step's loads as well as its arithmetic.
//
// TAF: per particle, a window of the last hsize accurate outputs (four
// components) in shared memory, column per thread; the statistic is the RSD
// of the window's potentials; a prediction repeats the newest output.
// iACT: the inputs are the particle's coordinates scaled to single precision;
// tables of tsize slots (scaled coordinates, four outputs) shared by
// 32 / tperwarp lanes; read, decide, execute and write phases with the write
// by the farthest exact lane of each table (a butterfly over its lanes).
// Decisions at warp and block level use the majority rules of the other
// regions (ballots, or block-wide counts at a barrier).
#include <math.h>

#include "fast_exp.cuh"
#include "hpac_internal.cuh"
#include "regions.cuh"

namespace hpac {
namespace {

enum { LMD_EXACT = 0, LMD_TAF = 1, LMD_IACT = 2 };
constexpr int kMaxParPerBox = 1024;
constexpr int kMaxBoxes1d = 1290;  // B^3 blocks stay below 2^31

struct LmdArgs {
  const double *rq;
  double *fv;
  uint8_t *mask;
  unsigned long long *counters;  // [0] approximated, [1] borderline
  int64_t P;
  int B, NP;
  double na2;  // -a2
  // TAF
  int h, p, reset, thr_inf;
  double thr;
  // iACT
  int tsize, g, L;
  float thr_f;
  double sc[3];
  ExpTang ex;  // the exponential's table and reduction constants
};

// Shared memory of a block of NL threads: the staged box (x, y, z, q rows of
// NP doubles), then the TAF windows (h x 4 x NL doubles) or the iACT tables
// (ntab x tsize x 4 output doubles, ntab x tsize x 3 key floats, ntab fill
// counts and ntab round-robin pointers).
__host__ __device__ inline size_t lmd_smem(int tech, int NP, int NL, int h, int tsize, int g) {
  size_t b = (size_t)32 * NP;
  if (tech == LMD_TAF) b += (size_t)32 * h * NL;
  if (tech == LMD_IACT) {
    const size_t ntab = (size_t)(NL / 32) * g;
    b += ntab * tsize * 32 + ((ntab * tsize * 12 + 7) & ~(size_t)7) + ntab * 8;
  }
  return b;
}

// The contribution of the staged box to every computing lane's particle,
// computed by the whole warp. The computing lanes' particles go in groups of
// eight; within a group four lanes share a particle, each sums the pair terms
// j = quarter + 4 t, and the four partial sums meet by two shuffle levels. So
// c computing lanes cost the warp ceil(c / 8) ceil(NP / 4) rounds of the pair
// loop, where one lane per particle would cost NP rounds whatever c is: a
// warp with a few computing lanes (thread-level decisions, or the last,
// partly filled warp of a box) is not held for a full pass. The exponential
// is Tang's table-driven one (10 FP64 operations against 15 for the
// library's) while every active lane's argument lies within +-700, the
// library's otherwise. Called by all lanes of the warp; y is written on the
// computing lanes only.
__device__ __forceinline__ void box_force(const double *__restrict__ sx, const double *__restrict__ sy,
                                          const double *__restrict__ sz, const double *__restrict__ sq,
                                          int NP, double na2, bool compute, double xp, double yp,
                                          double zp, const double *__restrict__ etab, double inv_l,
                                          double l1, double l2, double (&y)[4]) {
  constexpr unsigned kAll = 0xffffffffu;
  const int lane = threadIdx.x & 31, sub = lane >> 2, quarter = lane & 3;
  unsigned rest = __ballot_sync(kAll, compute);
  while (rest) {
    // this group: the next (up to) eight computing lanes, the s-th on sub-group s
    unsigned group = 0;
    int src = -1;
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const unsigned low = rest & (0u - rest);
      if (s == sub && low) src = __ffs(low) - 1;
      group |= low;
      rest ^= low;
    }
    const int from = src >= 0 ? src : lane;
    const double px = __shfl_sync(kAll, xp, from), py = __shfl_sync(kAll, yp, from),
                 pz = __shfl_sync(kAll, zp, from);
    double pot = 0.0, fx = 0.0, fy = 0.0, fz = 0.0;
    if (src >= 0) {
#pragma unroll 4
      for (int m = quarter; m < NP; m += 4) {
        const double dx = px - sx[m], dy = py - sy[m], dz = pz - sz[m];
        const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
        const double u = na2 * r2;
        const bool fast = exp_tang_in_range(u);
        double v;
        if (__all_sync(__activemask(), fast))
          v = exp_tang(u, etab, inv_l, l1, l2);
        else
          v = fast ? exp_tang(u, etab, inv_l, l1, l2) : exp(u);
        const double qv = sq[m] * v;
        const double t = qv + qv;  // q fs with fs = 2 v
        pot += qv;
        fx = fma(t, dx, fx);
        fy = fma(t, dy, fy);
        fz = fma(t, dz, fz);
      }
    }
#pragma unroll
    for (int off = 1; off < 4; off <<= 1) {
      pot += __shfl_xor_sync(kAll, pot, off);
      fx += __shfl_xor_sync(kAll, fx, off);
      fy += __shfl_xor_sync(kAll, fy, off);
      fz += __shfl_xor_sync(kAll, fz, off);
    }
    // each computing lane of the group takes its sub-group's sums
    const bool mine = (group >> lane) & 1u;
    const int at = mine ? 4 * __popc(group & ((1u << lane) - 1u)) : lane;
    const double r0 = __shfl_sync(kAll, pot, at), r1 = __shfl_sync(kAll, fx, at),
                 r2 = __shfl_sync(kAll, fy, at), r3 = __shfl_sync(kAll, fz, at);
    if (mine) {
      y[0] = r0;
      y[1] = r1;
      y[2] = r2;
      y[3] = r3;
    }
  }
}

template <int TECH, int LEVEL, int MAXT>
__global__ void __launch_bounds__(MAXT) lavamd_kernel(LmdArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ long long s_nb[27];
  __shared__ double s_exp[64];
  __shared__ int s_nn;
  __shared__ unsigned long long s_cnt[2];
  const int tid = threadIdx.x, lane = tid & 31, NL = blockDim.x, NP = a.NP;
  const int64_t hb = blockIdx.x, P = a.P;
  double *sx = reinterpret_cast<double *>(smem_raw);
  double *sy = sx + NP, *sz = sy + NP, *sq = sz + NP;
  double *win = sq + NP;  // TAF windows / iACT table outputs
  const int ntab = TECH == LMD_IACT ? (NL / 32) * a.g : 0;
  float *tkey = reinterpret_cast<float *>(win + (size_t)ntab * a.tsize * 4);
  int *tfill = reinterpret_cast<int *>(
      reinterpret_cast<unsigned char *>(win + (size_t)ntab * a.tsize * 4) +
      (((size_t)ntab * a.tsize * 12 + 7) & ~(size_t)7));
  int *trr = tfill + ntab;

  if (tid == 0) {
    const int B = a.B;
    const int hx = (int)(hb % B), hy = (int)((hb / B) % B), hz = (int)(hb / ((int64_t)B * B));
    int nn = 0;
    s_nb[nn++] = hb;
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          if (dx == 0 && dy == 0 && dz == 0) continue;
          const int x = hx + dx, y = hy + dy, z = hz + dz;
          if (x < 0 || y < 0 || z < 0 || x >= B || y >= B || z >= B) continue;
          s_nb[nn++] = ((long long)z * B + y) * B + x;
        }
    s_nn = nn;
    s_cnt[0] = s_cnt[1] = 0;
  }
  if (TECH == LMD_IACT)
    for (int t = tid; t < ntab; t += NL) tfill[t] = trr[t] = 0;
  for (int t = tid; t < 64; t += NL) s_exp[t] = a.ex.t[t];
  __syncthreads();

  const bool act = tid < NP;
  const int64_t pidx = hb * NP + tid;
  double xp = 0.0, yp = 0.0, zp = 0.0;
  if (act) {
    xp = a.rq[pidx];
    yp = a.rq[P + pidx];
    zp = a.rq[2 * P + pidx];
  }
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  unsigned long long n_apx = 0, n_border = 0;
  // TAF state
  int head = 0, cnt = 0, pred = 0;
  const double inv_h = TECH == LMD_TAF ? 1.0 / (double)a.h : 1.0;
  // iACT state: the lane's scaled coordinates and its table
  float z[3] = {0.0f, 0.0f, 0.0f};
  int tab = 0;
  if (TECH == LMD_IACT) {
    tab = (tid >> 5) * a.g + lane / a.L;
    z[0] = __double2float_rn(__dmul_rn(a.sc[0], xp));
    z[1] = __double2float_rn(__dmul_rn(a.sc[1], yp));
    z[2] = __double2float_rn(__dmul_rn(a.sc[2], zp));
  }

  const int nn = s_nn;
  for (int k = 0; k < nn; ++k) {
    const int64_t b = s_nb[k];
    double y[4] = {0.0, 0.0, 0.0, 0.0};
    bool compute = act, apx = false;
    // iACT read phase and decision
    float dmin = INFINITY;
    int near = -1;
    if (TECH == LMD_IACT) {
      bool has = false, wants = false;
      if (act) {
        const int f = tfill[tab];
        const float *kt = tkey + (size_t)tab * a.tsize * 3;
        float best = INFINITY;
        for (int j = 0; j < f; ++j) {
          float s = 0.0f;
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            const float df = __fsub_rn(z[d], kt[3 * j + d]);
            s = __fadd_rn(s, __fmul_rn(df, df));
          }
          if (near < 0 || s < best) {
            best = s;
            near = j;
          }
        }
        has = f > 0;
        if (has) {
          dmin = __fsqrt_rn(best);
          wants = dmin < a.thr_f;
          if (a.counters && borderline((double)dmin, a.thr)) ++n_border;
        }
      }
      if (LEVEL == HPAC_LEVEL_THREAD) {
        apx = act && wants;
      } else if (LEVEL == HPAC_LEVEL_WARP) {
        const int na = __popc(__ballot_sync(0xffffffffu, act));
        const int nw = __popc(__ballot_sync(0xffffffffu, act && wants));
        apx = 2 * nw > na && act && has;
      } else {
        const int na = __syncthreads_count(act);
        const int nw = __syncthreads_count(act && wants);
        apx = 2 * nw > na && act && has;
      }
      compute = act && !apx;
    }
    const bool predict = TECH == LMD_TAF && act && pred > 0;
    if (TECH == LMD_TAF) compute = act && !predict;

    // execute: stage the neighbour box if any thread computes
    if (__syncthreads_or(compute)) {
      const int64_t j0 = b * NP;
      for (int m = tid; m < NP; m += NL) {
        sx[m] = a.rq[j0 + m];
        sy[m] = a.rq[P + j0 + m];
        sz[m] = a.rq[2 * P + j0 + m];
        sq[m] = a.rq[3 * P + j0 + m];
      }
      __syncthreads();
    }
    box_force(sx, sy, sz, sq, NP, a.na2, compute, xp, yp, zp, s_exp, a.ex.inv_l, a.ex.l1, a.ex.l2, y);
    bool decided = false, wants = false;
    if (compute) {
      if (a.mask) a.mask[(int64_t)k * P + pidx] = HPAC_MASK_EXACT;
      if (TECH == LMD_TAF) {
        int slot;
        if (cnt < a.h) {
          slot = head + cnt;
          if (slot >= a.h) slot -= a.h;
          ++cnt;
        } else {
          slot = head;
          head = head + 1 == a.h ? 0 : head + 1;
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) win[(size_t)(slot * 4 + c) * NL + tid] = y[c];
        decided = true;
        if (cnt == a.h) {
          const double s = window_rsd<double>(win + tid, 4 * NL, head, a.h, inv_h);
          if (a.counters && borderline(s, a.thr)) ++n_border;
          wants = a.thr_inf || s < a.thr;
        }
      }
    } else if (predict) {
      int newest = head + cnt - 1;
      if (newest >= a.h) newest -= a.h;
#pragma unroll
      for (int c = 0; c < 4; ++c) y[c] = win[(size_t)(newest * 4 + c) * NL + tid];
      if (a.mask) a.mask[(int64_t)k * P + pidx] = HPAC_MASK_APPROX;
      ++n_apx;
      if (--pred == 0 && a.reset) cnt = 0;
    } else if (apx) {
      const double *yt = win + ((size_t)tab * a.tsize + near) * 4;
#pragma unroll
      for (int c = 0; c < 4; ++c) y[c] = yt[c];
      if (a.mask) a.mask[(int64_t)k * P + pidx] = HPAC_MASK_APPROX;
      ++n_apx;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[c] += y[c];

    if (TECH == LMD_TAF) {
      // decision at the requested level
      if (LEVEL == HPAC_LEVEL_THREAD) {
        if (decided && wants) pred = a.p;
      } else if (LEVEL == HPAC_LEVEL_WARP) {
        const int nd = __popc(__ballot_sync(0xffffffffu, decided));
        const int nw = __popc(__ballot_sync(0xffffffffu, decided && wants));
        if (2 * nw > nd && decided && cnt == a.h) pred = a.p;
      } else {
        const int nd = __syncthreads_count(decided);
        const int nw = __syncthreads_count(decided && wants);
        if (2 * nw > nd && decided && cnt == a.h) pred = a.p;
      }
    }
    if (TECH == LMD_IACT) {
      // write phase: per table, the exact lane farthest from it (lowest lane
      // on ties) stores its coordinates and outputs in the round-robin slot
      float key = compute ? dmin : -1.0f;
      int who = lane;
      for (int off = 1; off < a.L; off <<= 1) {
        const float ok = __shfl_xor_sync(0xffffffffu, key, off);
        const int ow = __shfl_xor_sync(0xffffffffu, who, off);
        if (ok > key || (ok == key && ow < who)) {
          key = ok;
          who = ow;
        }
      }
      if (key >= 0.0f && who == lane) {
        const int s = trr[tab];
        double *yt = win + ((size_t)tab * a.tsize + s) * 4;
        float *kt = tkey + ((size_t)tab * a.tsize + s) * 3;
#pragma unroll
        for (int c = 0; c < 4; ++c) yt[c] = y[c];
#pragma unroll
        for (int d = 0; d < 3; ++d) kt[d] = z[d];
        trr[tab] = s + 1 == a.tsize ? 0 : s + 1;
        if (tfill[tab] < a.tsize) tfill[tab] = tfill[tab] + 1;
      }
      __syncwarp();
    }
  }
  if (act) {
#pragma unroll
    for (int c = 0; c < 4; ++c) a.fv[(int64_t)c * P + pidx] = acc[c];
  }
  if (a.counters) {
    warp_count(s_cnt, n_apx, n_border);
    __syncthreads();
    if (tid == 0) {
      if (s_cnt[0]) atomicAdd(&a.counters[0], s_cnt[0]);
      if (s_cnt[1]) atomicAdd(&a.counters[1], s_cnt[1]);
    }
  }
}

template <int TECH, int LEVEL, int MAXT>
hpac_status launch_one(const LmdArgs &a, int64_t nbox, int NL, size_t smem, cudaStream_t st) {
  auto fn = lavamd_kernel<TECH, LEVEL, MAXT>;
  HPAC_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  fn<<<(unsigned)nbox, NL, smem, st>>>(a);
  HPAC_CUDA_TRY(cudaGetLastError());
  return HPAC_OK;
}

template <int TECH, int MAXT>
hpac_status launch_level(int level, const LmdArgs &a, int64_t nbox, int NL, size_t smem, cudaStream_t st) {
  switch (level) {
    case HPAC_LEVEL_WARP: return launch_one<TECH, HPAC_LEVEL_WARP, MAXT>(a, nbox, NL, smem, st);
    case HPAC_LEVEL_BLOCK: return launch_one<TECH, HPAC_LEVEL_BLOCK, MAXT>(a, nbox, NL, smem, st);
    default: return launch_one<TECH, HPAC_LEVEL_THREAD, MAXT>(a, nbox, NL, smem, st);
  }
}

template <int MAXT>
hpac_status launch_tech(int tech, int level, const LmdArgs &a, int64_t nbox, int NL, size_t smem,
                        cudaStream_t st) {
  if (tech == LMD_TAF) return launch_level<LMD_TAF, MAXT>(level, a, nbox, NL, smem, st);
  if (tech == LMD_IACT) return launch_level<LMD_IACT, MAXT>(level, a, nbox, NL, smem, st);
  return launch_one<LMD_EXACT, HPAC_LEVEL_THREAD, MAXT>(a, nbox, NL, smem, st);
}

}  // namespace
}  // namespace hpac

extern "C" hpac_status hpac_lavamd_run(const hpac_lavamd_desc *desc, int32_t technique,
                                       const void *knobs, const double *d_rq, double *d_fv,
                                       uint8_t *d_mask, hpac_stats *h_stats, void *cuda_stream) {
  using namespace hpac;
  TraceRange trace_("hpac_lavamd_run");
  if (!desc) return set_error(HPAC_EINVAL, "desc is NULL");
  const int B = desc->boxes1d, NP = desc->par_per_box;
  if (B < 0 || B > kMaxBoxes1d) return set_error(HPAC_EINVAL, "boxes1d %d outside 0..%d", B, kMaxBoxes1d);
  if (NP < 1 || NP > kMaxParPerBox)
    return set_error(HPAC_EINVAL, "par_per_box %d outside 1..%d", NP, kMaxParPerBox);
  if (!(desc->a2 >= 0.0) || isinf(desc->a2)) return set_error(HPAC_EINVAL, "a2 must be finite and >= 0");
  if (technique < LMD_EXACT || technique > LMD_IACT) return set_error(HPAC_EINVAL, "technique %d", technique);
  if (technique != LMD_EXACT && !knobs) return set_error(HPAC_EINVAL, "knobs are NULL");
  const int64_t nbox = (int64_t)B * B * B, P = nbox * NP;
  const int NL = (NP + 31) / 32 * 32;
  static const ExpTang kExp = exp_tang_constants();
  LmdArgs a{};
  a.ex = kExp;
  a.P = P;
  a.B = B;
  a.NP = NP;
  a.na2 = -desc->a2;
  a.mask = d_mask;
  int level = HPAC_LEVEL_THREAD;
  if (technique == LMD_TAF) {
    const hpac_taf_knobs *k = static_cast<const hpac_taf_knobs *>(knobs);
    if (k->hsize < 1 || k->hsize > kMaxHsize) return set_error(HPAC_EINVAL, "hsize %d", k->hsize);
    if (k->psize < 0) return set_error(HPAC_EINVAL, "psize %d", k->psize);
    if (!(k->thresh >= 0.0)) return set_error(HPAC_EINVAL, "thresh must be >= 0");
    if (k->reset_on_exit != 0 && k->reset_on_exit != 1) return set_error(HPAC_EINVAL, "reset_on_exit");
    level = k->level;
    a.h = k->hsize;
    a.p = k->psize;
    a.reset = k->reset_on_exit;
    a.thr = k->thresh;
    a.thr_inf = isinf(k->thresh) ? 1 : 0;
  } else if (technique == LMD_IACT) {
    const hpac_iact_knobs *k = static_cast<const hpac_iact_knobs *>(knobs);
    if (k->tsize < 1 || k->tsize > kMaxTsize) return set_error(HPAC_EINVAL, "tsize %d", k->tsize);
    const int g = k->tperwarp;
    if (g < 1 || g > 32 || (g & (g - 1)) != 0) return set_error(HPAC_EINVAL, "tperwarp %d", g);
    if (!(k->thresh >= 0.0)) return set_error(HPAC_EINVAL, "thresh must be >= 0");
    level = k->level;
    a.tsize = k->tsize;
    a.g = g;
    a.L = 32 / g;
    a.thr = k->thresh;
    a.thr_f = (float)k->thresh;
    for (int d = 0; d < 3; ++d) a.sc[d] = k->in_scale ? k->in_scale[d] : 1.0;
  }
  if (level < HPAC_LEVEL_THREAD || level > HPAC_LEVEL_BLOCK) return set_error(HPAC_EINVAL, "level %d", level);
  if (h_stats) *h_stats = hpac_stats{0, 0, 0, 0};
  if (P == 0) return HPAC_OK;
  if (!d_rq || !d_fv) return set_error(HPAC_EINVAL, "d_rq or d_fv is NULL");
  if (((uintptr_t)d_rq | (uintptr_t)d_fv) & 7) return set_error(HPAC_EINVAL, "d_rq and d_fv must be 8-byte aligned");
  int dev = 0;
  HPAC_CUDA_TRY(cudaGetDevice(&dev));
  const size_t smem = lmd_smem(technique, NP, NL, a.h, a.tsize, a.g);
  if (smem > (size_t)max_dyn_smem(dev))
    return set_error(HPAC_EINVAL, "the configuration needs %zu bytes of shared memory per block (limit %d)",
                     smem, max_dyn_smem(dev));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  unsigned long long *d_cnt = nullptr;
  if (h_stats) {
    HPAC_CUDA_TRY(cudaMallocAsync((void **)&d_cnt, 2 * sizeof(unsigned long long), st));
    HPAC_CUDA_TRY(cudaMemsetAsync(d_cnt, 0, 2 * sizeof(unsigned long long), st));
  }
  a.counters = d_cnt;
  a.rq = d_rq;
  a.fv = d_fv;
  hpac_status s = NL <= 256 ? launch_tech<256>(technique, level, a, nbox, NL, smem, st)
                            : launch_tech<1024>(technique, level, a, nbox, NL, smem, st);
  if (h_stats) {
    unsigned long long c[2] = {0, 0};
    if (s == HPAC_OK) {
      HPAC_CUDA_TRY(cudaMemcpyAsync(c, d_cnt, sizeof(c), cudaMemcpyDeviceToHost, st));
    }
    HPAC_CUDA_TRY(cudaFreeAsync(d_cnt, st));
    HPAC_CUDA_TRY(cudaStreamSynchronize(st));
    const int64_t per = 3 * (int64_t)B - 2;
    *h_stats = hpac_stats{per * per * per * NP, (int64_t)c[0], 0, (int64_t)c[1]};
  }
  return s;
}
