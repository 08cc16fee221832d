// Binomial Options region (Table 1): an American call priced on a
// Cox-Ross-Rubinstein tree, one option per team of 32 lanes (the paper gives a
// whole block to one option and decides per block, Section 4.2). The logical
// schedule counts teams: team t prices options i = t + k T in turn, and TAF /
// iACT / perforation decide per team at each of its steps k, exactly as the
// other regions' logical threads do at thread level.
//
// Tree layout: node j of the current level lives in register slot j / 32 of
// lane j % 32, so every lane keeps working while the level shrinks from N + 1
// nodes to one; a backward step reads the upper neighbour j + 1 with one
// shuffle per slot (lane 31 takes lane 0's next slot). No block barrier: a
// team is one warp. Four teams share a block.
#include <math.h>

#include "hpac_internal.cuh"
#include "perfo_rule.cuh"
#include "regions.cuh"

namespace hpac {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kTeams = 4;  // teams (warps) per block

struct TreeC {
  float puA, pdA, uf;
  double v;
};

// Per-option constants in double, rounded once: dt = T/N, v = sigma sqrt(dt),
// u = e^v, d = 1/u, a = e^{r dt}, pu = (a - d)/(u - d), weights pu/a, (1-pu)/a.
__device__ __forceinline__ TreeC tree_constants(float Tm, float sig, double r, int N) {
  const double dt = (double)Tm / N;
  const double v = (double)sig * sqrt(dt);
  const double u = exp(v), d = 1.0 / u, a = exp(r * dt);
  const double pu = (a - d) / (u - d), pd = 1.0 - pu;
  return TreeC{(float)(pu / a), (float)(pd / a), (float)u, v};
}

// Price of one option by the whole warp (all lanes return it). NPL register
// slots per lane hold 32 NPL >= N + 1 nodes.
template <int NPL>
__device__ __forceinline__ float team_price(float S0, float X, float Tm, float sig, double r, int N) {
  const int lane = threadIdx.x & 31;
  const TreeC c = tree_constants(Tm, sig, r, N);
  float V[NPL], S[NPL];
  // leaves S_j = S0 e^{v (2j - N)}: the lane's first by exp, the next slots by
  // the factor e^{64 v}, in double (a few double ulps from each leaf's own exp)
  double Sd = (double)S0 * exp(c.v * (double)(2 * lane - N));
  const double step = exp(64.0 * c.v);
#pragma unroll
  for (int s = 0; s < NPL; ++s) {
    const int j = 32 * s + lane;
    const float Sj = j <= N ? (float)Sd : 0.0f;
    Sd *= step;
    S[s] = Sj;
    V[s] = fmaxf(__fsub_rn(Sj, X), 0.0f);
  }
  const unsigned long long pu2 = f32x2_pack(c.puA, c.puA), pd2 = f32x2_pack(c.pdA, c.pdA);
  const unsigned long long uf2 = f32x2_pack(c.uf, c.uf), x2 = f32x2_pack(X, X);
  for (int n = N - 1; n >= 0; --n) {
    // slots in groups of four with one warp-uniform test per group (the level
    // has nodes 0..n; up to three slots past it are computed and never read),
    // so the four shuffles of a group issue back to back
#pragma unroll
    for (int s0 = 0; s0 < NPL; s0 += 4) {
      if (32 * s0 > n) break;
      float up[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int s = s0 + q;
        if (s < NPL) {
          const float send = lane == 0 ? (s + 1 < NPL ? V[s + 1] : 0.0f) : V[s];
          up[q] = __shfl_sync(kFull, send, (lane + 1) & 31);
        }
      }
      // two slots per packed instruction (each half rounded as the scalar
      // operation would be): continuation, the node's price and its exercise
#pragma unroll
      for (int q = 0; q < 4; q += 2) {
        const int s = s0 + q;
        if (s + 1 < NPL) {
          const unsigned long long cont =
              f32x2_fma(pu2, f32x2_pack(up[q], up[q + 1]), f32x2_mul(pd2, f32x2_pack(V[s], V[s + 1])));
          const unsigned long long sp = f32x2_mul(f32x2_pack(S[s], S[s + 1]), uf2);
          const unsigned long long ex = f32x2_sub(sp, x2);
          float c0, c1, e0, e1;
          f32x2_unpack(cont, c0, c1);
          f32x2_unpack(sp, S[s], S[s + 1]);
          f32x2_unpack(ex, e0, e1);
          V[s] = fmaxf(c0, e0);  // early exercise
          V[s + 1] = fmaxf(c1, e1);
        } else if (s < NPL) {
          const float cont = __fmaf_rn(c.puA, up[q], __fmul_rn(c.pdA, V[s]));
          S[s] = __fmul_rn(S[s], c.uf);
          V[s] = fmaxf(cont, __fsub_rn(S[s], X));
        }
      }
    }
  }
  return __shfl_sync(kFull, V[0], 0);
}

enum { TECH_EXACT = 0, TECH_TAF = 1, TECH_IACT = 2, TECH_PERFO = 3 };

struct BinoArgs {
  const float *in;
  int64_t stride, n, T;
  float *out;
  uint8_t *mask;
  float *stat;
  double r;
  int N;
  // TAF
  int h, p, thr_inf, reset;
  float thr;
  double thr_d;
  // iACT
  int tsize;
  float scale[4];
  // perforation
  DropRule rule;
  unsigned long long *counters;
};

// Shared memory per team: TAF window (h floats) or iACT table (tsize x 4
// scaled inputs, then tsize outputs).
template <int NPL, int TECH>
__global__ void __launch_bounds__(32 * kTeams) binomial_kernel(BinoArgs a) {
  extern __shared__ __align__(16) float sm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t team = (int64_t)blockIdx.x * kTeams + warp;
  const int per = TECH == TECH_TAF ? a.h : TECH == TECH_IACT ? 5 * a.tsize : 0;
  float *mine = sm + warp * per;
  unsigned long long n_alt = 0, n_border = 0;
  if (team < a.T) {
    // TAF state (uniform across the team's lanes)
    int pos = 0, cnt = 0, pred = 0;
    const float inv_h = TECH == TECH_TAF ? 1.0f / (float)a.h : 1.0f;
    // iACT state
    int filled = 0, rr = 0;
    for (int64_t k = 0, i = team; i < a.n; ++k, i += a.T) {
      if (TECH == TECH_PERFO) {
        bool drop;
        if (a.rule.kind == HPAC_PERFO_INI || a.rule.kind == HPAC_PERFO_FINI)
          drop = i < a.rule.lo || i >= a.rule.hi;
        else
          drop = a.rule.drop_key(a.rule.herded ? k : i);
        if (drop) {
          if (lane == 0 && a.mask) a.mask[i] = HPAC_MASK_SKIPPED;
          ++n_alt;
          continue;  // the output keeps the caller's value
        }
      }
      const float S0 = a.in[i], X = a.in[a.stride + i], Tm = a.in[2 * a.stride + i],
                  sig = a.in[3 * a.stride + i];
      if (TECH == TECH_TAF) {
        if (pred > 0) {
          const float y = mine[pos == 0 ? a.h - 1 : pos - 1];
          if (lane == 0) {
            a.out[i] = y;
            if (a.mask) a.mask[i] = HPAC_MASK_APPROX;
            if (a.stat) a.stat[i] = nan_v<float>();
          }
          --pred;
          ++n_alt;
          if (a.reset && pred == 0) cnt = 0;
          continue;
        }
        const float y = team_price<NPL>(S0, X, Tm, sig, a.r, a.N);
        __syncwarp();
        if (lane == 0) {
          a.out[i] = y;
          if (a.mask) a.mask[i] = HPAC_MASK_EXACT;
          mine[pos] = y;
        }
        __syncwarp();
        pos = pos + 1 == a.h ? 0 : pos + 1;
        cnt = cnt < a.h ? cnt + 1 : a.h;
        if (cnt == a.h) {
          bool wants;
          if (a.stat == nullptr && a.counters == nullptr && !a.thr_inf) {
            wants = rsd_below_fast<float>(mine, 1, pos, a.h, a.thr, inv_h);
          } else {
            const float s = window_rsd<float>(mine, 1, pos, a.h, inv_h);
            if (lane == 0 && a.stat) a.stat[i] = s;
            if (a.counters && borderline((double)s, a.thr_d)) ++n_border;
            wants = a.thr_inf || s < a.thr;
          }
          if (wants) pred = a.p;
        } else if (lane == 0 && a.stat) {
          a.stat[i] = nan_v<float>();
        }
        continue;
      }
      if (TECH == TECH_IACT) {
        const float z[4] = {__fmul_rn(a.scale[0], S0), __fmul_rn(a.scale[1], X),
                            __fmul_rn(a.scale[2], Tm), __fmul_rn(a.scale[3], sig)};
        // distances to the valid slots, two per lane, then the lowest-index minimum
        float best = INFINITY;
        int near = -1;
        for (int j = lane; j < filled; j += 32) {
          float acc = 0.0f;
#pragma unroll
          for (int d = 0; d < 4; ++d) {
            const float df = __fsub_rn(z[d], mine[4 * j + d]);
            acc = __fadd_rn(acc, __fmul_rn(df, df));
          }
          if (near < 0 || acc < best) {
            best = acc;
            near = j;
          }
        }
        for (int off = 16; off > 0; off >>= 1) {
          const float ob = __shfl_xor_sync(kFull, best, off);
          const int on = __shfl_xor_sync(kFull, near, off);
          if (on >= 0 && (near < 0 || ob < best || (ob == best && on < near))) {
            best = ob;
            near = on;
          }
        }
        const bool has = filled > 0;
        const float dmin = has ? __fsqrt_rn(best) : INFINITY;
        if (lane == 0 && a.stat) a.stat[i] = dmin;
        if (a.counters && has && borderline((double)dmin, a.thr_d)) ++n_border;
        if (has && dmin < a.thr) {
          if (lane == 0) {
            a.out[i] = mine[4 * a.tsize + near];
            if (a.mask) a.mask[i] = HPAC_MASK_APPROX;
          }
          ++n_alt;
          continue;
        }
        const float y = team_price<NPL>(S0, X, Tm, sig, a.r, a.N);
        __syncwarp();
        if (lane == 0) {
          a.out[i] = y;
          if (a.mask) a.mask[i] = HPAC_MASK_EXACT;
#pragma unroll
          for (int d = 0; d < 4; ++d) mine[4 * rr + d] = z[d];
          mine[4 * a.tsize + rr] = y;
        }
        __syncwarp();
        rr = rr + 1 == a.tsize ? 0 : rr + 1;
        filled = filled < a.tsize ? filled + 1 : a.tsize;
        continue;
      }
      const float y = team_price<NPL>(S0, X, Tm, sig, a.r, a.N);
      if (lane == 0) {
        a.out[i] = y;
        if (a.mask) a.mask[i] = HPAC_MASK_EXACT;
      }
    }
  }
  if (a.counters && lane == 0) {
    if (n_alt) atomicAdd(&a.counters[0], n_alt);
    if (n_border) atomicAdd(&a.counters[1], n_border);
  }
}

template <int NPL>
hpac_status launch_npl(const hpac_region *r, int tech, const BinoArgs &a, size_t smem) {
  const int64_t blocks = (a.T + kTeams - 1) / kTeams;
  if (blocks > 0x7fffffffLL) return set_error(HPAC_EINVAL, "too many logical teams");
  const dim3 grid((unsigned)blocks), block(32 * kTeams);
  switch (tech) {
    case TECH_TAF: binomial_kernel<NPL, TECH_TAF><<<grid, block, smem, r->stream>>>(a); break;
    case TECH_IACT: binomial_kernel<NPL, TECH_IACT><<<grid, block, smem, r->stream>>>(a); break;
    case TECH_PERFO: binomial_kernel<NPL, TECH_PERFO><<<grid, block, smem, r->stream>>>(a); break;
    default: binomial_kernel<NPL, TECH_EXACT><<<grid, block, smem, r->stream>>>(a); break;
  }
  HPAC_CUDA_TRY(cudaGetLastError());
  return HPAC_OK;
}

}  // namespace

hpac_status launch_binomial(hpac_region *r, int technique, const void *knobs, const void *in,
                            void *out, uint8_t *mask, void *stat, unsigned long long *counters) {
  const hpac_region_desc &d = r->d;
  if (d.n == 0) return HPAC_OK;
  BinoArgs a{};
  a.in = static_cast<const float *>(in);
  a.stride = d.in_stride;
  a.n = d.n;
  a.T = logical_threads(d);
  a.out = static_cast<float *>(out);
  a.mask = mask;
  a.stat = static_cast<float *>(stat);
  a.r = d.param;
  a.N = d.arg;
  a.counters = counters;
  a.rule.kind = -1;
  size_t smem = 0;
  if (technique == TECH_TAF) {
    const hpac_taf_knobs *k = static_cast<const hpac_taf_knobs *>(knobs);
    a.h = k->hsize;
    a.p = k->psize;
    a.thr = (float)k->thresh;
    a.thr_d = k->thresh;
    a.thr_inf = isinf(k->thresh) ? 1 : 0;
    a.reset = k->reset_on_exit;
    smem = (size_t)kTeams * a.h * sizeof(float);
  } else if (technique == TECH_IACT) {
    const hpac_iact_knobs *k = static_cast<const hpac_iact_knobs *>(knobs);
    a.tsize = k->tsize;
    a.thr = (float)k->thresh;
    a.thr_d = k->thresh;
    for (int j = 0; j < 4; ++j) a.scale[j] = k->in_scale ? (float)k->in_scale[j] : 1.0f;
    smem = (size_t)kTeams * 5 * a.tsize * sizeof(float);
  } else if (technique == TECH_PERFO) {
    const hpac_perfo_knobs *k = static_cast<const hpac_perfo_knobs *>(knobs);
    a.rule.kind = k->kind;
    a.rule.herded = k->herded ? 1 : 0;
    a.rule.m = k->m_or_percent;
    a.rule.seed = k->seed;
    a.rule.cut = (uint32_t)floor(k->rate * 16777216.0);
    a.rule.T = a.T;
    const int64_t cut = (d.n * (int64_t)k->m_or_percent) / 100;
    a.rule.lo = k->kind == HPAC_PERFO_INI ? cut : 0;
    a.rule.hi = k->kind == HPAC_PERFO_FINI ? d.n - cut : d.n;
  }
  const int nodes = a.N + 1;
  if (nodes <= 32 * 9) return launch_npl<9>(r, technique, a, smem);
  if (nodes <= 32 * 17) return launch_npl<17>(r, technique, a, smem);
  return launch_npl<33>(r, technique, a, smem);
}

}  // namespace hpac
