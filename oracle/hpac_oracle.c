/*
 * CPU oracle of the approximate-region hot path of HPAC-Offload
 * (Fink, Parasyris, Georgakoudis, Menon; arXiv 2308.16877).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path links, loads or calls
 * this file: only the tests, the smoke check of the entry module and the CPU
 * baseline leg of the benchmark do. It shares no code, header, table or
 * constant with the CUDA library; it is built from the paper's statement of
 * each technique, written out plainly and slowly.
 *
 * Compiled with -ffp-contract=off: every floating-point operation below is one
 * IEEE-rounded operation in the written order, so the decision statistics
 * (RSD, distances) are reproducible bit for bit by any implementation that
 * performs the same operations in the same order.
 *
 * Logical schedule (Section 3.1.3, Figure 3(d)): T logical threads; thread t
 * performs invocations i = t + k*T for k = 0, 1, ... while i < N (the
 * grid-stride loop). Warps are 32 consecutive logical threads, blocks are B
 * consecutive logical threads. All lanes of a block advance one step k
 * together; a lane with t >= T or i >= N is inactive at that step.
 *
 * Parity status: every function here is pinned by tests that do not reuse
 * this code (closed forms, brute force, library routines, textbook values).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORC_F32 = 0, ORC_F64 = 1 };
enum { ORC_BLACKSCHOLES = 0, ORC_EOS = 1, ORC_IDENTITY = 3, ORC_BINOMIAL = 4, ORC_KMEANS = 5 };
enum { ORC_THREAD = 0, ORC_WARP = 1, ORC_BLOCK = 2 };
enum { ORC_SMALL = 0, ORC_LARGE = 1, ORC_INI = 2, ORC_FINI = 3, ORC_RANDOM = 4 };
enum { ORC_EXACT = 0, ORC_APPROX = 1, ORC_SKIPPED = 2 };

#define ORC_WARP_SIZE 32
#define ORC_BORDER_REL 1e-6

typedef struct {
  int32_t kind;        /* ORC_BLACKSCHOLES / ORC_EOS / ORC_IDENTITY            */
  int32_t dtype;       /* ORC_F32 / ORC_F64                                    */
  int64_t n;           /* trip count N                                          */
  int32_t n_in;        /* D                                                     */
  int32_t n_out;       /* O (1 for every region here)                           */
  int64_t in_stride;   /* element d of invocation i at in[d*in_stride + i]      */
  int64_t out_stride;
  int64_t threads;     /* T; 0 means N                                          */
  int32_t block;       /* B, a multiple of 32                                   */
  double param;        /* r for Black-Scholes and Binomial, gamma for the EOS  */
  int32_t arg;         /* Binomial: tree steps; K-Means: clusters K; else 0    */
  int32_t pad;
  const float *aux;    /* K-Means: centroids [K][8]; NULL otherwise            */
} orc_region;

static int64_t logical_threads(const orc_region *R) {
  return R->threads > 0 ? R->threads : (R->n > 0 ? R->n : 1);
}

/* ------------------------------------------------------------------------ */
/* Exact regions                                                             */
/* ------------------------------------------------------------------------ */

/* European call under Black-Scholes (the Black-Scholes benchmark of Table 1):
 * C = S N(d1) - K e^{-rT} N(d2), d1 = (ln(S/K) + (r + sigma^2/2) T)/(sigma sqrt T),
 * d2 = d1 - sigma sqrt T, with N(x) = erfc(-x/sqrt 2)/2. */
static float bs_call_f32(float S, float K, float T, float sig, float r) {
  float sq = sqrtf(T);
  float sst = sig * sq;
  float d1 = (logf(S / K) + (r + 0.5f * sig * sig) * T) / sst;
  float d2 = d1 - sst;
  float n1 = 0.5f * erfcf(-d1 * 0.70710678118654752440f);
  float n2 = 0.5f * erfcf(-d2 * 0.70710678118654752440f);
  return S * n1 - K * expf(-r * T) * n2;
}

static double bs_call_f64(double S, double K, double T, double sig, double r) {
  double sq = sqrt(T);
  double sst = sig * sq;
  double d1 = (log(S / K) + (r + 0.5 * sig * sig) * T) / sst;
  double d2 = d1 - sst;
  double n1 = 0.5 * erfc(-d1 * 0.70710678118654752440);
  double n2 = 0.5 * erfc(-d2 * 0.70710678118654752440);
  return S * n1 - K * exp(-r * T) * n2;
}

/* Ideal-gas equation of state with an implicit trapezoid energy update.
 * Inputs: e_n (energy per reference volume), v_{n+1} (relative volume),
 * dv = v_{n+1} - v_n, q_{n+1} (artificial viscosity); output p_{n+1}.
 * e_{n+1} = e_n - (p_n + p_{n+1} + 2 q) dv / 2 with p = (gamma-1) e / v solves to
 * e_{n+1} = (e_n - dv (p_n + 2 q)/2) / (1 + (gamma-1) dv / (2 v_{n+1})),
 * clamped at zero; p_{n+1} = (gamma-1) e_{n+1} / v_{n+1}. */
static double eos_pressure(double e, double v1, double dv, double q, double g) {
  double v0 = v1 - dv;
  double p0 = (g - 1.0) * e / v0;
  double e1 = (e - 0.5 * dv * (p0 + 2.0 * q)) / (1.0 + 0.5 * (g - 1.0) * dv / v1);
  if (e1 < 0.0) e1 = 0.0;
  return (g - 1.0) * e1 / v1;
}

/* American call on a Cox-Ross-Rubinstein tree (Table 1, Binomial Options:
 * a portfolio of American options; tree after Podlozhnyuk 2008), single
 * precision, N steps. Per option, in double and then rounded: dt = T/N,
 * v = sigma sqrt(dt), u = e^v, d = 1/u, a = e^{r dt}, pu = (a - d)/(u - d),
 * pd = 1 - pu, the discounted weights pu/a and pd/a, and the leaf prices
 * S_j = S0 e^{v (2j - N)}, j = 0..N. Leaves V_j = max(S_j - X, 0). Each
 * backward step n = N-1 .. 0 moves every node price one level up (S_j <- S_j u,
 * since S0 u^{2j-n} = S0 u^{2j-(n+1)} u) and sets
 * V_j <- max(fma(pu/a, V_{j+1}, (pd/a) V_j), S_j - X) for j = 0..n (early
 * exercise). Returns V_0. Every single-precision operation is one IEEE
 * operation in this order (fmaf is the fused multiply-add). */
static float binomial_call_f32(float S0, float X, float T, float sig, double r, int N) {
  float V[4097], S[4097];
  if (N < 1 || N > 4096) return NAN;
  double dt = (double)T / N;
  double v = (double)sig * sqrt(dt);
  double u = exp(v), d = 1.0 / u, a = exp(r * dt);
  double pu = (a - d) / (u - d), pd = 1.0 - pu;
  float puA = (float)(pu / a), pdA = (float)(pd / a), uf = (float)u;
  for (int j = 0; j <= N; ++j) {
    S[j] = (float)((double)S0 * exp(v * (double)(2 * j - N)));
    V[j] = fmaxf(S[j] - X, 0.0f);
  }
  for (int n = N - 1; n >= 0; --n)
    for (int j = 0; j <= n; ++j) {
      float cont = fmaf(puA, V[j + 1], pdA * V[j]);
      S[j] = S[j] * uf;
      V[j] = fmaxf(cont, S[j] - X);
    }
  return V[0];
}

/* K-Means assignment (Table 1, K-Means: the cluster id of each observation;
 * Section 4.2 approximates the distance kernel): the index of the nearest of
 * the K centroids in squared Euclidean distance over the 8 features, each
 * distance summed in single precision over d = 0..7 in order, ties to the
 * lowest index. Returned as a float holding the integer id. */
static float kmeans_assign_f32(const float *x, const float *cent, int K) {
  int best = 0;
  float bd = 0.0f;
  for (int k = 0; k < K; ++k) {
    float acc = 0.0f;
    for (int d = 0; d < 8; ++d) {
      float df = x[d] - cent[k * 8 + d];
      float sq = df * df;
      acc = acc + sq;
    }
    if (k == 0 || acc < bd) {
      bd = acc;
      best = k;
    }
  }
  return (float)best;
}

static double in_at(const orc_region *R, const void *in, int d, int64_t i) {
  if (R->dtype == ORC_F32) return (double)((const float *)in)[d * R->in_stride + i];
  return ((const double *)in)[d * R->in_stride + i];
}

/* Exact output of invocation i (as a double holding the region-precision value). */
static double region_eval(const orc_region *R, const void *in, int64_t i) {
  switch (R->kind) {
    case ORC_BLACKSCHOLES:
      if (R->dtype == ORC_F32)
        return (double)bs_call_f32((float)in_at(R, in, 0, i), (float)in_at(R, in, 1, i),
                                   (float)in_at(R, in, 2, i), (float)in_at(R, in, 3, i),
                                   (float)R->param);
      return bs_call_f64(in_at(R, in, 0, i), in_at(R, in, 1, i), in_at(R, in, 2, i),
                         in_at(R, in, 3, i), R->param);
    case ORC_EOS:
      return eos_pressure(in_at(R, in, 0, i), in_at(R, in, 1, i), in_at(R, in, 2, i),
                          in_at(R, in, 3, i), R->param);
    case ORC_BINOMIAL:
      return (double)binomial_call_f32((float)in_at(R, in, 0, i), (float)in_at(R, in, 1, i),
                                       (float)in_at(R, in, 2, i), (float)in_at(R, in, 3, i),
                                       R->param, R->arg);
    case ORC_KMEANS: {
      float x[8];
      for (int d = 0; d < 8; ++d) x[d] = (float)in_at(R, in, d, i);
      return (double)kmeans_assign_f32(x, R->aux, R->arg);
    }
    case ORC_IDENTITY:
    default:
      return in_at(R, in, 0, i);
  }
}

static void out_put(const orc_region *R, void *out, int64_t i, double y) {
  if (R->dtype == ORC_F32) ((float *)out)[i] = (float)y;
  else ((double *)out)[i] = y;
}

static void stat_put(const orc_region *R, void *stat, int64_t i, double s) {
  if (!stat) return;
  if (R->dtype == ORC_F32) ((float *)stat)[i] = (float)s;
  else ((double *)stat)[i] = s;
}

static int check_region(const orc_region *R) {
  if (R->n < 0 || R->n_in < 1 || R->n_in > 8 || R->n_out != 1) return 1;
  if (R->in_stride < R->n || R->out_stride < R->n) return 1;
  if (R->block < 32 || R->block % 32 != 0 || R->threads < 0) return 1;
  if (R->dtype != ORC_F32 && R->dtype != ORC_F64) return 1;
  if (R->kind == ORC_BLACKSCHOLES && R->n_in != 4) return 1;
  if (R->kind == ORC_EOS && (R->n_in != 4 || R->dtype != ORC_F64)) return 1;
  if (R->kind == ORC_BINOMIAL && (R->n_in != 4 || R->dtype != ORC_F32 || R->arg < 1 || R->arg > 4096))
    return 1;
  if (R->kind == ORC_KMEANS && (R->n_in != 8 || R->dtype != ORC_F32 || R->arg < 1 || R->arg > 64 || !R->aux))
    return 1;
  return 0;
}

int orc_run_exact(const orc_region *R, const void *in, void *out) {
  if (check_region(R)) return 1;
  int64_t i;
#pragma omp parallel for schedule(static)
  for (i = 0; i < R->n; ++i) out_put(R, out, i, region_eval(R, in, i));
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Loop perforation (Section 2.3; herded variant Section 3.1.5;             */
/* runtime encounter counter Section 3.3)                                    */
/* ------------------------------------------------------------------------ */

/* SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): one counter-based draw. */
static uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Does invocation i (step k of its logical thread) get dropped?
 *  small:M   drop the M-th, 2M-th, ... encounter:        key mod M == M-1
 *  large:M   keep only the 1st, (M+1)-th, ... encounter: key mod M != 0 drops
 *  ini:P     drop the first floor(N P / 100) iterations of the loop
 *  fini:P    drop the last  floor(N P / 100) iterations of the loop
 *  random:r  drop iff the top 24 bits of splitmix64(seed ^ key) < floor(r 2^24)
 * key = k (the thread's encounter counter) when herded, so every thread of the
 * grid drops the same steps; key = i (the iteration index) otherwise. */
static int perfo_drop(int kind, int64_t m, double rate, uint64_t seed, int herded,
                      int64_t i, int64_t k, int64_t n) {
  int64_t key = herded ? k : i;
  switch (kind) {
    case ORC_SMALL: return key % m == m - 1;
    case ORC_LARGE: return key % m != 0;
    case ORC_INI: return i < (n * m) / 100;
    case ORC_FINI: return i >= n - (n * m) / 100;
    case ORC_RANDOM: {
      uint64_t cut = (uint64_t)floor(rate * 16777216.0);
      return (splitmix64(seed ^ (uint64_t)key) >> 40) < cut;
    }
  }
  return 0;
}

int orc_run_perfo(const orc_region *R, const void *in, int32_t kind, int32_t m_or_percent,
                  double rate, uint64_t seed, int32_t herded, void *out, uint8_t *mask,
                  int64_t *counters) {
  if (check_region(R)) return 1;
  if (kind < ORC_SMALL || kind > ORC_RANDOM) return 1;
  if ((kind == ORC_SMALL || kind == ORC_LARGE) && m_or_percent < 1) return 1;
  if ((kind == ORC_INI || kind == ORC_FINI) && (m_or_percent < 0 || m_or_percent > 100)) return 1;
  if (kind == ORC_RANDOM && !(rate >= 0.0 && rate <= 1.0)) return 1;
  int64_t T = logical_threads(R);
  int64_t skipped = 0;
  int64_t i;
#pragma omp parallel for schedule(static) reduction(+ : skipped)
  for (i = 0; i < R->n; ++i) {
    int64_t k = i / T;
    if (perfo_drop(kind, m_or_percent, rate, seed, herded, i, k, R->n)) {
      if (mask) mask[i] = ORC_SKIPPED;
      skipped++;
    } else {
      out_put(R, out, i, region_eval(R, in, i));
      if (mask) mask[i] = ORC_EXACT;
    }
  }
  if (counters) {
    counters[0] = R->n;
    counters[1] = 0;
    counters[2] = skipped;
    counters[3] = 0;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* TAF: temporal approximate function memoization                            */
/* (Section 2.3; GPU algorithm Section 3.1.3 / Figure 3(d); runtime 3.3)     */
/* ------------------------------------------------------------------------ */

/* Relative standard deviation of a window (oldest first), population moments,
 * two passes, in single precision: RSD = sigma/|mu|; 0/0 reads as 0 and
 * sigma/0 with sigma > 0 as +inf. */
static float rsd_f32(const float *w, int h) {
  float sum = 0.0f;
  for (int j = 0; j < h; ++j) sum = sum + w[j];
  float mu = sum / (float)h;
  float acc = 0.0f;
  for (int j = 0; j < h; ++j) {
    float d = w[j] - mu;
    float d2 = d * d;
    acc = acc + d2;
  }
  float var = acc / (float)h;
  float sd = sqrtf(var);
  float amu = fabsf(mu);
  if (amu == 0.0f) return var == 0.0f ? 0.0f : INFINITY;
  return sd / amu;
}

static double rsd_f64(const double *w, int h) {
  double sum = 0.0;
  for (int j = 0; j < h; ++j) sum = sum + w[j];
  double mu = sum / (double)h;
  double acc = 0.0;
  for (int j = 0; j < h; ++j) {
    double d = w[j] - mu;
    double d2 = d * d;
    acc = acc + d2;
  }
  double var = acc / (double)h;
  double sd = sqrt(var);
  double amu = fabs(mu);
  if (amu == 0.0) return var == 0.0 ? 0.0 : INFINITY;
  return sd / amu;
}

static int is_borderline(double s, double thr) {
  if (isinf(thr) || isnan(s)) return 0;
  return fabs(s - thr) <= ORC_BORDER_REL * thr;
}

/* Per logical thread: a FIFO window of the last h accurate outputs (cnt of them
 * filled) and the number of predictions still owed (pred). Everything starts
 * empty at kernel start: the state is scoped to one kernel launch
 * (Section 3.1.1). At each step:
 *   pred > 0:  output the newest window value, pred -= 1, window unchanged;
 *   otherwise: compute exactly, push the output (dropping the oldest when full);
 *              once the window is full the thread wants to predict iff
 *              RSD(window) < thr (or thr is +inf).
 * Level thread: a thread that wants to predict sets pred = p. Level warp/block
 * (Section 3.3, majority rules): among the group's lanes that computed exactly
 * at this step, if more than half want to, every one of them with a full
 * window sets pred = p; otherwise none does. After the p predictions the
 * window is kept, so the next accurate output slides it and re-tests (the
 * default reading; with reset = 1, the alternative reading, it is emptied and
 * h accurate outputs refill it before the next test). */
/* Replay (force != NULL): the decisions are read from a mask produced
 * elsewhere instead of being taken; the state advances along that mask (an
 * invocation marked approximate outputs the newest window value), and at
 * every decision point (a group step whose lanes computed exactly) the
 * oracle's own decision is compared with the mask's, read from each deciding
 * lane's next invocation. disagree[i] = 1 at the decision invocation of a lane
 * whose mask decision differs from the oracle's; counts[0] = deciding lanes
 * compared, counts[1] = disagreements, counts[2] = structural errors (the mask
 * approximates where no prediction can be owed, or breaks a prediction run). */
static int taf_core(const orc_region *R, const void *in, int32_t hsize, int32_t psize, double thr,
                    int32_t level, int32_t reset, const uint8_t *force, void *out, uint8_t *mask, void *stat,
                    uint8_t *disagree, int64_t *counters, int64_t *counts, double *st_vals,
                    int32_t *st_cnt, int32_t *st_pred) {
  if (check_region(R)) return 1;
  if (hsize < 1 || hsize > 64 || psize < 0 || !(thr >= 0.0)) return 1;
  if (level < ORC_THREAD || level > ORC_BLOCK || (reset != 0 && reset != 1)) return 1;
  const int64_t N = R->n, T = logical_threads(R);
  const int B = R->block, h = hsize;
  const int64_t nblocks = (T + B - 1) / B;
  const int f32 = R->dtype == ORC_F32;
  const float thr_f = (float)thr;
  const int thr_inf = isinf(thr);
  int64_t approx_total = 0, border_total = 0, n_cmp = 0, n_dis = 0, n_bad = 0;
  int64_t b;
#pragma omp parallel for schedule(dynamic, 1) \
    reduction(+ : approx_total, border_total, n_cmp, n_dis, n_bad)
  for (b = 0; b < nblocks; ++b) {
    double *win = (double *)calloc((size_t)B * h, sizeof(double));
    int *head = (int *)calloc(B, sizeof(int));   /* slot of the oldest value   */
    int *cnt = (int *)calloc(B, sizeof(int));
    int64_t *pred = (int64_t *)calloc(B, sizeof(int64_t));
    int *act = (int *)calloc(B, sizeof(int));
    int *decided = (int *)calloc(B, sizeof(int)); /* computed exactly this step */
    int *wants = (int *)calloc(B, sizeof(int));
    int *own = (int *)calloc(B, sizeof(int));     /* the oracle's own decision */
    float wf[64];
    double wd[64];
    if (st_cnt) /* persistent state: each logical thread resumes where it stopped */
      for (int l = 0; l < B && b * B + l < T; ++l) {
        int64_t t = b * B + l;
        cnt[l] = st_cnt[t];
        pred[l] = st_pred[t];
        head[l] = 0;
        for (int j = 0; j < cnt[l]; ++j) win[(size_t)l * h + j] = st_vals[(int64_t)j * T + t];
      }
    for (int64_t k = 0; b * B + k * T < N; ++k) {
      /* phase 1: per-thread path */
      for (int l = 0; l < B; ++l) {
        int64_t t = b * B + l, i = t + k * T;
        act[l] = (t < T) && (i < N);
        decided[l] = 0;
        wants[l] = 0;
        if (!act[l]) continue;
        double *w = win + (size_t)l * h;
        if (force) {
          /* the mask's decision; an owed prediction must be honoured */
          int apx = force[i] == ORC_APPROX;
          if (apx != (pred[l] > 0)) {
            n_bad++;
            if (apx && cnt[l] == 0) apx = 0;  /* nothing to repeat: compute */
          }
          pred[l] = apx ? (pred[l] > 0 ? pred[l] : 1) : 0;
        }
        if (pred[l] > 0) {
          int newest = (head[l] + cnt[l] - 1) % h;
          out_put(R, out, i, w[newest]);
          if (mask) mask[i] = ORC_APPROX;
          stat_put(R, stat, i, NAN);
          pred[l] -= 1;
          approx_total++;
          /* alternative reading: the window is emptied when a run ends */
          if (reset && pred[l] == 0) cnt[l] = 0;
          continue;
        }
        double y = region_eval(R, in, i);
        out_put(R, out, i, y);
        if (mask) mask[i] = ORC_EXACT;
        decided[l] = 1;
        if (cnt[l] < h) {
          w[(head[l] + cnt[l]) % h] = y;
          cnt[l] += 1;
        } else {
          w[head[l]] = y;
          head[l] = (head[l] + 1) % h;
        }
        if (cnt[l] == h) {
          double s;
          int want;
          if (f32) {
            for (int j = 0; j < h; ++j) wf[j] = (float)w[(head[l] + j) % h];
            float sf = rsd_f32(wf, h);
            s = sf;
            want = thr_inf || sf < thr_f;
          } else {
            for (int j = 0; j < h; ++j) wd[j] = w[(head[l] + j) % h];
            s = rsd_f64(wd, h);
            want = thr_inf || s < thr;
          }
          stat_put(R, stat, i, s);
          border_total += is_borderline(s, thr);
          wants[l] = want;
        } else {
          stat_put(R, stat, i, NAN);
        }
      }
      /* phase 2: decision at the requested level */
      for (int l = 0; l < B; ++l) own[l] = 0;
      if (level == ORC_THREAD) {
        for (int l = 0; l < B; ++l) own[l] = decided[l] && wants[l];
      } else {
        int gsize = level == ORC_WARP ? ORC_WARP_SIZE : B;
        for (int g0 = 0; g0 < B; g0 += gsize) {
          int n_dec = 0, n_want = 0;
          for (int l = g0; l < g0 + gsize; ++l) {
            n_dec += decided[l];
            n_want += decided[l] && wants[l];
          }
          if (2 * n_want > n_dec)
            for (int l = g0; l < g0 + gsize; ++l) own[l] = decided[l] && cnt[l] == h;
        }
      }
      for (int l = 0; l < B; ++l) {
        if (!decided[l]) continue;
        if (!force) {
          if (own[l]) pred[l] = psize;
          continue;
        }
        /* replay: the mask's decision shows at the lane's next invocation */
        int64_t t = b * B + l, inext = t + (k + 1) * T;
        if (inext >= N) continue;
        int mask_yes = force[inext] == ORC_APPROX;
        int own_yes = own[l] && psize > 0;
        n_cmp++;
        if (mask_yes != own_yes) {
          n_dis++;
          if (disagree) disagree[t + k * T] = 1;
        }
        pred[l] = mask_yes ? psize : 0;
        if (mask_yes && psize == 0) n_bad++;
      }
    }
    if (st_cnt)
      for (int l = 0; l < B && b * B + l < T; ++l) {
        int64_t t = b * B + l;
        st_cnt[t] = cnt[l];
        st_pred[t] = (int32_t)pred[l];
        for (int j = 0; j < cnt[l]; ++j)
          st_vals[(int64_t)j * T + t] = win[(size_t)l * h + (head[l] + j) % h];
      }
    free(win); free(head); free(cnt); free(pred); free(act); free(decided); free(wants); free(own);
  }
  if (counters) {
    counters[0] = N;
    counters[1] = approx_total;
    counters[2] = 0;
    counters[3] = border_total;
  }
  if (counts) {
    counts[0] = n_cmp;
    counts[1] = n_dis;
    counts[2] = n_bad;
  }
  return 0;
}

int orc_run_taf(const orc_region *R, const void *in, int32_t hsize, int32_t psize, double thr,
                int32_t level, int32_t reset, void *out, uint8_t *mask, void *stat,
                int64_t *counters) {
  return taf_core(R, in, hsize, psize, thr, level, reset, NULL, out, mask, stat, NULL, counters,
                  NULL, NULL, NULL, NULL);
}

/* TAF with state kept across calls (not in the paper, whose state is scoped to
 * one kernel, Section 3.1.1): per logical thread t the window (st_vals[j*T + t],
 * oldest first, j < st_cnt[t]) and the predictions still owed (st_pred[t]) are
 * read at the start and written back at the end. Zeroed arrays are the empty
 * state of a first call. */
int orc_run_taf_persist(const orc_region *R, const void *in, int32_t hsize, int32_t psize,
                        double thr, int32_t level, int32_t reset, double *st_vals,
                        int32_t *st_cnt, int32_t *st_pred, void *out, uint8_t *mask, void *stat,
                        int64_t *counters) {
  if (!st_vals || !st_cnt || !st_pred) return 1;
  return taf_core(R, in, hsize, psize, thr, level, reset, NULL, out, mask, stat, NULL, counters,
                  NULL, st_vals, st_cnt, st_pred);
}

/* Replay of a TAF run along a given mask (see taf_core). */
int orc_replay_taf(const orc_region *R, const void *in, int32_t hsize, int32_t psize, double thr,
                   int32_t level, int32_t reset, const uint8_t *force, void *out, void *stat,
                   uint8_t *disagree, int64_t *counts) {
  if (!force) return 1;
  return taf_core(R, in, hsize, psize, thr, level, reset, force, out, NULL, stat, disagree, NULL,
                  counts, NULL, NULL, NULL);
}

/* ------------------------------------------------------------------------ */
/* iACT: approximate input memoization with tables shared within a warp      */
/* (Section 2.3; sharing Section 3.1.4; read/write phases Section 3.3)       */
/* ------------------------------------------------------------------------ */

/* Scaled input of dimension d, rounded to single precision: the product
 * in_scale[d] * x_d is formed in the region's precision. */
static float scaled_input(const orc_region *R, const void *in, const double *scale, int d,
                          int64_t i) {
  double s = scale ? scale[d] : 1.0;
  if (R->dtype == ORC_F32) {
    float x = ((const float *)in)[d * R->in_stride + i];
    return (float)s * x;
  }
  double x = ((const double *)in)[d * R->in_stride + i];
  return (float)(s * x);
}

/* g = tperwarp tables per warp; lanes [j*32/g, (j+1)*32/g) share table j. A
 * table holds tsize slots of (scaled input z, output y), all invalid at kernel
 * start, and a round-robin pointer. At each step:
 *   read:   each active lane finds the nearest valid slot, Euclidean distance
 *           d = sqrt(sum_d (z_d - slot_d)^2) in single precision (ties to the
 *           lowest slot); it wants to approximate iff a slot exists and d < thr;
 *   decide: thread level - lanes that want do; warp/block level - if more than
 *           half of the group's active lanes want, every active lane that has a
 *           valid slot takes its nearest slot's output, the rest compute;
 *   write:  (after the phase barrier) per table, among the lanes that computed
 *           exactly, the one farthest from the table (largest d, +inf for an
 *           empty table; ties to the lowest lane) stores (z, y) in the
 *           round-robin slot, which then advances. One write per table per step. */
static int iact_core(const orc_region *R, const void *in, int32_t tsize, int32_t tperwarp,
                     double thr, int32_t level, const double *in_scale, void *out, uint8_t *mask,
                     void *stat, int64_t *counters, float *st_z, double *st_y, int32_t *st_valid,
                     int32_t *st_rr) {
  if (check_region(R)) return 1;
  if (tsize < 1 || tsize > 64 || !(thr >= 0.0)) return 1;
  if (tperwarp < 1 || tperwarp > 32 || 32 % tperwarp != 0) return 1;
  if (level < ORC_THREAD || level > ORC_BLOCK) return 1;
  const int64_t N = R->n, T = logical_threads(R);
  const int B = R->block, D = R->n_in, L = 32 / tperwarp;
  const int ntab = (B / 32) * tperwarp;
  const int64_t nblocks = (T + B - 1) / B;
  const float thr_f = (float)thr;
  int64_t approx_total = 0, border_total = 0;
  int64_t b;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : approx_total, border_total)
  for (b = 0; b < nblocks; ++b) {
    float *tz = (float *)calloc((size_t)ntab * tsize * D, sizeof(float));
    double *ty = (double *)calloc((size_t)ntab * tsize, sizeof(double));
    int *tvalid = (int *)calloc((size_t)ntab * tsize, sizeof(int));
    int *rr = (int *)calloc(ntab, sizeof(int));
    int *act = (int *)calloc(B, sizeof(int));
    int *has = (int *)calloc(B, sizeof(int));
    int *wants = (int *)calloc(B, sizeof(int));
    int *apx = (int *)calloc(B, sizeof(int));
    int *near = (int *)calloc(B, sizeof(int));
    float *dmin = (float *)calloc(B, sizeof(float));
    float *z = (float *)calloc((size_t)B * D, sizeof(float));
    double *yv = (double *)calloc(B, sizeof(double));
    /* persistent state: the tables of logical warp w are st_*[w][table][slot] */
    const int64_t nwarps = (T + 31) / 32;
    if (st_rr)
      for (int tab = 0; tab < ntab; ++tab) {
        int64_t w = (b * B) / 32 + tab / tperwarp;
        if (w >= nwarps) break;
        int64_t g = w * tperwarp + tab % tperwarp;
        rr[tab] = st_rr[g];
        for (int j = 0; j < tsize; ++j) {
          size_t s = (size_t)tab * tsize + j;
          int64_t gs = g * tsize + j;
          tvalid[s] = st_valid[gs];
          ty[s] = st_y[gs];
          for (int d = 0; d < D; ++d) tz[s * D + d] = st_z[gs * D + d];
        }
      }
    for (int64_t k = 0; b * B + k * T < N; ++k) {
      /* read phase */
      for (int l = 0; l < B; ++l) {
        int64_t t = b * B + l, i = t + k * T;
        act[l] = (t < T) && (i < N);
        has[l] = wants[l] = apx[l] = 0;
        dmin[l] = INFINITY;
        near[l] = -1;
        if (!act[l]) continue;
        int tab = (l / 32) * tperwarp + (l % 32) / L;
        for (int d = 0; d < D; ++d) z[l * D + d] = scaled_input(R, in, in_scale, d, i);
        float best = INFINITY;
        for (int j = 0; j < tsize; ++j) {
          size_t s = (size_t)tab * tsize + j;
          if (!tvalid[s]) continue;
          float acc = 0.0f;
          for (int d = 0; d < D; ++d) {
            float df = z[l * D + d] - tz[s * D + d];
            float sq = df * df;
            acc = acc + sq;
          }
          if (!has[l] || acc < best) {
            best = acc;
            near[l] = j;
          }
          has[l] = 1;
        }
        if (has[l]) {
          dmin[l] = sqrtf(best);
          wants[l] = dmin[l] < thr_f;
        }
      }
      /* decision */
      if (level == ORC_THREAD) {
        for (int l = 0; l < B; ++l) apx[l] = act[l] && wants[l];
      } else {
        int gsize = level == ORC_WARP ? ORC_WARP_SIZE : B;
        for (int g0 = 0; g0 < B; g0 += gsize) {
          int n_act = 0, n_want = 0;
          for (int l = g0; l < g0 + gsize; ++l) {
            n_act += act[l];
            n_want += act[l] && wants[l];
          }
          int maj = 2 * n_want > n_act;
          for (int l = g0; l < g0 + gsize; ++l) apx[l] = maj && act[l] && has[l];
        }
      }
      /* execute */
      for (int l = 0; l < B; ++l) {
        if (!act[l]) continue;
        int64_t i = b * B + l + k * T;
        int tab = (l / 32) * tperwarp + (l % 32) / L;
        if (apx[l]) {
          yv[l] = ty[(size_t)tab * tsize + near[l]];
          if (mask) mask[i] = ORC_APPROX;
          approx_total++;
        } else {
          yv[l] = region_eval(R, in, i);
          if (mask) mask[i] = ORC_EXACT;
        }
        out_put(R, out, i, yv[l]);
        stat_put(R, stat, i, (double)dmin[l]);
        if (has[l]) border_total += is_borderline((double)dmin[l], thr);
      }
      /* write phase */
      for (int tab = 0; tab < ntab; ++tab) {
        int l0 = (tab / tperwarp) * 32 + (tab % tperwarp) * L;
        int writer = -1;
        for (int l = l0; l < l0 + L; ++l) {
          if (!act[l] || apx[l]) continue;
          if (writer < 0 || dmin[l] > dmin[writer]) writer = l;
        }
        if (writer < 0) continue;
        size_t s = (size_t)tab * tsize + rr[tab];
        for (int d = 0; d < D; ++d) tz[s * D + d] = z[writer * D + d];
        ty[s] = yv[writer];
        tvalid[s] = 1;
        rr[tab] = (rr[tab] + 1) % tsize;
      }
    }
    if (st_rr)
      for (int tab = 0; tab < ntab; ++tab) {
        int64_t w = (b * B) / 32 + tab / tperwarp;
        if (w >= nwarps) break;
        int64_t g = w * tperwarp + tab % tperwarp;
        st_rr[g] = rr[tab];
        for (int j = 0; j < tsize; ++j) {
          size_t s = (size_t)tab * tsize + j;
          int64_t gs = g * tsize + j;
          st_valid[gs] = tvalid[s];
          st_y[gs] = ty[s];
          for (int d = 0; d < D; ++d) st_z[gs * D + d] = tz[s * D + d];
        }
      }
    free(tz); free(ty); free(tvalid); free(rr); free(act); free(has); free(wants);
    free(apx); free(near); free(dmin); free(z); free(yv);
  }
  if (counters) {
    counters[0] = N;
    counters[1] = approx_total;
    counters[2] = 0;
    counters[3] = border_total;
  }
  return 0;
}

int orc_run_iact(const orc_region *R, const void *in, int32_t tsize, int32_t tperwarp,
                 double thr, int32_t level, const double *in_scale, void *out, uint8_t *mask,
                 void *stat, int64_t *counters) {
  return iact_core(R, in, tsize, tperwarp, thr, level, in_scale, out, mask, stat, counters, NULL,
                   NULL, NULL, NULL);
}

/* iACT with the tables kept across calls (not in the paper, Section 3.1.1
 * scopes them to one kernel): for logical warp w and its table j (g = w *
 * tperwarp + j), slot s holds st_z[(g*tsize + s)*D + d], st_y[g*tsize + s] and
 * st_valid[g*tsize + s]; st_rr[g] is the round-robin slot. Read at the start,
 * written back at the end; zeroed arrays are the empty state. */
int orc_run_iact_persist(const orc_region *R, const void *in, int32_t tsize, int32_t tperwarp,
                         double thr, int32_t level, const double *in_scale, float *st_z,
                         double *st_y, int32_t *st_valid, int32_t *st_rr, void *out,
                         uint8_t *mask, void *stat, int64_t *counters) {
  if (!st_z || !st_y || !st_valid || !st_rr) return 1;
  return iact_core(R, in, tsize, tperwarp, thr, level, in_scale, out, mask, stat, counters, st_z,
                   st_y, st_valid, st_rr);
}

/* K-Means centroid update (the exact step between two assignments): each
 * centroid becomes the mean of the observations assigned to it, summed in
 * double over i in order and rounded once; a cluster without observations
 * keeps its centroid. changed (if prev is given) = observations whose id
 * differs from prev. x: 8 rows of `stride` floats; assign: ids as floats. */
int orc_kmeans_update(int64_t n, int32_t K, const float *x, int64_t stride, const float *assign,
                      const float *prev, float *cent, int64_t *changed) {
  if (n < 0 || K < 1 || K > 64 || stride < n) return 1;
  double sum[64 * 8];
  int64_t cnt[64];
  memset(sum, 0, sizeof(sum));
  memset(cnt, 0, sizeof(cnt));
  int64_t ch = 0;
  for (int64_t i = 0; i < n; ++i) {
    int k = (int)assign[i];
    if (k < 0 || k >= K) return 1;
    cnt[k] += 1;
    for (int d = 0; d < 8; ++d) sum[k * 8 + d] += (double)x[d * stride + i];
    if (prev && prev[i] != assign[i]) ch++;
  }
  for (int k = 0; k < K; ++k)
    if (cnt[k] > 0)
      for (int d = 0; d < 8; ++d) cent[k * 8 + d] = (float)(sum[k * 8 + d] / (double)cnt[k]);
  if (changed) *changed = ch;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Quality metrics (Section 4, Eq. 1 MAPE, Eq. 2 MCR; RMSE)                  */
/* ------------------------------------------------------------------------ */

/* Neumaier-compensated running sum. */
typedef struct { double s, c; } ksum;
static void kadd(ksum *k, double x) {
  double t = k->s + x;
  if (fabs(k->s) >= fabs(x)) k->c += (k->s - t) + x;
  else k->c += (x - t) + k->s;
  k->s = t;
}
static double kval(const ksum *k) { return k->s + k->c; }

/* metric 0: MAPE = mean over i with a_i != 0 of |a_i - b_i| / |a_i| (Eq. 1 with
 *           the zero-denominator terms set aside); res[1] = max |b_i| over the
 *           a_i == 0 terms; aux[0] = #(a_i == 0), aux[1] = #(a_i == 0, b_i != 0).
 * metric 1: RMSE = sqrt(mean (a_i - b_i)^2).
 * metric 2: MCR = mean of [a_i != b_i] (Eq. 2). */
int orc_quality(int64_t n, const double *a, const double *b, int32_t metric, double *res,
                int64_t *aux) {
  if (n < 0 || metric < 0 || metric > 2) return 1;
  ksum acc = {0.0, 0.0};
  int64_t zeros = 0, zeros_bad = 0, used = 0;
  double zmax = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    if (metric == 0) {
      if (a[i] == 0.0) {
        zeros++;
        if (b[i] != 0.0) zeros_bad++;
        if (fabs(b[i]) > zmax) zmax = fabs(b[i]);
        continue;
      }
      kadd(&acc, fabs(a[i] - b[i]) / fabs(a[i]));
      used++;
    } else if (metric == 1) {
      double d = a[i] - b[i];
      kadd(&acc, d * d);
      used++;
    } else {
      kadd(&acc, a[i] != b[i] ? 1.0 : 0.0);
      used++;
    }
  }
  double v = used ? kval(&acc) / (double)used : 0.0;
  if (metric == 1) v = sqrt(v);
  res[0] = v;
  res[1] = zmax;
  if (aux) {
    aux[0] = zeros;
    aux[1] = zeros_bad;
  }
  return 0;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads of the following parallel regions (n < 1: one per processor). */
void orc_set_threads(int n) {
#ifdef _OPENMP
  omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
#else
  (void)n;
#endif
}
