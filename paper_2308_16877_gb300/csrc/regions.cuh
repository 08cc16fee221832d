// Device-side regions and the IEEE-rounded decision statistics.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace hpac {

// ---------------------------------------------------------------------------
// Regions. Each has the value type T, the number of inputs its exact
// evaluation reads (kReads) and operator() over those inputs.
// ---------------------------------------------------------------------------

// Standard normal CDF N(x) = erfc(-x / sqrt 2) / 2 in single precision, with
// erfc from the Chebyshev-fitted form of Press, Teukolsky, Vetterling and
// Flannery (Numerical Recipes in C, 2nd ed., section 6.2, "erfcc"):
// erfc(z) = t exp(-z^2 + P(t)), t = 1 / (1 + z/2), fractional error below
// 1.2e-7 for z >= 0. z^2 is split into its rounded value and the rounding
// error (one FMA) so the exponent argument keeps full precision.
__device__ __forceinline__ float normal_cdf(float x) {
  const float z = fabsf(x) * 0.70710678118654752440f;
  const float t = __fdividef(1.0f, fmaf(0.5f, z, 1.0f));
  float p = 0.17087277f;
  p = fmaf(p, t, -0.82215223f);
  p = fmaf(p, t, 1.48851587f);
  p = fmaf(p, t, -1.13520398f);
  p = fmaf(p, t, 0.27886807f);
  p = fmaf(p, t, -0.18628806f);
  p = fmaf(p, t, 0.09678418f);
  p = fmaf(p, t, 0.37409196f);
  p = fmaf(p, t, 1.00002368f);
  p = fmaf(p, t, -1.26551223f);
  const float zz = z * z;
  const float zz_err = fmaf(z, z, -zz);
  const float half_erfc = 0.5f * t * __expf((p - zz) - zz_err);
  return x >= 0.0f ? 1.0f - half_erfc : half_erfc;
}

// European call (Table 1, Black-Scholes): C = S N(d1) - K e^{-rT} N(d2),
// d1 = (ln(S/K) + (r + sigma^2/2) T) / (sigma sqrt T), d2 = d1 - sigma sqrt T.
// Single precision with the hardware reciprocal square root, fast divide,
// log2/exp2 units and the normal CDF above: about 60 instructions per option,
// below the roughly 110 that keep the kernel at HBM speed on GB300.
struct BlackScholes32 {
  using T = float;
  static constexpr int kReads = 4;
  float r;
  __device__ __forceinline__ float operator()(const float *x) const {
    const float S = x[0], K = x[1], Tm = x[2], sig = x[3];
    const float rs = rsqrtf(Tm);
    const float sst = sig * (Tm * rs);
    const float d1 = (__logf(__fdividef(S, K)) + (r + 0.5f * sig * sig) * Tm) * __fdividef(rs, sig);
    const float d2 = d1 - sst;
    return S * normal_cdf(d1) - K * __expf(-r * Tm) * normal_cdf(d2);
  }
};

struct BlackScholes64 {
  using T = double;
  static constexpr int kReads = 4;
  double r;
  __device__ __forceinline__ double operator()(const double *x) const {
    const double S = x[0], K = x[1], Tm = x[2], sig = x[3];
    const double sst = sig * sqrt(Tm);
    const double d1 = (log(S / K) + (r + 0.5 * sig * sig) * Tm) / sst;
    const double d2 = d1 - sst;
    const double n1 = 0.5 * erfc(-0.70710678118654752440 * d1);
    const double n2 = 0.5 * erfc(-0.70710678118654752440 * d2);
    return S * n1 - K * exp(-r * Tm) * n2;
  }
};

// Ideal-gas EOS with the implicit trapezoid energy update solved in closed form.
struct Eos64 {
  using T = double;
  static constexpr int kReads = 4;
  double gamma;
  // p_{n+1} = (g-1) e_{n+1} / v_{n+1} with the implicit trapezoid energy
  // e_{n+1} = (e - dv (p_n + 2q)/2) / (1 + (g-1) dv / (2 v_{n+1})), p_n =
  // (g-1) e / v_n, v_n = v_{n+1} - dv, clamped at zero. Multiplying through by
  // v_n v_{n+1} leaves one division: p = (g-1) N / (v_n (v_{n+1} + (g-1) dv/2)),
  // N = e v_n - dv ((g-1) e + 2 q v_n) / 2; N has the sign of e_{n+1} (v_n > 0).
  // A double division costs about ten FP64 instructions on a pipe that issues
  // one warp instruction per ~16 cycles, so this form runs about 3x faster.
  __device__ __forceinline__ double operator()(const double *x) const {
    const double e = x[0], v1 = x[1], dv = x[2], q = x[3];
    const double gm1 = gamma - 1.0;
    const double v0 = v1 - dv;
    const double N = e * v0 - 0.5 * dv * (gm1 * e + 2.0 * q * v0);
    const double D = v0 * (v1 + 0.5 * gm1 * dv);
    return N < 0.0 ? 0.0 : gm1 * N / D;
  }
};

// K-Means assignment (Table 1, K-Means; Section 4.2 approximates this
// distance kernel): the nearest of K centroids (cent[k * 8 + d], read-only
// cache) in squared Euclidean distance over 8 features, summed over d in order
// in IEEE single precision, ties to the lowest index; the id as a float.
// Packed single-precision pairs (one IEEE round-to-nearest operation per
// half): two observations' distances advance in one instruction.
__device__ __forceinline__ unsigned long long f32x2_pack(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f32x2_unpack(unsigned long long v, float &lo, float &hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long f32x2_sub(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long f32x2_mul(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long f32x2_fma(unsigned long long a, unsigned long long b,
                                                        unsigned long long c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
__device__ __forceinline__ unsigned long long f32x2_add(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}

struct KMeans32 {
  using T = float;
  static constexpr int kReads = 8;
  static constexpr bool kGroup4 = true;  // has group4()
  const float *cent;
  int K;
  __device__ __forceinline__ float operator()(const float *x) const {
    int best = 0;
    float bd = 0.0f;
    // a centroid is two 16-byte loads (the pointer is 16-byte aligned, checked
    // when it is set); the distance sums d = 0..7 in order, as defined
    const float4 *c4 = reinterpret_cast<const float4 *>(cent);
    for (int k = 0; k < K; ++k) {
      const float4 lo = __ldg(c4 + 2 * k), hi = __ldg(c4 + 2 * k + 1);
      const float c[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
      float acc = 0.0f;
#pragma unroll
      for (int d = 0; d < 8; ++d) {
        const float df = __fsub_rn(x[d], c[d]);
        acc = __fadd_rn(acc, __fmul_rn(df, df));
      }
      if (k == 0 || acc < bd) {
        bd = acc;
        best = k;
      }
    }
    return (float)best;
  }
  // Four observations at once (x[d][j]: feature d of observation j), each
  // with exactly the operations and order of operator(): the pairs (0, 1) and
  // (2, 3) share every packed subtract, square and add.
  __device__ __forceinline__ void group4(const float (&x)[8][4], float (&y)[4]) const {
    unsigned long long xp[8][2];
#pragma unroll
    for (int d = 0; d < 8; ++d) {
      xp[d][0] = f32x2_pack(x[d][0], x[d][1]);
      xp[d][1] = f32x2_pack(x[d][2], x[d][3]);
    }
    int best[4] = {0, 0, 0, 0};
    float bd[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    const float4 *c4 = reinterpret_cast<const float4 *>(cent);
    for (int k = 0; k < K; ++k) {
      const float4 lo = __ldg(c4 + 2 * k), hi = __ldg(c4 + 2 * k + 1);
      const float c[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
      unsigned long long acc0 = 0ull, acc1 = 0ull;  // (+0, +0)
#pragma unroll
      for (int d = 0; d < 8; ++d) {
        const unsigned long long cc = f32x2_pack(c[d], c[d]);
        const unsigned long long d0 = f32x2_sub(xp[d][0], cc), d1 = f32x2_sub(xp[d][1], cc);
        acc0 = f32x2_add(acc0, f32x2_mul(d0, d0));
        acc1 = f32x2_add(acc1, f32x2_mul(d1, d1));
      }
      float a[4];
      f32x2_unpack(acc0, a[0], a[1]);
      f32x2_unpack(acc1, a[2], a[3]);
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (k == 0 || a[j] < bd[j]) {
          bd[j] = a[j];
          best[j] = k;
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) y[j] = (float)best[j];
  }
};

// Regions that evaluate a vector group of four invocations in one call
// (group4) use it in the maps; the others are called once per invocation.
template <class R, class = void>
struct HasGroup4 {
  static constexpr bool value = false;
};
template <class R>
struct HasGroup4<R, decltype(void(R::kGroup4))> {
  static constexpr bool value = R::kGroup4;
};

template <class R, int V>
__device__ __forceinline__ void eval_group(const R &reg, const typename R::T (&x)[R::kReads][V],
                                           typename R::T (&y)[V]) {
  if constexpr (V == 4 && HasGroup4<R>::value) {
    reg.group4(x, y);
  } else {
#pragma unroll
    for (int j = 0; j < V; ++j) {
      typename R::T xi[R::kReads];
#pragma unroll
      for (int d = 0; d < R::kReads; ++d) xi[d] = x[d][j];
      y[j] = reg(xi);
    }
  }
}

template <typename T_>
struct Identity {
  using T = T_;
  static constexpr int kReads = 1;
  __device__ __forceinline__ T operator()(const T *x) const { return x[0]; }
};

// ---------------------------------------------------------------------------
// IEEE-rounded arithmetic (no contraction), one overload set per precision, so
// that the decision statistics are bit-reproducible.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float div_rn(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float sqrt_rn(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double div_rn(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double sqrt_rn(double a) { return __dsqrt_rn(a); }

template <typename T>
__device__ __forceinline__ T inf_v() { return (T)INFINITY; }
template <typename T>
__device__ __forceinline__ T nan_v() { return (T)NAN; }

// Relative standard deviation of the h window values held in shared memory
// at win[slot * ld] (slot order oldest .. newest starting at `oldest`,
// wrapping at h): two passes, population moments, RSD = sigma / |mu|;
// 0/0 reads as 0 and sigma/0 (sigma > 0) as +inf.
// x / h correctly rounded, with inv_h = 1/h. For h a power of two, x inv_h is
// the same real number rounded once, so the product is the identical result
// without a division.
template <typename T>
__device__ __forceinline__ T div_count(T x, int h, T inv_h) {
  return (h & (h - 1)) == 0 ? mul_rn(x, inv_h) : div_rn(x, (T)h);
}

// RSD from the IEEE moments: sigma / |mu| with var = acc / h.
template <typename T>
__device__ __forceinline__ T rsd_from_moments(T mu, T acc, int h, T inv_h) {
  const T var = div_count(acc, h, inv_h);
  const T sd = sqrt_rn(var);
  const T amu = mu < (T)0 ? -mu : mu;
  if (amu == (T)0) return var == (T)0 ? (T)0 : inf_v<T>();
  return div_rn(sd, amu);
}

template <typename T>
__device__ __forceinline__ T window_rsd(const T *win, int ld, int oldest, int h, T inv_h) {
  T sum = (T)0;
  int s = oldest;
  for (int j = 0; j < h; ++j) {
    sum = add_rn(sum, win[s * ld]);
    s = (s + 1 == h) ? 0 : s + 1;
  }
  const T mu = div_count(sum, h, inv_h);
  T acc = (T)0;
  s = oldest;
  for (int j = 0; j < h; ++j) {
    const T d = sub_rn(win[s * ld], mu);
    acc = add_rn(acc, mul_rn(d, d));
    s = (s + 1 == h) ? 0 : s + 1;
  }
  return rsd_from_moments(mu, acc, h, inv_h);
}

// RSD < thr from the IEEE moments, the correctly rounded statistic taken only
// inside the guard band (see rsd_below_fast).
// The fast test needs (thr mu)^2 far inside the normal range: a subnormal
// square keeps too few bits for the guard band (and the absolute error of
// acc / h, at most one subnormal spacing, must stay far below 2e-5 of it).
template <typename T>
__device__ __forceinline__ T fast_test_floor() { return sizeof(T) == 4 ? (T)1e-30 : (T)1e-290; }

template <typename T>
__device__ __forceinline__ bool rsd_below_moments(T mu, T acc, int h, T thr, T inv_h) {
  const T var = acc * inv_h;
  const T tm = thr * mu;
  const T lim = tm * tm;
  if (mu != (T)0 && isfinite(lim) && lim < (T)1e30 && lim > fast_test_floor<T>()) {
    if (var < lim * (T)(1.0 - 2e-5)) return true;
    if (var > lim * (T)(1.0 + 2e-5)) return false;
  }
  return rsd_from_moments(mu, acc, h, inv_h) < thr;
}

// Decision RSD(window) < thr without the correctly rounded division and square
// root when it is clear: with mu the same IEEE mean as window_rsd (so the
// second pass is identical), var ~ acc / h and the test var < (thr mu)^2 carry
// a few ulps of error, far inside the 2e-5 relative guard band on the squared
// statistic; inside the band, for mu = 0, and where (thr mu)^2 is not a
// comfortably normal number, the IEEE statistic decides. The decision
// therefore equals window_rsd(...) < thr exactly.
template <typename T>
__device__ __forceinline__ bool rsd_below_fast(const T *win, int ld, int oldest, int h, T thr, T inv_h) {
  T sum = (T)0;
  int s = oldest;
  for (int j = 0; j < h; ++j) {
    sum = add_rn(sum, win[s * ld]);
    s = (s + 1 == h) ? 0 : s + 1;
  }
  const T mu = div_count(sum, h, inv_h);
  T acc = (T)0;
  s = oldest;
  for (int j = 0; j < h; ++j) {
    const T d = sub_rn(win[s * ld], mu);
    acc = add_rn(acc, mul_rn(d, d));
    s = (s + 1 == h) ? 0 : s + 1;
  }
  return rsd_below_moments(mu, acc, h, thr, inv_h);
}

// Decision RSD(w) < thr for a double-precision window of compile-time size KH
// (2, 4 or 8) settled, where it is clear, in single precision from the copy
// wf[j] = (float)w[j]; GB300 issues double-precision arithmetic at a small
// fraction of its single-precision rate. With u = 2^-24 and M = max |wf_j|
// (in [1e-10, 1e15]), the single-precision mean m = fl(sum wf_j) / KH and
// standard deviation sqrt(var), var = fl(sum fl(wf_j - m)^2) / KH, are within
// (KH + 1) u M and (2 KH + 3) u M of the exact mean and standard deviation of
// w (rounding of the copy, of the KH-term sums and of the squares; the
// deviation is at most 2 M). The test widens those bounds to Em = 4 (KH + 1) u M
// and Es = 8 (KH + 2) u M, so that the double-precision statistic's own
// rounding (relative 2^-53) also lies inside, takes the threshold 1e-5
// relative further (rounding of thr to single precision and of the test's own
// few operations) and decides only when the whole interval is on one side:
// below when sqrt(var) < thr (|m| - Em) - Es, not below when
// sqrt(var) > thr (|m| + Em) + Es, compared as squares. The subtraction is
// used only while Es is at most half of thr (|m| - Em), which keeps its
// relative rounding error within 5u. Returns 1 (below), 0 (not below) or -1
// (the double-precision test decides): always -1 for a window with a NaN or
// an infinity or outside the magnitude range, and for thresholds outside
// [1e-7, 1e12] (the caller passes thr_ok). An all-zero window has statistic 0
// and is decided exactly.
template <int KH>
__device__ __forceinline__ int rsd_below_f32(const float (&wf)[KH], const double (&w)[KH], float thr,
                                             bool thr_ok) {
  if (!thr_ok) return -1;
  float M = 0.0f;
#pragma unroll
  for (int j = 0; j < KH; ++j) M = fmaxf(M, fabsf(wf[j]));
  if (M == 0.0f) {
    bool zero = true;  // exact test on the double-precision values (+0 or -0)
#pragma unroll
    for (int j = 0; j < KH; ++j) zero &= (__double_as_longlong(w[j]) << 1) == 0;
    return zero ? 1 : -1;
  }
  if (!(M >= 1e-10f && M <= 1e15f)) return -1;
  float S = 0.0f;
#pragma unroll
  for (int j = 0; j < KH; ++j) S = __fadd_rn(S, wf[j]);
  const float m = __fmul_rn(S, 1.0f / KH);
  float a = 0.0f;
#pragma unroll
  for (int j = 0; j < KH; ++j) {
    const float d = __fsub_rn(wf[j], m);
    a = __fadd_rn(a, __fmul_rn(d, d));
  }
  const float var = __fmul_rn(a, 1.0f / KH);
  constexpr float u = 5.9604644775390625e-8f;  // 2^-24
  const float Es = __fmul_rn((float)(8 * (KH + 2)) * u, M);
  const float Em = __fmul_rn((float)(4 * (KH + 1)) * u, M);
  const float am = fabsf(m);
  const float xlo = __fmul_rn(thr, __fsub_rn(am, Em));
  if (Es <= 0.5f * xlo) {
    const float t = __fsub_rn(xlo, Es);
    if (t >= 1e-15f && t <= 1e15f && var < __fmul_rn(__fmul_rn(t, t), 1.0f - 1e-5f)) return 1;
  }
  const float t = __fadd_rn(__fmul_rn(thr, __fadd_rn(am, Em)), Es);
  if (t >= 1e-15f && t <= 1e15f && var > __fmul_rn(__fmul_rn(t, t), 1.0f + 1e-5f)) return 0;
  return -1;
}

// The window held in registers, oldest first (compile-time size): the same
// two IEEE passes in the same order as window_rsd.
template <typename T, int KH>
__device__ __forceinline__ void reg_window_moments(const T (&w)[KH], T inv_h, T &mu, T &acc) {
  T sum = (T)0;
#pragma unroll
  for (int j = 0; j < KH; ++j) sum = add_rn(sum, w[j]);
  mu = div_count(sum, KH, inv_h);
  acc = (T)0;
#pragma unroll
  for (int j = 0; j < KH; ++j) {
    const T d = sub_rn(w[j], mu);
    acc = add_rn(acc, mul_rn(d, d));
  }
}

__device__ __forceinline__ bool borderline(double s, double thr) {
  if (isinf(thr) || isnan(s)) return false;
  return fabs(s - thr) <= 1e-6 * thr;
}

// Warp-aggregated add of two per-thread counts into a block-wide shared pair,
// then (by the caller, after a barrier) one global add per block.
__device__ __forceinline__ void warp_count(unsigned long long *sm, unsigned long long a,
                                           unsigned long long b) {
  for (int off = 16; off > 0; off >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, off);
    b += __shfl_down_sync(0xffffffffu, b, off);
  }
  if ((threadIdx.x & 31) == 0) {
    if (a) atomicAdd(&sm[0], a);
    if (b) atomicAdd(&sm[1], b);
  }
}

}  // namespace hpac
