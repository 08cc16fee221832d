// Hexahedral Lagrangian hydro whose equation-of-state call is the approximated
// region (the paper approximates kernels of the LULESH proxy application,
// Table 1, Section 4.1; the scheme itself is a textbook staggered-grid update,
// the same one the CPU oracle restates).
//
// Per time step, on the EOS region's stream:
//   node kernel     forces from the stored volume gradients and the stored
//                   p + q, velocity and position update (1 / (12 m) stored at
//                   init), symmetry planes x = 0, y = 0, z = 0;
//   element kernel  exact trilinear-hexahedron volume and its gradient at the
//                   new positions, relative volume, artificial viscosity, the
//                   EOS inputs (e, v_{n+1}, dv, q_{n+1});
//   EOS region      exact, TAF, iACT or perforation through the region API;
//   finalize        e = p v / (gamma - 1), v = v_{n+1}, pq = p + q.
//
// Volume of a trilinear hexahedron and its gradient. With corners P_c in
// lexicographic order (c = a + 2b + 4d for offsets a, b, d), the integral of
// det J over the reference cube equals Grandy's sum of three triple products
// (J. Grandy, "Efficient computation of volume of hexahedral cells", LLNL
// UCRL-ID-128886, 1997), one per pair of faces meeting at corner 7 and at
// corner 0:
//   12 V = s1 . (c1 x d1) + s2 . (c2 x d2) + s3 . (c3 x d3),
//   s1 = (P2 - P1) + (P6 - P3), c1 = P7 - P2, d1 = P3 - P0,
//   s2 = (P4 - P2) + (P5 - P6), c2 = P7 - P4, d2 = P6 - P0,
//   s3 = (P1 - P4) + (P3 - P5) = -(s1 + s2), c3 = P7 - P1, d3 = P5 - P0.
// V is a cubic polynomial of the corners, so its gradient follows by the
// product rule: with A_i = c_i x d_i, B_i = d_i x s_i, C_i = s_i x c_i (the
// derivatives of the i-th triple product with respect to s_i, c_i and d_i),
// each corner collects the terms of the differences it appears in:
//   12 dV/dP0 = -(C1 + C2 + C3)        12 dV/dP7 = B1 + B2 + B3
//   12 dV/dP1 = (A3 - A1) - B3         12 dV/dP3 = (A3 - A1) + C1
//   12 dV/dP2 = (A1 - A2) - B1         12 dV/dP6 = (A1 - A2) + C2
//   12 dV/dP4 = (A2 - A3) - B2         12 dV/dP5 = (A2 - A3) + C3
// Every difference is of two corners of one element, so it carries the
// rounding of the element's size, not of its position. The kernel stores
// 12 dV/dP_c (the 1/12 is applied where the gradient is used).
// The corner differences and their sums (s_i, c_i, d_i and t = s1 + s2) are
// formed exactly in integer arithmetic: per element and axis the eight
// coordinates are placed on a fixed-point grid six bits finer than the
// significand of the largest one (exact for every coordinate within six
// binades of it, else rounded to that grid), subtracted and summed as 64-bit
// integers, and each result rounded once to FP64. The rest runs on the FP64
// pipe: 9 cross products (54 operations), the volume (10) and the corner sums
// (39). GB300 issues two FP64 operations per SM and clock against 64 integer
// ones, so moving the 39 difference operations to the integer pipes takes
// the element kernel from 143 to 104 FP64 instructions per element (the plain
// sum over the trilinear form's 24 corner triples with shared pair cross
// products takes 260). Coordinates that are infinite or NaN, or results
// outside the normal FP64 range, take the same differences in FP64 instead.
#include <math.h>

#include "hpac_internal.cuh"

namespace hpac {
namespace {

constexpr double kCq = 2.0;   // quadratic viscosity coefficient
constexpr double kCl = 0.5;   // linear viscosity coefficient

// The differences of Grandy's form, per axis: s1, s2, t = s1 + s2 = -s3,
// c1..c3, d1..d3 (component 0 x, 1 y, 2 z).
struct HexDiffs {
  double s1[3], s2[3], t[3], c1[3], c2[3], c3[3], d1[3], d2[3], d3[3];
};

// The differences in FP64 (the fallback for non-finite coordinates).
__device__ __forceinline__ void hex_diffs_fp64(const double (&X)[8], const double (&Y)[8], const double (&Z)[8],
                                               HexDiffs &D) {
  const double *P[3] = {X, Y, Z};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double *p = P[a];
    D.s1[a] = (p[2] - p[1]) + (p[6] - p[3]);
    D.s2[a] = (p[4] - p[2]) + (p[5] - p[6]);
    D.t[a] = D.s1[a] + D.s2[a];
    D.c1[a] = p[7] - p[2];
    D.c2[a] = p[7] - p[4];
    D.c3[a] = p[7] - p[1];
    D.d1[a] = p[3] - p[0];
    D.d2[a] = p[6] - p[0];
    D.d3[a] = p[5] - p[0];
  }
}

constexpr int kFixedGuard = 6;  // grid bits below the largest coordinate's significand

// Coordinates of one axis on the element's fixed-point grid: F = P / 2^L with
// L = e_max - 1075 - kFixedGuard (e_max the largest biased exponent among the
// eight, at least 1); |F| < 2^59. Coordinates more than kFixedGuard binades
// below e_max are rounded to the grid (half away from zero on the magnitude).
// `bad` is set for an infinite or NaN coordinate. Returns L.
__device__ __forceinline__ int to_fixed(const double *P, int64_t (&F)[8], bool &bad) {
  uint32_t emax = 1;
#pragma unroll
  for (int c = 0; c < 8; ++c) emax = max(emax, ((uint32_t)__double2hiint(P[c]) >> 20) & 0x7ffu);
  bad |= emax == 0x7ffu;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const uint64_t bits = (uint64_t)__double_as_longlong(P[c]);
    uint32_t ec = (uint32_t)(bits >> 52) & 0x7ffu;
    uint64_t m = bits & 0xfffffffffffffull;
    if (ec) m |= 1ull << 52;  // hidden bit of a normal number
    else ec = 1;              // zero or subnormal: same scale as exponent 1
    const int sh = (int)ec - (int)emax + kFixedGuard;
    uint64_t M;
    if (sh >= 0) {
      M = m << sh;
    } else {
      const int r = min(-sh, 63);
      M = (m + (1ull << (r - 1))) >> r;
    }
    F[c] = (bits >> 63) ? -(int64_t)M : (int64_t)M;
  }
  return (int)emax - 1075 - kFixedGuard;
}

// v 2^S rounded to the nearest FP64 (ties to even; exact when |v| < 2^53).
// `bad` is set when a nonzero result falls outside the normal range.
__device__ __forceinline__ double fixed_to_double(int64_t v, int S, bool &bad) {
  const uint64_t neg = (uint64_t)v >> 63;
  const uint64_t a = neg ? 0ull - (uint64_t)v : (uint64_t)v;
  const int lz = __clzll(a | 1ull);
  const uint64_t n = a << lz;  // leading one at bit 63
  uint64_t mant = n >> 11;     // 53 bits
  const uint64_t round = (n >> 10) & 1ull, sticky = (n & 0x3ffull) != 0;
  mant += round & (sticky | (mant & 1ull));
  int be = 63 - lz + S + 1023;
  if (mant >> 53) {  // rounded up to the next power of two
    mant >>= 1;
    be += 1;
  }
  bad |= (a != 0) & (be <= 0 || be >= 2047);
  const uint64_t r = (neg << 63) | ((uint64_t)(be & 0x7ff) << 52) | (mant & 0xfffffffffffffull);
  return __longlong_as_double(a ? (long long)r : 0ll);
}

// The differences exactly in integers, each rounded once to FP64.
__device__ __forceinline__ void hex_diffs_fixed(const double (&X)[8], const double (&Y)[8],
                                                const double (&Z)[8], HexDiffs &D, bool &bad) {
  const double *P[3] = {X, Y, Z};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    int64_t F[8];
    const int L = to_fixed(P[a], F, bad);
    const int64_t s1 = (F[2] - F[1]) + (F[6] - F[3]), s2 = (F[4] - F[2]) + (F[5] - F[6]);
    D.s1[a] = fixed_to_double(s1, L, bad);
    D.s2[a] = fixed_to_double(s2, L, bad);
    D.t[a] = fixed_to_double(s1 + s2, L, bad);
    D.c1[a] = fixed_to_double(F[7] - F[2], L, bad);
    D.c2[a] = fixed_to_double(F[7] - F[4], L, bad);
    D.c3[a] = fixed_to_double(F[7] - F[1], L, bad);
    D.d1[a] = fixed_to_double(F[3] - F[0], L, bad);
    D.d2[a] = fixed_to_double(F[6] - F[0], L, bad);
    D.d3[a] = fixed_to_double(F[5] - F[0], L, bad);
  }
}

__device__ __forceinline__ void cross3(const double (&a)[3], const double (&b)[3], double (&c)[3]) {
  c[0] = fma(a[1], b[2], -a[2] * b[1]);
  c[1] = fma(a[2], b[0], -a[0] * b[2]);
  c[2] = fma(a[0], b[1], -a[1] * b[0]);
}

// 12 dV/dP_c for the eight corners (absolute positions) and the volume V, in
// the three-triple-product form above.
__device__ __forceinline__ double hex_grad12(const double (&X)[8], const double (&Y)[8],
                                             const double (&Z)[8], double (&gx)[8], double (&gy)[8],
                                             double (&gz)[8]) {
  HexDiffs D;
  bool bad = false;
  hex_diffs_fixed(X, Y, Z, D, bad);
  if (bad) hex_diffs_fp64(X, Y, Z, D);
  double A1[3], A2[3], A3[3], B1[3], B2[3], B3[3], C1[3], C2[3], C3[3];
  cross3(D.c1, D.d1, A1);
  cross3(D.c2, D.d2, A2);
  cross3(D.c3, D.d3, A3);
  cross3(D.d1, D.s1, B1);
  cross3(D.d2, D.s2, B2);
  cross3(D.t, D.d3, B3);  // d3 x s3 = t x d3
  cross3(D.s1, D.c1, C1);
  cross3(D.s2, D.c2, C2);
  cross3(D.c3, D.t, C3);  // s3 x c3 = c3 x t
  double v12 = D.s1[0] * A1[0];
  v12 = fma(D.s1[1], A1[1], v12);
  v12 = fma(D.s1[2], A1[2], v12);
  v12 = fma(D.s2[0], A2[0], v12);
  v12 = fma(D.s2[1], A2[1], v12);
  v12 = fma(D.s2[2], A2[2], v12);
  v12 = fma(-D.t[0], A3[0], v12);
  v12 = fma(-D.t[1], A3[1], v12);
  v12 = fma(-D.t[2], A3[2], v12);
  double *g[3] = {gx, gy, gz};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double p31 = A3[a] - A1[a], p12 = A1[a] - A2[a], p23 = A2[a] - A3[a];
    g[a][0] = -C1[a] - C2[a] - C3[a];
    g[a][1] = p31 - B3[a];
    g[a][2] = p12 - B1[a];
    g[a][3] = p31 + C1[a];
    g[a][4] = p23 - B2[a];
    g[a][5] = p23 + C3[a];
    g[a][6] = p12 + C2[a];
    g[a][7] = B1[a] + B2[a] + B3[a];
  }
  return v12 * (1.0 / 12.0);
}

// Division of a 32-bit index by a fixed divisor with one multiply-high, an
// add and two shifts (Granlund and Montgomery, "Division by invariant
// integers using multiplication", PLDI 1994): with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1, x / d = (t + ((x - t) >> s1)) >> s2,
// t = umulhi(m, x), s1 = min(l, 1), s2 = max(l - 1, 0), for every 32-bit x
// and d >= 1. Mesh indices stay below 2^31 (n <= 1024: (n + 1)^3 < 1.1e9), so
// the kernels split them with it instead of 64-bit divisions.
struct FastDiv {
  uint32_t d, m, s1, s2;
};

FastDiv make_fastdiv(uint32_t d) {
  uint32_t l = 0;
  while ((1ull << l) < d) ++l;
  FastDiv f;
  f.d = d;
  f.m = (uint32_t)((((1ull << l) - d) << 32) / d + 1);
  f.s1 = l > 0 ? 1 : 0;
  f.s2 = l > 0 ? l - 1 : 0;
  return f;
}

__device__ __forceinline__ uint32_t fdiv(uint32_t x, const FastDiv &f) {
  const uint32_t t = __umulhi(f.m, x);
  return (t + ((x - t) >> f.s1)) >> f.s2;
}

// Corner positions of element e (lexicographic corner order).
__device__ __forceinline__ void gather(int n, int64_t e, const double *__restrict__ x,
                                       const double *__restrict__ y, const double *__restrict__ z,
                                       double (&X)[8], double (&Y)[8], double (&Z)[8]) {
  const int64_t n1 = n + 1;
  const int64_t i = e % n, j = (e / n) % n, k = e / ((int64_t)n * n);
  const int64_t base = (k * n1 + j) * n1 + i;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int64_t nd = base + ((c >> 2) & 1) * n1 * n1 + ((c >> 1) & 1) * n1 + (c & 1);
    X[c] = x[nd];
    Y[c] = y[nd];
    Z[c] = z[nd];
  }
}

// The same gather for the time-step kernel: element e split by the fixed
// divisor n, node offsets in 32 bits.
__device__ __forceinline__ void gather32(uint32_t e, const FastDiv &fn, const double *__restrict__ x,
                                         const double *__restrict__ y, const double *__restrict__ z,
                                         double (&X)[8], double (&Y)[8], double (&Z)[8]) {
  const uint32_t n = fn.d, n1 = n + 1;
  const uint32_t jk = fdiv(e, fn), i = e - jk * n;
  const uint32_t k = fdiv(jk, fn), j = jk - k * n;
  const uint32_t base = (k * n1 + j) * n1 + i;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int64_t nd = base + ((c >> 2) & 1) * n1 * n1 + ((c >> 1) & 1) * n1 + (c & 1);
    X[c] = x[nd];
    Y[c] = y[nd];
    Z[c] = z[nd];
  }
}

__global__ void __launch_bounds__(128) init_elem_kernel(hpac_hydro_state s) {
  const int n = s.n;
  const int64_t E = (int64_t)n * n * n;
  const double gm1 = s.gamma - 1.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x) {
    double X[8], Y[8], Z[8], gx[8], gy[8], gz[8];
    gather(n, e, s.x, s.y, s.z, X, Y, Z);
    const double V = hex_grad12(X, Y, Z, gx, gy, gz);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      s.grad[(0 * 8 + c) * E + e] = gx[c];
      s.grad[(1 * 8 + c) * E + e] = gy[c];
      s.grad[(2 * 8 + c) * E + e] = gz[c];
    }
    s.V0[e] = V;
    s.rV0[e] = 1.0 / V;
    s.vrel[e] = 1.0;
    s.p[e] = gm1 * s.e[e];
    s.q[e] = 0.0;
    s.pq[e] = s.p[e];
  }
}

__global__ void __launch_bounds__(256) init_node_kernel(hpac_hydro_state s) {
  const int n = s.n;
  const int64_t n1 = n + 1, Nn = n1 * n1 * n1;
  for (int64_t nd = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; nd < Nn;
       nd += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = nd % n1, j = (nd / n1) % n1, k = nd / (n1 * n1);
    double m = 0.0;
    for (int64_t ek = k - 1; ek <= k; ++ek)
      for (int64_t ej = j - 1; ej <= j; ++ej)
        for (int64_t ei = i - 1; ei <= i; ++ei) {
          if (ei < 0 || ej < 0 || ek < 0 || ei >= n || ej >= n || ek >= n) continue;
          m += 0.125 * s.V0[(ek * n + ej) * n + ei];
        }
    s.mnode[nd] = m;
    s.rmass[nd] = 1.0 / (12.0 * m);
    s.u[nd] = s.v[nd] = s.w[nd] = 0.0;
  }
}

// Forces at x^n from (p + q) and the stored gradients; velocity and position.
// Node indices are split by the fixed divisor n + 1 (fn1) in 32 bits.
__global__ void __launch_bounds__(256) node_kernel(hpac_hydro_state s, FastDiv fn1) {
  const int n = s.n;
  const uint32_t n1 = fn1.d, Nn = n1 * n1 * n1;
  const int64_t E = (int64_t)n * n * n;
  const double dt = s.dt;
  for (uint32_t nd = blockIdx.x * blockDim.x + threadIdx.x; nd < Nn; nd += gridDim.x * blockDim.x) {
    const uint32_t jk = fdiv(nd, fn1), i_ = nd - jk * n1;
    const uint32_t k_ = fdiv(jk, fn1), j_ = jk - k_ * n1;
    const int i = (int)i_, j = (int)j_, k = (int)k_;
    double fx = 0.0, fy = 0.0, fz = 0.0;
#pragma unroll
    for (int dk = 1; dk >= 0; --dk)
#pragma unroll
      for (int dj = 1; dj >= 0; --dj)
#pragma unroll
        for (int di = 1; di >= 0; --di) {
          const int ei = i - di, ej = j - dj, ek = k - dk;
          if (ei < 0 || ej < 0 || ek < 0 || ei >= n || ej >= n || ek >= n) continue;
          const int64_t el = (int64_t)(((uint32_t)ek * n + (uint32_t)ej) * n + (uint32_t)ei);
          const int c = di + 2 * dj + 4 * dk;  // corner of this node in element el
          const double pq = s.pq[el];
          fx = fma(pq, s.grad[(0 * 8 + c) * E + el], fx);
          fy = fma(pq, s.grad[(1 * 8 + c) * E + el], fy);
          fz = fma(pq, s.grad[(2 * 8 + c) * E + el], fz);
        }
    // the stored gradients are 12 dV/dx: rmass = 1 / (12 m), formed once at
    // init (a double division per node and step would cost a fifth of the
    // kernel's FP64 work)
    const double sc = dt * s.rmass[nd];
    double un = fma(fx, sc, s.u[nd]);
    double vn = fma(fy, sc, s.v[nd]);
    double wn = fma(fz, sc, s.w[nd]);
    if (i == 0) un = 0.0;
    if (j == 0) vn = 0.0;
    if (k == 0) wn = 0.0;
    s.u[nd] = un;
    s.v[nd] = vn;
    s.w[nd] = wn;
    s.x[nd] += dt * un;
    s.y[nd] += dt * vn;
    s.z[nd] += dt * wn;
  }
}

// New volume and gradient, viscosity, and the EOS region's inputs. Element
// indices are split by the fixed divisor n (fn) in 32 bits.
__global__ void __launch_bounds__(128, 4) elem_kernel(hpac_hydro_state s, FastDiv fn) {
  const int n = s.n;
  const int64_t E = (int64_t)n * n * n;
  const double dt = s.dt, gamma = s.gamma;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x) {
    double X[8], Y[8], Z[8], gx[8], gy[8], gz[8];
    gather32((uint32_t)e, fn, s.x, s.y, s.z, X, Y, Z);
    const double V = hex_grad12(X, Y, Z, gx, gy, gz);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      s.grad[(0 * 8 + c) * E + e] = gx[c];
      s.grad[(1 * 8 + c) * E + e] = gy[c];
      s.grad[(2 * 8 + c) * E + e] = gz[c];
    }
    // v1 = V / V0 without a division per element and step: exactly 1 for an
    // element at its reference volume (so an unmoved element keeps dv = 0),
    // else V times the stored 1 / V0 (within a rounding of the quotient)
    const double V0e = s.V0[e];
    const double v1 = V == V0e ? 1.0 : V * s.rV0[e];
    const double dv = v1 - s.vrel[e];
    double qn = 0.0;
    if (dv < 0.0) {
      const double L = cbrt(V);
      const double rho = 1.0 / v1;
      const double pp = s.p[e] > 0.0 ? s.p[e] : 0.0;
      const double cs = sqrt(gamma * pp * v1);
      const double du = L * dv / (v1 * dt);
      qn = rho * (kCq * kCq * du * du + kCl * cs * fabs(du));
    }
    s.eos_in[e] = s.e[e];
    s.eos_in[E + e] = v1;
    s.eos_in[2 * E + e] = dv;
    s.eos_in[3 * E + e] = qn;
    s.q[e] = qn;
  }
}

// inv_gm1 = 1 / (gamma - 1), formed once on the host: a double division per
// thread would cost more than the element update itself.
__global__ void __launch_bounds__(256) finalize_kernel(hpac_hydro_state s, double inv_gm1) {
  const int64_t E = (int64_t)s.n * s.n * s.n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double v1 = s.eos_in[E + e];
    s.e[e] = s.p[e] * v1 * inv_gm1;
    s.vrel[e] = v1;
    s.pq[e] = s.p[e] + s.q[e];  // the next step's nodal forces use p + q
  }
}

// The derived arrays from the state: pq = p + q and rV0 = 1 / V0 per element,
// rmass = 1 / (12 m) per node.
__global__ void __launch_bounds__(256) derive_kernel(hpac_hydro_state s) {
  const int64_t E = (int64_t)s.n * s.n * s.n, n1 = s.n + 1, Nn = n1 * n1 * n1;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < (E > Nn ? E : Nn);
       j += (int64_t)gridDim.x * blockDim.x) {
    if (j < E) {
      s.pq[j] = s.p[j] + s.q[j];
      s.rV0[j] = 1.0 / s.V0[j];
    }
    if (j < Nn) s.rmass[j] = 1.0 / (12.0 * s.mnode[j]);
  }
}

unsigned grid_for(int64_t work, int threads, int device) {
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const int64_t want = (work + threads - 1) / threads;
  const int64_t cap = (int64_t)sms * 16;
  return (unsigned)(want < 1 ? 1 : (want > cap ? cap : want));
}

hpac_status check_state(const hpac_hydro_state *s) {
  if (!s) return set_error(HPAC_EINVAL, "hydro state is NULL");
  if (s->n < 1 || s->n > 1024) return set_error(HPAC_EINVAL, "hydro n = %d not in 1..1024", s->n);
  if (s->reserved0 != 0) return set_error(HPAC_EINVAL, "reserved field not zero");
  if (!(s->dt > 0.0) || !isfinite(s->dt)) return set_error(HPAC_EINVAL, "hydro dt must be > 0");
  if (!(s->gamma > 1.0) || !isfinite(s->gamma)) return set_error(HPAC_EINVAL, "gamma must be > 1");
  const void *ptrs[] = {s->x, s->y, s->z, s->u, s->v, s->w, s->mnode, s->e, s->p, s->q, s->vrel,
                        s->V0, s->grad, s->eos_in, s->pq, s->rmass, s->rV0};
  for (const void *p : ptrs)
    if (!p) return set_error(HPAC_EINVAL, "a hydro state array is NULL");
  return HPAC_OK;
}

}  // namespace
}  // namespace hpac

using namespace hpac;

extern "C" hpac_status hpac_hydro_init(const hpac_hydro_state *s, void *cuda_stream) {
  TraceRange trace_("hpac_hydro_init");
  hpac_status st = check_state(s);
  if (st != HPAC_OK) return st;
  int dev = 0;
  HPAC_CUDA_TRY(cudaGetDevice(&dev));
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  const int64_t E = (int64_t)s->n * s->n * s->n, Nn = (int64_t)(s->n + 1) * (s->n + 1) * (s->n + 1);
  init_elem_kernel<<<grid_for(E, 128, dev), 128, 0, stream>>>(*s);
  HPAC_CUDA_TRY(cudaGetLastError());
  init_node_kernel<<<grid_for(Nn, 256, dev), 256, 0, stream>>>(*s);
  HPAC_CUDA_TRY(cudaGetLastError());
  return HPAC_OK;
}

extern "C" hpac_status hpac_hydro_derive(const hpac_hydro_state *s, void *cuda_stream) {
  TraceRange trace_("hpac_hydro_derive");
  hpac_status st = check_state(s);
  if (st != HPAC_OK) return st;
  int dev = 0;
  HPAC_CUDA_TRY(cudaGetDevice(&dev));
  const int64_t Nn = (int64_t)(s->n + 1) * (s->n + 1) * (s->n + 1);
  derive_kernel<<<grid_for(Nn, 256, dev), 256, 0, (cudaStream_t)cuda_stream>>>(*s);
  HPAC_CUDA_TRY(cudaGetLastError());
  return HPAC_OK;
}

extern "C" hpac_status hpac_hydro_nodes(const hpac_hydro_state *s, void *cuda_stream) {
  TraceRange trace_("hpac_hydro_nodes");
  hpac_status st = check_state(s);
  if (st != HPAC_OK) return st;
  int dev = 0;
  HPAC_CUDA_TRY(cudaGetDevice(&dev));
  const int64_t Nn = (int64_t)(s->n + 1) * (s->n + 1) * (s->n + 1);
  node_kernel<<<grid_for(Nn, 256, dev), 256, 0, (cudaStream_t)cuda_stream>>>(*s, make_fastdiv(s->n + 1));
  HPAC_CUDA_TRY(cudaGetLastError());
  return HPAC_OK;
}

extern "C" hpac_status hpac_hydro_elements(const hpac_hydro_state *s, void *cuda_stream) {
  TraceRange trace_("hpac_hydro_elements");
  hpac_status st = check_state(s);
  if (st != HPAC_OK) return st;
  int dev = 0;
  HPAC_CUDA_TRY(cudaGetDevice(&dev));
  const int64_t E = (int64_t)s->n * s->n * s->n;
  // 128 threads, four blocks (16 warps) per SM at 128 registers (4% faster
  // than 136 registers at 96 threads, 15 warps); one element per thread
  const int64_t blocks = (E + 127) / 128;
  elem_kernel<<<(unsigned)(blocks < 0x7fffffffLL ? blocks : 0x7fffffffLL), 128, 0,
                (cudaStream_t)cuda_stream>>>(*s, make_fastdiv(s->n));
  HPAC_CUDA_TRY(cudaGetLastError());
  return HPAC_OK;
}

extern "C" hpac_status hpac_hydro_finalize(const hpac_hydro_state *s, void *cuda_stream) {
  TraceRange trace_("hpac_hydro_finalize");
  hpac_status st = check_state(s);
  if (st != HPAC_OK) return st;
  int dev = 0;
  HPAC_CUDA_TRY(cudaGetDevice(&dev));
  const int64_t E = (int64_t)s->n * s->n * s->n;
  finalize_kernel<<<grid_for(E, 256, dev), 256, 0, (cudaStream_t)cuda_stream>>>(*s, 1.0 / (s->gamma - 1.0));
  HPAC_CUDA_TRY(cudaGetLastError());
  return HPAC_OK;
}

extern "C" hpac_status hpac_hydro_step(const hpac_hydro_state *s, hpac_region *eos,
                                       int32_t technique, const void *knobs, uint8_t *d_mask,
                                       hpac_stats *h_stats) {
  TraceRange trace_("hpac_hydro_step");
  hpac_status st = check_state(s);
  if (st != HPAC_OK) return st;
  if (!eos) return set_error(HPAC_EINVAL, "EOS region is NULL");
  const int64_t E = (int64_t)s->n * s->n * s->n;
  const hpac_region_desc &d = eos->d;
  if (d.kind != HPAC_REGION_EOS || d.dtype != HPAC_F64 || d.n != E || d.in_stride != E)
    return set_error(HPAC_EINVAL, "EOS region must be kind EOS, F64, n = in_stride = n^3 = %lld",
                     (long long)E);
  if (d.param != s->gamma) return set_error(HPAC_EINVAL, "EOS gamma differs from the hydro gamma");
  if (technique < 0 || technique > 3) return set_error(HPAC_EINVAL, "technique %d", technique);
  if (technique > 0 && !knobs) return set_error(HPAC_EINVAL, "knobs are NULL");
  cudaStream_t stream = eos->stream;
  st = hpac_hydro_nodes(s, stream);
  if (st != HPAC_OK) return st;
  st = hpac_hydro_elements(s, stream);
  if (st != HPAC_OK) return st;
  switch (technique) {
    case 0:
      st = hpac_run_exact(eos, s->eos_in, s->p);
      if (st == HPAC_OK && h_stats) {
        HPAC_CUDA_TRY(cudaStreamSynchronize(stream));
        *h_stats = hpac_stats{E, 0, 0, 0};
      }
      break;
    case 1:
      st = hpac_run_taf(eos, static_cast<const hpac_taf_knobs *>(knobs), s->eos_in, s->p, d_mask,
                        nullptr, h_stats);
      break;
    case 2:
      st = hpac_run_iact(eos, static_cast<const hpac_iact_knobs *>(knobs), s->eos_in, s->p, d_mask,
                         nullptr, h_stats);
      break;
    default:
      st = hpac_run_perfo(eos, static_cast<const hpac_perfo_knobs *>(knobs), s->eos_in, s->p,
                          d_mask, h_stats);
      break;
  }
  if (st != HPAC_OK) return st;
  return hpac_hydro_finalize(s, stream);
}

extern "C" hpac_status hpac_hydro_run(const hpac_hydro_state *s, hpac_region *eos, int32_t steps,
                                      int32_t technique, const void *knobs) {
  TraceRange trace_("hpac_hydro_run");
  if (steps < 0) return set_error(HPAC_EINVAL, "steps < 0");
  for (int32_t k = 0; k < steps; ++k) {
    hpac_status st = hpac_hydro_step(s, eos, technique, knobs, nullptr, nullptr);
    if (st != HPAC_OK) return st;
  }
  return HPAC_OK;
}
