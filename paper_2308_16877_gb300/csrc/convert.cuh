// Conversions between double and single precision on the integer pipes.
// GB300 executes the hardware conversions (and double comparisons) on its
// narrow FP64 pipe, about two per SM and clock; these give the same bits with
// integer operations, for every input (normal, subnormal, zero, infinite and
// NaN). The common cases take a few instructions; a warp with a rare input
// takes the full integer conversion for it, so no FP64 instruction is issued,
// not even a predicated one.
#pragma once

#include <stdint.h>

namespace hpac {

// Double to single precision, rounded to nearest even, for every input. A NaN
// keeps its sign and the top 22 bits of its payload, with the quiet bit set.
__device__ __forceinline__ float double_to_float_full(double x) {
  const uint64_t u = (uint64_t)__double_as_longlong(x);
  const uint32_t hi = (uint32_t)(u >> 32), sign = hi & 0x80000000u;
  const uint32_t ed = (hi >> 20) & 0x7ffu;
  const uint64_t m = (u & 0xfffffffffffffull) | (1ull << 52);  // significand of a normal double
  // normal single: keep 24 of the 53 bits, ties to even; a carry out of the
  // fraction raises the exponent (to infinity from 254)
  const int e = (int)ed - (1023 - 127);
  const uint32_t frac = (uint32_t)((u >> 29) & 0x7fffffu);
  const uint32_t rem = (uint32_t)(u & 0x1fffffffu);
  const uint32_t up = (rem > 0x10000000u) | ((rem == 0x10000000u) & (frac & 1u));
  const uint32_t normal = ((uint32_t)(e < 1 ? 1 : e) << 23) + frac + up;
  // subnormal single (or zero): m 2^(ed - 1075) in units of 2^-149 is
  // m >> (926 - ed), rounded to nearest even; a result of 2^23 is the
  // smallest normal single, which the same bits encode
  const int s = 926 - (int)ed;  // 30 when e = 0
  const int sc = s < 1 ? 1 : (s > 63 ? 63 : s);
  const uint64_t q = m >> sc, r = m & ((1ull << sc) - 1ull), half = 1ull << (sc - 1);
  const uint32_t sub = (uint32_t)q + (uint32_t)((r > half) | ((r == half) & (q & 1ull)));
  uint32_t res = e >= 1 ? normal : (s > 54 ? 0u : sub);
  if (e > 254) res = 0x7f800000u;                                   // overflow to infinity
  if (ed == 0x7ffu)  // infinity, or NaN
    res = (u & 0xfffffffffffffull) ? 0x7fc00000u | (uint32_t)((u >> 29) & 0x3fffffu) : 0x7f800000u;
  return __uint_as_float(sign | res);
}

// Single to double precision (exact) for every input. A NaN keeps its
// payload with the quiet bit set.
__device__ __forceinline__ double float_to_double_full(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  const uint64_t sign = (uint64_t)(u & 0x80000000u) << 32;
  // normal
  uint64_t r = ((uint64_t)(e + (1023 - 127)) << 52) | ((uint64_t)m << 29);
  // subnormal: leading bit of m at p = 31 - clz(m); value 1.f x 2^(p - 149)
  const int lz = __clz(m | 1u);
  const uint32_t p = 31u - (uint32_t)lz;
  const uint64_t fs = ((uint64_t)(m << (23u - p)) & 0x7fffffull) << 29;
  const uint64_t rs = ((uint64_t)(p + (1023u - 149u)) << 52) | fs;
  if (e == 0u) r = m ? rs : 0ull;
  if (e == 0xffu) r = (0x7ffull << 52) | ((uint64_t)m << 29) | (m ? (1ull << 51) : 0ull);
  return __longlong_as_double((long long)(sign | r));
}

// The common cases in a few integer operations: double to single where the
// result is a normal single or a zero, single to double for normal singles
// and zeros. A warp with any other input takes the full conversion for it (a
// warp-uniform branch, so warps without one skip it).
__device__ __forceinline__ float double_to_float_rn(double x) {
  const uint64_t u = (uint64_t)__double_as_longlong(x);
  const uint32_t hi = (uint32_t)(u >> 32), sign = hi & 0x80000000u;
  const uint32_t ed = (hi >> 20) & 0x7ffu;
  const int e = (int)ed - (1023 - 127);
  const uint32_t frac = (uint32_t)((u >> 29) & 0x7fffffu);
  const uint32_t rem = (uint32_t)(u & 0x1fffffffu);
  const uint32_t up = (rem > 0x10000000u) | ((rem == 0x10000000u) & (frac & 1u));
  uint32_t r = sign | ((((uint32_t)e << 23) + frac + up) & (ed ? 0xffffffffu : 0u));
  const bool rare = ed != 0u && (e < 1 || e > 254);
  if (__any_sync(__activemask(), rare)) {
    if (rare) r = __float_as_uint(double_to_float_full(x));
  }
  return __uint_as_float(r);
}

__device__ __forceinline__ double float_to_double(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xffu;
  const uint64_t sign = (uint64_t)(u & 0x80000000u) << 32;
  uint64_t r = sign | ((((uint64_t)(e + (1023 - 127)) << 52) | ((uint64_t)(u & 0x7fffffu) << 29)) &
                       ((u << 1) ? ~0ull : 0ull));
  const bool rare = e == 0xffu || (e == 0u && (u & 0x7fffffu) != 0u);
  if (__any_sync(__activemask(), rare)) {
    if (rare) r = (uint64_t)__double_as_longlong(float_to_double_full(f));
  }
  return __longlong_as_double((long long)r);
}

// Double to single precision, rounded to nearest even: the integer fast path
// for normal-single results and zeros, the hardware conversion for the rest,
// without a warp vote. The compiler may issue that conversion predicated in
// every warp; in a kernel with slack on its FP64 pipe this costs less than
// the vote (the kept-state iACT kernel is bound by issue and latency).
__device__ __forceinline__ float double_to_float_rn_novote(double x) {
  const uint64_t u = (uint64_t)__double_as_longlong(x);
  const uint32_t hi = (uint32_t)(u >> 32), sign = hi & 0x80000000u;
  const uint32_t ed = (hi >> 20) & 0x7ffu;
  if (ed == 0u) return __uint_as_float(sign);
  const int e = (int)ed - (1023 - 127);
  if (e < 1 || e > 254) return __double2float_rn(x);
  const uint32_t frac = (uint32_t)((u >> 29) & 0x7fffffu);
  const uint32_t rem = (uint32_t)(u & 0x1fffffffu);
  const uint32_t up = (rem > 0x10000000u) | ((rem == 0x10000000u) & (frac & 1u));
  return __uint_as_float(sign | (((uint32_t)e << 23) + frac + up));
}

}  // namespace hpac
