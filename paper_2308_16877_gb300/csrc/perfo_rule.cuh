// Drop rule of the loop-perforation patterns (Sections 2.3, 3.1.5, 3.3),
// shared by the perforation kernel and the knob-sweep kernel.
#pragma once

#include <stdint.h>

#include "hpac.h"

namespace hpac {

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Drop rule of one perforation pattern (see hpac.h). SplitMix64 above is the
// counter-based generator of Steele, Lea and Flood (2014).
struct DropRule {
  int kind;          // -1: nothing dropped (accurate path)
  int herded;
  int64_t m;         // M for small/large
  int64_t lo, hi;    // kept range [lo, hi) for ini/fini
  uint64_t seed;
  uint32_t cut;      // floor(rate * 2^24)
  int64_t T;         // logical threads

  __device__ __forceinline__ bool drop_key(int64_t key) const {
    switch (kind) {
      case HPAC_PERFO_SMALL: return key % m == m - 1;
      case HPAC_PERFO_LARGE: return key % m != 0;
      case HPAC_PERFO_RANDOM: return (uint32_t)(splitmix64(seed ^ (uint64_t)key) >> 40) < cut;
      default: return false;
    }
  }
  // Drop decisions for V consecutive invocations starting at i0.
  template <int V>
  __device__ __forceinline__ void drops(int64_t i0, bool (&d)[V]) const {
    if (kind < 0) {
#pragma unroll
      for (int j = 0; j < V; ++j) d[j] = false;
      return;
    }
    if (kind == HPAC_PERFO_INI || kind == HPAC_PERFO_FINI) {
#pragma unroll
      for (int j = 0; j < V; ++j) d[j] = (i0 + j < lo) || (i0 + j >= hi);
      return;
    }
    if (!herded) {
#pragma unroll
      for (int j = 0; j < V; ++j) d[j] = drop_key(i0 + j);
      return;
    }
    // herded: key = step index k = i / T
    const int64_t k0 = i0 / T;
    const int64_t r0 = i0 - k0 * T;
    if (r0 + V <= T) {
      const bool dd = drop_key(k0);
#pragma unroll
      for (int j = 0; j < V; ++j) d[j] = dd;
    } else {
#pragma unroll
      for (int j = 0; j < V; ++j) d[j] = drop_key((i0 + j) / T);
    }
  }
};

// drops<V> for a thread that visits the groups i0, i0 + G, i0 + 2G, ... of a
// grid-stride loop. The step k = i0 / T of a herded pattern and the residues
// modulo M of the small and large patterns are carried from one group to the
// next by additions, so the loop divides only once per thread, at its start.
template <int V>
struct DropWalk {
  int64_t k, r;      // herded: i0 = k T + r with 0 <= r < T
  int64_t dk, dr;
  int res;           // small / large: k mod M (herded) or i0 mod M (per invocation)
  int dres, m;

  __device__ __forceinline__ void init(const DropRule &R, int64_t i0, int64_t G) {
    k = r = res = dk = dr = dres = 0;
    m = (R.kind == HPAC_PERFO_SMALL || R.kind == HPAC_PERFO_LARGE) ? (int)R.m : 1;
    if (R.kind < 0 || R.kind == HPAC_PERFO_INI || R.kind == HPAC_PERFO_FINI) return;
    if (R.herded) {
      k = i0 / R.T;
      r = i0 - k * R.T;
      dk = G / R.T;
      dr = G - dk * R.T;
      res = (int)(k % m);
      dres = (int)(dk % m);
    } else {
      res = (int)(i0 % m);
      dres = (int)(G % m);
    }
  }
  __device__ __forceinline__ void advance(const DropRule &R) {
    if (R.herded) {
      k += dk;
      r += dr;
      res += dres;
      if (r >= R.T) {
        r -= R.T;
        ++k;
        ++res;
      }
    } else {
      res += dres;
    }
    if (res >= m) res -= m;  // res < 2M here (M < 2^31)
  }
  // The whole group's decision when it is the same for its V invocations: a
  // herded pattern with T a multiple of V (no group straddles two steps), or
  // ini / fini with no group straddling an end of the kept range.
  __device__ __forceinline__ bool uniform(const DropRule &R, int64_t i0) const {
    if (R.kind == HPAC_PERFO_INI || R.kind == HPAC_PERFO_FINI) return i0 < R.lo || i0 >= R.hi;
    return (R.kind == HPAC_PERFO_SMALL || R.kind == HPAC_PERFO_LARGE) ? drop_res(R, res)
                                                                      : R.drop_key(k);
  }
  __device__ __forceinline__ bool drop_res(const DropRule &R, int q) const {
    return R.kind == HPAC_PERFO_SMALL ? q == m - 1 : q != 0;
  }
  __device__ __forceinline__ void drops(const DropRule &R, int64_t i0, bool (&d)[V]) const {
    const bool modm = R.kind == HPAC_PERFO_SMALL || R.kind == HPAC_PERFO_LARGE;
    if (R.kind < 0 || R.kind == HPAC_PERFO_INI || R.kind == HPAC_PERFO_FINI ||
        (!R.herded && !modm)) {
      R.drops<V>(i0, d);  // no division on these paths
      return;
    }
    if (R.herded) {
      if (r + V <= R.T) {
        const bool dd = modm ? drop_res(R, res) : R.drop_key(k);
#pragma unroll
        for (int j = 0; j < V; ++j) d[j] = dd;
      } else {  // the group straddles steps: walk them invocation by invocation
        int64_t rr = r, kk = k;
        int q = res;
#pragma unroll
        for (int j = 0; j < V; ++j) {
          d[j] = modm ? drop_res(R, q) : R.drop_key(kk);
          if (++rr == R.T) {
            rr = 0;
            ++kk;
            q = q + 1 == m ? 0 : q + 1;
          }
        }
      }
      return;
    }
    int q = res;
#pragma unroll
    for (int j = 0; j < V; ++j) {
      d[j] = drop_res(R, q);
      q = q + 1 == m ? 0 : q + 1;
    }
  }
};

}  // namespace hpac
