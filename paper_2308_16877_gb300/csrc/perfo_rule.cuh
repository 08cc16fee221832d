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

}  // namespace hpac
