// Internal declarations shared by the translation units of libhpac.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "hpac.h"

struct hpac_region {
  hpac_region_desc d;
  cudaStream_t stream;
  int device;
  unsigned long long *d_counters;  // [0] approximated, [1] borderline
  int persist;                     // TAF windows / iACT tables kept across calls
  void *d_state;                   // their device copy (region-owned)
  size_t state_bytes;
  int64_t state_key[6];            // technique and shape the copy holds
  const void *aux;                 // K-Means: the caller's centroids (device)
};

namespace hpac {

constexpr int kWarp = 32;
constexpr int kMaxIn = 8;
constexpr int kMaxHsize = 64;
constexpr int kMaxTsize = 64;
constexpr int kMaxBinomialSteps = 1024;
constexpr int kMaxClusters = 64;
constexpr double kBorderRel = 1e-6;

// Thread-local error reporting (hpac_last_error).
hpac_status set_error(hpac_status s, const char *fmt, ...);
hpac_status cuda_error(cudaError_t e, const char *what);

inline int64_t logical_threads(const hpac_region_desc &d) {
  return d.logical_threads > 0 ? d.logical_threads : (d.n > 0 ? d.n : 1);
}

// Launchers (one translation unit each). All validate nothing: the C ABI layer
// has checked the descriptor and knobs before calling them.
hpac_status launch_exact(const hpac_region *r, const void *in, void *out);
hpac_status launch_perfo(const hpac_region *r, const hpac_perfo_knobs *k, const void *in, void *out,
                         uint8_t *mask, unsigned long long *counters);
hpac_status launch_taf(hpac_region *r, const hpac_taf_knobs *k, const void *in, void *out,
                       uint8_t *mask, void *stat, unsigned long long *counters);
hpac_status launch_iact(hpac_region *r, const hpac_iact_knobs *k, const void *in, void *out,
                        uint8_t *mask, void *stat, unsigned long long *counters);

// The Binomial region: every technique runs in binomial.cu's team kernels
// (technique 0 exact, 1 TAF, 2 iACT, 3 perforation; knobs of that technique).
hpac_status launch_binomial(hpac_region *r, int technique, const void *knobs, const void *in,
                            void *out, uint8_t *mask, void *stat, unsigned long long *counters);

// The persistent state buffer of a TAF or iACT run: nullptr when the region
// keeps no state; otherwise a zeroed buffer of `bytes` the first time a shape
// (key) is seen, the previous run's buffer when the key repeats.
hpac_status region_state(hpac_region *r, const int64_t (&key)[6], size_t bytes, void **out);

inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// A named NVTX range around a library call, for timeline tools (Nsight
// Systems, ncu --nvtx); without a tool attached the push and pop return at
// once.
struct TraceRange {
  explicit TraceRange(const char *name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange &) = delete;
  TraceRange &operator=(const TraceRange &) = delete;
};

// Largest dynamic shared memory a block of this device may use.
int max_dyn_smem(int device);

// Number of SMs of the device.
int sm_count(int device);

// Physical block size (a multiple of 32, at most b) for a launch of `threads`
// threads whose block is not part of the semantics (plain maps, thread- and
// warp-level decisions): small enough to give every SM about eight blocks.
// The work of a region is often uneven along the invocation index (a shock
// front, a run of approximations), and double-precision work runs at a small
// fraction of the single-precision rate, so a few large blocks left on a few
// SMs would set the kernel time.
int balanced_block(int64_t threads, int b, int device);

}  // namespace hpac

#define HPAC_CUDA_TRY(call)                                   \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return hpac::cuda_error(e_, #call); \
  } while (0)
