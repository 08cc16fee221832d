// C ABI of libhpac: argument checking, region handles, statistics readback.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "hpac_internal.cuh"

namespace hpac {

static thread_local char g_err[512] = "";

hpac_status set_error(hpac_status s, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}

hpac_status cuda_error(cudaError_t e, const char *what) {
  return set_error(HPAC_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

int max_dyn_smem(int device) {
  static int cached[64] = {0};
  if (device < 0 || device >= 64) return 48 * 1024;
  if (!cached[device]) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess ||
        v <= 0)
      v = 48 * 1024;
    cached[device] = v - 1024;  // headroom for the kernels' static shared memory
  }
  return cached[device];
}

int sm_count(int device) {
  static int cached[64] = {0};
  if (device < 0 || device >= 64) return 148;
  if (!cached[device]) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || v <= 0)
      v = 148;
    cached[device] = v;
  }
  return cached[device];
}

int balanced_block(int64_t threads, int b, int device) {
  const int64_t want = (int64_t)sm_count(device) * 8;
  int64_t per = (threads + want - 1) / want;
  per = (per + 31) / 32 * 32;
  if (per < 32) per = 32;
  return per < b ? (int)per : b;
}

static hpac_status check_desc(const hpac_region_desc *d) {
  if (!d) return set_error(HPAC_EINVAL, "descriptor is NULL");
  if (d->n < 0) return set_error(HPAC_EINVAL, "n = %lld < 0", (long long)d->n);
  if (d->n_out != 1) return set_error(HPAC_EINVAL, "n_out = %d, must be 1", d->n_out);
  if (d->n_in < 1 || d->n_in > kMaxIn) return set_error(HPAC_EINVAL, "n_in = %d not in 1..8", d->n_in);
  if (d->in_stride < d->n || d->out_stride < d->n)
    return set_error(HPAC_EINVAL, "stride smaller than n");
  if (d->logical_threads < 0) return set_error(HPAC_EINVAL, "logical_threads < 0");
  if (d->block_threads < 32 || d->block_threads > 1024 || d->block_threads % 32)
    return set_error(HPAC_EINVAL, "block_threads = %d, must be a multiple of 32 in 32..1024",
                     d->block_threads);
  if (d->dtype != HPAC_F32 && d->dtype != HPAC_F64) return set_error(HPAC_EINVAL, "dtype %d", d->dtype);
  if (d->kind != HPAC_REGION_BINOMIAL && d->kind != HPAC_REGION_KMEANS && d->arg != 0)
    return set_error(HPAC_EINVAL, "arg must be 0 for region kind %d", d->kind);
  if (!isfinite(d->param)) return set_error(HPAC_EINVAL, "param is not finite");
  switch (d->kind) {
    case HPAC_REGION_BLACKSCHOLES:
      if (d->n_in != 4) return set_error(HPAC_EINVAL, "Black-Scholes takes 4 inputs");
      break;
    case HPAC_REGION_EOS:
      if (d->n_in != 4) return set_error(HPAC_EINVAL, "EOS takes 4 inputs");
      if (d->dtype != HPAC_F64) return set_error(HPAC_EUNSUPPORTED, "EOS is double precision only");
      break;
    case HPAC_REGION_IDENTITY:
      break;
    case HPAC_REGION_KMEANS:
      if (d->n_in != 8) return set_error(HPAC_EINVAL, "K-Means takes 8 features");
      if (d->dtype != HPAC_F32) return set_error(HPAC_EUNSUPPORTED, "K-Means is single precision only");
      if (d->arg < 1 || d->arg > kMaxClusters)
        return set_error(HPAC_EINVAL, "K-Means clusters %d not in 1..%d", d->arg, kMaxClusters);
      break;
    case HPAC_REGION_BINOMIAL:
      if (d->n_in != 4) return set_error(HPAC_EINVAL, "Binomial takes 4 inputs");
      if (d->dtype != HPAC_F32) return set_error(HPAC_EUNSUPPORTED, "Binomial is single precision only");
      if (d->arg < 1 || d->arg > kMaxBinomialSteps)
        return set_error(HPAC_EINVAL, "Binomial steps %d not in 1..%d", d->arg, kMaxBinomialSteps);
      break;
    default:
      return set_error(HPAC_EINVAL, "unknown region kind %d", d->kind);
  }
  return HPAC_OK;
}

static hpac_status check_call(hpac_region *r, const void *in, const void *out) {
  if (!r) return set_error(HPAC_EINVAL, "region is NULL");
  if (r->d.n > 0 && (!in || !out)) return set_error(HPAC_EINVAL, "input or output pointer is NULL");
  if (r->d.kind == HPAC_REGION_KMEANS && !r->aux)
    return set_error(HPAC_EINVAL, "K-Means region without centroids (hpac_region_set_aux)");
  int dev = -1;
  HPAC_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != r->device)
    return set_error(HPAC_EINVAL, "current device %d differs from the region's device %d", dev,
                     r->device);
  return HPAC_OK;
}

static hpac_status begin_counters(hpac_region *r, const void *h_stats) {
  if (!h_stats) return HPAC_OK;
  HPAC_CUDA_TRY(cudaMemsetAsync(r->d_counters, 0, 2 * sizeof(unsigned long long), r->stream));
  return HPAC_OK;
}

static hpac_status end_counters(hpac_region *r, hpac_stats *h, int64_t skipped_known) {
  if (!h) return HPAC_OK;
  unsigned long long c[3] = {0, 0, 0};
  HPAC_CUDA_TRY(cudaMemcpyAsync(c, r->d_counters, sizeof(c), cudaMemcpyDeviceToHost, r->stream));
  HPAC_CUDA_TRY(cudaStreamSynchronize(r->stream));
  if (c[2]) {  // a bounded device-side wait of an earlier call gave up
    HPAC_CUDA_TRY(cudaMemsetAsync(r->d_counters + 2, 0, sizeof(unsigned long long), r->stream));
    return set_error(HPAC_ETIMEOUT, "a bounded device-side wait of the region's kernels gave up");
  }
  h->invocations = r->d.n;
  h->approximated = (int64_t)c[0];
  h->skipped = skipped_known;
  h->borderline = (int64_t)c[1];
  return HPAC_OK;
}

}  // namespace hpac

namespace hpac {

hpac_status region_state(hpac_region *r, const int64_t (&key)[6], size_t bytes, void **out) {
  *out = nullptr;
  if (!r->persist) return HPAC_OK;
  if (r->d_state && r->state_bytes == bytes && memcmp(r->state_key, key, sizeof(key)) == 0) {
    *out = r->d_state;
    return HPAC_OK;
  }
  // a new shape: the previous state cannot continue, start empty
  if (r->d_state) {
    HPAC_CUDA_TRY(cudaStreamSynchronize(r->stream));
    HPAC_CUDA_TRY(cudaFree(r->d_state));
    r->d_state = nullptr;
    r->state_bytes = 0;
  }
  HPAC_CUDA_TRY(cudaMalloc(&r->d_state, bytes));
  r->state_bytes = bytes;
  memcpy(r->state_key, key, sizeof(key));
  HPAC_CUDA_TRY(cudaMemsetAsync(r->d_state, 0, bytes, r->stream));
  *out = r->d_state;
  return HPAC_OK;
}

}  // namespace hpac

using namespace hpac;

extern "C" {

const char *hpac_last_error(void) { return g_err; }

const char *hpac_version(void) { return "hpac-gb300 0.1 (sm_103a)"; }

hpac_status hpac_region_create(const hpac_region_desc *desc, void *cuda_stream, hpac_region **out) {
  if (!out) return set_error(HPAC_EINVAL, "out is NULL");
  *out = nullptr;
  hpac_status s = check_desc(desc);
  if (s != HPAC_OK) return s;
  hpac_region *r = (hpac_region *)calloc(1, sizeof(hpac_region));
  if (!r) return set_error(HPAC_ENOMEM, "host allocation of the region handle failed");
  r->d = *desc;
  r->stream = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaGetDevice(&r->device);
  if (e == cudaSuccess) e = cudaMalloc(&r->d_counters, 4 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(r->d_counters, 0, 4 * sizeof(unsigned long long));
  if (e != cudaSuccess) {
    free(r);
    return cuda_error(e, "hpac_region_create");
  }
  *out = r;
  return HPAC_OK;
}

hpac_status hpac_region_destroy(hpac_region *r) {
  if (!r) return HPAC_OK;
  cudaError_t e = cudaStreamSynchronize(r->stream);
  cudaError_t f = cudaFree(r->d_counters);
  if (r->d_state) {
    const cudaError_t g = cudaFree(r->d_state);
    if (f == cudaSuccess) f = g;
  }
  free(r);
  if (e != cudaSuccess) return cuda_error(e, "hpac_region_destroy: stream");
  if (f != cudaSuccess) return cuda_error(f, "hpac_region_destroy: free");
  return HPAC_OK;
}

hpac_status hpac_region_set_persistent(hpac_region *r, int32_t enable) {
  if (!r) return set_error(HPAC_EINVAL, "region is NULL");
  if (enable != 0 && enable != 1) return set_error(HPAC_EINVAL, "enable %d not 0 or 1", enable);
  if (!enable && r->d_state) {
    HPAC_CUDA_TRY(cudaStreamSynchronize(r->stream));
    HPAC_CUDA_TRY(cudaFree(r->d_state));
    r->d_state = nullptr;
    r->state_bytes = 0;
    memset(r->state_key, 0, sizeof(r->state_key));
  }
  r->persist = enable;
  return HPAC_OK;
}

hpac_status hpac_region_set_aux(hpac_region *r, const void *d_aux) {
  if (!r) return set_error(HPAC_EINVAL, "region is NULL");
  if (r->d.kind != HPAC_REGION_KMEANS) return set_error(HPAC_EINVAL, "region kind %d takes no aux", r->d.kind);
  if (!d_aux) return set_error(HPAC_EINVAL, "aux is NULL");
  if ((uintptr_t)d_aux % 16) return set_error(HPAC_EINVAL, "centroids not 16-byte aligned");
  r->aux = d_aux;
  return HPAC_OK;
}

hpac_status hpac_region_reset_state(hpac_region *r) {
  if (!r) return set_error(HPAC_EINVAL, "region is NULL");
  if (r->d_state) HPAC_CUDA_TRY(cudaMemsetAsync(r->d_state, 0, r->state_bytes, r->stream));
  return HPAC_OK;
}

hpac_status hpac_region_set_stream(hpac_region *r, void *cuda_stream) {
  if (!r) return set_error(HPAC_EINVAL, "region is NULL");
  r->stream = (cudaStream_t)cuda_stream;
  return HPAC_OK;
}

hpac_status hpac_run_exact(hpac_region *r, const void *d_in, void *d_out) {
  TraceRange trace_("hpac_run_exact");
  hpac_status s = check_call(r, d_in, d_out);
  if (s != HPAC_OK) return s;
  if (r->d.kind == HPAC_REGION_BINOMIAL)
    return launch_binomial(r, 0, nullptr, d_in, d_out, nullptr, nullptr, nullptr);
  return launch_exact(r, d_in, d_out);
}

hpac_status hpac_run_perfo(hpac_region *r, const hpac_perfo_knobs *k, const void *d_in, void *d_out,
                           uint8_t *d_mask, hpac_stats *h_stats) {
  TraceRange trace_("hpac_run_perfo");
  hpac_status s = check_call(r, d_in, d_out);
  if (s != HPAC_OK) return s;
  if (!k) return set_error(HPAC_EINVAL, "knobs are NULL");
  switch (k->kind) {
    case HPAC_PERFO_SMALL:
    case HPAC_PERFO_LARGE:
      if (k->m_or_percent < 1) return set_error(HPAC_EINVAL, "perforation M = %d < 1", k->m_or_percent);
      break;
    case HPAC_PERFO_INI:
    case HPAC_PERFO_FINI:
      if (k->m_or_percent < 0 || k->m_or_percent > 100)
        return set_error(HPAC_EINVAL, "perforation percent %d not in 0..100", k->m_or_percent);
      break;
    case HPAC_PERFO_RANDOM:
      if (!(k->rate >= 0.0 && k->rate <= 1.0))
        return set_error(HPAC_EINVAL, "perforation rate %g not in [0, 1]", k->rate);
      break;
    default:
      return set_error(HPAC_EINVAL, "unknown perforation kind %d", k->kind);
  }
  if (k->reserved0 != 0) return set_error(HPAC_EINVAL, "reserved field not zero");
  s = begin_counters(r, h_stats);
  if (s != HPAC_OK) return s;
  s = r->d.kind == HPAC_REGION_BINOMIAL
          ? launch_binomial(r, 3, k, d_in, d_out, d_mask, nullptr, h_stats ? r->d_counters : nullptr)
          : launch_perfo(r, k, d_in, d_out, d_mask, h_stats ? r->d_counters : nullptr);
  if (s != HPAC_OK) return s;
  s = end_counters(r, h_stats, 0);
  if (s == HPAC_OK && h_stats) {
    // the perforation kernel counts dropped invocations in the first counter
    h_stats->skipped = h_stats->approximated;
    h_stats->approximated = 0;
    h_stats->borderline = 0;
  }
  return s;
}

hpac_status hpac_run_taf(hpac_region *r, const hpac_taf_knobs *k, const void *d_in, void *d_out,
                         uint8_t *d_mask, void *d_stat, hpac_stats *h_stats) {
  TraceRange trace_("hpac_run_taf");
  hpac_status s = check_call(r, d_in, d_out);
  if (s != HPAC_OK) return s;
  if (!k) return set_error(HPAC_EINVAL, "knobs are NULL");
  if (k->hsize < 1 || k->hsize > kMaxHsize)
    return set_error(HPAC_EINVAL, "hsize %d not in 1..%d", k->hsize, kMaxHsize);
  if (k->psize < 0) return set_error(HPAC_EINVAL, "psize %d < 0", k->psize);
  if (!(k->thresh >= 0.0)) return set_error(HPAC_EINVAL, "threshold must be >= 0 (got %g)", k->thresh);
  if (k->level < HPAC_LEVEL_THREAD || k->level > HPAC_LEVEL_BLOCK)
    return set_error(HPAC_EINVAL, "level %d", k->level);
  if (k->reset_on_exit != 0 && k->reset_on_exit != 1)
    return set_error(HPAC_EINVAL, "reset_on_exit %d not 0 or 1", k->reset_on_exit);
  if (r->d.kind == HPAC_REGION_BINOMIAL) {
    if (k->level != HPAC_LEVEL_BLOCK)
      return set_error(HPAC_EUNSUPPORTED, "Binomial decides per team: level must be HPAC_LEVEL_BLOCK");
    if (r->persist) return set_error(HPAC_EUNSUPPORTED, "Binomial keeps no state across calls");
  }
  s = begin_counters(r, h_stats);
  if (s != HPAC_OK) return s;
  s = r->d.kind == HPAC_REGION_BINOMIAL
          ? launch_binomial(r, 1, k, d_in, d_out, d_mask, d_stat, h_stats ? r->d_counters : nullptr)
          : launch_taf(r, k, d_in, d_out, d_mask, d_stat, h_stats ? r->d_counters : nullptr);
  if (s != HPAC_OK) return s;
  return end_counters(r, h_stats, 0);
}

hpac_status hpac_run_iact(hpac_region *r, const hpac_iact_knobs *k, const void *d_in, void *d_out,
                          uint8_t *d_mask, void *d_stat, hpac_stats *h_stats) {
  TraceRange trace_("hpac_run_iact");
  hpac_status s = check_call(r, d_in, d_out);
  if (s != HPAC_OK) return s;
  if (!k) return set_error(HPAC_EINVAL, "knobs are NULL");
  if (k->tsize < 1 || k->tsize > kMaxTsize)
    return set_error(HPAC_EINVAL, "tsize %d not in 1..%d", k->tsize, kMaxTsize);
  if (k->tperwarp < 1 || k->tperwarp > 32 || (32 % k->tperwarp) != 0)
    return set_error(HPAC_EINVAL, "tperwarp %d must divide 32", k->tperwarp);
  if (!(k->thresh >= 0.0)) return set_error(HPAC_EINVAL, "threshold must be >= 0 (got %g)", k->thresh);
  if (k->level < HPAC_LEVEL_THREAD || k->level > HPAC_LEVEL_BLOCK)
    return set_error(HPAC_EINVAL, "level %d", k->level);
  if (k->reserved0 != 0) return set_error(HPAC_EINVAL, "reserved field not zero");
  if (k->in_scale)
    for (int j = 0; j < r->d.n_in; ++j)
      if (!isfinite(k->in_scale[j])) return set_error(HPAC_EINVAL, "in_scale[%d] is not finite", j);
  if (r->d.kind == HPAC_REGION_BINOMIAL) {
    if (k->level != HPAC_LEVEL_BLOCK || k->tperwarp != 32)
      return set_error(HPAC_EUNSUPPORTED,
                       "Binomial keeps one table per team: level HPAC_LEVEL_BLOCK, tperwarp 32");
    if (r->persist) return set_error(HPAC_EUNSUPPORTED, "Binomial keeps no state across calls");
  }
  s = begin_counters(r, h_stats);
  if (s != HPAC_OK) return s;
  s = r->d.kind == HPAC_REGION_BINOMIAL
          ? launch_binomial(r, 2, k, d_in, d_out, d_mask, d_stat, h_stats ? r->d_counters : nullptr)
          : launch_iact(r, k, d_in, d_out, d_mask, d_stat, h_stats ? r->d_counters : nullptr);
  if (s != HPAC_OK) return s;
  return end_counters(r, h_stats, 0);
}

}  // extern "C"
