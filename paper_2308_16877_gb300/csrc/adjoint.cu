// Adjoint (input derivatives) of the exact regions: the derivative targets of
// the learned surrogate, and, scaled by an upstream gradient, the backward
// pass of a differentiable region call (vector-Jacobian product). One thread
// per invocation, grid-stride.
#include <math.h>

#include "hpac_internal.cuh"
#include "regions.cuh"

namespace hpac {
namespace {

// Black-Scholes call partials with respect to (S, K, T, sigma):
// dC/dS = N(d1), dC/dK = -e^{-rT} N(d2),
// dC/dT = S phi(d1) sigma / (2 sqrt T) + r K e^{-rT} N(d2), dC/dsigma = S phi(d1) sqrt T.
__global__ void bs32_adjoint(const float *__restrict__ in, int64_t stride, int64_t n, float r,
                             const float *__restrict__ gout, float *__restrict__ g) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float S = in[i], K = in[stride + i], Tm = in[2 * stride + i], sig = in[3 * stride + i];
    const float sq = sqrtf(Tm), sst = sig * sq;
    const float d1 = (__logf(__fdividef(S, K)) + (r + 0.5f * sig * sig) * Tm) / sst;
    const float d2 = d1 - sst;
    const float disc = __expf(-r * Tm);
    const float phi1 = 0.3989422804014327f * __expf(-0.5f * d1 * d1);
    const float n2 = normal_cdf(d2);
    const float w = gout ? gout[i] : 1.0f;
    g[i] = w * normal_cdf(d1);
    g[n + i] = w * (-disc * n2);
    g[2 * n + i] = w * (S * phi1 * sig * 0.5f / sq + r * K * disc * n2);
    g[3 * n + i] = w * (S * phi1 * sq);
  }
}

__global__ void bs64_adjoint(const double *__restrict__ in, int64_t stride, int64_t n, double r,
                             const double *__restrict__ gout, double *__restrict__ g) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double S = in[i], K = in[stride + i], Tm = in[2 * stride + i], sig = in[3 * stride + i];
    const double sq = sqrt(Tm), sst = sig * sq;
    const double d1 = (log(S / K) + (r + 0.5 * sig * sig) * Tm) / sst;
    const double d2 = d1 - sst;
    const double disc = exp(-r * Tm);
    const double phi1 = 0.39894228040143267794 * exp(-0.5 * d1 * d1);
    const double n1 = 0.5 * erfc(-0.70710678118654752440 * d1);
    const double n2 = 0.5 * erfc(-0.70710678118654752440 * d2);
    const double w = gout ? gout[i] : 1.0;
    g[i] = w * n1;
    g[n + i] = w * (-disc * n2);
    g[2 * n + i] = w * (S * phi1 * sig * 0.5 / sq + r * K * disc * n2);
    g[3 * n + i] = w * (S * phi1 * sq);
  }
}

// EOS: p = (g-1) num / Dn with num = e - dv (p0 + 2q)/2, p0 = (g-1) e / (v1 - dv),
// Dn = v1 + (g-1) dv / 2 (the closed form of the implicit update times v1);
// zero where num < 0 (the energy clamp).
__global__ void eos_adjoint(const double *__restrict__ in, int64_t stride, int64_t n, double gamma,
                            const double *__restrict__ gout, double *__restrict__ g) {
  const double g1 = gamma - 1.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double e = in[i], v1 = in[stride + i], dv = in[2 * stride + i], q = in[3 * stride + i];
    const double v0 = v1 - dv;
    const double p0 = g1 * e / v0;
    const double num = e - 0.5 * dv * (p0 + 2.0 * q);
    const double Dn = v1 + 0.5 * g1 * dv;
    double de = 0.0, dv1 = 0.0, ddv = 0.0, dq = 0.0;
    if (num >= 0.0) {
      const double dp0_dv1 = -g1 * e / (v0 * v0);
      const double num_e = 1.0 - 0.5 * dv * g1 / v0;
      const double num_v1 = -0.5 * dv * dp0_dv1;
      const double num_dv = -0.5 * p0 - 0.5 * dv * (-dp0_dv1) - q;
      const double inv = 1.0 / Dn;
      de = g1 * num_e * inv;
      dq = -g1 * dv * inv;
      dv1 = g1 * (num_v1 * Dn - num) * inv * inv;
      ddv = g1 * (num_dv * Dn - 0.5 * g1 * num) * inv * inv;
    }
    const double w = gout ? gout[i] : 1.0;
    g[i] = w * de;
    g[n + i] = w * dv1;
    g[2 * n + i] = w * ddv;
    g[3 * n + i] = w * dq;
  }
}

template <typename T>
__global__ void identity_adjoint(int64_t n, int D, const T *__restrict__ gout, T *__restrict__ g) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    for (int d = 0; d < D; ++d) g[d * n + i] = d == 0 ? (gout ? gout[i] : (T)1) : (T)0;
}

}  // namespace
}  // namespace hpac

using namespace hpac;

namespace {

hpac_status adjoint_launch(hpac_region *r, const void *d_in, const void *d_gout, void *d_grad) {
  if (!r) return set_error(HPAC_EINVAL, "region is NULL");
  const hpac_region_desc &d = r->d;
  if (d.n == 0) return HPAC_OK;
  if (!d_in || !d_grad) return set_error(HPAC_EINVAL, "NULL pointer");
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, r->device);
  int64_t blocks = (d.n + 255) / 256;
  if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
  if (d.kind == HPAC_REGION_BINOMIAL || d.kind == HPAC_REGION_KMEANS)
    return set_error(HPAC_EUNSUPPORTED, "no adjoint of region kind %d", d.kind);
  const bool f32 = d.dtype == HPAC_F32;
  const float *gf = static_cast<const float *>(d_gout);
  const double *gd = static_cast<const double *>(d_gout);
  switch (d.kind) {
    case HPAC_REGION_BLACKSCHOLES:
      if (f32)
        bs32_adjoint<<<(unsigned)blocks, 256, 0, r->stream>>>(
            static_cast<const float *>(d_in), d.in_stride, d.n, (float)d.param, gf,
            static_cast<float *>(d_grad));
      else
        bs64_adjoint<<<(unsigned)blocks, 256, 0, r->stream>>>(
            static_cast<const double *>(d_in), d.in_stride, d.n, d.param, gd,
            static_cast<double *>(d_grad));
      break;
    case HPAC_REGION_EOS:
      eos_adjoint<<<(unsigned)blocks, 256, 0, r->stream>>>(
          static_cast<const double *>(d_in), d.in_stride, d.n, d.param, gd,
          static_cast<double *>(d_grad));
      break;
    default:
      if (f32)
        identity_adjoint<float><<<(unsigned)blocks, 256, 0, r->stream>>>(d.n, d.n_in, gf,
                                                                         static_cast<float *>(d_grad));
      else
        identity_adjoint<double><<<(unsigned)blocks, 256, 0, r->stream>>>(d.n, d.n_in, gd,
                                                                          static_cast<double *>(d_grad));
  }
  HPAC_CUDA_TRY(cudaGetLastError());
  return HPAC_OK;
}

}  // namespace

extern "C" hpac_status hpac_region_adjoint(hpac_region *r, const void *d_in, void *d_grad) {
  TraceRange trace_("hpac_region_adjoint");
  return adjoint_launch(r, d_in, nullptr, d_grad);
}

extern "C" hpac_status hpac_region_vjp(hpac_region *r, const void *d_in, const void *d_gout,
                                       void *d_grad) {
  TraceRange trace_("hpac_region_vjp");
  if (r && r->d.n > 0 && !d_gout) return set_error(HPAC_EINVAL, "upstream gradient is NULL");
  return adjoint_launch(r, d_in, d_gout, d_grad);
}
