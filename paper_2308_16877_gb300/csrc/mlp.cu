// Learned surrogate of a region: a D -> H -> H -> 1 MLP with GELU (tanh form,
// Hendrycks & Gimpel 2016), BF16 weights and activations, FP32 accumulation,
// trained with Adam (Kingma & Ba 2014) by the library's own forward and
// backward kernels, with the exact region as fallback. Not from the paper: it
// stands beside TAF and iACT as a third way to skip the region's arithmetic.
//
// Three kernels:
//  - inference (mlp_tc_infer): layer 2 (H x H, the contraction) as one
//    128-row tcgen05 product per tile into tensor memory, layers 1 and 3 and
//    the GELUs on the CUDA cores in packed single-precision pairs, one
//    invocation per thread;
//  - training gradient (mlp_tc_grad): the forward product, the backward
//    product dh1 = dz2 W2, and the weight-gradient contractions over the
//    samples (dW2 with db2, dW3, dW1 with db1) as tcgen05 products
//    accumulated in tensor memory across a block's tiles; the same pass with
//    a caller's per-sample d(loss)/d(output) in place of the squared error's
//    gives the parameter half of a vector-Jacobian product;
//  - input derivatives (mlp_tc_input_grad): the forward product and the
//    backward product dh1 = dz2 W2 on tcgen05, one invocation per thread,
//    then the chain rule from the features to the region inputs on the CUDA
//    cores (the input half of a vector-Jacobian product scales it by the
//    caller's per-sample derivative).
#include <cuda_bf16.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "hpac_internal.cuh"
#include "regions.cuh"

struct hpac_mlp {
  hpac_mlp_desc d;
  int device;
  cudaStream_t stream;
  int n_params;
  float *params;   // FP32 master copy
  float *grad;
  float *m, *v;    // Adam moments
  float *loss;     // device scalar: sum of squared errors of the last gradient pass
  unsigned long long *counters;
  int64_t step;
};

namespace hpac {
namespace {

constexpr float kGeluA = 0.7978845608028654f;  // sqrt(2/pi)
constexpr float kGeluB = 0.044715f;

__device__ __forceinline__ float tanh_fast(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&v);
}
__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

struct MlpArgs {
  const void *in;       // region inputs (SoA, in_stride)
  int64_t stride, n;
  double param;         // r (Black-Scholes) or gamma (EOS)
  const float *target;  // gradient: region outputs
  float *out;           // inference: region outputs; input gradient: D x n derivatives
  uint8_t *mask;        // inference (nullable)
  float fallback_below; // inference: exact region where the prediction is below (NaN: never)
  const float *params;
  float *grad;
  float *loss;
  unsigned long long *counters;  // [0] fallbacks, [2] status (a tensor-core wait gave up)
  float inv_n;          // gradient: 1 / total samples of the batch
  const float *gout;    // vector-Jacobian products: per-sample d(loss)/d(region output);
                        // the gradient takes it instead of the squared error, the input
                        // gradient multiplies each input derivative by it (nullable)
};

// Feature count of a region kind (the descriptor's n_feat is checked against it
// at creation), a compile-time constant in the kernels.
template <int KIND>
constexpr int n_feat_of() {
  return KIND == HPAC_REGION_BLACKSCHOLES ? 5 : 4;
}

// Features of one invocation (FP32) and the output multiplier of the region.
template <int KIND>
__device__ __forceinline__ void features(const void *in, int64_t stride, int64_t i, double param,
                                         const hpac_mlp_desc &d, float (&f)[8], float &mult,
                                         float (&raw)[4]) {
  if (KIND == HPAC_REGION_BLACKSCHOLES) {
    const float *x = static_cast<const float *>(in);
    const float S = x[i], K = x[stride + i], T = x[2 * stride + i], sig = x[3 * stride + i];
    raw[0] = S, raw[1] = K, raw[2] = T, raw[3] = sig;
    const float r = (float)param;
    f[0] = __logf(__fdividef(S, K));
    f[1] = sig * sqrtf(T);
    f[2] = r * T;
    f[3] = fminf(fmaxf(__fdividef(f[0] + (r + 0.5f * sig * sig) * T, f[1]), -10.f), 10.f);  // d1
    f[4] = sig;
    mult = S;
  } else {
    // EOS: the output multiplier is the ideal-gas pressure of the energy after
    // the viscous work, (gamma - 1) max(e - dv q, 0) / v1, so the network learns
    // a ratio near 1 and an untouched element (e = q = 0) gives exactly 0
    const double *x = static_cast<const double *>(in);
    const double e = x[i], v1 = x[stride + i], dv = x[2 * stride + i], q = x[3 * stride + i];
    raw[0] = (float)e, raw[1] = (float)v1, raw[2] = (float)dv, raw[3] = (float)q;
#pragma unroll
    for (int k = 0; k < 4; ++k) f[k] = raw[k];
    const double u = e - dv * q;
    mult = u > 0.0 ? (float)((param - 1.0) * u / v1) : 0.f;
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) f[k] = k < n_feat_of<KIND>() ? (f[k] - d.feat_shift[k]) * d.feat_scale[k] : 0.f;
}

// ---------------------------------------------------------------------------
// Inference on the fifth-generation tensor cores (tcgen05, accumulators in
// tensor memory). One thread owns one invocation of a 128-invocation tile:
// features, layer 1 and GELU in FP32 on the CUDA cores, the BF16 activations
// written as row `thread` of the layer-2 A operand in shared memory; one
// elected thread issues the H x H product (M = 128 rows, N = H, K = H in
// steps of 16) into an FP32 accumulator of H tensor-memory columns and
// commits it to an mbarrier; every thread then reads its own row back
// (tcgen05.ld, 32 lanes per warp) for bias, GELU and the layer-3 dot product.
//
// Operands in shared memory use the canonical no-swizzle K-major layout of
// 8-row x 16-byte core matrices: element (r, k) of an R x H BF16 matrix at
// byte (r / 8) * 16 H + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2, so the
// leading-dimension offset (between core matrices along K) is 128 bytes and
// the stride offset (between 8-row groups) 16 H bytes. A is the tile's
// activations (128 x H), B is W2 as stored, [out][in] (N x K, K-major).
//
// Every wait on the mbarrier is bounded: after kWaitLimit polls the block
// sets the status word (counters[2] = 1), waits once more (bounded) for the
// product in flight, frees its tensor memory and returns; hpac_mlp_infer
// reports HPAC_ETIMEOUT at its next synchronizing call.
// ---------------------------------------------------------------------------
constexpr int kTile = 128;
constexpr int kWaitLimit = 1 << 20;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start address, leading and stride byte
// offsets (all in 16-byte units), descriptor version 1 (bits 46-47), no
// swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3fff) | ((uint64_t)((lbo >> 4) & 0x3fff) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3fff) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16
// A and B (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N / 8 at
// bits 17-22, M / 16 at bits 24-28.
template <int N>
__host__ __device__ constexpr uint32_t umma_idesc_bf16_m128() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kTile >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  for (int it = 0; it < kWaitLimit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// 32 consecutive FP32 accumulator columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

template <int H>
struct TcLayout {
  static constexpr int kA = 0;                        // 128 x H BF16 activations
  static constexpr int kB = kTile * H * 2;            // H x H BF16 W2 [out][in]
  static constexpr int kW1 = kB + H * H * 2;          // H / 2 unit pairs x 8 features, float pairs
  static constexpr int kB1 = kW1 + H * 8 * 4;
  static constexpr int kB2 = kB1 + H * 4;
  static constexpr int kW3 = kB2 + H * 4;
  static constexpr int kB3 = kW3 + H * 4;
  static constexpr int kBar = (kB3 + 4 + 7) & ~7;     // mbarrier (8 bytes)
  static constexpr int kSlot = kBar + 8;              // tensor-memory address
  static constexpr int kBytes = kSlot + 8;
};

// Byte offset of element (r, k) in the canonical K-major layout of an
// R x H BF16 operand (8-element chunk k / 8).
template <int H>
__device__ __forceinline__ int kmajor_off(int r, int k) {
  return (r >> 3) * (16 * H) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// GELU of two values in packed single-precision pairs,
// 0.5 z (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))), one IEEE rounding per
// operation and half, the hyperbolic tangent per value.
__device__ __forceinline__ unsigned long long gelu2(unsigned long long z) {
  const unsigned long long kA2 = f32x2_pack(kGeluA, kGeluA), kB2 = f32x2_pack(kGeluB, kGeluB);
  const unsigned long long half2 = f32x2_pack(0.5f, 0.5f), one2 = f32x2_pack(1.0f, 1.0f);
  const unsigned long long arg = f32x2_mul(kA2, f32x2_fma(f32x2_mul(kB2, z), f32x2_mul(z, z), z));
  float a0, a1;
  f32x2_unpack(arg, a0, a1);
  const unsigned long long th = f32x2_pack(tanh_fast(a0), tanh_fast(a1));
  return f32x2_mul(f32x2_mul(half2, z), f32x2_add(one2, th));
}

template <int H, int KIND>
__global__ void __launch_bounds__(kTile) mlp_tc_infer(MlpArgs a, hpac_mlp_desc d) {
  using L = TcLayout<H>;
  extern __shared__ __align__(1024) unsigned char sm[];
  float *w1 = reinterpret_cast<float *>(sm + L::kW1);
  float *b1 = reinterpret_cast<float *>(sm + L::kB1);
  float *b2 = reinterpret_cast<float *>(sm + L::kB2);
  float *w3 = reinterpret_cast<float *>(sm + L::kW3);
  float *b3 = reinterpret_cast<float *>(sm + L::kB3);
  const uint32_t bar = smem_u32(sm + L::kBar);
  uint32_t *slot = reinterpret_cast<uint32_t *>(sm + L::kSlot);
  __shared__ unsigned long long fallbacks;
  const int tid = threadIdx.x, warp = tid >> 5;
  constexpr int D = n_feat_of<KIND>();
  {
    const float *p = a.params;
    const int oW1 = 0, ob1 = H * D, oW2 = ob1 + H, ob2 = oW2 + H * H, oW3 = ob2 + H, ob3 = oW3 + H;
    for (int j = tid; j < H * H; j += kTile) {
      const int o = j / H, k = j % H;
      *reinterpret_cast<__nv_bfloat16 *>(sm + L::kB + kmajor_off<H>(o, k)) = __float2bfloat16_rn(p[oW2 + j]);
    }
    for (int j = tid; j < H * 8; j += kTile) {  // (pair, feature, half): w1[2 pair + half][feature]
      const int pr = j / 16, k = (j / 2) % 8, h = j % 2;
      w1[j] = k < D ? bf16r(p[oW1 + (2 * pr + h) * D + k]) : 0.f;
    }
    for (int j = tid; j < H; j += kTile) {
      b1[j] = p[ob1 + j];
      b2[j] = p[ob2 + j];
      w3[j] = bf16r(p[oW3 + j]);
    }
    if (tid == 0) {
      *b3 = p[ob3];
      fallbacks = 0;
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar));
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {  // H columns of tensor memory (a power of two >= 32)
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                   "r"(H));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
  }
  // W2 was written by the generic proxy; the tensor core reads it through the
  // async proxy
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *slot;
  const uint64_t adesc = umma_desc(smem_u32(sm + L::kA), 128, 16 * H);
  const uint64_t bdesc = umma_desc(smem_u32(sm + L::kB), 128, 16 * H);
  constexpr uint32_t idesc = umma_idesc_bf16_m128<H>();
  uint32_t parity = 0;
  bool failed = false;
  const int64_t tiles = (a.n + kTile - 1) / kTile;
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t i = tile * kTile + tid;
    const bool valid = i < a.n;
    float f[8], mult = 0.f, raw[4];
    features<KIND>(a.in, a.stride, valid ? i : 0, a.param, d, f, mult, raw);
    // layer 1 and GELU into row tid of A, 8 units (16 bytes) at a time; two
    // units advance together in packed pairs (the same fused multiply-adds
    // over k in order as one unit at a time), weights read 16 bytes at once
    unsigned long long fp[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) fp[k] = f32x2_pack(f[k], f[k]);
    const ulonglong2 *w1v = reinterpret_cast<const ulonglong2 *>(w1);
#pragma unroll 2
    for (int kc = 0; kc < H / 8; ++kc) {
      uint32_t pk[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int pr = 4 * kc + q;
        unsigned long long z = *reinterpret_cast<const unsigned long long *>(b1 + 2 * pr);
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) {
          const ulonglong2 w = w1v[pr * 4 + k2];
          if (2 * k2 < D) z = f32x2_fma(w.x, fp[2 * k2], z);
          if (2 * k2 + 1 < D) z = f32x2_fma(w.y, fp[2 * k2 + 1], z);
        }
        float g0, g1;
        f32x2_unpack(gelu2(z), g0, g1);
        pk[q] = pack_bf16(g0, g1);
      }
      *reinterpret_cast<uint4 *>(sm + L::kA + kmajor_off<H>(tid, 8 * kc)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
#pragma unroll
      for (int ks = 0; ks < H / 16; ++ks)  // K = 16 per product: two core matrices (256 bytes) along K
        umma_bf16(tmem, adesc + (uint64_t)((ks * 256) >> 4), bdesc + (uint64_t)((ks * 256) >> 4), idesc,
                  ks > 0 ? 1u : 0u);
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                   : "memory");
    }
    const bool ok = mbar_wait_bounded(bar, parity);
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    parity ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // row tid of the accumulator: lane 32 warp + (tid % 32) of this warp's quarter
    // bias, GELU, BF16 rounding and the layer-3 dot product in packed pairs
    // (even and odd units summed apart, then added)
    unsigned long long y2 = 0ull;
#pragma unroll
    for (int c = 0; c < H; c += 32) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
#pragma unroll
      for (int j = 0; j < 32; j += 4) {
        const float4 bb = *reinterpret_cast<const float4 *>(b2 + c + j);
        const float4 ww = *reinterpret_cast<const float4 *>(w3 + c + j);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const unsigned long long z =
              f32x2_add(f32x2_pack(v[j + 2 * h], v[j + 2 * h + 1]), h ? f32x2_pack(bb.z, bb.w) : f32x2_pack(bb.x, bb.y));
          float g0, g1;
          f32x2_unpack(gelu2(z), g0, g1);
          const float2 hb = __bfloat1622float2(__floats2bfloat162_rn(g0, g1));
          y2 = f32x2_fma(f32x2_pack(hb.x, hb.y), h ? f32x2_pack(ww.z, ww.w) : f32x2_pack(ww.x, ww.y), y2);
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    float y_even, y_odd;
    f32x2_unpack(y2, y_even, y_odd);
    float y = (y_even + y_odd) + *b3;
    if (valid) {
      const float pred = mult * fmaf(d.out_scale, y, d.out_shift);
      float o = pred;
      uint8_t mk = HPAC_MASK_APPROX;
      if (pred < a.fallback_below) {  // calibrated exact fallback (NaN never falls back)
        if (KIND == HPAC_REGION_BLACKSCHOLES) o = BlackScholes32{(float)a.param}(raw);
        mk = HPAC_MASK_EXACT;
        atomicAdd(&fallbacks, 1ull);
      }
      if (KIND == HPAC_REGION_EOS)  // the region's own dtype; pressure is non-negative
        reinterpret_cast<double *>(a.out)[i] = (double)fmaxf(o, 0.f);
      else
        a.out[i] = o;
      if (a.mask) a.mask[i] = mk;
    }
  }
  if (failed) {
    // the product in flight must land before its tensor memory is freed
    mbar_wait_bounded(bar, parity);
    if (tid == 0 && a.counters) atomicExch(&a.counters[2], 1ull);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(H));
  if (tid == 0 && fallbacks && a.counters) atomicAdd(&a.counters[0], fallbacks);
}

// ---------------------------------------------------------------------------
// Training gradients on tcgen05. One thread owns one sample of a 128-sample
// tile; five tensor-core products per tile, all M = 128 with BF16 operands in
// the canonical no-swizzle K-major layout and FP32 accumulators in tensor
// memory:
//   1. z2 = h1 W2^T            A1 = h1 (rows: samples, K = hidden), B1 = W2
//   2. dh1 = dz2 W2            A1 = dz2, B2 = W2^T (K = the layer-2 outputs)
//   3. [dW2 | db2] += dz2^T [h1 | 1]   A3 = dz2^T (rows: units, K = samples),
//                                      B3 = h1^T with a row of ones
//   4. dW3 += h2^T dy          A4 = h2^T, B4 rows 0 and 1 = dy split into its
//                              BF16 value and the BF16 of the remainder
//   5. [dW1 | db1] += dz1^T [f | 1]    A3 = dz1^T, B4 = the features and ones
// Products 3-5 contract over the samples (K = 128 per tile) and accumulate in
// tensor memory across the block's tiles; the block adds its totals to the
// gradient once at the end. Operands with the samples along K are written
// element by element (column `thread` of a K-major matrix). Rows beyond H of
// A3 and A4 stay zero (H = 64). Products 1, 2 and 3-4 are each committed to
// the block's mbarrier and waited for (bounded, as in the inference kernel);
// 5 as well. dy, db3 and the loss are reduced in FP32 through shuffles.
// ---------------------------------------------------------------------------
template <int H>
struct TcGradLayout {
  static constexpr int kA1 = 0;                            // 128 x H: h1, then dz2
  static constexpr int kB1 = kA1 + kTile * H * 2;          // H x H: W2 [out][in]
  static constexpr int kB2 = kB1 + H * H * 2;              // H x H: W2^T [in][out]
  static constexpr int kA3 = kB2 + H * H * 2;              // 128 x 128: dz2^T, then dz1^T
  static constexpr int kA4 = kA3 + kTile * kTile * 2;      // 128 x 128: h2^T
  static constexpr int kB3 = kA4 + kTile * kTile * 2;      // (H + 16) x 128: h1^T, ones, zeros
  static constexpr int kB4 = kB3 + (H + 16) * kTile * 2;   // 16 x 128: dy, then features and ones
  static constexpr int kW1 = kB4 + 16 * kTile * 2;         // unit pairs x 8 features (float pairs)
  static constexpr int kB1v = kW1 + H * 8 * 4;
  static constexpr int kB2v = kB1v + H * 4;
  static constexpr int kW3 = kB2v + H * 4;
  static constexpr int kRed = kW3 + H * 4;                 // loss, db3
  static constexpr int kBar = (kRed + 8 + 7) & ~7;
  static constexpr int kSlot = kBar + 8;
  static constexpr int kBytes = kSlot + 8;
  static constexpr int kCols = (2 * H + 48) <= 256 ? 256 : 512;  // tensor-memory columns
};

// Byte offset of element (r, s) of an R x 128 K-major operand (K = samples).
__device__ __forceinline__ int kmajor128_off(int r, int s) {
  return (r >> 3) * 2048 + (s >> 3) * 128 + (r & 7) * 16 + (s & 7) * 2;
}

template <int N>
__host__ __device__ constexpr uint32_t idesc_m128() { return umma_idesc_bf16_m128<N>(); }

// 16 consecutive FP32 accumulator columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// GELU derivative of two values in packed pairs.
__device__ __forceinline__ unsigned long long gelu_grad2(unsigned long long z) {
  const unsigned long long kA2 = f32x2_pack(kGeluA, kGeluA), kB2 = f32x2_pack(kGeluB, kGeluB);
  const unsigned long long k3B2 = f32x2_pack(3.0f * kGeluB, 3.0f * kGeluB);
  const unsigned long long half2 = f32x2_pack(0.5f, 0.5f), one2 = f32x2_pack(1.0f, 1.0f);
  const unsigned long long zz = f32x2_mul(z, z);
  const unsigned long long arg = f32x2_mul(kA2, f32x2_fma(f32x2_mul(kB2, z), zz, z));
  float a0, a1;
  f32x2_unpack(arg, a0, a1);
  const unsigned long long th = f32x2_pack(tanh_fast(a0), tanh_fast(a1));
  const unsigned long long t1 = f32x2_mul(half2, f32x2_add(one2, th));
  const unsigned long long sech2 = f32x2_sub(one2, f32x2_mul(th, th));
  const unsigned long long t2 =
      f32x2_mul(f32x2_mul(f32x2_mul(f32x2_mul(half2, z), sech2), kA2), f32x2_fma(k3B2, zz, one2));
  return f32x2_add(t1, t2);
}

// GELU and its derivative of two values in packed pairs from one hyperbolic
// tangent per value: the same operations, in the same order, as gelu2 and
// gelu_grad2 (bit-identical results).
__device__ __forceinline__ void gelu_both2(unsigned long long z, unsigned long long &g,
                                           unsigned long long &dg) {
  const unsigned long long kA2 = f32x2_pack(kGeluA, kGeluA), kB2 = f32x2_pack(kGeluB, kGeluB);
  const unsigned long long k3B2 = f32x2_pack(3.0f * kGeluB, 3.0f * kGeluB);
  const unsigned long long half2 = f32x2_pack(0.5f, 0.5f), one2 = f32x2_pack(1.0f, 1.0f);
  const unsigned long long zz = f32x2_mul(z, z);
  const unsigned long long arg = f32x2_mul(kA2, f32x2_fma(f32x2_mul(kB2, z), zz, z));
  float a0, a1;
  f32x2_unpack(arg, a0, a1);
  const unsigned long long th = f32x2_pack(tanh_fast(a0), tanh_fast(a1));
  const unsigned long long hz = f32x2_mul(half2, z);
  const unsigned long long opt = f32x2_add(one2, th);
  g = f32x2_mul(hz, opt);
  const unsigned long long t1 = f32x2_mul(half2, opt);
  const unsigned long long sech2 = f32x2_sub(one2, f32x2_mul(th, th));
  const unsigned long long t2 = f32x2_mul(f32x2_mul(f32x2_mul(hz, sech2), kA2), f32x2_fma(k3B2, zz, one2));
  dg = f32x2_add(t1, t2);
}

__device__ __forceinline__ void st_bf16(unsigned char *base, int off, float v) {
  *reinterpret_cast<__nv_bfloat16 *>(base + off) = __float2bfloat16_rn(v);
}

// Issue `steps` K = 16 products (256 bytes along K per step) and commit them.
__device__ __forceinline__ void umma_k(uint32_t d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int steps,
                                       bool accumulate) {
  for (int ks = 0; ks < steps; ++ks)
    umma_bf16(d, adesc + (uint64_t)((ks * 256) >> 4), bdesc + (uint64_t)((ks * 256) >> 4), idesc,
              (accumulate || ks > 0) ? 1u : 0u);
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void sync_for_umma() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

template <int H, int KIND>
__global__ void __launch_bounds__(kTile) mlp_tc_grad(MlpArgs a, hpac_mlp_desc d) {
  using L = TcGradLayout<H>;
  extern __shared__ __align__(1024) unsigned char sm[];
  float *w1 = reinterpret_cast<float *>(sm + L::kW1);
  float *b1 = reinterpret_cast<float *>(sm + L::kB1v);
  float *b2 = reinterpret_cast<float *>(sm + L::kB2v);
  float *w3 = reinterpret_cast<float *>(sm + L::kW3);
  float *red = reinterpret_cast<float *>(sm + L::kRed);
  const uint32_t bar = smem_u32(sm + L::kBar);
  uint32_t *slot = reinterpret_cast<uint32_t *>(sm + L::kSlot);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int D = n_feat_of<KIND>();
  const float *p = a.params;
  const int oW1 = 0, ob1 = H * D, oW2 = ob1 + H, ob2 = oW2 + H * H, oW3 = ob2 + H, ob3 = oW3 + H;
  // operands: W2 and its transpose, zeroed sample-major operands, the row of
  // ones of B3, the weight vectors
  for (int j = tid; j < H * H; j += kTile) {
    const int o = j / H, k = j % H;
    const __nv_bfloat16 w = __float2bfloat16_rn(p[oW2 + j]);
    *reinterpret_cast<__nv_bfloat16 *>(sm + L::kB1 + kmajor_off<H>(o, k)) = w;
    *reinterpret_cast<__nv_bfloat16 *>(sm + L::kB2 + kmajor_off<H>(k, o)) = w;
  }
  // zeros where no tile writes: rows H.. of A3 and A4 (H = 64), rows H..
  // of B3 and all of B4 (each row group of 8 is 2048 contiguous bytes)
  {
    const uint4 z4 = make_uint4(0u, 0u, 0u, 0u);
    constexpr int kPad = (kTile - H) * kTile * 2 / 16;  // 16-byte words of rows H..127
    for (int j = tid; j < kPad; j += kTile) {
      reinterpret_cast<uint4 *>(sm + L::kA3 + H * kTile * 2)[j] = z4;
      reinterpret_cast<uint4 *>(sm + L::kA4 + H * kTile * 2)[j] = z4;
    }
    for (int j = tid; j < (16 * kTile * 2 + 16 * kTile * 2) / 16; j += kTile)
      reinterpret_cast<uint4 *>(sm + L::kB3 + H * kTile * 2)[j] = z4;  // B3 rows H..H+15, then B4
  }
  __syncthreads();  // the zeros land before the row of ones is written into them
  st_bf16(sm + L::kB3, kmajor128_off(H, tid), 1.0f);
  for (int j = tid; j < H * 8; j += kTile) {
    const int pr = j / 16, k = (j / 2) % 8, h = j % 2;
    w1[j] = k < D ? bf16r(p[oW1 + (2 * pr + h) * D + k]) : 0.f;
  }
  for (int j = tid; j < H; j += kTile) {
    b1[j] = p[ob1 + j];
    b2[j] = p[ob2 + j];
    w3[j] = bf16r(p[oW3 + j]);
  }
  if (tid == 0) {
    red[0] = red[1] = 0.f;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(L::kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  sync_for_umma();
  const uint32_t tmem = *slot;
  const uint32_t d12 = tmem, d3 = tmem + H, d4 = tmem + 2 * H + 16, d5 = tmem + 2 * H + 32;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  const uint64_t a1 = umma_desc(smem_u32(sm + L::kA1), 128, 16 * H);
  const uint64_t b1d = umma_desc(smem_u32(sm + L::kB1), 128, 16 * H);
  const uint64_t b2d = umma_desc(smem_u32(sm + L::kB2), 128, 16 * H);
  const uint64_t a3 = umma_desc(smem_u32(sm + L::kA3), 128, 2048);
  const uint64_t a4 = umma_desc(smem_u32(sm + L::kA4), 128, 2048);
  const uint64_t b3d = umma_desc(smem_u32(sm + L::kB3), 128, 2048);
  const uint64_t b4d = umma_desc(smem_u32(sm + L::kB4), 128, 2048);
  const float b3 = p[ob3];
  uint32_t parity = 0;
  bool failed = false, any = false;
  const int64_t tiles = (a.n + kTile - 1) / kTile;
  for (int64_t tile = blockIdx.x; tile < tiles && !failed; tile += gridDim.x) {
    const int64_t i = tile * kTile + tid;
    const bool valid = i < a.n;
    float f[8], mult = 0.f, raw[4];
    features<KIND>(a.in, a.stride, valid ? i : 0, a.param, d, f, mult, raw);
    unsigned long long fp[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) fp[k] = f32x2_pack(f[k], f[k]);
    const ulonglong2 *w1v = reinterpret_cast<const ulonglong2 *>(w1);
    // ---- phase F: layer 1 and GELU; h1 into row tid of A1 and column tid of B3
#pragma unroll 2
    for (int kc = 0; kc < H / 8; ++kc) {
      uint32_t pk[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int pr = 4 * kc + q;
        unsigned long long z = *reinterpret_cast<const unsigned long long *>(b1 + 2 * pr);
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) {
          const ulonglong2 w = w1v[pr * 4 + k2];
          if (2 * k2 < D) z = f32x2_fma(w.x, fp[2 * k2], z);
          if (2 * k2 + 1 < D) z = f32x2_fma(w.y, fp[2 * k2 + 1], z);
        }
        float g0, g1;
        f32x2_unpack(gelu2(z), g0, g1);
        pk[q] = pack_bf16(g0, g1);
        *reinterpret_cast<uint16_t *>(sm + L::kB3 + kmajor128_off(2 * pr, tid)) = (uint16_t)(pk[q] & 0xffffu);
        *reinterpret_cast<uint16_t *>(sm + L::kB3 + kmajor128_off(2 * pr + 1, tid)) = (uint16_t)(pk[q] >> 16);
      }
      *reinterpret_cast<uint4 *>(sm + L::kA1 + kmajor_off<H>(tid, 8 * kc)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
    sync_for_umma();
    if (tid == 0) {
      umma_k(d12, a1, b1d, idesc_m128<H>(), H / 16, false);
      umma_commit(bar);
    }
    if (__syncthreads_or(!mbar_wait_bounded(bar, parity))) {
      failed = true;
      break;
    }
    parity ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // ---- phase B, pass 1: the network output and the loss derivative dy
    unsigned long long y2 = 0ull;
#pragma unroll
    for (int c = 0; c < H; c += 32) {
      float v[32];
      tmem_ld32(d12 + lane_base + (uint32_t)c, v);
#pragma unroll
      for (int j = 0; j < 32; j += 2) {
        const unsigned long long z = f32x2_add(f32x2_pack(v[j], v[j + 1]), *reinterpret_cast<const unsigned long long *>(b2 + c + j));
        float g0, g1;
        f32x2_unpack(gelu2(z), g0, g1);
        const float2 hb = __bfloat1622float2(__floats2bfloat162_rn(g0, g1));
        y2 = f32x2_fma(f32x2_pack(hb.x, hb.y), *reinterpret_cast<const unsigned long long *>(w3 + c + j), y2);
      }
    }
    float ye, yo;
    f32x2_unpack(y2, ye, yo);
    const float y = (ye + yo) + b3;
    float dy, e2 = 0.f;
    if (a.gout) {
      const float o = mult * fmaf(d.out_scale, y, d.out_shift);
      const bool k = valid && (KIND != HPAC_REGION_EOS || o > 0.f);
      dy = k ? a.gout[i] * mult * d.out_scale : 0.f;
    } else {
      // rows whose multiplier is 0 (an untouched EOS element) carry no target
      const bool u = valid && mult != 0.f;
      const float t = u ? (a.target[i] / mult - d.out_shift) / d.out_scale : 0.f;
      const float e = u ? y - t : 0.f;
      dy = 2.f * e * a.inv_n;
      e2 = e * e;
    }
    {
      float s_dy = dy, s_e2 = e2;
      for (int off = 16; off > 0; off >>= 1) {
        s_dy += __shfl_xor_sync(0xffffffffu, s_dy, off);
        s_e2 += __shfl_xor_sync(0xffffffffu, s_e2, off);
      }
      if (lane == 0) {
        atomicAdd(&red[1], s_dy);
        atomicAdd(&red[0], s_e2);
      }
    }
    // ---- phase B, pass 2: dz2 = dy w3 gelu'(z2) into row tid of A1 (as
    // BF16) and column tid of A3; h2 into column tid of A4; dy into B4
    const unsigned long long dyp = f32x2_pack(dy, dy);
#pragma unroll
    for (int c = 0; c < H; c += 32) {
      float v[32];
      tmem_ld32(d12 + lane_base + (uint32_t)c, v);
#pragma unroll
      for (int j = 0; j < 32; j += 8) {
        uint32_t pk[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int u = c + j + 2 * q;
          const unsigned long long z = f32x2_add(f32x2_pack(v[j + 2 * q], v[j + 2 * q + 1]),
                                                 *reinterpret_cast<const unsigned long long *>(b2 + u));
          unsigned long long gz, dgz;
          gelu_both2(z, gz, dgz);
          float g0, g1;
          f32x2_unpack(gz, g0, g1);
          const uint32_t h2 = pack_bf16(g0, g1);
          *reinterpret_cast<uint16_t *>(sm + L::kA4 + kmajor128_off(u, tid)) = (uint16_t)(h2 & 0xffffu);
          *reinterpret_cast<uint16_t *>(sm + L::kA4 + kmajor128_off(u + 1, tid)) = (uint16_t)(h2 >> 16);
          const unsigned long long dz =
              f32x2_mul(f32x2_mul(dyp, *reinterpret_cast<const unsigned long long *>(w3 + u)), dgz);
          float d0, d1;
          f32x2_unpack(dz, d0, d1);
          pk[q] = pack_bf16(d0, d1);
          *reinterpret_cast<uint16_t *>(sm + L::kA3 + kmajor128_off(u, tid)) = (uint16_t)(pk[q] & 0xffffu);
          *reinterpret_cast<uint16_t *>(sm + L::kA3 + kmajor128_off(u + 1, tid)) = (uint16_t)(pk[q] >> 16);
        }
        *reinterpret_cast<uint4 *>(sm + L::kA1 + kmajor_off<H>(tid, c + j)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
      }
    }
    {
      const float hi = bf16r(dy);
      st_bf16(sm + L::kB4, kmajor128_off(0, tid), hi);
      st_bf16(sm + L::kB4, kmajor128_off(1, tid), dy - hi);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    sync_for_umma();
    if (tid == 0) {
      umma_k(d12, a1, b2d, idesc_m128<H>(), H / 16, false);                 // dh1 = dz2 W2
      umma_k(d3, a3, b3d, idesc_m128<H + 16>(), kTile / 16, any);           // [dW2 | db2]
      umma_k(d4, a4, b4d, idesc_m128<16>(), kTile / 16, any);               // dW3
      umma_commit(bar);
    }
    if (__syncthreads_or(!mbar_wait_bounded(bar, parity))) {
      failed = true;
      break;
    }
    parity ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // ---- phase C: dz1 = dh1 gelu'(z1) (z1 recomputed) into column tid of
    // A3; the features and a one into column tid of B4
#pragma unroll
    for (int c = 0; c < H; c += 32) {
      float v[32];
      tmem_ld32(d12 + lane_base + (uint32_t)c, v);
#pragma unroll
      for (int j = 0; j < 32; j += 2) {
        const int pr = (c + j) / 2;
        unsigned long long z = *reinterpret_cast<const unsigned long long *>(b1 + 2 * pr);
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) {
          const ulonglong2 w = w1v[pr * 4 + k2];
          if (2 * k2 < D) z = f32x2_fma(w.x, fp[2 * k2], z);
          if (2 * k2 + 1 < D) z = f32x2_fma(w.y, fp[2 * k2 + 1], z);
        }
        const unsigned long long dz1 = f32x2_mul(f32x2_pack(v[j], v[j + 1]), gelu_grad2(z));
        float d0, d1;
        f32x2_unpack(dz1, d0, d1);
        st_bf16(sm + L::kA3, kmajor128_off(c + j, tid), d0);
        st_bf16(sm + L::kA3, kmajor128_off(c + j + 1, tid), d1);
      }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (k < D) st_bf16(sm + L::kB4, kmajor128_off(k, tid), valid ? f[k] : 0.f);
    st_bf16(sm + L::kB4, kmajor128_off(D, tid), 1.0f);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    sync_for_umma();
    if (tid == 0) {
      umma_k(d5, a3, b4d, idesc_m128<16>(), kTile / 16, any);               // [dW1 | db1]
      umma_commit(bar);
    }
    if (__syncthreads_or(!mbar_wait_bounded(bar, parity))) {
      failed = true;
      break;
    }
    parity ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    any = true;
    // the next tile overwrites B4's rows 0 and 1 (dy) and leaves the feature
    // rows 2..D of this one, which only columns 2..D of product 4 read
  }
  if (failed) {
    mbar_wait_bounded(bar, parity);
    if (tid == 0 && a.counters) atomicExch(&a.counters[2], 1ull);
  } else if (any) {
    // accumulator row tid: unit tid of dW2 / db2, dW3, dW1 / db1
    const int j = tid;
#pragma unroll
    for (int c = 0; c < H; c += 32) {
      float v[32];
      tmem_ld32(d3 + lane_base + (uint32_t)c, v);
      if (j < H)
#pragma unroll
        for (int q = 0; q < 32; ++q) atomicAdd(&a.grad[oW2 + j * H + c + q], v[q]);
    }
    float v16[16];
    tmem_ld16(d3 + lane_base + (uint32_t)H, v16);
    if (j < H) atomicAdd(&a.grad[ob2 + j], v16[0]);
    tmem_ld16(d4 + lane_base, v16);
    if (j < H) atomicAdd(&a.grad[oW3 + j], v16[0] + v16[1]);
    tmem_ld16(d5 + lane_base, v16);
    if (j < H) {
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (k < D) atomicAdd(&a.grad[oW1 + j * D + k], v16[k]);
      atomicAdd(&a.grad[ob1 + j], v16[D < 8 ? D : 7]);
    }
    __syncthreads();
    if (tid == 0) {
      atomicAdd(&a.grad[ob3], red[1]);
      if (a.loss) atomicAdd(a.loss, red[0]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(L::kCols));
}

// ---------------------------------------------------------------------------
// Input derivatives on tcgen05 (hpac_mlp_input_grad, the input half of
// hpac_mlp_vjp): per 128-sample tile the forward product z2 = h1 W2^T and the
// backward product dh1 = dz2 W2 (dz2 = w3 gelu'(z2), the derivative of the
// network output), each into the same H tensor-memory columns; then per
// thread dz1 = dh1 gelu'(z1), d(net)/d(features) = dz1 W1 and the chain rule
// from the features to the region inputs, scaled by the caller's per-sample
// derivative when one is given.
// ---------------------------------------------------------------------------
template <int H>
struct TcIgLayout {
  static constexpr int kA1 = 0;                      // 128 x H: h1, then dz2
  static constexpr int kB1 = kA1 + kTile * H * 2;    // W2 [out][in]
  static constexpr int kB2 = kB1 + H * H * 2;        // W2^T [in][out]
  static constexpr int kW1 = kB2 + H * H * 2;        // unit pairs x 8 features (float pairs)
  static constexpr int kB1v = kW1 + H * 8 * 4;
  static constexpr int kB2v = kB1v + H * 4;
  static constexpr int kW3 = kB2v + H * 4;
  static constexpr int kBar = (kW3 + H * 4 + 7) & ~7;
  static constexpr int kSlot = kBar + 8;
  static constexpr int kBytes = kSlot + 8;
};

template <int H, int KIND>
__global__ void __launch_bounds__(kTile) mlp_tc_input_grad(MlpArgs a, hpac_mlp_desc d) {
  using L = TcIgLayout<H>;
  extern __shared__ __align__(1024) unsigned char sm[];
  float *w1 = reinterpret_cast<float *>(sm + L::kW1);
  float *b1 = reinterpret_cast<float *>(sm + L::kB1v);
  float *b2 = reinterpret_cast<float *>(sm + L::kB2v);
  float *w3 = reinterpret_cast<float *>(sm + L::kW3);
  const uint32_t bar = smem_u32(sm + L::kBar);
  uint32_t *slot = reinterpret_cast<uint32_t *>(sm + L::kSlot);
  const int tid = threadIdx.x, warp = tid >> 5;
  constexpr int D = n_feat_of<KIND>();
  const float *p = a.params;
  const int oW1 = 0, ob1 = H * D, oW2 = ob1 + H, ob2 = oW2 + H * H, oW3 = ob2 + H, ob3 = oW3 + H;
  for (int j = tid; j < H * H; j += kTile) {
    const int o = j / H, k = j % H;
    const __nv_bfloat16 w = __float2bfloat16_rn(p[oW2 + j]);
    *reinterpret_cast<__nv_bfloat16 *>(sm + L::kB1 + kmajor_off<H>(o, k)) = w;
    *reinterpret_cast<__nv_bfloat16 *>(sm + L::kB2 + kmajor_off<H>(k, o)) = w;
  }
  for (int j = tid; j < H * 8; j += kTile) {
    const int pr = j / 16, k = (j / 2) % 8, h = j % 2;
    w1[j] = k < D ? bf16r(p[oW1 + (2 * pr + h) * D + k]) : 0.f;
  }
  for (int j = tid; j < H; j += kTile) {
    b1[j] = p[ob1 + j];
    b2[j] = p[ob2 + j];
    w3[j] = bf16r(p[oW3 + j]);
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(H));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  sync_for_umma();
  const uint32_t tmem = *slot;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  const uint64_t a1 = umma_desc(smem_u32(sm + L::kA1), 128, 16 * H);
  const uint64_t b1d = umma_desc(smem_u32(sm + L::kB1), 128, 16 * H);
  const uint64_t b2d = umma_desc(smem_u32(sm + L::kB2), 128, 16 * H);
  const float b3 = p[ob3];
  const ulonglong2 *w1v = reinterpret_cast<const ulonglong2 *>(w1);
  uint32_t parity = 0;
  bool failed = false;
  const int64_t tiles = (a.n + kTile - 1) / kTile;
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t i = tile * kTile + tid;
    const bool valid = i < a.n;
    float f[8], mult = 0.f, raw[4];
    features<KIND>(a.in, a.stride, valid ? i : 0, a.param, d, f, mult, raw);
    unsigned long long fp[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) fp[k] = f32x2_pack(f[k], f[k]);
    // layer 1 and GELU into row tid of A1
#pragma unroll 2
    for (int kc = 0; kc < H / 8; ++kc) {
      uint32_t pk[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int pr = 4 * kc + q;
        unsigned long long z = *reinterpret_cast<const unsigned long long *>(b1 + 2 * pr);
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) {
          const ulonglong2 w = w1v[pr * 4 + k2];
          if (2 * k2 < D) z = f32x2_fma(w.x, fp[2 * k2], z);
          if (2 * k2 + 1 < D) z = f32x2_fma(w.y, fp[2 * k2 + 1], z);
        }
        float g0, g1;
        f32x2_unpack(gelu2(z), g0, g1);
        pk[q] = pack_bf16(g0, g1);
      }
      *reinterpret_cast<uint4 *>(sm + L::kA1 + kmajor_off<H>(tid, 8 * kc)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
    sync_for_umma();
    if (tid == 0) {
      umma_k(tmem, a1, b1d, idesc_m128<H>(), H / 16, false);
      umma_commit(bar);
    }
    if (__syncthreads_or(!mbar_wait_bounded(bar, parity))) {
      failed = true;
      break;
    }
    parity ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // the network output, then dz2 = w3 gelu'(z2) into row tid of A1
    unsigned long long y2 = 0ull;
#pragma unroll
    for (int c = 0; c < H; c += 32) {
      float v[32];
      tmem_ld32(tmem + lane_base + (uint32_t)c, v);
#pragma unroll
      for (int j = 0; j < 32; j += 8) {
        uint32_t pk[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int u = c + j + 2 * q;
          const unsigned long long z = f32x2_add(f32x2_pack(v[j + 2 * q], v[j + 2 * q + 1]),
                                                 *reinterpret_cast<const unsigned long long *>(b2 + u));
          const unsigned long long w3p = *reinterpret_cast<const unsigned long long *>(w3 + u);
          unsigned long long gz, dgz;
          gelu_both2(z, gz, dgz);
          float g0, g1;
          f32x2_unpack(gz, g0, g1);
          const float2 hb = __bfloat1622float2(__floats2bfloat162_rn(g0, g1));
          y2 = f32x2_fma(f32x2_pack(hb.x, hb.y), w3p, y2);
          float d0, d1;
          f32x2_unpack(f32x2_mul(w3p, dgz), d0, d1);
          pk[q] = pack_bf16(valid ? d0 : 0.f, valid ? d1 : 0.f);
        }
        *reinterpret_cast<uint4 *>(sm + L::kA1 + kmajor_off<H>(tid, c + j)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
      }
    }
    float ye, yo;
    f32x2_unpack(y2, ye, yo);
    const float net = (ye + yo) + b3;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    sync_for_umma();
    if (tid == 0) {
      umma_k(tmem, a1, b2d, idesc_m128<H>(), H / 16, false);  // dh1 = dz2 W2
      umma_commit(bar);
    }
    if (__syncthreads_or(!mbar_wait_bounded(bar, parity))) {
      failed = true;
      break;
    }
    parity ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // dz1 = dh1 gelu'(z1) (z1 recomputed) and d(net)/d(features) = dz1 W1,
    // two units per packed pair, the halves summed at the end
    unsigned long long df2[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) df2[k] = 0ull;
#pragma unroll
    for (int c = 0; c < H; c += 32) {
      float v[32];
      tmem_ld32(tmem + lane_base + (uint32_t)c, v);
#pragma unroll
      for (int j = 0; j < 32; j += 2) {
        const int pr = (c + j) / 2;
        unsigned long long z = *reinterpret_cast<const unsigned long long *>(b1 + 2 * pr);
        ulonglong2 w[4];
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) {
          w[k2] = w1v[pr * 4 + k2];
          if (2 * k2 < D) z = f32x2_fma(w[k2].x, fp[2 * k2], z);
          if (2 * k2 + 1 < D) z = f32x2_fma(w[k2].y, fp[2 * k2 + 1], z);
        }
        const unsigned long long dz1 = f32x2_mul(f32x2_pack(v[j], v[j + 1]), gelu_grad2(z));
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) {
          if (2 * k2 < D) df2[2 * k2] = f32x2_fma(dz1, w[k2].x, df2[2 * k2]);
          if (2 * k2 + 1 < D) df2[2 * k2 + 1] = f32x2_fma(dz1, w[k2].y, df2[2 * k2 + 1]);
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    if (valid) {
      float df[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        float lo, hi;
        f32x2_unpack(df2[k], lo, hi);
        df[k] = (lo + hi) * d.feat_scale[k];
      }
      float gin[4];
      if (KIND == HPAC_REGION_BLACKSCHOLES) {
        // region output C = S (shift + scale net); features ln(S/K),
        // sigma sqrt(T), r T, d1 (clamped to [-10, 10]), sigma
        const float S = raw[0], K = raw[1], Tm = raw[2], sig = raw[3];
        const float sc = d.out_scale, sq = sqrtf(Tm), r = (float)a.param;
        const float sst = sig * sq;
        const float d1 = (logf(S / K) + (r + 0.5f * sig * sig) * Tm) / sst;
        const float g3 = (d1 > -10.f && d1 < 10.f) ? df[3] : 0.f;  // clamp
        const float dnet_dS = df[0] / S + g3 / (S * sst);
        const float dnet_dK = -df[0] / K - g3 / (K * sst);
        const float dnet_dT = df[1] * sig * 0.5f / sq + df[2] * r +
                              g3 * ((r + 0.5f * sig * sig) / sst - 0.5f * d1 / Tm);
        const float dnet_dsig = df[1] * sq + df[4] + g3 * (sq - d1 / sig);
        gin[0] = fmaf(sc, net, d.out_shift) + S * sc * dnet_dS;
        gin[1] = S * sc * dnet_dK;
        gin[2] = S * sc * dnet_dT;
        gin[3] = S * sc * dnet_dsig;
      } else {
        // p = mult (shift + scale net), mult = (g - 1) (e - dv q) / v1 where positive
        const float v1 = raw[1], dv = raw[2], q = raw[3];
        const float g1 = (float)a.param - 1.f;
        const float ratio = fmaf(d.out_scale, net, d.out_shift);
        const bool on = mult > 0.f;
        const float dm[4] = {on ? g1 / v1 : 0.f, on ? -mult / v1 : 0.f, on ? -g1 * q / v1 : 0.f,
                             on ? -g1 * dv / v1 : 0.f};
#pragma unroll
        for (int k = 0; k < 4; ++k) gin[k] = ratio * dm[k] + mult * d.out_scale * df[k];
      }
      if (a.gout) {
        // the caller's d(loss)/d(output); zero where the EOS output is clamped
        const float o = mult * fmaf(d.out_scale, net, d.out_shift);
        const float go = (KIND != HPAC_REGION_EOS || o > 0.f) ? a.gout[i] : 0.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) gin[k] *= go;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) a.out[k * a.n + i] = gin[k];
    }
  }
  if (failed) {
    mbar_wait_bounded(bar, parity);
    if (tid == 0 && a.counters) atomicExch(&a.counters[2], 1ull);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(H));
}

// Sums of the features, their squares and the per-invocation targets
// (region output / multiplier) for the normalisation statistics.
template <int KIND>
__global__ void moments_kernel(const void *in, int64_t stride, int64_t n, double param,
                               const float *target, hpac_mlp_desc d, double *acc) {
  __shared__ double s[18];
  if (threadIdx.x < 18) s[threadIdx.x] = 0.0;
  __syncthreads();
  double loc[18];
#pragma unroll
  for (int k = 0; k < 18; ++k) loc[k] = 0.0;
  hpac_mlp_desc id = d;  // raw (unnormalised) features
#pragma unroll
  for (int k = 0; k < 8; ++k) id.feat_shift[k] = 0.f, id.feat_scale[k] = 1.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float f[8], mult, raw[4];
    features<KIND>(in, stride, i, param, id, f, mult, raw);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      loc[k] += f[k];
      loc[8 + k] += (double)f[k] * f[k];
    }
    if (mult != 0.f) {
      const double t = (double)target[i] / mult;
      loc[16] += t;
      loc[17] += t * t;
      loc[7] += 1.0;  // count of targets (feature slot 7 is unused: n_feat <= 5)
    }
  }
#pragma unroll
  for (int k = 0; k < 18; ++k) {
    double v = loc[k];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(&s[k], v);
  }
  __syncthreads();
  if (threadIdx.x < 18) atomicAdd(&acc[threadIdx.x], s[threadIdx.x]);
}

__global__ void adam_kernel(float *p, const float *g, float *m, float *v, int n, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

int n_params_of(const hpac_mlp_desc &d) {
  const int H = d.hidden, D = d.n_feat;
  return H * D + H + H * H + H + H + 1;
}

// The tensor-core inference: persistent blocks of 128 threads, as many per
// SM as registers, threads and shared memory allow while their tensor-memory
// columns (H each) fit in the SM's 512; extra shared memory is requested
// until they do, so no block waits for columns another resident block holds.
// Residency is computed here from the function's attributes and the device
// limits (the runtime's occupancy query reported one block per SM for this
// kernel, a quarter of what its resources allow).
template <int H, int KIND>
hpac_status launch_tc_infer(hpac_mlp *m, const MlpArgs &a) {
  auto fn = mlp_tc_infer<H, KIND>;
  cudaFuncAttributes fa;
  HPAC_CUDA_TRY(cudaFuncGetAttributes(&fa, fn));
  int sm_smem = 0, sm_regs = 0, sm_threads = 0, reserved = 0;
  HPAC_CUDA_TRY(cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, m->device));
  HPAC_CUDA_TRY(cudaDeviceGetAttribute(&sm_regs, cudaDevAttrMaxRegistersPerMultiprocessor, m->device));
  HPAC_CUDA_TRY(cudaDeviceGetAttribute(&sm_threads, cudaDevAttrMaxThreadsPerMultiProcessor, m->device));
  HPAC_CUDA_TRY(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, m->device));
  const int regs = ((fa.numRegs + 7) / 8) * 8 * kTile;
  int smem = TcLayout<H>::kBytes;
  int per_sm = 0;
  for (;;) {
    const int by_smem = sm_smem / (smem + (int)fa.sharedSizeBytes + reserved);
    const int by_regs = regs > 0 ? sm_regs / regs : 32;
    const int by_threads = sm_threads / kTile;
    per_sm = by_smem < by_regs ? by_smem : by_regs;
    per_sm = per_sm < by_threads ? per_sm : by_threads;
    if (per_sm * H <= 512 || per_sm <= 1) break;
    smem += 1024;
  }
  if (per_sm < 1) return set_error(HPAC_EUNSUPPORTED, "surrogate inference kernel does not fit an SM");
  HPAC_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  const int64_t tiles = (a.n + kTile - 1) / kTile;
  int64_t blocks = (int64_t)sm_count(m->device) * per_sm;
  if (blocks > tiles) blocks = tiles < 1 ? 1 : tiles;
  fn<<<(unsigned)blocks, kTile, smem, m->stream>>>(a, m->d);
  HPAC_CUDA_TRY(cudaGetLastError());
  return HPAC_OK;
}

// The tensor-core training gradient: one 128-thread block per SM at most
// (its operands take most of the shared memory), one tile of 128 samples per
// block and iteration.
template <int H, int KIND>
hpac_status launch_tc_grad(hpac_mlp *m, const MlpArgs &a) {
  auto fn = mlp_tc_grad<H, KIND>;
  const int smem = TcGradLayout<H>::kBytes;
  HPAC_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  const int64_t tiles = (a.n + kTile - 1) / kTile;
  int64_t blocks = sm_count(m->device);
  if (blocks > tiles) blocks = tiles < 1 ? 1 : tiles;
  fn<<<(unsigned)blocks, kTile, smem, m->stream>>>(a, m->d);
  HPAC_CUDA_TRY(cudaGetLastError());
  return HPAC_OK;
}

hpac_status launch_grad(hpac_mlp *m, const MlpArgs &a) {
  const bool bs = m->d.kind == HPAC_REGION_BLACKSCHOLES;
  if (m->d.hidden == 64)
    return bs ? launch_tc_grad<64, HPAC_REGION_BLACKSCHOLES>(m, a) : launch_tc_grad<64, HPAC_REGION_EOS>(m, a);
  return bs ? launch_tc_grad<128, HPAC_REGION_BLACKSCHOLES>(m, a) : launch_tc_grad<128, HPAC_REGION_EOS>(m, a);
}

hpac_status launch_infer(hpac_mlp *m, const MlpArgs &a) {
  const bool bs = m->d.kind == HPAC_REGION_BLACKSCHOLES;
  if (m->d.hidden == 64)
    return bs ? launch_tc_infer<64, HPAC_REGION_BLACKSCHOLES>(m, a) : launch_tc_infer<64, HPAC_REGION_EOS>(m, a);
  return bs ? launch_tc_infer<128, HPAC_REGION_BLACKSCHOLES>(m, a) : launch_tc_infer<128, HPAC_REGION_EOS>(m, a);
}

// The tensor-core input derivatives: residency as for the inference kernel.
template <int H, int KIND>
hpac_status launch_tc_input_grad(hpac_mlp *m, const MlpArgs &a) {
  auto fn = mlp_tc_input_grad<H, KIND>;
  cudaFuncAttributes fa;
  HPAC_CUDA_TRY(cudaFuncGetAttributes(&fa, fn));
  int sm_smem = 0, sm_regs = 0, sm_threads = 0, reserved = 0;
  HPAC_CUDA_TRY(cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, m->device));
  HPAC_CUDA_TRY(cudaDeviceGetAttribute(&sm_regs, cudaDevAttrMaxRegistersPerMultiprocessor, m->device));
  HPAC_CUDA_TRY(cudaDeviceGetAttribute(&sm_threads, cudaDevAttrMaxThreadsPerMultiProcessor, m->device));
  HPAC_CUDA_TRY(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, m->device));
  const int regs = ((fa.numRegs + 7) / 8) * 8 * kTile;
  int smem = TcIgLayout<H>::kBytes;
  int per_sm = 0;
  for (;;) {
    const int by_smem = sm_smem / (smem + (int)fa.sharedSizeBytes + reserved);
    const int by_regs = regs > 0 ? sm_regs / regs : 32;
    per_sm = by_smem < by_regs ? by_smem : by_regs;
    per_sm = per_sm < sm_threads / kTile ? per_sm : sm_threads / kTile;
    if (per_sm * H <= 512 || per_sm <= 1) break;
    smem += 1024;
  }
  if (per_sm < 1) return set_error(HPAC_EUNSUPPORTED, "surrogate input-gradient kernel does not fit an SM");
  HPAC_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  const int64_t tiles = (a.n + kTile - 1) / kTile;
  int64_t blocks = (int64_t)sm_count(m->device) * per_sm;
  if (blocks > tiles) blocks = tiles < 1 ? 1 : tiles;
  fn<<<(unsigned)blocks, kTile, smem, m->stream>>>(a, m->d);
  HPAC_CUDA_TRY(cudaGetLastError());
  return HPAC_OK;
}

hpac_status launch_input_grad(hpac_mlp *m, const MlpArgs &a) {
  const bool bs = m->d.kind == HPAC_REGION_BLACKSCHOLES;
  if (m->d.hidden == 64)
    return bs ? launch_tc_input_grad<64, HPAC_REGION_BLACKSCHOLES>(m, a)
              : launch_tc_input_grad<64, HPAC_REGION_EOS>(m, a);
  return bs ? launch_tc_input_grad<128, HPAC_REGION_BLACKSCHOLES>(m, a)
            : launch_tc_input_grad<128, HPAC_REGION_EOS>(m, a);
}

uint64_t sm64(uint64_t &s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

hpac_status check_io(hpac_mlp *m, int64_t n, const void *in, int64_t stride) {
  if (!m) return set_error(HPAC_EINVAL, "surrogate is NULL");
  if (n < 0 || stride < n) return set_error(HPAC_EINVAL, "n < 0 or stride < n");
  if (n > 0 && !in) return set_error(HPAC_EINVAL, "inputs are NULL");
  return HPAC_OK;
}

}  // namespace
}  // namespace hpac

using namespace hpac;

extern "C" hpac_status hpac_mlp_create(const hpac_mlp_desc *desc, const float *h_params,
                                       uint64_t seed, void *cuda_stream, hpac_mlp **out) {
  if (!out || !desc) return set_error(HPAC_EINVAL, "NULL argument");
  *out = nullptr;
  const hpac_mlp_desc &d = *desc;
  if (d.kind != HPAC_REGION_BLACKSCHOLES && d.kind != HPAC_REGION_EOS)
    return set_error(HPAC_EINVAL, "surrogate region kind %d", d.kind);
  if ((d.kind == HPAC_REGION_BLACKSCHOLES && d.n_feat != 5) || (d.kind == HPAC_REGION_EOS && d.n_feat != 4))
    return set_error(HPAC_EINVAL, "n_feat must be 5 (Black-Scholes) or 4 (EOS)");
  if (d.hidden != 64 && d.hidden != 128) return set_error(HPAC_EINVAL, "hidden must be 64 or 128");
  if (!(d.out_scale != 0.f) || !isfinite(d.out_scale)) return set_error(HPAC_EINVAL, "out_scale");
  hpac_mlp *m = (hpac_mlp *)calloc(1, sizeof(hpac_mlp));
  if (!m) return set_error(HPAC_ENOMEM, "host allocation failed");
  m->d = d;
  m->stream = (cudaStream_t)cuda_stream;
  m->n_params = n_params_of(d);
  cudaError_t e = cudaGetDevice(&m->device);
  const size_t pb = sizeof(float) * m->n_params;
  if (e == cudaSuccess) e = cudaMalloc(&m->params, pb);
  if (e == cudaSuccess) e = cudaMalloc(&m->grad, pb);
  if (e == cudaSuccess) e = cudaMalloc(&m->m, pb);
  if (e == cudaSuccess) e = cudaMalloc(&m->v, pb);
  if (e == cudaSuccess) e = cudaMalloc(&m->loss, sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->counters, 4 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(m->counters, 0, 4 * sizeof(unsigned long long));
  if (e != cudaSuccess) {
    hpac_mlp_destroy(m);
    return cuda_error(e, "hpac_mlp_create");
  }
  float *h = (float *)malloc(pb);
  if (!h) {
    hpac_mlp_destroy(m);
    return set_error(HPAC_ENOMEM, "host allocation failed");
  }
  if (h_params) {
    memcpy(h, h_params, pb);
  } else {
    // uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases
    const int H = d.hidden, D = d.n_feat;
    uint64_t st = seed;
    auto uni = [&](float bound) {
      return (float)((double)(sm64(st) >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0) * bound;
    };
    int o = 0;
    for (int i = 0; i < H * D; ++i) h[o++] = uni(1.f / sqrtf((float)D));
    for (int i = 0; i < H; ++i) h[o++] = 0.f;
    for (int i = 0; i < H * H; ++i) h[o++] = uni(1.f / sqrtf((float)H));
    for (int i = 0; i < H; ++i) h[o++] = 0.f;
    for (int i = 0; i < H; ++i) h[o++] = uni(1.f / sqrtf((float)H));
    h[o++] = 0.f;
  }
  e = cudaMemcpy(m->params, h, pb, cudaMemcpyHostToDevice);
  free(h);
  if (e == cudaSuccess) e = cudaMemset(m->m, 0, pb);
  if (e == cudaSuccess) e = cudaMemset(m->v, 0, pb);
  if (e != cudaSuccess) {
    hpac_mlp_destroy(m);
    return cuda_error(e, "hpac_mlp_create upload");
  }
  *out = m;
  return HPAC_OK;
}

extern "C" hpac_status hpac_mlp_destroy(hpac_mlp *m) {
  if (!m) return HPAC_OK;
  cudaStreamSynchronize(m->stream);
  cudaFree(m->params);
  cudaFree(m->grad);
  cudaFree(m->m);
  cudaFree(m->v);
  cudaFree(m->loss);
  cudaFree(m->counters);
  free(m);
  return HPAC_OK;
}

extern "C" int32_t hpac_mlp_num_params(const hpac_mlp *m) { return m ? m->n_params : 0; }

extern "C" hpac_status hpac_mlp_get_params(hpac_mlp *m, float *h_params) {
  if (!m || !h_params) return set_error(HPAC_EINVAL, "NULL argument");
  HPAC_CUDA_TRY(cudaMemcpyAsync(h_params, m->params, sizeof(float) * m->n_params,
                                cudaMemcpyDeviceToHost, m->stream));
  HPAC_CUDA_TRY(cudaStreamSynchronize(m->stream));
  return HPAC_OK;
}

extern "C" hpac_status hpac_mlp_set_params(hpac_mlp *m, const float *h_params) {
  if (!m || !h_params) return set_error(HPAC_EINVAL, "NULL argument");
  HPAC_CUDA_TRY(cudaMemcpyAsync(m->params, h_params, sizeof(float) * m->n_params,
                                cudaMemcpyHostToDevice, m->stream));
  HPAC_CUDA_TRY(cudaStreamSynchronize(m->stream));
  m->step = 0;
  HPAC_CUDA_TRY(cudaMemsetAsync(m->m, 0, sizeof(float) * m->n_params, m->stream));
  HPAC_CUDA_TRY(cudaMemsetAsync(m->v, 0, sizeof(float) * m->n_params, m->stream));
  return HPAC_OK;
}

extern "C" hpac_status hpac_mlp_infer(hpac_mlp *m, int64_t n, const void *d_in, int64_t in_stride,
                                      double param, void *d_out_, float fallback_below,
                                      uint8_t *d_mask, hpac_stats *h_stats) {
  TraceRange trace_("hpac_mlp_infer");
  hpac_status s = check_io(m, n, d_in, in_stride);
  if (s != HPAC_OK) return s;
  float *d_out = static_cast<float *>(d_out_);
  if (n > 0 && !d_out) return set_error(HPAC_EINVAL, "output is NULL");
  if (m->d.kind != HPAC_REGION_BLACKSCHOLES && !isnan(fallback_below))
    return set_error(HPAC_EUNSUPPORTED, "exact fallback is implemented for Black-Scholes only");
  if (h_stats) HPAC_CUDA_TRY(cudaMemsetAsync(m->counters, 0, sizeof(unsigned long long), m->stream));
  if (n > 0) {
    MlpArgs a{};
    a.in = d_in, a.stride = in_stride, a.n = n, a.param = param, a.out = d_out, a.mask = d_mask;
    a.fallback_below = fallback_below;
    a.params = m->params;
    a.counters = m->counters;
    s = launch_infer(m, a);
    if (s != HPAC_OK) return s;
  }
  if (h_stats) {
    unsigned long long c[3] = {0, 0, 0};
    HPAC_CUDA_TRY(cudaMemcpyAsync(c, m->counters, sizeof(c), cudaMemcpyDeviceToHost, m->stream));
    HPAC_CUDA_TRY(cudaStreamSynchronize(m->stream));
    if (c[2]) {
      HPAC_CUDA_TRY(cudaMemsetAsync(m->counters + 2, 0, sizeof(unsigned long long), m->stream));
      return set_error(HPAC_ETIMEOUT, "surrogate inference: a tensor-core product did not complete "
                                      "within the kernel's wait limit");
    }
    *h_stats = hpac_stats{n, n - (int64_t)c[0], 0, 0};
  }
  return HPAC_OK;
}

extern "C" hpac_status hpac_mlp_grad(hpac_mlp *m, int64_t n, const void *d_in, int64_t in_stride,
                                     double param, const float *d_target, float *d_grad,
                                     float *h_loss) {
  TraceRange trace_("hpac_mlp_grad");
  hpac_status s = check_io(m, n, d_in, in_stride);
  if (s != HPAC_OK) return s;
  if (n < 1 || !d_target) return set_error(HPAC_EINVAL, "empty batch or NULL targets");
  float *grad = d_grad ? d_grad : m->grad;
  HPAC_CUDA_TRY(cudaMemsetAsync(grad, 0, sizeof(float) * m->n_params, m->stream));
  HPAC_CUDA_TRY(cudaMemsetAsync(m->loss, 0, sizeof(float), m->stream));
  MlpArgs a{};
  a.in = d_in, a.stride = in_stride, a.n = n, a.param = param, a.target = d_target;
  a.params = m->params;
  a.grad = grad;
  a.loss = m->loss;
  a.counters = m->counters;
  a.inv_n = 1.0f / (float)n;
  s = launch_grad(m, a);
  if (s != HPAC_OK) return s;
  if (h_loss) {
    float l = 0.f;
    unsigned long long status = 0;
    HPAC_CUDA_TRY(cudaMemcpyAsync(&l, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    HPAC_CUDA_TRY(cudaMemcpyAsync(&status, m->counters + 2, sizeof(status), cudaMemcpyDeviceToHost, m->stream));
    HPAC_CUDA_TRY(cudaStreamSynchronize(m->stream));
    if (status) {
      HPAC_CUDA_TRY(cudaMemsetAsync(m->counters + 2, 0, sizeof(unsigned long long), m->stream));
      return set_error(HPAC_ETIMEOUT, "surrogate gradient: a tensor-core product did not complete within "
                                      "the kernel's wait limit");
    }
    *h_loss = l / (float)n;
  }
  return HPAC_OK;
}

extern "C" hpac_status hpac_mlp_train(hpac_mlp *m, int64_t n, const void *d_in, int64_t in_stride,
                                      double param, const float *d_target, int32_t batch,
                                      int32_t epochs, float lr, float *h_loss) {
  TraceRange trace_("hpac_mlp_train");
  hpac_status s = check_io(m, n, d_in, in_stride);
  if (s != HPAC_OK) return s;
  if (n < 1 || !d_target || batch < 16 || epochs < 0 || !(lr > 0.f))
    return set_error(HPAC_EINVAL, "bad training arguments");
  const int64_t nb = (n + batch - 1) / batch;
  const int64_t total = nb * epochs;
  int64_t it = 0;
  for (int ep = 0; ep < epochs; ++ep) {
    for (int64_t b = 0; b < nb; ++b, ++it) {
      const int64_t lo = b * batch, cnt = (n - lo) < batch ? (n - lo) : batch;
      // the batch is a column window of the structure-of-arrays inputs
      const void *in_b = m->d.kind == HPAC_REGION_BLACKSCHOLES
                             ? (const void *)((const float *)d_in + lo)
                             : (const void *)((const double *)d_in + lo);
      s = hpac_mlp_grad(m, cnt, in_b, in_stride, param, d_target + lo, nullptr, nullptr);
      if (s != HPAC_OK) return s;
      // cosine-decayed learning rate
      const float lr_t = 0.5f * lr * (1.0f + cosf(3.14159265f * (float)it / (float)total));
      ++m->step;
      const float c1 = 1.f - powf(0.9f, (float)m->step), c2 = 1.f - powf(0.999f, (float)m->step);
      adam_kernel<<<(m->n_params + 255) / 256, 256, 0, m->stream>>>(
          m->params, m->grad, m->m, m->v, m->n_params, lr_t, 0.9f, 0.999f, 1e-8f, c1, c2);
      HPAC_CUDA_TRY(cudaGetLastError());
    }
  }
  if (h_loss) {
    // loss of the whole set with the final parameters
    s = hpac_mlp_grad(m, n, d_in, in_stride, param, d_target, nullptr, h_loss);
    if (s != HPAC_OK) return s;
  }
  return HPAC_OK;
}

extern "C" hpac_status hpac_mlp_input_grad(hpac_mlp *m, int64_t n, const void *d_in,
                                           int64_t in_stride, double param, float *d_grad) {
  TraceRange trace_("hpac_mlp_input_grad");
  hpac_status s = check_io(m, n, d_in, in_stride);
  if (s != HPAC_OK) return s;
  if (n > 0 && !d_grad) return set_error(HPAC_EINVAL, "output is NULL");
  if (n == 0) return HPAC_OK;
  MlpArgs a{};
  a.in = d_in, a.stride = in_stride, a.n = n, a.param = param, a.out = d_grad;
  a.params = m->params;
  a.counters = m->counters;
  return launch_input_grad(m, a);
}

extern "C" hpac_status hpac_mlp_vjp(hpac_mlp *m, int64_t n, const void *d_in, int64_t in_stride,
                                    double param, const float *d_gout, float *d_grad_params,
                                    float *d_grad_in) {
  TraceRange trace_("hpac_mlp_vjp");
  hpac_status s = check_io(m, n, d_in, in_stride);
  if (s != HPAC_OK) return s;
  if (n > 0 && !d_gout) return set_error(HPAC_EINVAL, "upstream gradient is NULL");
  if (d_grad_params) {
    HPAC_CUDA_TRY(cudaMemsetAsync(d_grad_params, 0, sizeof(float) * m->n_params, m->stream));
    if (n > 0) {
      MlpArgs a{};
      a.in = d_in, a.stride = in_stride, a.n = n, a.param = param, a.gout = d_gout;
      a.params = m->params;
      a.grad = d_grad_params;
      a.counters = m->counters;
      s = launch_grad(m, a);
      if (s != HPAC_OK) return s;
    }
  }
  if (d_grad_in && n > 0) {
    MlpArgs a{};
    a.in = d_in, a.stride = in_stride, a.n = n, a.param = param, a.out = d_grad_in, a.gout = d_gout;
    a.params = m->params;
    a.counters = m->counters;
    s = launch_input_grad(m, a);
    if (s != HPAC_OK) return s;
  }
  return HPAC_OK;
}

extern "C" hpac_status hpac_mlp_set_params_device(hpac_mlp *m, const float *d_params) {
  if (!m || !d_params) return set_error(HPAC_EINVAL, "NULL argument");
  HPAC_CUDA_TRY(cudaMemcpyAsync(m->params, d_params, sizeof(float) * m->n_params,
                                cudaMemcpyDeviceToDevice, m->stream));
  return HPAC_OK;
}

extern "C" hpac_status hpac_mlp_fit_normalization(hpac_mlp *m, int64_t n, const void *d_in,
                                                  int64_t in_stride, double param,
                                                  const float *d_target) {
  hpac_status s = check_io(m, n, d_in, in_stride);
  if (s != HPAC_OK) return s;
  if (n < 2 || !d_target) return set_error(HPAC_EINVAL, "need at least 2 samples and targets");
  double *acc = nullptr;
  HPAC_CUDA_TRY(cudaMalloc(&acc, 18 * sizeof(double)));
  cudaError_t e = cudaMemsetAsync(acc, 0, 18 * sizeof(double), m->stream);
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device);
  int64_t blocks = (n + 255) / 256;
  if (blocks > (int64_t)sms * 4) blocks = (int64_t)sms * 4;
  if (e == cudaSuccess) {
    if (m->d.kind == HPAC_REGION_BLACKSCHOLES)
      moments_kernel<HPAC_REGION_BLACKSCHOLES><<<(unsigned)blocks, 256, 0, m->stream>>>(
          d_in, in_stride, n, param, d_target, m->d, acc);
    else
      moments_kernel<HPAC_REGION_EOS><<<(unsigned)blocks, 256, 0, m->stream>>>(
          d_in, in_stride, n, param, d_target, m->d, acc);
    e = cudaGetLastError();
  }
  double h[18];
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  cudaFree(acc);
  if (e != cudaSuccess) return cuda_error(e, "hpac_mlp_fit_normalization");
  for (int k = 0; k < m->d.n_feat; ++k) {
    const double mu = h[k] / n, var = h[8 + k] / n - mu * mu;
    m->d.feat_shift[k] = (float)mu;
    m->d.feat_scale[k] = var > 0 ? (float)(1.0 / sqrt(var)) : 1.f;
  }
  const double nt = h[7] > 0 ? h[7] : 1.0;
  const double mu = h[16] / nt, var = h[17] / nt - mu * mu;
  m->d.out_shift = (float)mu;
  m->d.out_scale = var > 0 ? (float)sqrt(var) : 1.f;
  return HPAC_OK;
}

extern "C" hpac_status hpac_mlp_get_desc(const hpac_mlp *m, hpac_mlp_desc *out) {
  if (!m || !out) return set_error(HPAC_EINVAL, "NULL argument");
  *out = m->d;
  return HPAC_OK;
}
