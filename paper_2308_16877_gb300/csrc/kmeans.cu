// K-Means centroid update, the exact step between two (approximated)
// assignments (Table 1, K-Means: iterate until no observation changes
// cluster). One pass over the observations accumulates the per-cluster
// feature sums (double) and counts in shared memory: one column per thread up
// to 32 clusters, one copy per warp beyond; each block adds its columns or
// copies and then the workspace with one atomic per value; a second tiny
// kernel divides. Changed assignments are counted in the same pass.
#include "hpac_internal.cuh"

namespace hpac {
namespace {

constexpr int kThreads = 256;

// Each warp accumulates into its own copy of the per-cluster sums, so the
// shared-memory double-precision atomics of one instruction collide only among
// lanes of the same warp and cluster; the copies are then added once per block.
constexpr int kWarps = kThreads / 32;

__global__ void __launch_bounds__(kThreads) kmeans_sums(const float *__restrict__ x, int64_t stride,
                                                        int64_t n, int K,
                                                        const float *__restrict__ assign,
                                                        const float *__restrict__ prev,
                                                        double *__restrict__ sum,
                                                        unsigned long long *__restrict__ cnt,
                                                        unsigned long long *__restrict__ changed) {
  __shared__ double s_sum[kWarps][kMaxClusters * 8];
  __shared__ unsigned s_cnt[kWarps][kMaxClusters];
  const int warp = threadIdx.x >> 5;
  for (int j = threadIdx.x; j < kWarps * K * 8; j += blockDim.x) s_sum[j / (K * 8)][j % (K * 8)] = 0.0;
  for (int j = threadIdx.x; j < kWarps * K; j += blockDim.x) s_cnt[j / K][j % K] = 0;
  __syncthreads();
  double *ws = s_sum[warp];
  unsigned *wc = s_cnt[warp];
  unsigned ch = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float a = assign[i];
    const int k = (int)a;
    if (k >= 0 && k < K) {  // ids are produced in range; anything else is left out
      atomicAdd(&wc[k], 1u);
#pragma unroll
      for (int d = 0; d < 8; ++d) atomicAdd(&ws[k * 8 + d], (double)x[d * stride + i]);
    }
    if (prev && prev[i] != a) ++ch;
  }
  ch = __reduce_add_sync(0xffffffffu, ch);
  if ((threadIdx.x & 31) == 0 && ch) atomicAdd(changed, (unsigned long long)ch);
  __syncthreads();
  for (int j = threadIdx.x; j < K * 8; j += blockDim.x) {
    double v = 0.0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) v += s_sum[w][j];
    if (v != 0.0) atomicAdd(&sum[j], v);
  }
  for (int j = threadIdx.x; j < K; j += blockDim.x) {
    unsigned long long c = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) c += s_cnt[w][j];
    if (c) atomicAdd(&cnt[j], c);
  }
}

// For up to 32 clusters: every thread keeps its own column of per-cluster
// sums and counts in shared memory ([cluster * 8 + d][thread], conflict-free),
// so the pass needs no atomics; the block then adds its columns (each thread
// starting at its own column, so the reads spread over the banks) and the
// workspace gets one atomic per value.
template <int L>
__global__ void __launch_bounds__(L) kmeans_sums_private(const float *__restrict__ x, int64_t stride,
                                                         int64_t n, int K,
                                                         const float *__restrict__ assign,
                                                         const float *__restrict__ prev,
                                                         double *__restrict__ sum,
                                                         unsigned long long *__restrict__ cnt,
                                                         unsigned long long *__restrict__ changed) {
  extern __shared__ __align__(16) double s_acc[];             // [K * 8][L]
  unsigned *s_n = reinterpret_cast<unsigned *>(s_acc + K * 8 * L);  // [K][L]
  const int tid = threadIdx.x;
  for (int j = 0; j < K * 8; ++j) s_acc[j * L + tid] = 0.0;
  for (int j = 0; j < K; ++j) s_n[j * L + tid] = 0;
  unsigned ch = 0;
  // the next observation's id and features are loaded before this one's
  // additions, so each thread keeps two observations' loads in flight (the
  // columns leave room for few threads per SM)
  const int64_t step = (int64_t)gridDim.x * L;
  int64_t i = (int64_t)blockIdx.x * L + tid;
  float a = 0.0f, pa = 0.0f, xv[8];
  if (i < n) {
    a = assign[i];
    if (prev) pa = prev[i];
#pragma unroll
    for (int d = 0; d < 8; ++d) xv[d] = x[d * stride + i];
  }
  while (i < n) {
    const int64_t nx = i + step;
    float an = 0.0f, pn = 0.0f, xn[8];
    if (nx < n) {
      an = assign[nx];
      if (prev) pn = prev[nx];
#pragma unroll
      for (int d = 0; d < 8; ++d) xn[d] = x[d * stride + nx];
    }
    const int k = (int)a;
    if (k >= 0 && k < K) {  // ids are produced in range; anything else is left out
      s_n[k * L + tid] += 1;
      double *col = s_acc + (size_t)k * 8 * L + tid;
#pragma unroll
      for (int d = 0; d < 8; ++d) col[d * L] += (double)xv[d];
    }
    if (prev && pa != a) ++ch;
    a = an;
    pa = pn;
#pragma unroll
    for (int d = 0; d < 8; ++d) xv[d] = xn[d];
    i = nx;
  }
  ch = __reduce_add_sync(0xffffffffu, ch);
  if ((tid & 31) == 0 && ch) atomicAdd(changed, (unsigned long long)ch);
  __syncthreads();
  for (int j = tid; j < K * 8; j += L) {
    double v = 0.0;
    for (int l = 0; l < L; ++l) v += s_acc[j * L + ((l + tid) & (L - 1))];
    if (v != 0.0) atomicAdd(&sum[j], v);
  }
  for (int j = tid; j < K; j += L) {
    unsigned long long c = 0;
    for (int l = 0; l < L; ++l) c += s_n[j * L + ((l + tid) & (L - 1))];
    if (c) atomicAdd(&cnt[j], c);
  }
}

__global__ void kmeans_divide(int K, const double *__restrict__ sum,
                              const unsigned long long *__restrict__ cnt, float *__restrict__ cent) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= K * 8) return;
  const unsigned long long c = cnt[j / 8];
  if (c) cent[j] = (float)(sum[j] / (double)c);  // an empty cluster keeps its centroid
}

}  // namespace
}  // namespace hpac

using namespace hpac;

extern "C" size_t hpac_kmeans_workspace_bytes(int32_t clusters) {
  if (clusters < 1 || clusters > kMaxClusters) return 0;
  return (size_t)(clusters * 8 + clusters + 1) * 8;
}

extern "C" hpac_status hpac_kmeans_update(int64_t n, int32_t clusters, const float *d_x,
                                          int64_t stride, const float *d_assign,
                                          const float *d_prev, float *d_cent, void *d_work,
                                          int64_t *h_changed, void *cuda_stream) {
  TraceRange trace_("hpac_kmeans_update");
  if (n < 0 || clusters < 1 || clusters > kMaxClusters || stride < n)
    return set_error(HPAC_EINVAL, "K-Means update: bad n, clusters or stride");
  if (!d_cent || !d_work || (n > 0 && (!d_x || !d_assign)))
    return set_error(HPAC_EINVAL, "K-Means update: NULL pointer");
  if ((uintptr_t)d_work % 8) return set_error(HPAC_EINVAL, "workspace not 8-byte aligned");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  double *sum = static_cast<double *>(d_work);
  unsigned long long *cnt = reinterpret_cast<unsigned long long *>(sum + clusters * 8);
  unsigned long long *changed = cnt + clusters;
  HPAC_CUDA_TRY(cudaMemsetAsync(d_work, 0, hpac_kmeans_workspace_bytes(clusters), s));
  int dev = 0, sms = 148;
  HPAC_CUDA_TRY(cudaGetDevice(&dev));
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (clusters <= 32) {
    // thread-private columns: 64 threads per block up to 16 clusters, 32 up to 32
    const int L = clusters <= 16 ? 64 : 32;
    const size_t smem = (size_t)clusters * 8 * L * sizeof(double) + (size_t)clusters * L * sizeof(unsigned);
    auto fn = L == 64 ? kmeans_sums_private<64> : kmeans_sums_private<32>;
    HPAC_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 1;
    HPAC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, L, smem));
    int64_t blocks = (n + L - 1) / L;
    const int64_t cap = (int64_t)sms * (per_sm < 1 ? 1 : per_sm);
    blocks = blocks < 1 ? 1 : blocks > cap ? cap : blocks;
    fn<<<(unsigned)blocks, L, smem, s>>>(d_x, stride, n, clusters, d_assign, d_prev, sum, cnt, changed);
  } else {
    int64_t blocks = (n + kThreads - 1) / kThreads;
    const int64_t cap = (int64_t)sms * 4;
    blocks = blocks < 1 ? 1 : blocks > cap ? cap : blocks;
    kmeans_sums<<<(unsigned)blocks, kThreads, 0, s>>>(d_x, stride, n, clusters, d_assign, d_prev, sum,
                                                        cnt, changed);
  }
  HPAC_CUDA_TRY(cudaGetLastError());
  kmeans_divide<<<(clusters * 8 + 255) / 256, 256, 0, s>>>(clusters, sum, cnt, d_cent);
  HPAC_CUDA_TRY(cudaGetLastError());
  if (h_changed) {
    unsigned long long c = 0;
    HPAC_CUDA_TRY(cudaMemcpyAsync(&c, changed, sizeof(c), cudaMemcpyDeviceToHost, s));
    HPAC_CUDA_TRY(cudaStreamSynchronize(s));
    *h_changed = (int64_t)c;
  }
  return HPAC_OK;
}
