// stats.cu - ensemble statistics of sampled fields on the device: the sample
// mean, variance, skewness and kurtosis, and the empirical PDF / CDF by
// histogram, as used to check simulated waves against their target moments
// (Sec. 6, the statistics of the bridge wind field).
//
// One pass over the values per call, HBM-bound: every CTA of a fixed grid
// walks 16-byte vectors in a grid-stride loop, four vectors per thread per
// step.  Power sums of d = u - shift go to FP64 per thread; FP32 input is
// summed in FP32 over the 16 values of a step first (one FP64 add per power
// per step: the FP64 pipe of this part is far narrower than its FP32 pipe),
// FP64 input in FP64 throughout.  Bins are b = floor((u - lo) * (nbins /
// (hi - lo))) in the input's precision, each operation rounded once; b < 0
// counts below, b >= nbins (or a NaN) above, as two extra slots of the
// shared histogram, so that every value costs one shared atomic and no
// branch.  Per-CTA shared histograms merge into the global one with integer
// atomics; the per-CTA power sums go to a partials array, added in a fixed
// order of runs.  The same values given in the same calls yield
// bit-identical results.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "srm3.h"
#include "srm3_internal.cuh"

struct srm3_stats {
  int nbins = 0;
  double lo = 0.0, hi = 1.0, shift = 0.0;
  int grid = 0;
  double count = 0.0;
  double *acc = nullptr;                 // [4] running power sums
  double *part = nullptr;                // [grid][4] per-CTA sums of one call
  unsigned long long *hist = nullptr;    // [nbins + 2]: bins, below, above
};

namespace srm3 {
namespace {

constexpr int kStatThreads = 256;
constexpr int kStatVec = 4;  // vectors per thread per step

template <typename T>
struct StatVec;
template <>
struct StatVec<float> {
  using V = float4;
  static constexpr int N = 4;
  static __device__ __forceinline__ float at(const float4 &v, int i) {
    return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
  }
};
template <>
struct StatVec<double> {
  using V = double2;
  static constexpr int N = 2;
  static __device__ __forceinline__ double at(const double2 &v, int i) { return i == 0 ? v.x : v.y; }
};

// The shared-histogram slot of a value: its bin, nbins for below lo,
// nbins + 1 at or above hi or for a NaN.
template <typename T>
__device__ __forceinline__ int stat_slot(T u, T lo, T scale, int nbins) {
  T t;
  if constexpr (sizeof(T) == sizeof(float))
    t = __fmul_rn(__fsub_rn(u, lo), scale);
  else
    t = __dmul_rn(__dsub_rn(u, lo), scale);
  return t < (T)0 ? nbins : (t < (T)nbins ? (int)t : nbins + 1);
}

// One value into the running FP32 (or FP64) power sums and the histogram.
template <typename T>
__device__ __forceinline__ void stat_one(T val, T sh, T lo, T scale, int nbins,
                                         unsigned int *hist, T &s1, T &s2, T &s3, T &s4) {
  const T d = val - sh, d2 = d * d;
  s1 += d;
  s2 += d2;
  s3 = fma(d2, d, s3);
  s4 = fma(d2, d2, s4);
  atomicAdd(hist + stat_slot<T>(val, lo, scale, nbins), 1u);
}

template <typename T>
__global__ void __launch_bounds__(kStatThreads) k_stats(const T *__restrict__ u, long long count,
                                                        T lo, T scale, int nbins, double shift,
                                                        double *__restrict__ part,
                                                        unsigned long long *__restrict__ hist) {
  using SV = StatVec<T>;
  using V = typename SV::V;
  extern __shared__ unsigned int sh_hist[];  // nbins + 2 slots
  __shared__ double sh_sum[kStatThreads / 32][4];
  for (int b = threadIdx.x; b < nbins + 2; b += blockDim.x) sh_hist[b] = 0;
  __syncthreads();
  const long long nv = count / SV::N;
  const long long nth = (long long)gridDim.x * blockDim.x;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const V *uv = reinterpret_cast<const V *>(u);
  const T sh = (T)shift;
  double a1 = 0.0, a2 = 0.0, a3 = 0.0, a4 = 0.0;
  // steps whose kStatVec vectors all exist, without per-value checks
  const long long full = nv / (nth * kStatVec) * (nth * kStatVec);
  for (long long v0 = tid; v0 < full; v0 += nth * kStatVec) {
    V x[kStatVec];
#pragma unroll
    for (int j = 0; j < kStatVec; ++j) x[j] = __ldcs(uv + v0 + (long long)j * nth);
    T s1 = 0, s2 = 0, s3 = 0, s4 = 0;
#pragma unroll
    for (int j = 0; j < kStatVec; ++j)
#pragma unroll
      for (int i = 0; i < SV::N; ++i)
        stat_one<T>(SV::at(x[j], i), sh, lo, scale, nbins, sh_hist, s1, s2, s3, s4);
    a1 += (double)s1;
    a2 += (double)s2;
    a3 += (double)s3;
    a4 += (double)s4;
  }
  // the last partial step: one vector at a time
  for (long long v = full + tid; v < nv; v += nth) {
    const V x = __ldcs(uv + v);
    T s1 = 0, s2 = 0, s3 = 0, s4 = 0;
#pragma unroll
    for (int i = 0; i < SV::N; ++i)
      stat_one<T>(SV::at(x, i), sh, lo, scale, nbins, sh_hist, s1, s2, s3, s4);
    a1 += (double)s1;
    a2 += (double)s2;
    a3 += (double)s3;
    a4 += (double)s4;
  }
  // the count % N trailing values: block 0, thread 0, in index order
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (long long e = nv * SV::N; e < count; ++e) {
      T s1 = 0, s2 = 0, s3 = 0, s4 = 0;
      stat_one<T>(u[e], sh, lo, scale, nbins, sh_hist, s1, s2, s3, s4);
      a1 += (double)s1;
      a2 += (double)s2;
      a3 += (double)s3;
      a4 += (double)s4;
    }
  }
  // CTA reduction in a fixed order: butterflies within warps, then warps in order
  double a[4] = {a1, a2, a3, a4};
#pragma unroll
  for (int p = 0; p < 4; ++p)
    for (int o = 16; o > 0; o >>= 1) a[p] += __shfl_xor_sync(0xffffffffu, a[p], o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
#pragma unroll
    for (int p = 0; p < 4; ++p) sh_sum[warp][p] = a[p];
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double s = 0.0;
    for (int w = 0; w < kStatThreads / 32; ++w) s += sh_sum[w][threadIdx.x];
    part[(size_t)blockIdx.x * 4 + threadIdx.x] = s;
  }
  for (int b = threadIdx.x; b < nbins + 2; b += blockDim.x)
    if (sh_hist[b]) atomicAdd(hist + b, (unsigned long long)sh_hist[b]);
}

// acc[p] += sum over CTAs in a fixed order: thread t sums power t & 3 over
// the t >> 2-th contiguous run of CTAs, then thread p < 4 adds the runs in
// order.
constexpr int kMergeThreads = 256;
__global__ void __launch_bounds__(kMergeThreads) k_stats_merge(const double *__restrict__ part,
                                                               int grid, double *__restrict__ acc) {
  __shared__ double run[kMergeThreads];
  const int t = threadIdx.x, p = t & 3, r = t >> 2, nr = kMergeThreads / 4;
  const int per = (grid + nr - 1) / nr, c0 = r * per, c1 = min(grid, c0 + per);
  double s = 0.0;
  for (int c = c0; c < c1; ++c) s += part[(size_t)c * 4 + p];
  run[t] = s;
  __syncthreads();
  if (t < 4) {
    double tot = 0.0;
    for (int q = 0; q < nr; ++q) tot += run[4 * q + t];
    acc[t] += tot;
  }
}

}  // namespace
}  // namespace srm3

using namespace srm3;

SRM3_API int srm3_stats_create(int32_t nbins, double lo, double hi, double shift,
                               srm3_stats **out) {
  if (!out) return fail(SRM3_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (nbins < 1 || nbins > SRM3_STATS_MAX_BINS)
    return fail(SRM3_ERR_INVALID_ARG, "nbins must be in [1, SRM3_STATS_MAX_BINS]");
  if (!(hi > lo) || !std::isfinite(lo) || !std::isfinite(hi) || !std::isfinite(shift))
    return fail(SRM3_ERR_INVALID_ARG, "need finite lo < hi and a finite shift");
  int dev = 0, nsm = 0;
  SRM3_CUDA(cudaGetDevice(&dev));
  SRM3_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  srm3_stats *s = new srm3_stats;
  s->nbins = nbins;
  s->lo = lo;
  s->hi = hi;
  s->shift = shift;
  s->grid = 4 * nsm;
  cudaError_t e = cudaMalloc(&s->acc, 4 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&s->part, (size_t)s->grid * 4 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&s->hist, (size_t)(nbins + 2) * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(s->acc, 0, 4 * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(s->hist, 0, (size_t)(nbins + 2) * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    srm3_stats_destroy(s);
    return cuda_fail(e, "srm3_stats_create");
  }
  *out = s;
  return SRM3_OK;
}

SRM3_API int srm3_stats_add(srm3_stats *s, const void *u, int32_t precision, int64_t count,
                            void *stream) {
  if (!s) return fail(SRM3_ERR_INVALID_ARG, "stats is NULL");
  if (count < 0) return fail(SRM3_ERR_INVALID_ARG, "count must be >= 0");
  if (count == 0) return SRM3_OK;
  if (!u) return fail(SRM3_ERR_INVALID_ARG, "u is NULL");
  if (precision != SRM3_FP32 && precision != SRM3_FP64)
    return fail(SRM3_ERR_INVALID_ARG, "precision must be SRM3_FP32 or SRM3_FP64");
  if (reinterpret_cast<uintptr_t>(u) % 16)
    return fail(SRM3_ERR_INVALID_ARG, "u must be 16-byte aligned");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t smem = ((size_t)s->nbins + 2) * sizeof(unsigned int);
  const double scale = (double)s->nbins / (s->hi - s->lo);
  if (precision == SRM3_FP32) {
    SRM3_CUDA(cudaFuncSetAttribute(k_stats<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
    k_stats<float><<<s->grid, kStatThreads, smem, st>>>(
        static_cast<const float *>(u), count, (float)s->lo, (float)scale, s->nbins, s->shift,
        s->part, s->hist);
  } else {
    SRM3_CUDA(cudaFuncSetAttribute(k_stats<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
    k_stats<double><<<s->grid, kStatThreads, smem, st>>>(
        static_cast<const double *>(u), count, s->lo, scale, s->nbins, s->shift, s->part,
        s->hist);
  }
  SRM3_CUDA(cudaGetLastError());
  k_stats_merge<<<1, kMergeThreads, 0, st>>>(s->part, s->grid, s->acc);
  SRM3_CUDA(cudaGetLastError());
  s->count += (double)count;
  return SRM3_OK;
}

SRM3_API int srm3_stats_read(srm3_stats *s, void *stream, srm3_stats_result *r, uint64_t *hist) {
  if (!s || !r) return fail(SRM3_ERR_INVALID_ARG, "stats and result must be non-NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double acc[4];
  std::vector<unsigned long long> h((size_t)s->nbins + 2);
  SRM3_CUDA(cudaMemcpyAsync(acc, s->acc, sizeof(acc), cudaMemcpyDeviceToHost, st));
  SRM3_CUDA(cudaMemcpyAsync(h.data(), s->hist, h.size() * sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, st));
  SRM3_CUDA(cudaStreamSynchronize(st));
  std::memset(r, 0, sizeof(*r));
  const double n = s->count;
  r->count = n;
  for (int p = 0; p < 4; ++p) r->power_sum[p] = acc[p];
  r->below = h[s->nbins];
  r->above = h[s->nbins + 1];
  if (hist) std::memcpy(hist, h.data(), (size_t)s->nbins * sizeof(uint64_t));
  if (n > 0) {
    // central moments about the mean from the moments about the shift
    const double m1 = acc[0] / n, e2 = acc[1] / n, e3 = acc[2] / n, e4 = acc[3] / n;
    const double c2 = e2 - m1 * m1;
    const double c3 = e3 - 3.0 * m1 * e2 + 2.0 * m1 * m1 * m1;
    const double c4 = e4 - 4.0 * m1 * e3 + 6.0 * m1 * m1 * e2 - 3.0 * m1 * m1 * m1 * m1;
    r->mean = s->shift + m1;
    r->variance = c2;
    r->skewness = c2 > 0 ? c3 / (c2 * std::sqrt(c2)) : 0.0;
    r->kurtosis = c2 > 0 ? c4 / (c2 * c2) : 0.0;
  }
  return SRM3_OK;
}

SRM3_API int srm3_stats_reset(srm3_stats *s, void *stream) {
  if (!s) return fail(SRM3_ERR_INVALID_ARG, "stats is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  SRM3_CUDA(cudaMemsetAsync(s->acc, 0, 4 * sizeof(double), st));
  SRM3_CUDA(cudaMemsetAsync(s->hist, 0, ((size_t)s->nbins + 2) * sizeof(unsigned long long), st));
  s->count = 0.0;
  return SRM3_OK;
}

SRM3_API void srm3_stats_destroy(srm3_stats *s) {
  if (!s) return;
  if (s->acc) cudaFree(s->acc);
  if (s->part) cudaFree(s->part);
  if (s->hist) cudaFree(s->hist);
  delete s;
}
