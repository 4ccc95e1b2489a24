// conv.cu - launches of the separable pair sum as an FFT self-convolution
// (kernels in conv.cuh), one instantiation per padded length.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "conv.cuh"
#include "srm3_internal.cuh"

namespace srm3 {
namespace {

int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

// f(std::integral_constant<int, l>) for the l in [L0, L1] equal to v.
template <int L0, int L1, class F>
void with_log2(int v, F &&f) {
  if constexpr (L0 <= L1) {
    if (v == L0)
      f(std::integral_constant<int, L0>{});
    else
      with_log2<L0 + 1, L1>(v, f);
  }
}

// The pair sum of n samples (y / y0 laid out for sspad_for(n)) on stream
// st, into C_out.  Shapes: the row passes as the output transform's rows
// (64-thread CTAs), the column pass TC columns per CTA (at most 16, at most
// 512 threads, both buffers within 96 KB), column stride chosen so that the
// TC columns of one access fall on distinct banks.
template <typename T>
int conv_pairsum_impl(srm3_plan *p, cudaStream_t st, int n, const void *y, const void *y0,
                      void *C_out) {
  using T2 = typename Vec2<T>::type;
  const int SS = 2 * n, sp = sspad_for(n);
  if (SS > p->zc_ss) return fail(SRM3_ERR_INVALID_ARG, "separable pair sum: workspace too small");
  constexpr bool f32 = std::is_same<T, float>::value;
  const T *e = f32 ? (const T *)p->env_e32 : (const T *)p->env_e;
  const T *eb = f32 ? (const T *)p->env_b32 : (const T *)p->env_b;
  const T2 *twk = (const T2 *)p->tw_conv, *tww = twk + tx_twlen(p->log2cNk);
  T2 *Z = (T2 *)p->Zc;
  const int Nk = p->cNk, Nw = p->cNw, lk = p->log2cNk, lw = p->log2cNw;
  const size_t e2 = sizeof(T2);
  const int rb = conv_rows_per_cta(lw);
  const size_t srow = (size_t)rb * (tx_len(Nw) + 1) * e2;
  const int wf = (int)(128 / e2);  // lanes of one shared-memory wavefront
  auto colstride = [&](int tc) {
    const int len = (tx_len(Nk) + wf - 1) / wf * wf;
    return len + (tc >= wf ? 1 : wf / tc);
  };
  int TC = 16;
  while (TC > 1 && (TC > Nw || 2 * (size_t)TC * colstride(TC) * e2 > 96 * 1024 ||
                    TC * tx_tpt(Nk) > 512))
    TC >>= 1;
  const int cs = colstride(TC);
  const size_t scol = 2 * (size_t)TC * cs * e2;
  if (srow > 200 * 1024 || scol > 200 * 1024)
    return fail(SRM3_ERR_NOT_SUPPORTED,
                "separable pair sum: a padded row or column does not fit in shared memory");
  const int lim = 200 * 1024;
  const T cb = (T)std::cos(p->beta), sb = (T)std::sin(p->beta);
  cudaError_t err = cudaSuccess;
  with_log2<1, 13>(lw, [&](auto c) {
    constexpr int L = decltype(c)::value;
    err = cudaFuncSetAttribute(k_conv_rows<L, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               lim);
    if (err == cudaSuccess) {
      k_conv_rows<L, T><<<dim3(cdiv(p->nk, rb), SS), rb * tx_tpt(1 << L), srow, st>>>(
          p->nk, p->nw, sp, p->rowstride, y, e, tww, Z);
      err = cudaGetLastError();
    }
  });
  if (err != cudaSuccess) return cuda_fail(err, "separable pair sum, rows");
  with_log2<1, 13>(lk, [&](auto c) {
    constexpr int L = decltype(c)::value;
    err = cudaFuncSetAttribute(k_conv_cols<L, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               lim);
    if (err == cudaSuccess) {
      k_conv_cols<L, T><<<dim3(Nw / TC, SS), TC * tx_tpt(1 << L), scol, st>>>(p->nk, Nw, TC, cs,
                                                                              twk, Z);
      err = cudaGetLastError();
    }
  });
  if (err != cudaSuccess) return cuda_fail(err, "separable pair sum, columns");
  with_log2<1, 13>(lw, [&](auto c) {
    constexpr int L = decltype(c)::value;
    err = cudaFuncSetAttribute(k_conv_out<L, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               lim);
    if (err == cudaSuccess) {
      k_conv_out<L, T><<<dim3(cdiv(p->nk, rb), SS), rb * tx_tpt(1 << L), srow, st>>>(
          p->nk, p->nw, Nk, sp, p->rowstride, y, (const T2 *)y0, e, eb, (const T *)p->Pk,
          (const T *)p->ck, cb, sb, tww, Z, (T2 *)C_out);
      err = cudaGetLastError();
    }
  });
  if (err != cudaSuccess) return cuda_fail(err, "separable pair sum, output rows");
  return SRM3_OK;
}

}  // namespace

int conv_pairsum_on(srm3_plan *p, cudaStream_t st, int n, const void *y, const void *y0,
                    void *C_out) {
  return p->precision == SRM3_FP32 ? conv_pairsum_impl<float>(p, st, n, y, y0, C_out)
                                   : conv_pairsum_impl<double>(p, st, n, y, y0, C_out);
}

}  // namespace srm3
