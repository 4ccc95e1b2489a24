// transform.cu - launches of the output transform (a6, FFT form, Sec. 4.3):
// the x stage over the coefficient columns and the half-length
// complex-to-real t stage (kernels in fft.cuh), one instantiation per
// transform length.
#include <algorithm>
#include <type_traits>

#include "fft.cuh"
#include "srm3_internal.cuh"

namespace srm3 {
namespace {

int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

// Launch shape of the two stages.  Stage 1: TC columns per CTA (at most 16,
// at most the power of two >= nw), column stride in shared memory chosen so
// that the TC columns of one access fall on distinct banks; stage 2: rows
// per CTA up to 64 threads (small CTAs: a row's passes wait at their own
// barriers only; 1, 2, 4 and 8 rows of 1024 measured 201, 219, 237 and
// 269 us on the 1024 x 2048 field).  Both within 72 KB of shared memory
// where one column or row allows it.
struct TxShape {
  int TC, colstride, rb, rowstride;
  size_t smem1, smem2;
};

TxShape tx_shape(const srm3_plan *p, size_t e2) {
  const size_t cap = 72 * 1024;
  const int wf = (int)(128 / e2);  // lanes of one shared-memory wavefront
  TxShape s{};
  const int L = p->nx, M = p->nt / 2;
  int TC = 16;
  while (TC > 1 && TC / 2 >= p->nw) TC >>= 1;
  auto colstride = [&](int tc) {
    const int len = (tx_len(L) + wf - 1) / wf * wf;
    return len + (tc >= wf ? 1 : wf / tc);
  };
  while (TC > 1 && ((size_t)TC * colstride(TC) * e2 > cap || TC * tx_tpt(L) > 512)) TC >>= 1;
  s.TC = TC;
  s.colstride = colstride(TC);
  s.smem1 = (size_t)TC * s.colstride * e2;
  s.rowstride = tx_len(M) + 1;
  int rb = std::max(1, 64 / tx_tpt(M));
  while (rb > 1 && ((size_t)rb * s.rowstride * e2 > cap || rb > p->nx)) rb >>= 1;
  s.rb = rb;
  s.smem2 = (size_t)rb * s.rowstride * e2;
  return s;
}

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

// Nonzero input blocks of a stage's first pass (tx_in_mask): a length-2^l
// transform whose inputs vanish except at the n indices of each end of the
// spectrum (kk < nk or nx - kk < nk in x; m < nw or M - m < nw in t).  The
// smallest of 1, 2, 4 blocks (of 2^l / R each, R the first radix) that
// covers them, else 0 (all).  Pruned passes are compiled for FP32 and
// transforms of 64 points or more.
int tx_nz(int l, int n, bool fp32) {
  if (!fp32 || l < 6) return 0;
  const int R = 1 << tx_lr(l, 0), LR = (1 << l) / R;
  for (int nz = 1; nz <= 4 && 2 * nz < R; nz *= 2)
    if ((long long)nz * LR >= n) return nz;
  return 0;
}

// f(integral_constant NZ) for NZ in {0, 1, 2, 4} equal to nz (0 alone when
// the pruned forms are not compiled for this type and length).
template <bool PRUNE, class F>
void with_nz(int nz, F &&f) {
  if constexpr (PRUNE) {
    if (nz == 1) return f(std::integral_constant<int, 1>{});
    if (nz == 2) return f(std::integral_constant<int, 2>{});
    if (nz == 4) return f(std::integral_constant<int, 4>{});
  }
  f(std::integral_constant<int, 0>{});
}

template <typename T, typename T2>
int transform_impl(srm3_plan *p, cudaStream_t st, const T2 *C, int n, T *out, T2 *G) {
  const TxShape s = tx_shape(p, sizeof(T2));
  const int lim = 200 * 1024;
  const T2 *tw1 = (const T2 *)p->tw, *tw2 = tw1 + tx_twlen(p->log2nx);
  const T2 *twz = tw2 + tx_twlen(p->log2nt - 1);
  cudaError_t e = cudaSuccess;
  constexpr bool f32 = std::is_same<T, float>::value;
  with_log2<1, 13>(p->log2nx, [&](auto c) {
    constexpr int l = decltype(c)::value;
    with_nz<f32 && l >= 6>(tx_nz(l, p->nk, f32), [&](auto z) {
      constexpr int nz = decltype(z)::value;
      e = cudaFuncSetAttribute(k_tx_cols<l, T2, nz>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               lim);
      if (e == cudaSuccess) {
        k_tx_cols<l, T2, nz><<<dim3(cdiv(p->nw, s.TC), n), s.TC * tx_tpt(1 << l), s.smem1, st>>>(
            p->nk, p->nw, s.TC, s.colstride, C, tw1, G);
        e = cudaGetLastError();
      }
    });
  });
  if (e != cudaSuccess) return cuda_fail(e, "output transform, x stage");
  with_log2<0, 12>(p->log2nt - 1, [&](auto c) {
    constexpr int l = decltype(c)::value;
    with_nz<f32 && l >= 6>(tx_nz(l, p->nw, f32), [&](auto z) {
      constexpr int nz = decltype(z)::value;
      e = cudaFuncSetAttribute(k_tx_rows<l, T, T2, nz>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
      if (e == cudaSuccess) {
        k_tx_rows<l, T, T2, nz><<<dim3(p->nx / s.rb, n), s.rb * tx_tpt(1 << l), s.smem2, st>>>(
            p->nx, p->nw, s.rowstride, G, tw2, twz, out);
        e = cudaGetLastError();
      }
    });
  });
  if (e != cudaSuccess) return cuda_fail(e, "output transform, t stage");
  return SRM3_OK;
}

}  // namespace

// The transform of n coefficient sets with the x-stage columns in H
// (n * transform_elems(p) complex), on stream st.
int transform_on(srm3_plan *p, cudaStream_t st, const void *C, int n, void *out, void *H) {
  if (p->log2nx < 1 || p->log2nx > 13 || p->log2nt < 1 || p->log2nt > 13)
    return fail(SRM3_ERR_GRID_CONSTRAINT, "output transform: n_x, n_t outside [2, 8192]");
  if (p->precision == SRM3_FP32)
    return transform_impl<float, float2>(p, st, (const float2 *)C, n, (float *)out,
                                         (float2 *)H);
  return transform_impl<double, double2>(p, st, (const double2 *)C, n, (double *)out,
                                         (double2 *)H);
}

}  // namespace srm3
