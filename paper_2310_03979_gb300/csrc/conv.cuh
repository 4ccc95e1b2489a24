// conv.cuh - the pair sum of a separable envelope as an FFT self-convolution
// (a4 + a5 for g(i,j) = a(i) a(j) b(i+j)).  Included by sample.cu after
// fft.cuh, whose register-resident Stockham passes it runs.
//
// With W_ij = c_k a_i a_j b_k the pair part of C_k is
//   c_k e^{i beta} b_k sum_{Pi(k)} z_i z_j,   z = a y  (z_0 = 0),
// and over unordered pairs {i, j}, i + j = k,
//   sum_{Pi(k)} z_i z_j = ((z * z)_k + [k even] z_{k/2}^2) / 2,
// with (z * z) the linear 2-D self-convolution on the quadrant lattice.  It
// is taken on a zero-padded Nk x Nw grid (powers of two, Nk >= 2 n_kappa - 1,
// Nw >= 2 n_omega - 1) with one transform direction only (here e^{+}, the
// direction of the output transform's passes):
//   G(G(z)^2)[m] = Nk Nw (z * z)[-m mod (Nk, Nw)],
// so the second transform is read back at negated indices.  Three passes
// per sheet-sample: rows of z (k_conv_rows), columns, square, columns again
// (k_conv_cols, which also negates the row index on its way out), rows and
// the coefficient epilogue (k_conv_out).  The inputs of the first row and
// column transforms are zero past n_omega, n_kappa <= half the length: their
// first passes skip the upper half of the blocks (tx_mask_low_half).  Rows
// of the grid at kk >= n_kappa are zero and never stored; only the n_kappa
// rows and n_omega columns the lattice needs are written back.
#pragma once

#include "fft.cuh"

namespace srm3 {
namespace {

// y of sheet-sample ss at lattice point (kk, kw), in the layout k_phases
// writes (FP32 pair-planar per sample pair, FP64 one complex per sheet-sample).
template <typename T>
__device__ __forceinline__ typename Vec2<T>::type conv_y(const void *y, int SSpad, int rowstride,
                                                         int kk, int kw, int ss) {
  const size_t row = (size_t)kk * rowstride + kPad + kw;
  if constexpr (sizeof(T) == sizeof(float)) {
    const float *yf = static_cast<const float *>(y) + (row * (SSpad / 2) + (ss >> 1)) * 4 + (ss & 1);
    return make_float2(yf[0], yf[2]);
  } else {
    return static_cast<const double2 *>(y)[row * SSpad + ss];
  }
}

// Rows per CTA of the row passes: 64-thread CTAs (tx_tpt(Nw) threads a row;
// one row of more than 64 threads for Nw > 1024).
__host__ __device__ constexpr int conv_rows_per_cta(int log2Nw) {
  return tx_tpt(1 << log2Nw) >= 64 ? 1 : 64 / tx_tpt(1 << log2Nw);
}

// Pass 1: z = a y along lattice row kk < n_kappa, zero-padded to Nw,
// transformed; rb rows of one sheet-sample per CTA (blockIdx.y = ss).
// Threads of rows past n_kappa take part in the passes' barriers only.
template <int LW, typename T>
__global__ void __launch_bounds__(512) k_conv_rows(int nk, int nw, int SSpad,
                                                  int rowstride, const void *__restrict__ y,
                                                  const T *__restrict__ e,
                                                  const typename Vec2<T>::type *__restrict__ tw,
                                                  typename Vec2<T>::type *__restrict__ Z) {
  using T2 = typename Vec2<T>::type;
  extern __shared__ __align__(16) unsigned char conv_smem[];
  constexpr int Nw = 1 << LW, tpt = tx_tpt(Nw), rb = conv_rows_per_cta(LW);
  const int row = threadIdx.x / tpt, jt = threadIdx.x & (tpt - 1), ss = blockIdx.y;
  const int kk = blockIdx.x * rb + row;
  const bool live = kk < nk;
  T2 *buf = reinterpret_cast<T2 *>(conv_smem) + row * (tx_len(Nw) + 1);
  T2 *out = Z + ((size_t)ss * nk + kk) * Nw;
  auto src = [&](int m) -> T2 {
    T2 v;
    v.x = 0;
    v.y = 0;
    if (live && m < nw) {
      const T2 yv = conv_y<T>(y, SSpad, rowstride, kk, m, ss);
      const T ev = e[(size_t)kk * nw + m];
      v.x = ev * yv.x;
      v.y = ev * yv.y;
    }
    return v;
  };
  auto dst = [&](int i, T2 v) {
    if (live) out[i] = v;
  };
  stockham_passes<LW, 0, tx_mask_low_half<LW>()>(1, 0, tpt, jt, tw, buf, src, dst);
}

// Pass 2: TC columns of one sheet-sample per CTA, thread (c, jt) = (t mod TC,
// t / TC): the column transformed along kappa (rows >= n_kappa zero),
// squared on its way out of the last pass into a second buffer, transformed
// again, and the n_kappa rows the lattice needs stored, row kk taking grid
// row (Nk - kk) mod Nk.  In place in Z ([ss][n_kappa][Nw]: the grid's rows
// past n_kappa are zero and not stored).  Shared memory: two buffers of
// colstride entries per column.
template <int LK, typename T>
__global__ void __launch_bounds__(512) k_conv_cols(int nk, int Nw, int TC, int colstride,
                                                   const typename Vec2<T>::type *__restrict__ tw,
                                                   typename Vec2<T>::type *__restrict__ Z) {
  using T2 = typename Vec2<T>::type;
  extern __shared__ __align__(16) unsigned char conv_smem[];
  constexpr int Nk = 1 << LK, tpt = tx_tpt(Nk);
  const int c = threadIdx.x & (TC - 1), jt = threadIdx.x / TC, ss = blockIdx.y;
  const int m = blockIdx.x * TC + c;
  T2 *colA = reinterpret_cast<T2 *>(conv_smem) + c * colstride;
  T2 *colB = reinterpret_cast<T2 *>(conv_smem) + (TC + c) * colstride;
  T2 *base = Z + (size_t)ss * nk * Nw + m;
  auto src1 = [&](int kk) -> T2 {
    T2 v;
    v.x = 0;
    v.y = 0;
    if (kk < nk) v = base[(size_t)kk * Nw];
    return v;
  };
  auto dst1 = [&](int i, T2 v) {  // the square, at the padded position of i
    T2 q;
    q.x = v.x * v.x - v.y * v.y;
    q.y = 2 * v.x * v.y;
    colB[sp16(i)] = q;
  };
  stockham_passes<LK, 0, tx_mask_low_half<LK>()>(1, 0, tpt, jt, tw, colA, src1, dst1);
  __syncthreads();
  auto src2 = [&](int i) -> T2 { return colB[sp16(i)]; };
  auto dst2 = [&](int i, T2 v) {
    const int kk = (Nk - i) & (Nk - 1);
    if (kk < nk) base[(size_t)kk * Nw] = v;
  };
  stockham_passes<LK, 0, 0u>(1, 0, tpt, jt, tw, colA, src2, dst2);
}

// Pass 3: lattice row kk of the twice-transformed grid, transformed along
// omega; the ordered self-convolution at (kk, kw) is its entry (Nw - kw) mod
// Nw over Nk Nw, taken straight from the last pass.  Epilogue as in the
// O(N^2) pair sums:
//   C_k = P_k y_k + c_k e^{i beta} b_k ((z * z)_k + [k even] z_{k/2}^2) / 2.
template <int LW, typename T>
__global__ void __launch_bounds__(512) k_conv_out(int nk, int nw, int Nk, int SSpad, int rowstride,
                                                 const void *__restrict__ y,
                                                 const typename Vec2<T>::type *__restrict__ y0,
                                                 const T *__restrict__ e, const T *__restrict__ eb,
                                                 const T *__restrict__ Pk,
                                                 const T *__restrict__ ck, T cb, T sb,
                                                 const typename Vec2<T>::type *__restrict__ tw,
                                                 const typename Vec2<T>::type *__restrict__ Z,
                                                 typename Vec2<T>::type *__restrict__ C) {
  using T2 = typename Vec2<T>::type;
  extern __shared__ __align__(16) unsigned char conv_smem[];
  constexpr int Nw = 1 << LW, tpt = tx_tpt(Nw), rb = conv_rows_per_cta(LW);
  const int row = threadIdx.x / tpt, jt = threadIdx.x & (tpt - 1), ss = blockIdx.y;
  const int kk = blockIdx.x * rb + row;
  const bool live = kk < nk;
  T2 *buf = reinterpret_cast<T2 *>(conv_smem) + row * (tx_len(Nw) + 1);
  const T2 *in = Z + ((size_t)ss * nk + (live ? kk : 0)) * Nw;
  const T inv = (T)1 / ((T)Nk * (T)Nw);
  auto src = [&](int i) -> T2 { return in[i]; };
  auto dst = [&](int i, T2 cv) {
    const int kw = (Nw - i) & (Nw - 1);
    if (!live || kw >= nw) return;
    T ar = cv.x * inv, ai = cv.y * inv;
    if ((kk & 1) == 0 && (kw & 1) == 0) {  // the diagonal pair {k/2, k/2}
      const int hk = kk >> 1, hw = kw >> 1;
      const T2 yh = conv_y<T>(y, SSpad, rowstride, hk, hw, ss);
      const T eh = e[(size_t)hk * nw + hw];
      const T zr = eh * yh.x, zi = eh * yh.y;
      ar += zr * zr - zi * zi;
      ai += 2 * zr * zi;
    }
    ar *= (T)0.5;
    ai *= (T)0.5;
    const size_t k = (size_t)kk * nw + kw;
    const T2 yk = (k == 0) ? y0[ss] : conv_y<T>(y, SSpad, rowstride, kk, kw, ss);
    const T f = ck[k] * eb[k], P = Pk[k];
    T2 out;
    out.x = P * yk.x + f * (ar * cb - ai * sb);
    out.y = P * yk.y + f * (ar * sb + ai * cb);
    C[((size_t)ss * nk + kk) * nw + kw] = out;
  };
  stockham_passes<LW, 0, 0u>(1, 0, tpt, jt, tw, buf, src, dst);
}

}  // namespace
}  // namespace srm3
