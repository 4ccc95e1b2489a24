// conv.cuh - the pair sum of a separable envelope as an FFT self-convolution
// (a4 + a5 for g(i,j) = a(i) a(j) b(i+j)).  Included by sample.cu after
// fft.cuh, whose radix-2 stages it reuses.
//
// With W_ij = c_k a_i a_j b_k the pair part of C_k is
//   c_k e^{i beta} b_k sum_{Pi(k)} z_i z_j,   z = a y  (z_0 = 0),
// and over unordered pairs {i, j}, i + j = k,
//   sum_{Pi(k)} z_i z_j = ((z * z)_k + [k even] z_{k/2}^2) / 2,
// with (z * z) the linear 2-D self-convolution on the quadrant lattice.  It
// is taken on a zero-padded Nk x Nw grid (powers of two, Nk >= 2 n_kappa - 1,
// Nw >= 2 n_omega - 1) with one transform direction only:
//   F(F(z)^2)[m] = Nk Nw (z * z)[-m mod (Nk, Nw)],
// so the second transform is read back at negated indices.  Three passes
// per sheet-sample: rows of z forward (k_conv_rows), columns forward, square,
// columns forward again (k_conv_cols, which also negates the row index on
// its way out), rows forward and the coefficient epilogue (k_conv_out).
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

// Pass 1: z = a y along each lattice row kk < n_kappa, zero-padded to Nw,
// transformed; block (kk, ss).  Rows kk >= n_kappa of the grid are zero
// and never stored.
template <typename T>
__global__ void k_conv_rows(int nk, int nw, int log2Nw, int Nk, int SSpad, int rowstride,
                            const void *__restrict__ y, const T *__restrict__ e,
                            const typename Vec2<T>::type *__restrict__ tw,
                            typename Vec2<T>::type *__restrict__ Z) {
  using T2 = typename Vec2<T>::type;
  extern __shared__ __align__(16) unsigned char conv_smem[];
  T2 *buf = reinterpret_cast<T2 *>(conv_smem);
  const int kk = blockIdx.x, ss = blockIdx.y, Nw = 1 << log2Nw;
  for (int m = threadIdx.x; m < Nw; m += blockDim.x) {
    T2 v;
    v.x = 0;
    v.y = 0;
    if (m < nw) {
      const T2 yv = conv_y<T>(y, SSpad, rowstride, kk, m, ss);
      const T ev = e[(size_t)kk * nw + m];
      v.x = ev * yv.x;
      v.y = ev * yv.y;
    }
    buf[rp(brev(m, log2Nw))] = v;
  }
  __syncthreads();
  fft_stages<false>(buf, 1, log2Nw, tw);
  T2 *out = Z + ((size_t)ss * Nk + kk) * Nw;
  for (int m = threadIdx.x; m < Nw; m += blockDim.x) out[m] = buf[rp(m)];
}

// Pass 2: TC columns of one sheet-sample: forward transform along kappa
// (rows >= n_kappa are zero), square, forward again, and store the n_kappa
// rows needed, row kk taking grid row (Nk - kk) mod Nk.  In place in Z.
template <typename T>
__global__ void k_conv_cols(int nk, int log2Nk, int Nw, int TC,
                            const typename Vec2<T>::type *__restrict__ tw,
                            typename Vec2<T>::type *__restrict__ Z) {
  using T2 = typename Vec2<T>::type;
  extern __shared__ __align__(16) unsigned char conv_smem[];
  T2 *buf = reinterpret_cast<T2 *>(conv_smem);  // [TC][Nk + 1]
  const int Nk = 1 << log2Nk, col0 = blockIdx.x * TC, ss = blockIdx.y, cs = fft_col_stride(Nk);
  T2 *base = Z + (size_t)ss * Nk * Nw + col0;
  for (int t = threadIdx.x; t < Nk * TC; t += blockDim.x) {
    const int r = t / TC, c = t - r * TC;
    T2 v;
    v.x = 0;
    v.y = 0;
    if (r < nk) v = base[(size_t)r * Nw + c];
    buf[c * cs + brev(r, log2Nk)] = v;
  }
  __syncthreads();
  fft_stages<true>(buf, TC, log2Nk, tw);
  // square, then back to bit-reversed order for the second transform
  for (int t = threadIdx.x; t < Nk * TC; t += blockDim.x) {
    const int c = t / Nk, r = t - c * Nk, rb = brev(r, log2Nk);
    if (r <= rb) {
      const T2 a = buf[c * cs + r], b = buf[c * cs + rb];
      T2 a2, b2;
      a2.x = a.x * a.x - a.y * a.y;
      a2.y = 2 * a.x * a.y;
      b2.x = b.x * b.x - b.y * b.y;
      b2.y = 2 * b.x * b.y;
      buf[c * cs + r] = b2;
      buf[c * cs + rb] = a2;
    }
  }
  __syncthreads();
  fft_stages<true>(buf, TC, log2Nk, tw);
  for (int t = threadIdx.x; t < nk * TC; t += blockDim.x) {
    const int r = t / TC, c = t - r * TC;
    base[(size_t)r * Nw + c] = buf[c * cs + ((Nk - r) & (Nk - 1))];
  }
}

// Pass 3: row kk of the twice-transformed grid, transformed along omega; the
// ordered self-convolution at (kk, kw) is its entry (Nw - kw) mod Nw over
// Nk Nw.  Epilogue as in the O(N^2) pair sums:
//   C_k = P_k y_k + c_k e^{i beta} b_k ((z * z)_k + [k even] z_{k/2}^2) / 2.
template <typename T>
__global__ void k_conv_out(int nk, int nw, int log2Nw, int Nk, int SSpad, int rowstride,
                           const void *__restrict__ y, const typename Vec2<T>::type *__restrict__ y0,
                           const T *__restrict__ e, const T *__restrict__ eb,
                           const T *__restrict__ Pk,
                           const T *__restrict__ ck, T cb, T sb,
                           const typename Vec2<T>::type *__restrict__ tw,
                           const typename Vec2<T>::type *__restrict__ Z,
                           typename Vec2<T>::type *__restrict__ C) {
  using T2 = typename Vec2<T>::type;
  extern __shared__ __align__(16) unsigned char conv_smem[];
  T2 *buf = reinterpret_cast<T2 *>(conv_smem);
  const int kk = blockIdx.x, ss = blockIdx.y, Nw = 1 << log2Nw;
  const T2 *in = Z + ((size_t)ss * Nk + kk) * Nw;
  for (int m = threadIdx.x; m < Nw; m += blockDim.x) buf[rp(brev(m, log2Nw))] = in[m];
  __syncthreads();
  fft_stages<false>(buf, 1, log2Nw, tw);
  const T inv = (T)1 / ((T)Nk * (T)Nw);
  for (int kw = threadIdx.x; kw < nw; kw += blockDim.x) {
    const T2 cv = buf[rp((Nw - kw) & (Nw - 1))];
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
  }
}

}  // namespace
}  // namespace srm3
