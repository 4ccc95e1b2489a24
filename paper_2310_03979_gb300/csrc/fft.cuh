// fft.cuh - the hand-written 2-D inverse FFT of the SRM3 field (t stage, then
// x stage), shared by the sampling entry points and the no-allocation
// transform.  Internal linkage: every translation unit that includes it
// gets its own copy of the kernels.
#pragma once

#include "srm3_internal.cuh"

namespace srm3 {
namespace {

// a6: inverse transform.  u[mx][mt] = Re sum_kk e^{2 pi i kk mx / nx}
//   sum_m F[kk][m] e^{2 pi i m mt / nt}, F[kk][kw] = C^+_k,
//   F[kk][(nt - kw) mod nt] += C^-_k (FFT form, Sec. 4.3).
// Radix-2 decimation in time in shared memory, input in bit-reversed order,
// twiddles from a table packed by stage: stage s (1-based) reads
// e^{+2 pi i j / 2^s}, j < 2^(s-1), at twp[2^(s-1) - 1 + j], so the lanes of
// a warp read consecutive entries in every stage.
template <typename T2>
__device__ __forceinline__ T2 cmul(T2 a, T2 b) {
  T2 r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}

// One radix-2 butterfly: (a, b) <- (a + w b, a - w b).
template <typename T2>
__device__ __forceinline__ void bfly(T2 &a, T2 &b, T2 w) {
  const T2 x1 = cmul(b, w);
  T2 o0, o1;
  o0.x = a.x + x1.x;
  o0.y = a.y + x1.y;
  o1.x = a.x - x1.x;
  o1.y = a.y - x1.y;
  a = o0;
  b = o1;
}

// Shared-memory layouts.  One transform (a row): element i at rp(i) = i XOR
// (((i >> 4) XOR (i >> 8)) & 15), a permutation of each 16-element (128-byte
// for FP32) group by the bits above it, which spreads over the banks both
// the bit-reversed scatter of a row's first entries (multiples of n / 32
// apart) and the stride-4 and stride-16 groups of the first two radix-4
// stage pairs.  Several transforms (columns): column c at
// c (n + 1); in the stages with h < 16 consecutive threads take consecutive
// columns (the lanes then meet different banks), in the later ones
// consecutive butterflies of one column (contiguous runs of 16 or more).
__host__ __device__ constexpr int fft_row_len(int n) { return n; }
__host__ __device__ constexpr int fft_col_stride(int n) { return n + 1; }
__device__ __forceinline__ int rp(int i) { return i ^ (((i >> 4) ^ (i >> 8)) & 15); }

// Stages s0..log2n of transforms of length n = 2^log2n in buf (input in
// bit-reversed order): one padded row (COLS = false, ncols = 1), or ncols
// (a power of two, 1 allowed) columns of stride n + 1 (COLS = true).  s0 > 1
// when the caller has done stages 1..s0-1 itself.  Stages go in
// pairs (s, s + 1) held in registers: four elements j, j + h, j + 2h, j + 3h
// of a block of 4h (h = 2^(s-1)) take the two butterflies of stage s and the
// two of stage s + 1 -- the same butterflies, in the same order, as one
// stage at a time, with half the shared-memory round trips and barriers.
// An odd last stage runs alone.
template <bool COLS, typename T2>
__device__ void fft_stages(T2 *buf, int ncols, int log2n, const T2 *__restrict__ twp,
                           int s0 = 1) {
  const int n = 1 << log2n, cs = fft_col_stride(n), lc = __ffs(ncols) - 1;
  auto at = [&](int col, int i) { return COLS ? col * cs + i : rp(i); };
  int s = s0;
  for (; s + 1 <= log2n; s += 2) {
    const int half = 1 << (s - 1);
    const int total = ncols * (n >> 2);
    const bool cf = COLS && half < 16;  // consecutive threads on consecutive columns
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      const int col = cf ? t & (ncols - 1) : t >> (log2n - 2);
      const int g = cf ? t >> lc : t & ((n >> 2) - 1);
      const int blk = g >> (s - 1);
      const int j = g & (half - 1);
      const int i0 = blk * 4 * half + j;
      const int a0 = at(col, i0), a1 = at(col, i0 + half), a2 = at(col, i0 + 2 * half),
                a3 = at(col, i0 + 3 * half);
      T2 e0 = buf[a0], e1 = buf[a1], e2 = buf[a2], e3 = buf[a3];
      const T2 ws = twp[half - 1 + j];
      bfly(e0, e1, ws);
      bfly(e2, e3, ws);
      bfly(e0, e2, twp[2 * half - 1 + j]);
      bfly(e1, e3, twp[3 * half - 1 + j]);
      buf[a0] = e0;
      buf[a1] = e1;
      buf[a2] = e2;
      buf[a3] = e3;
    }
    __syncthreads();
  }
  if (s == log2n) {  // odd number of stages: the last one alone
    const int half = 1 << (s - 1);
    const int total = ncols * (n >> 1);
    const bool cf = COLS && half < 16;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      const int col = cf ? t & (ncols - 1) : t >> (log2n - 1);
      const int bf = cf ? t >> lc : t & ((n >> 1) - 1);
      const int grp = bf >> (s - 1);
      const int j = bf & (half - 1);
      const int i0 = grp * 2 * half + j;
      const int a0 = at(col, i0), a1 = at(col, i0 + half);
      T2 a = buf[a0], b = buf[a1];
      bfly(a, b, twp[half - 1 + j]);
      buf[a0] = a;
      buf[a1] = b;
    }
    __syncthreads();
  }
}

__device__ __forceinline__ int brev(int m, int log2n) {
  return (int)(__brev((unsigned)m) >> (32 - log2n));
}

template <typename T2>
__global__ void k_fft_t(int nk, int nw, int nt, int log2nt,
                        const T2 *__restrict__ C, const T2 *__restrict__ tw, T2 *__restrict__ H) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T2 *buf = reinterpret_cast<T2 *>(smem_raw);
  const int kk = blockIdx.x, n = blockIdx.y;
  for (int m = threadIdx.x; m < fft_row_len(nt); m += blockDim.x) {
    buf[m].x = 0;
    buf[m].y = 0;
  }
  __syncthreads();
  const T2 *Cp = C + ((size_t)(2 * n) * nk + kk) * nw;
  const T2 *Cm = C + ((size_t)(2 * n + 1) * nk + kk) * nw;
  for (int kw = threadIdx.x; kw < nw; kw += blockDim.x) buf[rp(brev(kw, log2nt))] = Cp[kw];
  __syncthreads();
  for (int kw = threadIdx.x; kw < nw; kw += blockDim.x) {
    const int m = kw == 0 ? 0 : nt - kw;
    const int pos = rp(brev(m, log2nt));
    T2 v = buf[pos];
    const T2 c = Cm[kw];
    v.x += c.x;
    v.y += c.y;
    buf[pos] = v;
  }
  __syncthreads();
  fft_stages<false>(buf, 1, log2nt, tw);
  T2 *Hrow = H + ((size_t)n * nk + kk) * nt;
  for (int m = threadIdx.x; m < nt; m += blockDim.x) Hrow[m] = buf[rp(m)];
}

template <typename T, typename T2>
__global__ void k_fft_x(int nk, int nx, int nt, int log2nx, int TC,
                        const T2 *__restrict__ H, const T2 *__restrict__ tw, T *__restrict__ u) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T2 *buf = reinterpret_cast<T2 *>(smem_raw);
  const int mt0 = blockIdx.x * TC, n = blockIdx.y, cs = fft_col_stride(nx);
  // Inputs kk >= nk are zero.  With nk <= nkp = 2^q, the entries x[kk +
  // j nkp] (j < 2^r, r = log2nx - q) sit at bit-reversed positions brev(kk)
  // + brev_r(j), one aligned group of 2^r, and only j = 0 is nonzero; the
  // first r stages of butterflies turn such a group into 2^r copies of
  // x[kk].  The copies are written here and the stages start at r + 1;
  // every position is written, so the buffer needs no clearing.
  int q = 0;
  while ((1 << q) < nk) ++q;
  const int r = log2nx - q, rep = 1 << r;
  const T2 *Hn = H + (size_t)n * nk * nt + mt0;
  for (int idx = threadIdx.x; idx < (TC << q); idx += blockDim.x) {
    const int kk = idx / TC, c = idx - kk * TC;
    T2 v;
    v.x = 0;
    v.y = 0;
    if (kk < nk) v = Hn[(size_t)kk * nt + c];
    T2 *dst = buf + c * cs + brev(kk, log2nx);
    for (int j = 0; j < rep; ++j) dst[j] = v;
  }
  __syncthreads();
  fft_stages<true>(buf, TC, log2nx, tw, r + 1);
  T *un = u + (size_t)n * nx * nt + mt0;
  for (int idx = threadIdx.x; idx < nx * TC; idx += blockDim.x) {
    const int mx = idx / TC, c = idx - mx * TC;
    un[(size_t)mx * nt + c] = buf[c * cs + mx].x;
  }
}

}  // namespace
}  // namespace srm3
