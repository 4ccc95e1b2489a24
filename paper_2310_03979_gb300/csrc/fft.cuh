// fft.cuh - the hand-written FFTs: the 2-D inverse transform of the SRM3 field
// (x stage over the coefficient columns, then half-length complex-to-real
// rows), shared by the sampling entry points and the no-allocation
// transform, and the radix-2 shared-memory stages of the separable
// self-convolution.  Internal linkage: every translation unit that includes
// it gets its own copy of the kernels.
#pragma once

#include <utility>

#include "srm3_internal.cuh"

namespace srm3 {
namespace {

// Radix-2 decimation in time in shared memory (the separable
// self-convolution's transforms), input in bit-reversed order,
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

// ---------------------------------------------------------------------------
// a6: the output transform (FFT form, Sec. 4.3).  With F[kk][m] on the
// nx x nt grid (F[kk][kw] = C^+_k, F[kk][(nt - kw) mod nt] += C^-_k, zero
// for kk >= nk), the field is
//   u[mx][mt] = Re sum_{kk,m} F[kk][m] e^{2 pi i (kk mx / nx + m mt / nt)}.
// Re z = (z + conj z) / 2, so u is the plain inverse DFT of the Hermitian
// part F_h[kk][m] = (F[kk][m] + conj F[-kk][-m]) / 2 (indices mod nx, nt).
// In the columns m <= nt/2, F_h is nonzero only for m < nw (nt >= 2 nw - 1):
//   F_h[kk][m] = (P[kk][m] + conj P'[-kk][m]) / 2,
//   P[kk][m] = C^+[kk][m] + [m = 0] C^-[kk][0],
//   P'[kk][m] = C^-[kk][m] + [m = 0] C^+[kk][0]   (zero for kk >= nk).
// Stage 1 (x): G[mx][m] = sum_kk F_h[kk][m] e^{2 pi i kk mx / nx} for the nw
// columns m < nw only.  Stage 2 (t): each row X[m] = G[mx][m] is Hermitian
// in m (u is real), so with M = nt / 2 the row is one complex inverse DFT of
// length M: z[j] = u[mx][2j] + i u[mx][2j + 1] = sum_{m<M} Z[m] e^{2 pi i m j/M},
//   Z[m] = (X[m] + conj X[M - m]) + i e^{2 pi i m / nt} (X[m] - conj X[M - m])
// (the split of u into even and odd samples; X[M] = 0 as M >= nw).
// Compared with transforming all nt columns of H[kk][mt], stage 1 runs over
// nw columns and stage 2 over half-length rows.
//
// Both stages are Stockham autosort passes of radix R <= 16 (Govindaraju et
// al., SC 2008): pass item j < L/R of a length-L transform, with Ns the
// length already transformed, reads x[j + r L/R] (r < R), multiplies by
// w_{Ns R}^{(j mod Ns) r}, takes a radix-R DFT in registers and writes
// x[(j / Ns) Ns R + j mod Ns + r Ns].  Natural order in and out: the first
// pass reads its inputs straight from global memory (forming F_h or Z on
// the way), the last writes straight to global memory, the passes between
// go through shared memory in place.  A thread holds 16 values (one radix-16
// item, or 16/R items of radix R); log2 L splits into ceil(log2 L / 4)
// passes of near-equal radix.  w_N = e^{+2 pi i / N}.

// b * e^{2 pi i e / 16}, e in [0, 8) (e a constant after unrolling)
template <typename T2>
__device__ __forceinline__ T2 rot16(T2 b, int e) {
  using T = decltype(b.x);
  constexpr double c1 = 0.92387953251128675613;  // cos(pi / 8)
  constexpr double s1 = 0.38268343236508977173;  // sin(pi / 8)
  constexpr double h = 0.70710678118654752440;   // cos(pi / 4)
  T2 r;
  switch (e) {
    case 0:
      return b;
    case 2:
      r.x = (T)h * (b.x - b.y);
      r.y = (T)h * (b.x + b.y);
      return r;
    case 4:
      r.x = -b.y;
      r.y = b.x;
      return r;
    case 6:
      r.x = -(T)h * (b.x + b.y);
      r.y = (T)h * (b.x - b.y);
      return r;
    default: {
      const T c = e == 1 ? (T)c1 : e == 3 ? (T)s1 : e == 5 ? (T)-s1 : (T)-c1;
      const T s = (e == 1 || e == 7) ? (T)s1 : (T)c1;
      r.x = b.x * c - b.y * s;
      r.y = b.x * s + b.y * c;
      return r;
    }
  }
}

template <int R>
struct Log2R {
  static constexpr int v = R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : 4;
};

// v[r] <- sum_s v[s] e^{2 pi i r s / R}: radix-2 decimation in time on the
// bit-reversed copy, every index and twiddle a compile-time constant.
template <int R, typename T2>
__device__ __forceinline__ void dft_inv(T2 (&v)[R]) {
  constexpr int B = Log2R<R>::v;
  T2 a[R];
#pragma unroll
  for (int i = 0; i < R; ++i) {
    int rb = 0;
#pragma unroll
    for (int bit = 0; bit < B; ++bit) rb |= ((i >> bit) & 1) << (B - 1 - bit);
    a[i] = v[rb];
  }
#pragma unroll
  for (int st = 0; st < B; ++st) {
    const int h = 1 << st;
#pragma unroll
    for (int g = 0; g < R; g += 2 * h)
#pragma unroll
      for (int j = 0; j < h; ++j) {
        const T2 t = rot16(a[g + j + h], j * (8 >> st));  // w_{2h}^j
        const T2 x = a[g + j];
        a[g + j].x = x.x + t.x;
        a[g + j].y = x.y + t.y;
        a[g + j + h].x = x.x - t.x;
        a[g + j + h].y = x.y - t.y;
      }
  }
#pragma unroll
  for (int i = 0; i < R; ++i) v[i] = a[i];
}

// The same DFT when some inputs are zero by construction: bit r of VMASK is
// set when v[r] may be nonzero (the others must be zero).  Each butterfly
// of the decimation in time is resolved at compile time from the zero
// pattern its stage inherits: both operands zero, skipped; the rotated one
// zero, a copy (x +- 0 = x); the other zero, the rotated operand and its
// negation (0 +- t = +-t); else computed as in dft_inv.  IEEE arithmetic does
// not let the compiler drop the additions of zeros by itself.  The results
// equal dft_inv's up to the sign of zero outputs.
template <int R>
__host__ __device__ constexpr unsigned dit_in_mask(unsigned vmask) {
  unsigned m = 0;
  for (int i = 0; i < R; ++i) {
    int rb = 0;
    for (int bit = 0; bit < Log2R<R>::v; ++bit)
      rb |= ((i >> bit) & 1) << (Log2R<R>::v - 1 - bit);
    if ((vmask >> rb) & 1u) m |= 1u << i;
  }
  return m;
}
template <int R>
__host__ __device__ constexpr unsigned dit_next_mask(unsigned m, int st) {
  const int h = 1 << st;
  unsigned o = 0;
  for (int g = 0; g < R; g += 2 * h)
    for (int j = 0; j < h; ++j)
      if (((m >> (g + j)) & 1u) || ((m >> (g + j + h)) & 1u))
        o |= (1u << (g + j)) | (1u << (g + j + h));
  return o;
}
template <int R, int ST, unsigned M, int B, typename T2>
__device__ __forceinline__ void dit_bfly(T2 (&a)[R]) {
  constexpr int h = 1 << ST, j = B % h, i0 = (B / h) * 2 * h + j, i1 = i0 + h;
  constexpr bool n0 = (M >> i0) & 1u, n1 = (M >> i1) & 1u;
  if constexpr (n0 && n1) {
    const T2 t = rot16(a[i1], j * (8 >> ST));
    const T2 x = a[i0];
    a[i0].x = x.x + t.x;
    a[i0].y = x.y + t.y;
    a[i1].x = x.x - t.x;
    a[i1].y = x.y - t.y;
  } else if constexpr (n0) {
    a[i1] = a[i0];
  } else if constexpr (n1) {
    const T2 t = rot16(a[i1], j * (8 >> ST));
    a[i0] = t;
    a[i1].x = -t.x;
    a[i1].y = -t.y;
  }
}
template <int R, int ST, unsigned M, typename T2, int... Bs>
__device__ __forceinline__ void dit_stage(T2 (&a)[R], std::integer_sequence<int, Bs...>) {
  (dit_bfly<R, ST, M, Bs>(a), ...);
}
template <int R, int ST, unsigned M, typename T2>
__device__ __forceinline__ void dit_stages(T2 (&a)[R]) {
  if constexpr (ST < Log2R<R>::v) {
    dit_stage<R, ST, M>(a, std::make_integer_sequence<int, R / 2>{});
    dit_stages<R, ST + 1, dit_next_mask<R>(M, ST)>(a);
  }
}
template <int R, unsigned VMASK, typename T2>
__device__ __forceinline__ void dft_inv_masked(T2 (&v)[R]) {
  constexpr int B = Log2R<R>::v;
  T2 a[R];
#pragma unroll
  for (int i = 0; i < R; ++i) {
    int rb = 0;
#pragma unroll
    for (int bit = 0; bit < B; ++bit) rb |= ((i >> bit) & 1) << (B - 1 - bit);
    a[i] = v[rb];
  }
  dit_stages<R, 0, dit_in_mask<R>(VMASK)>(a);
#pragma unroll
  for (int i = 0; i < R; ++i) v[i] = a[i];
}

// Inputs of the first pass of a length-L transform that can be nonzero:
// with R the first radix, the blocks r < nz and r >= R - nz of the L/R-long
// input runs (both ends of the spectrum); nz = 0 or nz >= R/2: all.
__host__ __device__ constexpr unsigned tx_in_mask(int R, int nz) {
  return (nz <= 0 || 2 * nz >= R) ? (R >= 32 ? 0xffffffffu : (1u << R) - 1u)
                                   : ((1u << nz) - 1u) | (((1u << nz) - 1u) << (R - nz));
}

// Pass plan of a length-2^l transform: ceil(l / 4) passes, pass p of radix
// 2^tx_lr(l, p) (larger radices first).
__host__ __device__ constexpr int tx_npass(int l) { return (l + 3) >> 2; }
__host__ __device__ constexpr int tx_lr(int l, int p) {
  return l / tx_npass(l) + (p < l - (l / tx_npass(l)) * tx_npass(l) ? 1 : 0);
}
// Entries of the pass-twiddle table: passes p >= 1 in order, pass p holding
// w_{Ns R}^{k r} at k R + r (k < Ns, r < R; Ns = the length its earlier
// passes transformed), so that an item's R twiddles are one contiguous run.
__host__ __device__ constexpr int tx_twlen(int l) {
  int n = 0, ns = 1;
  for (int p = 0; p < tx_npass(l); ++p) {
    ns <<= tx_lr(l, p);
    if (p >= 1) n += ns;
  }
  return n;
}

// Shared-memory position of entry i of one transform: one pad entry per 16,
// which spreads the first pass's stride-R writes over the banks.
__device__ __forceinline__ int sp16(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int tx_len(int L) { return L + (L >> 4); }
__host__ __device__ constexpr int tx_tpt(int L) { return L >= 16 ? L >> 4 : 1; }

// The R twiddles of one item (16-byte loads; the tables start 16-byte aligned
// and every run is an even number of entries).
template <int R, typename T2>
__device__ __forceinline__ void load_tw(const T2 *__restrict__ p, T2 (&w)[R]) {
  if constexpr (sizeof(T2) == 8) {
    const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
    for (int i = 0; i < R / 2; ++i) {
      const float4 t = __ldg(q + i);
      w[2 * i].x = t.x;
      w[2 * i].y = t.y;
      w[2 * i + 1].x = t.z;
      w[2 * i + 1].y = t.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < R; ++i) w[i] = __ldg(p + i);
  }
}

// One Stockham pass of radix R (see above).  tpt threads per transform, jt
// this thread's index among them; items jt, jt + tpt, ... < L/R.  twp: this
// pass's run of the pass-twiddle table.  FIRST: inputs from src(i) (global);
// else from sm (shared, padded positions).  LAST: outputs to dst(i, v)
// (global); else to sm.
template <int R, bool FIRST, bool LAST, unsigned VMASK, typename T2, class Src, class Dst>
__device__ __forceinline__ void stockham_pass(int L, int Ns, int tpt, int jt,
                                              const T2 *__restrict__ twp, T2 *sm, Src &src,
                                              Dst &dst) {
  constexpr int NI = 16 / R;
  const int LR = L / R;
  T2 v[NI][R];
#pragma unroll
  for (int it = 0; it < NI; ++it) {
    const int j = jt + it * tpt;
    if (j < LR) {
      if constexpr (FIRST) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          if ((VMASK >> r) & 1u) {
            v[it][r] = src(j + r * LR);
          } else {
            v[it][r].x = 0;
            v[it][r].y = 0;
          }
        }
      } else {
        if (LR % 16 == 0) {  // (j + r LR) >> 4 = (j >> 4) + r LR / 16
          const int a = sp16(j), st = LR + (LR >> 4);
#pragma unroll
          for (int r = 0; r < R; ++r) v[it][r] = sm[a + r * st];
        } else {
#pragma unroll
          for (int r = 0; r < R; ++r) v[it][r] = sm[sp16(j + r * LR)];
        }
        T2 w[R];
        load_tw<R>(twp + (j & (Ns - 1)) * R, w);
#pragma unroll
        for (int r = 1; r < R; ++r) v[it][r] = cmul(v[it][r], w[r]);
      }
      if constexpr (FIRST && VMASK != tx_in_mask(R, 0))
        dft_inv_masked<R, VMASK>(v[it]);
      else
        dft_inv<R>(v[it]);
    }
  }
  if constexpr (!FIRST && !LAST) __syncthreads();  // in place: all reads before any write
#pragma unroll
  for (int it = 0; it < NI; ++it) {
    const int j = jt + it * tpt;
    if (j < LR) {
      const int k = j & (Ns - 1);
      const int b = (j - k) * R + k;
      if constexpr (LAST) {
#pragma unroll
        for (int r = 0; r < R; ++r) dst(b + r * Ns, v[it][r]);
      } else if (Ns % 16 == 0) {
        const int a = sp16(b), st = Ns + (Ns >> 4);
#pragma unroll
        for (int r = 0; r < R; ++r) sm[a + r * st] = v[it][r];
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) sm[sp16(b + r * Ns)] = v[it][r];
      }
    }
  }
  if constexpr (!LAST) __syncthreads();
}

// Passes p, p + 1, ... of the inverse DFT of length 2^l (1 <= l <= 13),
// unrolled at compile time so that each pass keeps only its own 16 values
// live; Ns is the length transformed by the passes before p, toff the
// offset of pass p's run in the pass-twiddle table tw.
// VM0: the inputs of the first pass that can be nonzero (bit r: the block
// r of L/R inputs, R the first radix; 0 = all).
template <int l, int p, unsigned VM0, typename T2, class Src, class Dst>
__device__ __forceinline__ void stockham_passes(int Ns, int toff, int tpt, int jt,
                                                const T2 *__restrict__ tw, T2 *sm, Src &src,
                                                Dst &dst) {
  if constexpr (p < tx_npass(l)) {
    constexpr int lr = tx_lr(l, p);
    constexpr unsigned vm = (p == 0 && VM0 != 0u) ? VM0 : tx_in_mask(1 << lr, 0);
    stockham_pass<(1 << lr), p == 0, p == tx_npass(l) - 1, vm>(1 << l, Ns, tpt, jt, tw + toff,
                                                               sm, src, dst);
    stockham_passes<l, p + 1, VM0>(Ns << lr, p == 0 ? 0 : toff + (Ns << lr), tpt, jt, tw, sm,
                                   src, dst);
  }
}

// The first pass's mask for inputs at both ends of the spectrum (nz blocks
// each, tx_in_mask) or at the low end only (the lower half of the blocks:
// a zero-padded sequence of at most L/2 entries).
template <int l>
__host__ __device__ constexpr unsigned tx_mask_ends(int nz) {
  return tx_in_mask(1 << tx_lr(l, 0), nz);
}
template <int l>
__host__ __device__ constexpr unsigned tx_mask_low_half() {
  return (1u << ((1 << tx_lr(l, 0)) / 2)) - 1u;
}

// Stage 1: TC columns m0 + c of one coefficient set per CTA (blockIdx.y =
// set), thread (c, jt) = (t mod TC, t / TC); TC consecutive columns make the
// reads of C and the writes of G runs of TC complex values.  G is
// [set][nx][nw].  Column stride in shared memory: colstride entries.  twp:
// the pass-twiddle table of length nx.
template <int LOG2NX, typename T2, int NZ = 0>
__global__ void __launch_bounds__(512) k_tx_cols(int nk, int nw, int TC, int colstride,
                                                  const T2 *__restrict__ C,
                                                  const T2 *__restrict__ twp,
                                                  T2 *__restrict__ G) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using T = decltype(T2::x);
  constexpr int L = 1 << LOG2NX;
  const int n = blockIdx.y;
  const int c = threadIdx.x & (TC - 1), jt = threadIdx.x / TC;
  const int m = blockIdx.x * TC + c;
  const bool live = m < nw;
  const T2 *Cp = C + (size_t)(2 * n) * nk * nw;
  const T2 *Cm = Cp + (size_t)nk * nw;
  T2 *col = reinterpret_cast<T2 *>(smem_raw) + c * colstride;
  T2 *Gn = G + (size_t)n * L * nw;
  auto src = [&](int kk) -> T2 {  // F_h[kk][m]
    T2 v;
    v.x = 0;
    v.y = 0;
    if (!live) return v;
    if (kk < nk) {
      v = Cp[(size_t)kk * nw + m];
      if (m == 0) {
        const T2 w = Cm[(size_t)kk * nw];
        v.x += w.x;
        v.y += w.y;
      }
    }
    const int k2 = kk == 0 ? 0 : L - kk;
    if (k2 < nk) {
      T2 w = Cm[(size_t)k2 * nw + m];
      if (m == 0) {
        const T2 a = Cp[(size_t)k2 * nw];
        w.x += a.x;
        w.y += a.y;
      }
      v.x += w.x;
      v.y -= w.y;
    }
    v.x *= (T)0.5;
    v.y *= (T)0.5;
    return v;
  };
  auto dst = [&](int i, T2 v) {
    if (live) Gn[(size_t)i * nw + m] = v;
  };
  stockham_passes<LOG2NX, 0, tx_mask_ends<LOG2NX>(NZ)>(1, 0, tx_tpt(L), jt, twp, col, src, dst);
}

// Stage 2: RB rows mx of one set per CTA, thread (row, jt) = (t / tpt,
// t mod tpt); the row's output is the nt = 2M real values u[set][mx][.].
// twp: the pass-twiddle table of length M; twz[m] = e^{2 pi i m / nt}, m < M.
template <int LOG2M, typename T, typename T2, int NZ = 0>
__global__ void __launch_bounds__(512) k_tx_rows(int nx, int nw, int rowstride,
                                                 const T2 *__restrict__ G,
                                                 const T2 *__restrict__ twp,
                                                 const T2 *__restrict__ twz, T *__restrict__ u) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int M = 1 << LOG2M, tpt = tx_tpt(M);
  const int n = blockIdx.y;
  const int row = threadIdx.x / tpt, jt = threadIdx.x & (tpt - 1);
  const int rb = blockDim.x / tpt, mx = blockIdx.x * rb + row;
  const T2 *X = G + ((size_t)n * nx + mx) * nw;
  T2 *buf = reinterpret_cast<T2 *>(smem_raw) + row * rowstride;
  T *urow = u + ((size_t)n * nx + mx) * (size_t)(2 * M);
  auto src = [&](int m) -> T2 {  // Z[m]
    T2 a, b;
    a.x = 0;
    a.y = 0;
    b = a;
    if (m < nw) a = X[m];
    if (M - m < nw) b = X[M - m];
    if (m >= nw && M - m >= nw) return a;  // zero
    const T2 w = twz[m];
    const T dx = a.x - b.x, dy = a.y + b.y;  // X[m] - conj X[M - m]
    const T wx = w.x * dx - w.y * dy, wy = w.x * dy + w.y * dx;
    T2 z;
    z.x = (a.x + b.x) - wy;
    z.y = (a.y - b.y) + wx;
    return z;
  };
  const bool vec = (reinterpret_cast<uintptr_t>(u) & (sizeof(T2) - 1)) == 0;
  auto dst = [&](int i, T2 v) {
    if (vec) {
      reinterpret_cast<T2 *>(urow)[i] = v;
    } else {
      urow[2 * i] = v.x;
      urow[2 * i + 1] = v.y;
    }
  };
  if constexpr (LOG2M == 0) {  // nt = 2: z[0] = Z[0]
    if (jt == 0) dst(0, src(0));
  } else {
    stockham_passes<LOG2M, 0, tx_mask_ends<LOG2M>(NZ)>(1, 0, tpt, jt, twp, buf, src, dst);
  }
}

}  // namespace
}  // namespace srm3
