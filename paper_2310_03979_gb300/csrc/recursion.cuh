// recursion.cuh - device side of the pure-spectrum / partial-bicoherence
// recursion (Eq. pure): one pass over the lattice as a persistent
// cooperative kernel, and the linear (q = 1) pass that brackets eps.
// Included by plan.cu only.
#pragma once

#include "fft.cuh"
#include "srm3_internal.cuh"

namespace srm3 {

constexpr int kRecThreads = 512;  // one CTA per SM
constexpr int kRecBL = 16;        // levels per block of the blocked pass
constexpr int kRecSmem = 64 << 10;  // dynamic shared memory of a pass in FFT form

struct RecArgs {
  int nk, nw, nlev;
  long long nl;
  const int2 *pts;      // lattice points in level order (level-major, kk ascending)
  const int *pt_off;    // first point of each level, nlev + 1 entries
  // bulk phase ph (D = ph BL) works on point pairs (kk, kw), (kk, kw + 1)
  // of its band of levels [D, min(2D, nlev)): starts pairs[pair_off[ph - 1]
  // .. pair_off[ph]), those of the fringe block [D, D + BL) that follows
  // the phase first (up to pair_mid[ph])
  const int2 *pairs;
  const int *pair_off;
  const int *pair_mid;
  int tk_def;           // bar[tk_def + ph]: ticket of the rest of bulk phase ph
  const double *S;
  void *q;              // [nl][M] of T: q = S/S_p (0 where S = 0), plane fastest
  void *acc;            // [nl][M] of T: pair sums gathered by the bulk phases
  double *sb2;          // [M][nl]
  const void *G2;       // T[nk][nw]: g^2 = EkSq[|ik-jk|] EwSq[|iw-jw|]
  const double *scal;   // [M]: eps^2 dk dw per plane
  // separable envelope (else NULL): e^2 per point.  The pair sums then run
  // over h = e^2 q (stored in q, G2 all ones), sum_b2(k) takes the factor
  // e_k^2, and the FP64 pass writes q itself to qout ([M][nl])
  const double *e2;   // a^2: h = a^2 q
  const double *e2k;  // b^2: the factor of sum_b2(k)
  double *qout;
  // separable envelope with the FFT form of the bulk (else NULL): the
  // product grid [M][2 L][Nc] of complex T, the packed twiddles (complex T)
  // for every length up to max(Nc, 2 L), log2 Nc, and the complex T elements
  // of dynamic shared memory
  void *zr;
  const void *twr;
  int log2Nc, zcap;
  // mixed-sign interactions (else NULL): the difference-pair sums of every
  // point, sum g^2 q_i q_j over its opposite-sheet pairs at the previous
  // iterate of the fixed point, added before q_k is formed (M = 1 only)
  const double *dsum;
  int *err;             // [M]: some S_p <= 0 on this plane
  unsigned int *bar;    // [0] grid barrier arrivals, [i] and [tk_def + i] tickets of bulk phase i (zero at launch)
  unsigned int *row_done;  // [nk]: 1 + the last fringe level each lattice row has finished (zero at launch)
  int *abort;           // barrier wait timed out
  unsigned long long *maxb;  // [M]: max_k sum_b2 per plane, as the bits of a double >= 0
};

// Grid-wide barrier for a cooperative launch (all CTAs resident): one
// arrival counter bar[0], zeroed on the stream before each launch.  After a
// CTA barrier, thread 0 of every CTA adds 1 with release semantics at GPU
// scope (ordering every write the CTA made before it) and polls with acquire
// loads until the counter reaches `target` (the barrier's number within the
// launch x gridDim.x), which orders every read after the barrier with every
// CTA's writes before it.  Waits are bounded: past ~2^22 polls a CTA raises
// *abort and sets kBarAbort in the counter, which every poll sees at once
// (the counter then exceeds any target), so every CTA returns false from
// this or its next barrier without a second memory read on the normal path.
constexpr unsigned int kBarAbort = 1u << 30;

__device__ __forceinline__ bool grid_barrier(unsigned int *bar, int *abort, unsigned int target,
                                             long long limit = 1ll << 22) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int v;
    asm volatile("atom.add.release.gpu.global.u32 %0, [%1], 1;" : "=r"(v) : "l"(bar) : "memory");
    bool ok = true;
    long long spins = 0;
    for (;;) {
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
      if (v >= target) break;
      if (++spins > limit) {
        ok = false;
        break;
      }
    }
    if (v & kBarAbort) ok = false;
    if (!ok) {
      atomicOr(bar, kBarAbort);
      atomicExch(abort, 1);
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <typename T, int M>
struct PlaneVec;
template <>
struct PlaneVec<double, 1> {
  static __device__ __forceinline__ void load(const double *p, double (&v)[1]) { v[0] = *p; }
};
template <>
struct PlaneVec<double, 3> {
  static __device__ __forceinline__ void load(const double *p, double (&v)[3]) {
    v[0] = p[0];
    v[1] = p[1];
    v[2] = p[2];
  }
};
// The eight FP32 planes of a point are one 32-byte aligned vector: one
// 256-bit load, so that the 16 points a half-warp reads on a lattice row
// are one contiguous 512-byte span per load instruction.
template <>
struct PlaneVec<float, 8> {
  static __device__ __forceinline__ void load(const float *p, float (&v)[8]) {
    asm volatile("ld.global.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]),
                   "=f"(v[6]), "=f"(v[7])
                 : "l"(p)
                 : "memory");
  }
};

// Four FP32 planes (the window pass around the coarse-lattice root): one
// 128-bit load.
template <>
struct PlaneVec<float, 4> {
  static __device__ __forceinline__ void load(const float *p, float (&v)[4]) {
    const float4 t = *reinterpret_cast<const float4 *>(p);
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
    v[3] = t.w;
  }
};

// One pair term g^2(i, j) q_i q_j added to acc (all planes).  SEP: the
// pair factor is carried by h = a^2 q (g^2 = a_i^2 a_j^2 b_k^2), so the term
// is h_i h_j and no g^2 is read.
template <typename T, int M, bool SEP>
__device__ __forceinline__ void add_pair(const RecArgs &A, int kk, int kw, int ia, int iw, int ja,
                                         int jw, T (&acc)[M]) {
  const int nw = A.nw;
  const T *q = static_cast<const T *>(A.q);
  T va[M], vb[M];
  PlaneVec<T, M>::load(q + ((size_t)ia * nw + iw) * M, va);
  PlaneVec<T, M>::load(q + ((size_t)ja * nw + jw) * M, vb);
  if constexpr (SEP) {
#pragma unroll
    for (int m = 0; m < M; ++m) acc[m] = fma(va[m], vb[m], acc[m]);
  } else {
    const T *G2 = static_cast<const T *>(A.G2);
    const int dk = 2 * ia - kk, dw = 2 * iw - kw;
    const T g2 = G2[(size_t)(dk < 0 ? -dk : dk) * nw + (dw < 0 ? -dw : dw)];
#pragma unroll
    for (int m = 0; m < M; ++m) acc[m] = fma(g2, va[m] * vb[m], acc[m]);
  }
}

template <typename T, int M>
__device__ __forceinline__ void warp_sum(T (&v)[M]) {
#pragma unroll
  for (int m = 0; m < M; ++m)
    for (int o = 16; o > 0; o >>= 1) v[m] += __shfl_xor_sync(0xffffffffu, v[m], o);
}

// q_k and sum_b2(k) of plane m from the point's complete pair sum t.
// 1/x, correctly rounded (the same value as the division)
__device__ __forceinline__ float recip_rn(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip_rn(double x) { return __drcp_rn(x); }

// ek2 = a_k^2, bk2 = b_k^2 (1 for non-separable envelopes), ds: the
// difference-pair sum of mixed plans (0 otherwise).
template <typename T, int M>
__device__ __forceinline__ T finalize_plane(const RecArgs &A, long long k, int m, T t, double ek2d,
                                            double bk2d, double ds) {
  T *q = static_cast<T *>(A.q);
  const T ek2 = (T)ek2d, bk2 = (T)bk2d;
  // t >= 0 (a sum of non-negative terms) up to the rounding of the FFT form,
  // which can leave a small negative value, of the order of the rounding of
  // the largest sums, where every term is zero; a NaN passes through
  if (M == 1 && A.dsum) t += (T)ds;
  const T s2r = (T)A.scal[m] * bk2 * t;
  const T s2 = s2r < (T)0 ? (T)0 : s2r;
  A.sb2[m * A.nl + k] = (double)s2;
  // non-negative doubles order as their bit patterns
  atomicMax(A.maxb + m, (unsigned long long)__double_as_longlong((double)s2));
  if (s2 < (T)1) {
    const T qk = recip_rn((T)1 - s2);
    // separable forms: h_0 = 0 (the origin is never part of a pair), so
    // that masked pair slots, which read the origin, add nothing
    const T h = A.e2 ? (k == 0 ? (T)0 : ek2 * qk) : qk;
    q[k * M + m] = h;
    if (A.qout) A.qout[m * A.nl + k] = (double)qk;
    return h;
  }
  q[k * M + m] = (T)0;
  if (A.qout) A.qout[m * A.nl + k] = 0.0;
  atomicOr(A.err + m, 1);
  return (T)0;
}

// All planes of a point (lane 0 only).
template <typename T, int M>
__device__ __forceinline__ void finalize(const RecArgs &A, long long k, const T (&t)[M]) {
  const double ek2 = A.e2 ? A.e2[k] : 1.0, bk2 = A.e2k ? A.e2k[k] : 1.0;
  const double ds = (M == 1 && A.dsum) ? A.dsum[k] : 0.0;
#pragma unroll
  for (int m = 0; m < M; ++m) finalize_plane<T, M>(A, k, m, t[m], ek2, bk2, ds);
}

template <typename T, int M>
__device__ __forceinline__ void point_zero(const RecArgs &A, long long k, int lane) {
  if (lane < M) {
    A.sb2[lane * A.nl + k] = 0.0;
    static_cast<T *>(A.q)[k * M + lane] = (T)0;
  }
  if (lane < M && A.qout) A.qout[lane * A.nl + k] = 0.0;
}

// Levels below kRecBL: the whole canonical pair sum of the point (one warp),
// rows a <= kk/2 laid end to end as a*(kw+1) + iw, the centre row a = kk - a
// keeping iw <= kw/2, i = 0 skipped.
template <typename T, int M, bool SEP>
__device__ void point_direct(const RecArgs &A, int kk, int kw, int lane) {
  const long long k = (long long)kk * A.nw + kw;
  if (!(A.S[k] > 0.0)) {
    point_zero<T, M>(A, k, lane);
    return;
  }
  T acc[M];
#pragma unroll
  for (int m = 0; m < M; ++m) acc[m] = (T)0;
  const int W = kw + 1, E = (kk / 2 + 1) * W;
  for (int e = lane; e < E; e += 32) {
    const int a = e / W, iw = e - a * W, b = kk - a;
    const int lim = (a == b) ? kw / 2 : kw;
    if ((a == 0 && iw == 0) || iw > lim) continue;
    add_pair<T, M, SEP>(A, kk, kw, a, iw, b, kw - iw, acc);
  }
  warp_sum<T, M>(acc);
  if (lane == 0) finalize<T, M>(A, k, acc);
}

// Bulk phase of block D for a point at level d in [D, 2D): the pairs whose
// higher-level element lies on a level in [D - BL, D).  For a row pair
// (a, b = kk - a) these are two slivers of at most BL omega indices:
//   right: i = (a, iw) is the higher element, iw = D - BL - a + u with
//          2 (D - BL + u) >= d;
//   left:  j = (b, jw) is the higher element, jw = D - BL - b + u with
//          2 (D - BL + u) > d.
// Lanes take (row, u) slots, 16 u per row and two rows per warp step; the
// canonical limits (centre row, i != 0, iw <= kw) mask the rest.  The loads
// of kBulkUnroll steps are issued before their products: a masked slot reads
// point (0, 0) and adds g^2 = 0, which leaves each lane's running sum and its
// order of additions exactly as if the slot were skipped.
constexpr int kBulkUnroll = 4;

// One sliver of a point's bulk pairs for this lane: rows v = v0, v0 + 2, ...
// < n with i = (a0 + v, iw0 - v) and j = k - i; uok: the lane's omega slot
// lies inside the sliver.  Offsets step linearly with v; the canonical
// limits (centre row, i != 0, iw <= kw) mask the rest.
template <typename T, int M, bool SEP>
__device__ __forceinline__ void bulk_rows(int kk, int kw, int nw, const T *__restrict__ G2,
                                          const T *__restrict__ q, int n, int v0, int a0,
                                          int iw0, bool uok, T (&acc)[M]) {
  const int qa0 = (a0 * nw + iw0) * M, qb0 = ((kk - a0) * nw + (kw - iw0)) * M;
  const int qstep = (nw - 1) * M;  // qa grows and qb shrinks by this per row
  for (int v = v0; v < n; v += 2 * kBulkUnroll) {
    T g2[kBulkUnroll], va[kBulkUnroll][M], vb[kBulkUnroll][M];
#pragma unroll
    for (int s = 0; s < kBulkUnroll; ++s) {
      const int vs = v + 2 * s;
      const int a = a0 + vs, iw = iw0 - vs, b = kk - a;
      const bool ok = uok && vs < n && iw >= (a == 0 ? 1 : 0) &&
                      iw <= ((a == b) ? kw / 2 : kw) && iw <= kw;
      const int dk = 2 * a - kk, dw = 2 * iw - kw;
      const int gi = ok ? (dk < 0 ? -dk : dk) * nw + (dw < 0 ? -dw : dw) : 0;
      const int qa = ok ? qa0 + vs * qstep : 0;
      const int qb = ok ? qb0 - vs * qstep : 0;
      if constexpr (!SEP) g2[s] = ok ? G2[gi] : (T)0;
      PlaneVec<T, M>::load(q + qa, va[s]);
      PlaneVec<T, M>::load(q + qb, vb[s]);
    }
#pragma unroll
    for (int s = 0; s < kBulkUnroll; ++s)
#pragma unroll
      for (int m = 0; m < M; ++m) {
        if constexpr (SEP)
          acc[m] = fma(va[s][m], vb[s][m], acc[m]);
        else
          acc[m] = fma(g2[s], va[s][m] * vb[s][m], acc[m]);
      }
  }
}

template <typename T, int M, bool SEP>
__device__ void point_bulk(const RecArgs &A, int kk, int kw, int D, int lane) {
  const long long k = (long long)kk * A.nw + kw;
  if (!(A.S[k] > 0.0)) return;
  const int d = kk + kw, base = D - kRecBL, arow = kk / 2 + 1;
  const int uR0 = max(0, (d + 1) / 2 - base);
  const int uL0 = max(0, d / 2 - base + 1);
  const int aR0 = max(0, base + uR0 - kw), aR1 = min(arow - 1, D - 1);
  const int aL0 = max(0, kk - D + 1), aL1 = arow - 1;
  const int nR = (uR0 < kRecBL && aR1 >= aR0) ? aR1 - aR0 + 1 : 0;
  const int nL = (uL0 < kRecBL && aL1 >= aL0) ? aL1 - aL0 + 1 : 0;
  if (nR + nL == 0) return;
  const int u = lane & (kRecBL - 1), rs = lane >> 4;
  T acc[M];
#pragma unroll
  for (int m = 0; m < M; ++m) acc[m] = (T)0;
  const int nw = A.nw;
  const T *G2 = static_cast<const T *>(A.G2);
  const T *q = static_cast<const T *>(A.q);
  // rows v < nR: right sliver, i = (aR0 + v, base - aR0 - v + u);
  // rows v = nR + m: left sliver, j = (kk - aL0 - m, base - kk + aL0 + m + u).
  // Each lane takes the rows of its parity rs, right then left: the order of
  // one sequence over v.
  bulk_rows<T, M, SEP>(kk, kw, nw, G2, q, nR, rs, aR0, base - aR0 + u, u >= uR0, acc);
  bulk_rows<T, M, SEP>(kk, kw, nw, G2, q, nL, (rs + nR) & 1, aL0, kw - base + kk - aL0 - u,
                       u >= uL0, acc);
  warp_sum<T, M>(acc);
  if (lane == 0) {
    T *ac = static_cast<T *>(A.acc);
#pragma unroll
    for (int m = 0; m < M; ++m) ac[k * M + m] += acc[m];
  }
}

// Bulk of two neighbouring points of a lattice row, k0 = (kk, kw) and
// k1 = (kk, kw + 1) (has1: k1 lies in the phase's band).  In both slivers
// the pair's element on the levels [D - BL, D) -- the higher one -- is the
// same for the two points at a given (row a, slot u), and their other
// elements are lattice neighbours (0, 1) apart: one load of the higher
// element and two adjacent loads of the lower ones serve both points, a
// quarter less traffic per pair than one point at a time.  RIGHT: the
// higher element is i = (a, base - a + u); else it is j = (kk - a, base -
// (kk - a) + u).  Rows a run over the union of the two points' ranges, the
// lanes of row parity rs taking every other row; each point keeps its own
// limits (the sliver's u and row ranges, i != 0, the centre row, iw <= kw),
// a masked slot reading point (0, 0) with weight 0.  Rows in flight per
// step: 4 with four planes (the eps-search window pass, room in its
// registers), else 2.
template <int M>
__host__ __device__ constexpr int pair_unroll() {
  return M == 4 ? 4 : 2;
}

template <bool RIGHT, typename T, int M, bool SEP>
__device__ __forceinline__ void bulk_rows2(int kk, int kw, int nw, const T *__restrict__ G2,
                                           const T *__restrict__ q, int base, int u, int rs,
                                           const int (&alo)[2], const int (&ahi)[2],
                                           const bool (&uok)[2], T (&acc0)[M], T (&acc1)[M]) {
  const int a_first = min(alo[0], alo[1]), a_last = max(ahi[0], ahi[1]);
  constexpr int kPairUnroll = pair_unroll<M>();
  for (int a00 = a_first + rs; a00 <= a_last; a00 += 2 * kPairUnroll) {
    T g2[kPairUnroll][2], vh[kPairUnroll][M], vl[kPairUnroll][2][M];
#pragma unroll
    for (int s = 0; s < kPairUnroll; ++s) {
      const int a = a00 + 2 * s, b = kk - a;
      // higher element (shared) and the lower elements' omega for point p
      const int hw = RIGHT ? base - a + u : base - b + u;
      bool okp[2];
      int gi[2], ql[2];
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const int kwp = kw + p;
        const int iw = RIGHT ? hw : kwp - hw;  // omega of i = (a, iw)
        okp[p] = uok[p] && a >= alo[p] && a <= ahi[p] && iw >= (a == 0 ? 1 : 0) &&
                 iw <= ((a == b) ? kwp / 2 : kwp) && iw <= kwp;
        const int dk = 2 * a - kk, dw = 2 * iw - kwp;
        gi[p] = okp[p] ? (dk < 0 ? -dk : dk) * nw + (dw < 0 ? -dw : dw) : 0;
        // the lower element: j = k_p - i (RIGHT) or i itself
        ql[p] = okp[p] ? (RIGHT ? (b * nw + (kwp - iw)) * M : (a * nw + iw) * M) : 0;
      }
      const bool any = okp[0] || okp[1];
      const int qh = any ? (RIGHT ? (a * nw + hw) * M : (b * nw + hw) * M) : 0;
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        if constexpr (!SEP) g2[s][p] = okp[p] ? G2[gi[p]] : (T)0;
        PlaneVec<T, M>::load(q + ql[p], vl[s][p]);
      }
      PlaneVec<T, M>::load(q + qh, vh[s]);
    }
#pragma unroll
    for (int s = 0; s < kPairUnroll; ++s)
#pragma unroll
      for (int m = 0; m < M; ++m) {
        if constexpr (SEP) {
          acc0[m] = fma(vh[s][m], vl[s][0][m], acc0[m]);
          acc1[m] = fma(vh[s][m], vl[s][1][m], acc1[m]);
        } else {
          acc0[m] = fma(g2[s][0], vh[s][m] * vl[s][0][m], acc0[m]);
          acc1[m] = fma(g2[s][1], vh[s][m] * vl[s][1][m], acc1[m]);
        }
      }
  }
}

template <typename T, int M, bool SEP>
__device__ void point2_bulk(const RecArgs &A, int kk, int kw, bool has1, int D, int lane) {
  const int base = D - kRecBL, arow = kk / 2 + 1, nw = A.nw;
  const int u = lane & (kRecBL - 1), rs = lane >> 4;
  int aRlo[2], aRhi[2], aLlo[2], aLhi[2];
  bool uR[2], uL[2];
  bool live[2];
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const int kwp = kw + p, d = kk + kwp;
    live[p] = (p == 0 || has1) && A.S[(long long)kk * nw + kwp] > 0.0;
    const int uR0 = max(0, (d + 1) / 2 - base), uL0 = max(0, d / 2 - base + 1);
    aRlo[p] = max(0, base + uR0 - kwp);
    aRhi[p] = min(arow - 1, D - 1);
    aLlo[p] = max(0, kk - D + 1);
    aLhi[p] = arow - 1;
    uR[p] = live[p] && uR0 < kRecBL && u >= uR0;
    uL[p] = live[p] && uL0 < kRecBL && u >= uL0;
    if (!(live[p] && uR0 < kRecBL)) aRhi[p] = -1;  // no right rows for this point
    if (!(live[p] && uL0 < kRecBL)) aLhi[p] = -1;
  }
  if (!live[0] && !live[1]) return;
  T acc0[M], acc1[M];
#pragma unroll
  for (int m = 0; m < M; ++m) acc0[m] = acc1[m] = (T)0;
  const T *G2 = static_cast<const T *>(A.G2);
  const T *q = static_cast<const T *>(A.q);
  if (max(aRhi[0], aRhi[1]) >= 0)
    bulk_rows2<true, T, M, SEP>(kk, kw, nw, G2, q, base, u, rs, aRlo, aRhi, uR, acc0, acc1);
  if (max(aLhi[0], aLhi[1]) >= 0)
    bulk_rows2<false, T, M, SEP>(kk, kw, nw, G2, q, base, u, rs, aLlo, aLhi, uL, acc0, acc1);
  warp_sum<T, M>(acc0);
  warp_sum<T, M>(acc1);
  if (lane == 0) {
    T *ac = static_cast<T *>(A.acc);
    const long long k0 = (long long)kk * nw + kw;
#pragma unroll
    for (int m = 0; m < M; ++m) {
      if (live[0]) ac[k0 * M + m] += acc0[m];
      if (live[1]) ac[(k0 + 1) * M + m] += acc1[m];
    }
  }
}

// The fringe runs by lattice rows: warp w of a CTA walks row kk = row0 + w
// (row0 = kRowWarps g for the CTA's row group g) through the block's levels
// in order.  A point (kk, kw) on level d needs, besides points of its own
// row (finished earlier by the same warp), the point (kk - 1, kw) on level
// d - 1 (the pair {(1, 0), k - (1, 0)}) and points (kk - lk, kw - lw) with
// lk, lw >= 1 on levels <= d - 2.  Finishing (kk - 1, kw) required (kk - 2,
// kw) finished, and so on down the rows, so row kk - 1 having finished level
// d - 1 implies that row kk - lk has finished level d - lk, and row kk - 1
// having finished level d - 2 (the point (kk - 1, kw - 1)) that row kk - lk
// has finished level d - 1 - lk: one wait on the row below covers every
// lower row.  Levels below the block are complete at its start (grid
// barrier).  A row's progress (1 + its last finished level) is kept in
// shared memory for the next warp of the CTA and, for the CTA's last row, in
// row_done for the first warp of the next row group.  Waits are bounded like
// the grid barrier; a warp that gives up raises the abort state and the grid
// barrier after the block then fails for every CTA.
//
// The values a point reads are on chip where they can be: the h (or q) of
// the group's points on the block's levels (written there as they are
// finalized), the lattice corner (levels < BL: the low element of every
// fringe pair), and each point's S and bulk sum (prefetched at the block's
// start).  Only partners on rows below the group come from global memory,
// through L2 (they were written by another SM).
constexpr int kRowWarps = kRecThreads / 32;

template <typename T, int M>
struct FringeSmem {
  T band[kRowWarps][kRecBL][M];    // by (row - row0, level - D)
  T corner[kRecBL][kRecBL][M];     // h(lk, lw) for lk + lw < BL, else 0
  T bulk[kRowWarps][kRecBL][M];    // bulk sum of the row's point on level D + t
  double S[kRowWarps][kRecBL];
  double e2[kRowWarps][kRecBL];    // a_k^2, b_k^2 (separable forms), difference sums (mixed)
  double e2k[kRowWarps][kRecBL];
  double ds[kRowWarps][kRecBL];
  // the low points (lk, lw), lw >= 1, of the fringe pairs in level order:
  // the first t (t + 1) / 2 entries are those of a point t levels into its block
  unsigned char pl[kRecBL * (kRecBL - 1) / 2][2];
  int colnz;  // some corner point (lk, 0), 1 <= lk < BL, has h != 0
};
constexpr int kFringeSmem = 33792;  // bytes, the larger of the FP32 and FP64 layouts
static_assert(sizeof(FringeSmem<float, 8>) <= kFringeSmem &&
                  sizeof(FringeSmem<double, 1>) <= kFringeSmem,
              "fringe shared memory");

// M planes of a point from shared or global memory (generic address); the
// global ones are read through L2 (ld.cg), never from a stale L1 line.
template <typename T, int M>
struct PlaneLd;
template <>
struct PlaneLd<float, 8> {
  static __device__ __forceinline__ void smem(const float *p, float (&v)[8]) {
    const float4 a = reinterpret_cast<const float4 *>(p)[0];
    const float4 b = reinterpret_cast<const float4 *>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  }
  static __device__ __forceinline__ void gmem(const float *p, float (&v)[8]) {
    const float4 a = __ldcg(reinterpret_cast<const float4 *>(p));
    const float4 b = __ldcg(reinterpret_cast<const float4 *>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  }
};
template <>
struct PlaneLd<float, 4> {
  static __device__ __forceinline__ void smem(const float *p, float (&v)[4]) {
    const float4 a = *reinterpret_cast<const float4 *>(p);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  }
  static __device__ __forceinline__ void gmem(const float *p, float (&v)[4]) {
    const float4 a = __ldcg(reinterpret_cast<const float4 *>(p));
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  }
};
template <>
struct PlaneLd<double, 1> {
  static __device__ __forceinline__ void smem(const double *p, double (&v)[1]) { v[0] = *p; }
  static __device__ __forceinline__ void gmem(const double *p, double (&v)[1]) { v[0] = __ldcg(p); }
};
template <>
struct PlaneLd<double, 3> {
  static __device__ __forceinline__ void smem(const double *p, double (&v)[3]) {
    v[0] = p[0];
    v[1] = p[1];
    v[2] = p[2];
  }
  static __device__ __forceinline__ void gmem(const double *p, double (&v)[3]) {
    v[0] = __ldcg(p);
    v[1] = __ldcg(p + 1);
    v[2] = __ldcg(p + 2);
  }
};

// One fringe pair {l, k - l}, l = (lk, lw): the partner p = k - l on level
// d - |l| from the band (rows of the group) or from global memory, zero
// when the pair does not exist (ok false); then its term into acc, with h_l
// from the corner.  The loads of several pairs are issued before their terms.
template <typename T, int M>
__device__ __forceinline__ void fringe_load(const RecArgs &A, const FringeSmem<T, M> &F, int kk,
                                            int kw, int D, int w, int lk, int lw, bool ok,
                                            T (&vp)[M]) {
  if (!ok) {
#pragma unroll
    for (int m = 0; m < M; ++m) vp[m] = (T)0;
    return;
  }
  const int ep = kk + kw - lk - lw - D;  // level of the partner - D
  if (lk <= w)
    PlaneLd<T, M>::smem(&F.band[w - lk][ep][0], vp);
  else
    PlaneLd<T, M>::gmem(static_cast<const T *>(A.q) + ((size_t)(kk - lk) * A.nw + kw - lw) * M,
                        vp);
}

template <typename T, int M, bool SEP>
__device__ __forceinline__ void fringe_fma(const RecArgs &A, const FringeSmem<T, M> &F, int kk,
                                           int kw, int lk, int lw, bool ok, const T (&vp)[M],
                                           T (&acc)[M]) {
  T vl[M];
  PlaneLd<T, M>::smem(&F.corner[ok ? lk : 0][ok ? lw : 0][0], vl);
  if constexpr (SEP) {
#pragma unroll
    for (int m = 0; m < M; ++m) acc[m] = fma(vl[m], vp[m], acc[m]);
  } else {
    const int dk = 2 * lk - kk, dw = 2 * lw - kw;
    const T g2 = ok ? static_cast<const T *>(A.G2)[(size_t)(dk < 0 ? -dk : dk) * A.nw +
                                                     (dw < 0 ? -dw : dw)]
                    : (T)0;
#pragma unroll
    for (int m = 0; m < M; ++m) acc[m] = fma(g2, vl[m] * vp[m], acc[m]);
  }
}

constexpr int kFringeUnroll = 3;

__device__ __forceinline__ bool wait_row(const RecArgs &A, const volatile unsigned int *s_done,
                                         int row, int row0, int lev, int lane,
                                         long long limit = 1ll << 22) {
  int ok = 1;
  if (lane == 0) {
    long long spins = 0;
    for (;;) {
      unsigned int v;
      if (row >= row0)
        v = s_done[row - row0];
      else
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(A.row_done + row)
                     : "memory");
      if (v > (unsigned int)lev) break;
      if ((++spins & 255) == 0 && *(volatile int *)A.abort) {
        ok = 0;
        break;
      }
      if (spins > limit) {
        ok = 0;
        atomicOr(A.bar, kBarAbort);
        atomicExch(A.abort, 1);
        break;
      }
    }
    __threadfence_block();
  }
  __syncwarp();
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

__device__ __forceinline__ void publish_row(const RecArgs &A, volatile unsigned int *s_done, int w,
                                            int kk, int d, int lane) {
  __syncwarp();
  if (lane == 0) {
    if (w == kRowWarps - 1)
      asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(A.row_done + kk), "r"(d + 1)
                   : "memory");
    __threadfence_block();
    s_done[w] = (unsigned int)(d + 1);
  }
}

// Fringe of a point at level d in [D, D + BL): the pairs whose higher
// element lies on a level in [D, d).  Their other element l has level
// 1 .. d - D < BL <= D, so each such pair is {l, k - l} for exactly one
// low lattice point l: the t(t+3)/2 points of levels 1..t, t = d - D.
// The t(t+1)/2 pairs with lw >= 1 are summed, reduced over the warp and
// added to the bulk sum once row kk - 1 has finished level d - 2; the t with
// lw = 0 (zero unless some corner point (lk, 0) has h != 0: the workloads'
// spectra vanish at omega = 0) once it has finished level d - 1, which also
// keeps the rows' progress a chain.  So after that last wait only the
// finalisation (and, where they are not zero, the column pairs) remain.
// Publishes the row's progress.  Returns false when a wait gave up (the
// point is then left unpublished).
template <typename T, int M, bool SEP>
__device__ bool point_fringe(const RecArgs &A, FringeSmem<T, M> &F, int kk, int kw, int D,
                             int row0, int w, volatile unsigned int *s_done, int lane) {
  const long long k = (long long)kk * A.nw + kw;
  const int d = kk + kw, t = d - D;
  T acc[M];
#pragma unroll
  for (int m = 0; m < M; ++m) acc[m] = (T)0;
  if (t >= 1 && kw >= 1) {
    if (kk >= 1 && d - 2 >= D && !wait_row(A, s_done, kk - 1, row0, d - 2, lane)) return false;
    const int e_end = t * (t + 1) / 2;
    for (int e0 = lane; e0 < e_end; e0 += 32 * kFringeUnroll) {
      T vp[kFringeUnroll][M];
      int2 lp[kFringeUnroll];
      bool ok[kFringeUnroll];
#pragma unroll
      for (int s = 0; s < kFringeUnroll; ++s) {
        const int e = e0 + 32 * s;
        const int ec = e < e_end ? e : 0;
        lp[s] = make_int2(F.pl[ec][0], F.pl[ec][1]);
        ok[s] = e < e_end && lp[s].x <= kk && lp[s].y <= kw;
        fringe_load<T, M>(A, F, kk, kw, D, w, lp[s].x, lp[s].y, ok[s], vp[s]);
      }
#pragma unroll
      for (int s = 0; s < kFringeUnroll; ++s)
        fringe_fma<T, M, SEP>(A, F, kk, kw, lp[s].x, lp[s].y, ok[s], vp[s], acc);
    }
  }
  warp_sum<T, M>(acc);  // every lane holds the sums of every plane
  T tt = (T)0;
#pragma unroll
  for (int m = 0; m < M; ++m)
    if (m == lane) tt = acc[m];
  if (lane < M) tt += F.bulk[w][t][lane];
  if (t >= 1 && kk >= 1) {
    if (!wait_row(A, s_done, kk - 1, row0, d - 1, lane)) return false;
    if (F.colnz) {  // the pairs {(lk, 0), (kk - lk, kw)}, lk = 1..t, one lane each
      const int lk = lane + 1;
      const bool ok = lk <= t && lk <= kk;
      T vp[M], c[M];
#pragma unroll
      for (int m = 0; m < M; ++m) c[m] = (T)0;
      fringe_load<T, M>(A, F, kk, kw, D, w, lk, 0, ok, vp);
      fringe_fma<T, M, SEP>(A, F, kk, kw, lk, 0, ok, vp, c);
      warp_sum<T, M>(c);
#pragma unroll
      for (int m = 0; m < M; ++m)
        if (m == lane) tt += c[m];
    }
  }
  if (lane < M) {
    T h = (T)0;
    if (!(F.S[w][t] > 0.0))
      point_zero<T, M>(A, k, lane);
    else
      h = finalize_plane<T, M>(A, k, lane, tt, F.e2[w][t], F.e2k[w][t], F.ds[w][t]);
    F.band[w][t][lane] = h;
  }
  publish_row(A, s_done, w, kk, d, lane);
  return true;
}

// The fringe of block [D, D + BL): row groups of kRowWarps rows over the
// CTAs (group g on CTA g - g_lo mod gridDim.x, a CTA's groups in increasing
// order, so every wait is on a group started earlier).  Returns false when a
// wait gave up.
template <typename T, int M, bool SEP>
__device__ bool fringe_rows(const RecArgs &A, FringeSmem<T, M> &F, int D,
                            volatile unsigned int *s_done, int lane) {
  const int w = threadIdx.x >> 5;
  const int dend = min(D + kRecBL, A.nlev);
  const int r_lo = max(0, D - A.nw + 1), r_hi = min(A.nk - 1, dend - 1);
  const int g_lo = r_lo / kRowWarps, g_hi = r_hi / kRowWarps;
  bool live = true;
  for (int g = g_lo + (int)blockIdx.x; g <= g_hi; g += gridDim.x) {  // uniform over the CTA
    const int row0 = g * kRowWarps, kk = row0 + w;
    if (lane == 0) s_done[w] = 0;
    __syncthreads();
    if (kk >= r_lo && kk <= r_hi) {
      const int kw0 = max(0, D - kk), kw1 = min(A.nw - 1, dend - 1 - kk);
      const int t0 = kk + kw0 - D, np = kw1 - kw0 + 1;
      // S and the bulk sums of the row's points (written by other SMs before
      // the grid barrier: read through L2); FFT form: half the diagonal term
      for (int i = lane; i < np * M; i += 32) {
        const int pi = i / M, m = i - pi * M, kw = kw0 + pi, t = t0 + pi;
        const long long k = (long long)kk * A.nw + kw;
        T b = __ldcg(static_cast<const T *>(A.acc) + k * M + m);
        if (A.zr && ((kk | kw) & 1) == 0) {
          const T hh = __ldcg(static_cast<const T *>(A.q) +
                              ((long long)(kk >> 1) * A.nw + (kw >> 1)) * M + m);
          b += (T)0.5 * hh * hh;
        }
        F.bulk[w][t][m] = b;
        if (m == 0) {
          F.S[w][t] = A.S[k];
          F.e2[w][t] = A.e2 ? A.e2[k] : 1.0;
          F.e2k[w][t] = A.e2k ? A.e2k[k] : 1.0;
          F.ds[w][t] = (M == 1 && A.dsum) ? __ldcg(A.dsum + k) : 0.0;
        }
      }
      __syncwarp();
      for (int kw = kw0; kw <= kw1 && live; ++kw)
        live = point_fringe<T, M, SEP>(A, F, kk, kw, D, row0, w, s_done, lane);
    }
    __syncthreads();
  }
  return live;
}

// The lattice corner (levels < BL, final after the direct levels) into the
// fringe's shared memory; visible after the next CTA barrier.
template <typename T, int M>
__device__ void load_corner(const RecArgs &A, FringeSmem<T, M> &F) {
  for (int i = threadIdx.x; i < kRecBL * kRecBL * M; i += blockDim.x) {
    const int lk = i / (kRecBL * M), lw = (i / M) % kRecBL, m = i % M;
    T v = (T)0;
    if (lk + lw < kRecBL && lk < A.nk && lw < A.nw)
      v = __ldcg(static_cast<const T *>(A.q) + ((size_t)lk * A.nw + lw) * M + m);
    F.corner[lk][lw][m] = v;
  }
  if (threadIdx.x == 0) {  // pair table: level L = 1..BL-1, lk = 0..L-1, lw = L - lk
    int e = 0;
    for (int L = 1; L < kRecBL; ++L)
      for (int lk = 0; lk < L; ++lk, ++e) {
        F.pl[e][0] = (unsigned char)lk;
        F.pl[e][1] = (unsigned char)(L - lk);
      }
    F.colnz = 0;
  }
  __syncthreads();
  if (threadIdx.x < 32) {  // column points (lk, 0), 1 <= lk < BL
    int nz = 0;
    for (int i = threadIdx.x; i < (kRecBL - 1) * M; i += 32) {
      const int lk = 1 + i / M, m = i % M;
      nz |= F.corner[lk][0][m] != (T)0;
    }
    nz = __any_sync(0xffffffffu, nz);
    if (threadIdx.x == 0) F.colnz = nz;
  }
}

// ---- separable envelope: the bulk as an online FFT self-convolution ----
// With g = a_i a_j b_k every pair term of a plane is h_i h_j (h = a^2 q), and
// i + j = k is d_i + d_j = d_k with kk_i + kk_j = kk_k, so the pairs of the
// points of a level form a 2-D self-convolution of h over (level, kk).  A
// divide and conquer over levels (leaves of kRecBL levels, sizes 2L = 2 BL,
// 4 BL, ...) supplies it online: before leaf [D, D + BL) the product of the
// node with mid D (L = BL 2^{v2(D / BL)}, l0 = D - L) adds to the levels
// [D, D + L) every ordered pair (d1, d2) with d1 in [l0, D) and d2 in
// [0, 2L) in either order (l0 > 0; then 2L <= l0), or with both in [0, L)
// (l0 = 0).  When leaf D starts, every ordered pair with both levels below D
// has been added exactly once (the pair's larger level and d first fall in
// different halves of one node, which adds it), so the leaf's bulk is half
// the ordered sum plus half the diagonal term h_{k/2}^2, and the fringe adds
// the pairs with a part in [D, d) as before.
//
// A product on a 2L x Nc grid over (level offset o, kk):
//   z[o][kk] = h(l0 + o, kk) [o < L] + i h(o, kk)   (l0 > 0),
//   z[o][kk] = h(o, kk) [o < L]                      (l0 = 0),
// so that Im (z * z) = 2 A * B and Re (z * z) = A * A; z * z comes from one
// transform direction, F(F(z)^2)[-o, -kk] = 2L Nc (z * z)[o, kk] (cyclic).
// The cyclic length 2L in o suffices: the wanted offsets [L, 2L) could only
// meet aliases from [3L, 4L), beyond the support [0, 3L - 1); Nc >= nk +
// min(2L, nk) - 1 keeps kk free of aliases.  Three phases, a grid barrier
// after each: rows along kk; columns along o, squared, along o again and
// stored at negated o; rows along kk again, read at negated kk, added to
// acc.  Returns false when a barrier gave up.
template <typename T, int M>
__device__ __forceinline__ T sep_h(const RecArgs &A, int d, int kk, int m) {
  const int kw = d - kk;
  if (d == 0 || kk >= A.nk || kw < 0 || kw >= A.nw) return (T)0;
  return static_cast<const T *>(A.q)[((long long)kk * A.nw + kw) * M + m];
}

template <typename T, int M>
__device__ bool sep_product(const RecArgs &A, int l0, int log2L, unsigned int &g,
                            typename Vec2<T>::type *buf) {
  using T2 = typename Vec2<T>::type;
  const int L = 1 << log2L, L2 = 2 * L, Nc = 1 << A.log2Nc;
  const unsigned int nb = gridDim.x;
  T2 *Z = static_cast<T2 *>(A.zr);
  const T2 *tw = static_cast<const T2 *>(A.twr);
  // rows: z along kk
  for (int it = blockIdx.x; it < L2 * M; it += gridDim.x) {
    const int m = it / L2, o = it - m * L2;
    T2 *row = Z + ((size_t)m * L2 + o) * Nc;
    if (l0 == 0 && o >= L) {  // a zero row (uniform over the CTA)
      for (int kk = threadIdx.x; kk < Nc; kk += blockDim.x) row[kk] = T2{};
      continue;
    }
    for (int kk = threadIdx.x; kk < Nc; kk += blockDim.x) {
      T2 v;
      v.x = o < L ? sep_h<T, M>(A, l0 + o, kk, m) : (T)0;
      v.y = l0 > 0 ? sep_h<T, M>(A, o, kk, m) : (T)0;
      buf[rp(brev(kk, A.log2Nc))] = v;
    }
    __syncthreads();
    fft_stages<false>(buf, 1, A.log2Nc, tw);
    for (int kk = threadIdx.x; kk < Nc; kk += blockDim.x) row[kk] = buf[rp(kk)];
    __syncthreads();
  }
  if (!grid_barrier(A.bar, A.abort, nb * g++)) return false;
  // columns: along o, square, along o, store at negated o (rows [L, 2L)),
  // TC columns per CTA: enough groups for every CTA where there are columns
  // for them (the FP64 pipe of one SM would otherwise carry a whole product)
  const int cs = fft_col_stride(L2);
  int TC = Nc;
  while (TC > 1 && (TC * cs > A.zcap || (Nc / TC) * M < (int)gridDim.x)) TC >>= 1;
  const int ng = Nc / TC;
  for (int it = blockIdx.x; it < ng * M; it += gridDim.x) {
    const int m = it / ng, c0 = (it - m * ng) * TC;
    T2 *base = Z + (size_t)m * L2 * Nc + c0;
    for (int t = threadIdx.x; t < L2 * TC; t += blockDim.x) {
      const int r = t / TC, c = t - r * TC;
      buf[c * cs + brev(r, log2L + 1)] = base[(size_t)r * Nc + c];
    }
    __syncthreads();
    fft_stages<true>(buf, TC, log2L + 1, tw);
    for (int t = threadIdx.x; t < L2 * TC; t += blockDim.x) {
      const int c = t >> (log2L + 1), r = t & (L2 - 1), rb = brev(r, log2L + 1);
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
    fft_stages<true>(buf, TC, log2L + 1, tw);
    for (int t = threadIdx.x; t < L * TC; t += blockDim.x) {
      const int r = L + t / TC, c = t % TC;
      base[(size_t)r * Nc + c] = buf[c * cs + ((L2 - r) & (L2 - 1))];
    }
    __syncthreads();
  }
  if (!grid_barrier(A.bar, A.abort, nb * g++)) return false;
  // rows again: along kk, read at negated kk, half the ordered sum into acc
  const T inv = (T)0.5 / ((T)L2 * (T)Nc);
  T *ac = static_cast<T *>(A.acc);
  for (int it = blockIdx.x; it < L * M; it += gridDim.x) {
    const int m = it / L, o = L + (it - m * L), d = l0 + o;
    if (d >= A.nlev) continue;  // uniform over the CTA
    const T2 *row = Z + ((size_t)m * L2 + o) * Nc;
    for (int kk = threadIdx.x; kk < Nc; kk += blockDim.x) buf[rp(brev(kk, A.log2Nc))] = row[kk];
    __syncthreads();
    fft_stages<false>(buf, 1, A.log2Nc, tw);
    const int kk0 = max(0, d - A.nw + 1), kk1 = min(d, A.nk - 1);
    for (int kk = kk0 + threadIdx.x; kk <= kk1; kk += blockDim.x) {
      const T2 v = buf[rp((Nc - kk) & (Nc - 1))];
      ac[((long long)kk * A.nw + (d - kk)) * M + m] += (l0 > 0 ? v.y : v.x) * inv;
    }
    __syncthreads();
  }
  return grid_barrier(A.bar, A.abort, nb * g++);
}

// Bulk items [b, e) of phase D (point pairs of the FP32 search pass, else
// points) drawn by whole warps from the ticket counter tk, the next ticket
// drawn while the current item is summed.  Tickets run from the end of the
// range: items of higher lattice rows (more row pairs, the longer ones) are
// drawn first, so that the short ones fill the tail before the barrier.
template <typename T, int M, bool SEP>
__device__ __forceinline__ void bulk_items(const RecArgs &A, unsigned int *tk, int b, int e,
                                           int D, int lane) {
  constexpr bool kPairs = sizeof(T) == sizeof(float);
  const int dend = min(2 * D, A.nlev);
  int t = 0;
  if (lane == 0) t = (int)atomicAdd(tk, 1u);
  t = __shfl_sync(0xffffffffu, t, 0);
  while (b + t < e) {
    int tn = 0;
    if (lane == 0) tn = (int)atomicAdd(tk, 1u);
    if constexpr (kPairs) {
      const int2 pt = A.pairs[e - 1 - t];
      const bool has1 = pt.y + 1 <= min(A.nw - 1, dend - 1 - pt.x);
      point2_bulk<T, M, SEP>(A, pt.x, pt.y, has1, D, lane);
    } else {
      const int2 pt = A.pts[e - 1 - t];
      point_bulk<T, M, SEP>(A, pt.x, pt.y, D, lane);
    }
    t = __shfl_sync(0xffffffffu, tn, 0);
  }
}

// One recursion pass.  Levels d = kk + kw: every part of a pair of Pi(k)
// lies on a lower level.  Each pair {i, j} of a point is assigned to the
// higher of its two levels, M(i, j) in [ceil(d/2), d).  The pass runs:
//   levels 0 .. BL-1 directly, one grid barrier per level;
//   then for D = BL, 2 BL, ...: a bulk phase adding every pair with
//   M in [D - BL, D) to every point of levels [D, 2D) (M >= d/2 bounds the
//   points that have any) -- its points of levels [D, D + BL) first, then
//   one barrier, then for each level d of [D, D + BL) the fringe (pairs with
//   M in [D, d)) and the finalisation of q by the CTAs of the lattice's row
//   groups while every other CTA adds the phase's pairs to the points of
//   levels [D + BL, 2D) (which no fringe level of the block reads; the
//   fringe CTAs join them when their rows are done), and a barrier.
// Per plane m (one eps value each)
//   sum_b2(k) = eps_m^2 dk dw sum_{Pi(k)} g^2 q_i q_j,  q_k = 1/(1 - sum_b2)
// (b_p^2 = eps^2 g^2 dk dw q_i q_j for |B| = eps g sqrt(S_i S_j S_k)).  Each
// point's sums are formed by one warp at a time in a fixed order, so the
// result does not depend on scheduling.  T = double, M = 1 is the exact
// pass, M = 3 the same at three eps values (the last pass of FP64 plans);
// T = float, M = 8 evaluates eight eps values at once to locate eps.
// SEP: the envelope is separable on i + j = k (g^2 = a_i^2 a_j^2 b_k^2), q
// holds h = a^2 q and the pair terms are h_i h_j (no g^2 read).
template <typename T, int M, bool SEP>
__global__ void __launch_bounds__(kRecThreads, 1) k_rec_pass(RecArgs A) {
  __shared__ unsigned int s_done[kRowWarps];
  // dynamic shared memory: the fringe's state, then (FFT form of the
  // separable bulk only) kRecSmem for its grids -- the other passes leave that
  // space to the L1 cache of their bulk loads
  extern __shared__ __align__(16) unsigned char rec_smem[];
  FringeSmem<T, M> &F = *reinterpret_cast<FringeSmem<T, M> *>(rec_smem);
  const int lane = threadIdx.x & 31;
  // consecutive points (neighbours on a level, of similar cost) go to
  // different SMs
  const int gw = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  unsigned int g = 1;  // barriers passed, counting the next one
  const unsigned int nb = gridDim.x;
  T *ac = static_cast<T *>(A.acc);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < A.nl * M;
       i += (long long)gridDim.x * blockDim.x)
    ac[i] = (T)0;
  if (!grid_barrier(A.bar, A.abort, nb * g++)) return;
  // the points of level d are kk = lo .. hi, lo = max(0, d - nw + 1),
  // hi = min(d, nk - 1), in the order of the level list; their coordinates
  // are formed here rather than loaded, which keeps a memory round trip off
  // every level's critical path
  const int d0 = min(kRecBL, A.nlev);
  for (int d = 0; d < d0; ++d) {
    const int lo = max(0, d - A.nw + 1), n = min(d, A.nk - 1) - lo + 1;
    for (int i = gw; i < n; i += nwarps) point_direct<T, M, SEP>(A, lo + i, d - lo - i, lane);
    if (!grid_barrier(A.bar, A.abort, nb * g++)) return;
  }
  load_corner<T, M>(A, F);  // levels < BL are final: read after the next barrier
  for (int D = kRecBL, ph = 1; D < A.nlev; D += kRecBL, ++ph) {
    if (A.zr) {  // separable envelope: the bulk by one FFT product
      const int log2L = (31 - __clz(kRecBL)) + (__ffs(D / kRecBL) - 1);
      if (!sep_product<T, M>(A, D - (1 << log2L), log2L, g,
                             reinterpret_cast<typename Vec2<T>::type *>(rec_smem + kFringeSmem)))
        return;
    } else {
      // bulk: warps take items in turn from the phase's ticket counters
      // (the FP32 search pass, bound by its q loads, takes the points in
      // pairs; the FP64 pass, bound by its FP64 pipe, one at a time); the
      // items of the fringe block [D, D + BL) before the barrier
      constexpr bool kPairs = sizeof(T) == sizeof(float);
      const int pb = kPairs ? A.pair_off[ph - 1] : A.pt_off[D];
      const int pm = kPairs ? A.pair_mid[ph] : A.pt_off[min(D + kRecBL, A.nlev)];
      bulk_items<T, M, SEP>(A, A.bar + ph, pb, pm, D, lane);
      if (!grid_barrier(A.bar, A.abort, nb * g++)) return;
    }
    // fringe levels by lattice rows (a warp that gave up skips its remaining
    // points; the grid barrier after the block then fails for every CTA)
    fringe_rows<T, M, SEP>(A, F, D, s_done, lane);
    if (!A.zr) {  // the rest of the bulk phase, beside the fringe
      constexpr bool kPairs = sizeof(T) == sizeof(float);
      const int pm = kPairs ? A.pair_mid[ph] : A.pt_off[min(D + kRecBL, A.nlev)];
      const int pe = kPairs ? A.pair_off[ph] : A.pt_off[min(2 * D, A.nlev)];
      bulk_items<T, M, SEP>(A, A.bar + A.tk_def + ph, pm, pe, D, lane);
    }
    if (!grid_barrier(A.bar, A.abort, nb * g++)) return;
  }
}

// Linear pass: L_k = dk dw sum_{Pi(k)} g^2 [S_i > 0][S_j > 0] (q == 1), the
// small-eps slope of sum_b2 used to bracket eps.  No level dependencies.  A
// CTA takes lattice row kk, kLinOut consecutive omega outputs (one thread
// each) and one part of the row's row pairs (a = part, part + nparts, ...):
// per row pair (a, b = kk - a) it stages the S > 0 masks of rows a and b in
// shared memory, and every thread sums
//   R(kw) = sum_iw EwSq[|2 iw - kw|] m_a[iw] m_b[kw - iw]
// over iw <= kw (iw <= kw/2 on the centre row, i = 0 skipped), weighted by
// EkSq[kk - 2a], into part[part][k].  Splitting a row's row pairs over
// kLinParts CTAs keeps the long rows (kk/2 + 1 row pairs) off the critical
// path; k_rec_linear_sum adds the parts in a fixed order.  FP32 terms (only
// the scale of eps is taken from it).  CTAs go in order of decreasing kk.
constexpr int kLinOut = 128;
constexpr int kLinParts = 8;

__global__ void __launch_bounds__(kLinOut) k_rec_linear(int nk, int nw, const double *__restrict__ S,
                                                        const float *__restrict__ EkSq,
                                                        const float *__restrict__ EwSq,
                                                        float *__restrict__ part) {
  extern __shared__ float lin_smem[];
  float *ma = lin_smem, *mb = lin_smem + nw, *ew = lin_smem + 2 * nw;  // [nw] each
  const int nblk = (nw + kLinOut - 1) / kLinOut;
  const int cta = (int)(blockIdx.x / kLinParts), prt = (int)(blockIdx.x % kLinParts);
  const int kk = nk - 1 - cta / nblk;
  const int kw = (cta % nblk) * kLinOut + threadIdx.x;
  const int kwmax = min(nw, (cta % nblk) * kLinOut + kLinOut);  // outputs < kwmax
  for (int i = threadIdx.x; i < nw; i += blockDim.x) ew[i] = EwSq[i];
  float acc = 0.f;
  for (int a = prt; a <= kk / 2; a += kLinParts) {
    const int b = kk - a;
    __syncthreads();
    for (int i = threadIdx.x; i < kwmax; i += blockDim.x) {
      ma[i] = S[(size_t)a * nw + i] > 0.0 ? 1.f : 0.f;
      mb[i] = S[(size_t)b * nw + i] > 0.0 ? 1.f : 0.f;
    }
    __syncthreads();
    if (kw < nw) {
      const int lim = (a == b) ? kw / 2 : kw;
      float r = 0.f;
      for (int iw = (a == 0 ? 1 : 0); iw <= lim; ++iw) {
        const int dw = 2 * iw - kw;
        r = fmaf(ew[dw < 0 ? -dw : dw], ma[iw] * mb[kw - iw], r);
      }
      acc = fmaf(EkSq[kk - 2 * a], r, acc);
    }
  }
  if (kw < nw) part[(size_t)prt * nk * nw + (size_t)kk * nw + kw] = acc;
}

__global__ void k_rec_linear_sum(long long n, const double *__restrict__ S,
                                 const float *__restrict__ part, double *__restrict__ sb2,
                                 double dkdw) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  float t = 0.f;
  for (int j = 0; j < kLinParts; ++j) t += part[(size_t)j * n + k];
  sb2[k] = S[k] > 0.0 ? dkdw * (double)t : 0.0;
}

// Difference-pair sums of the mixed-sign interactions for every point at the
// iterate q (FP64, q = 0 where S = 0): for k = (kk, kw), kw >= 1, S_k > 0,
//   D_k = sum_{ia=0..kk} EkSq[|2 ia - kk|] sum_{jw=1..nw-1-kw}
//         EwSq[kw + 2 jw] q(ia, kw + jw) q(kk - ia, jw)
// -- i = (ia, kw + jw) on the point's sheet, j = (kk - ia, jw) on the other,
// g^2 of the signed frequency difference kw + 2 jw (EwSq holds 2 nw
// entries); both sheets share q, so one D serves both.  One warp per point,
// lanes along jw (coalesced rows of q), a fixed order of additions.
__global__ void __launch_bounds__(256) k_rec_diff(int nk, int nw, const double *__restrict__ S,
                                                  const double *__restrict__ q,
                                                  const double *__restrict__ EkSq,
                                                  const double *__restrict__ EwSq,
                                                  double *__restrict__ D) {
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gw >= (long long)nk * nw) return;
  const int kk = (int)(gw / nw), kw = (int)(gw - (long long)kk * nw);
  double acc = 0.0;
  if (kw >= 1 && S[gw] > 0.0) {
    const int J = nw - 1 - kw;
    for (int ia = 0; ia <= kk; ++ia) {
      const double *qa = q + (size_t)ia * nw + kw;  // qa[jw] = q(ia, kw + jw)
      const double *qb = q + (size_t)(kk - ia) * nw;
      double r = 0.0;
      for (int jw = 1 + lane; jw <= J; jw += 32) r = fma(EwSq[kw + 2 * jw], qa[jw] * qb[jw], r);
      const int dk = 2 * ia - kk;
      acc = fma(EkSq[dk < 0 ? -dk : dk], r, acc);
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) D[gw] = acc;
}

}  // namespace srm3
