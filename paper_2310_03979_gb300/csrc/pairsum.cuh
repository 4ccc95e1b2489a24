// pairsum.cuh - the pair sum that assembles the coefficients C^s_k (FFT form,
// Sec. 4.3): the plain FP64 form and the FP32 form (persistent, warp-specialised,
// TMA-fed, packed two-lane arithmetic).  Included by sample.cu only.
#pragma once

#include <cuda.h>  // CUtensorMap

#include "srm3_internal.cuh"

namespace srm3 {

// ---------------------------------------------------------------------------
// a4 + a5, plain FP64 form: one warp per (k, sheet-sample), exact canonical
// half (centre row iw <= kw/2), W_ij = c_k Ek[|ik-jk|] Ew[iw-jw] rebuilt per
// pair:
//   A = sum_a sum_iw Ek[kk-2a] Ew[2iw-kw] y(a,iw) y(kk-a,kw-iw)
//   C = P_k y_k + c_k e^{i beta} A
// The point's terms are laid end to end (row pairs a <= kk/2 of kw + 1 terms,
// the centre row to kw/2), lane l taking terms l, l + 32, ...; a fixed
// butterfly adds the lanes' sums.  A warp per (k, sheet-sample) keeps every
// lane of the narrow FP64 pipe busy however few samples share a launch, and
// the order of every sum is the same for any launch.
// Mixed plans (mixed != 0) add the difference pairs: i = (a, kw + jw) on this
// sheet-sample's sheet and j = (kk - a, jw) on the other sheet of the same
// sample (sheet-sample ss ^ 1), 0 <= a <= kk, 1 <= jw <= nw - 1 - kw, kw >= 1,
// W = c_k Ek[|2a - kk|] Ew[kw + 2 jw] (the signed frequency difference), laid
// out after the sum pairs in the same way.
__global__ void __launch_bounds__(256) k_pairsum_f64(
    int nk, int nw, int SS, int SSpad, int rowstride, const double2 *__restrict__ y,
    const double2 *__restrict__ y0, const double *__restrict__ Ek,
    const double *__restrict__ Ews, int ew_off, const double *__restrict__ Pk,
    const double *__restrict__ ck, double cb, double sb, double2 *__restrict__ C,
    int mixed, int row_lo, int row_hi) {
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const long long nl = (long long)nk * nw;
  if (gw >= nl * SS) return;  // uniform over the warp
  const long long k = gw / SS;
  const int ss = (int)(gw - k * SS);
  const int kk = (int)(k / nw), kw = (int)(k - (long long)kk * nw);
  if (kk < row_lo || kk >= row_hi) return;  // rows of another shard
  const double2 *yl = y + ss;
  double ar = 0.0, ai = 0.0;
  const int W = kw + 1, E = (kk / 2 + 1) * W;
  for (int e = lane; e < E; e += 32) {
    const int a = e / W, iw = e - a * W, b = kk - a;
    if (iw > ((a == b) ? kw / 2 : kw)) continue;
    const double2 u = yl[(size_t)(a * rowstride + kPad + iw) * SSpad];
    const double2 v = yl[(size_t)(b * rowstride + kPad + kw - iw) * SSpad];
    const double w = Ek[kk - 2 * a] * Ews[ew_off + 2 * iw - kw];
    const double pr = u.x * v.x - u.y * v.y;
    const double pi = u.x * v.y + u.y * v.x;
    ar = fma(w, pr, ar);
    ai = fma(w, pi, ai);
  }
  if (mixed && kw >= 1 && kw < nw - 1) {
    const double2 *yo = y + (ss ^ 1);  // the other sheet of the same sample
    const int L = nw - 1 - kw, E2 = (kk + 1) * L;
    for (int e = lane; e < E2; e += 32) {
      const int a = e / L, jw = 1 + e - a * L;
      const double2 u = yl[(size_t)(a * rowstride + kPad + kw + jw) * SSpad];
      const double2 v = yo[(size_t)((kk - a) * rowstride + kPad + jw) * SSpad];
      const int dk = 2 * a - kk;
      const double w = Ek[dk < 0 ? -dk : dk] * Ews[ew_off + kw + 2 * jw];
      const double pr = u.x * v.x - u.y * v.y;
      const double pi = u.x * v.y + u.y * v.x;
      ar = fma(w, pr, ar);
      ai = fma(w, pi, ai);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    ar += __shfl_xor_sync(0xffffffffu, ar, o);
    ai += __shfl_xor_sync(0xffffffffu, ai, o);
  }
  if (lane != 0) return;
  double2 yk = (k == 0) ? y0[ss] : yl[((size_t)kk * rowstride + kPad + kw) * SSpad];
  double c = ck[k], P = Pk[k];
  double pr = c * (ar * cb - ai * sb), pim = c * (ar * sb + ai * cb);
  C[((size_t)ss * nk + kk) * nw + kw] = make_double2(P * yk.x + pr, P * yk.y + pim);
}


// ---------------------------------------------------------------------------
// a4 + a5, FP32 form: persistent, warp-specialised, packed two-lane
// arithmetic.
//
// Work unit: a super-tile of 32 outputs kws0..kws0+31 of lattice row kk for
// one group of 64 sheet-samples.  Units are ordered by decreasing cost and
// dealt to the resident CTAs in a snake order; a CTA walks its units one
// after another.  Every lane carries two sheet-samples, stored pair-planar
// as {x0, x1, y0, y1} (the layout k_phases writes for FP32 plans), so that
// fma.rn.f32x2 / mul.rn.f32x2 act on both samples at once.
//
// Warps 0-3 compute: warp w owns the 8-output tile kw0 = kws0 + 8w.  Per row
// pair (a, b = kk - a) a thread forms, for r < 8,
//   T_r = sum_iw w(r, iw) y_a[iw] y_b[kw0 + r - iw]
// in blocks of 4 iw: 4 values of y_a and a window of 11 values of y_b serve 32
// (r, iw) products; 7 of the 11 carry over to the next block.  A product is
// w*p*q with the minus sign of the complex product kept in a third
// accumulator:
//   Tx+ += (w px) qx,  Tx- += (w py) qy,  Ty += (w px) qy + (w py) qx,
// six packed instructions for two pair-terms.  Terms with iw > kw read zero
// padding; the centre row a = b runs the full range and is halved with its
// diagonal added back, T = (T_full + w y_{kw/2}^2) / 2.  Row partials are
// merged once per row pair into Kahan-compensated FP32 sums kept in shared
// memory.
//
// Warp 4 produces: the omega range [0, kws0 + 31] of each row pair is
// walked in chunks of 16, and for each chunk one lane stages the 16 y_a rows
// and 48 y_b rows (47 used) of the group with four TMA tile loads of 16 rows
// x 512 bytes through a 2-D tensor map over y (rows outside the lattice read
// the zero padding of y) into one of two stages, signalled by an mbarrier
// with a transaction count.  TABLE: the chunk's W rows of each tile reaching
// the chunk arrive on the same mbarrier by one 512-byte bulk copy per tile
// (the table is chunk-major; the producer's register round trip it replaced
// cost 3 % of the launch), four weights per 16-byte load on the compute side,
// each paired with itself (w, w) in registers for the packed products --
// half the shared-memory loads of storing the pairs, worth 4 % of the launch;
// otherwise the chunk's
// 64-entry window of the omega envelope table Ew is bulk-copied, w =
// Ew[2 iw - kw], each weight paired with itself in registers as above, with the kappa factor Ek[kk - 2a] applied
// per row pair and c_k at the end.
// Half-group mode (at most 32 sheet-samples, W recomputed): the lanes of a
// group would be half empty, so each half-warp takes one of two row pairs
// (a = 2i, 2i + 1) of a work item, on 256-byte rows staged by eight tile
// loads; at the end of the pair the upper half passes its terms to the lower
// half, which merges the two row pairs in order -- the same sums in the same
// order as the full form, so a sample's result does not depend on how many
// samples share its launch.
// The compute warps release a stage through a second mbarrier.  Every wait
// is bounded: past kWaitCycles the waiter raises the CTA's abort flag and
// the error word, all warps leave their loops, and the producer first waits
// (bounded again) for the copies it has in flight.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 f2_fma(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f32x2 f2_mul(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f32x2 f2_dup(float x) {
  f32x2 d;
  asm("mov.b64 %0, {%1, %1};" : "=l"(d) : "f"(x));
  return d;
}
__device__ __forceinline__ float2 f2_split(f32x2 v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}

namespace packed {
constexpr int R = kTileR;                 // outputs per thread (8)
constexpr int U = 4;                      // iw per register block
constexpr int CH = 16;                    // iw per chunk
constexpr int NB = CH / U;                // register blocks per chunk
constexpr int NV = R + U - 1;             // y_b window per block (11)
constexpr int NE = 2 * U + R - 2;         // envelope window per block (14)
constexpr int BOX_ROWS = 16;              // rows per TMA tile load
constexpr int LANES = 32;                 // sample pairs per group
constexpr int ROW_BYTES = LANES * 16;     // one staged row
constexpr int EWIN = 64;                  // (w, w) pairs per stage, envelope
constexpr int NK = 4 * R;                 // Kahan sums per compute thread
constexpr long long kWaitCycles = 4000000000LL;  // about 2 s at 2 GHz
static_assert(kTileU == CH && kTileR == R, "W table chunks: one 512-byte span per tile");
static_assert(NB * U == CH && (NE % 2) == 0 && CH == BOX_ROWS, "block shape");

// Tile shape of the FP32 pair sum: NC compute warps, each one 8-wide output
// tile, make one super-tile of SW = 8 NC outputs (a work unit with one
// sample group).  NC = 4 (32-wide) suits long rows; NC = 2 (16-wide) halves
// the triangle of work across a super-tile's warps in the last chunks of
// every row pair (the low tiles of a super-tile need fewer omega values), at
// the cost of staging 48 rows per chunk for two warps instead of 64 for four.
// The sums of an output and their order do not depend on NC: a warp walks
// the same chunks and register blocks of its tile either way.
template <int NC_>
struct Shape {
  static constexpr int NC = NC_;                    // compute warps = tiles per super-tile
  static constexpr int NCT = 32 * NC;               // compute threads
  static constexpr int NT = NCT + 32;               // plus the producer warp
  static constexpr int SW = NC * R;                 // super-tile width
  static constexpr int YB_ROWS = CH + SW - 1;       // y_b rows per chunk
  static constexpr int YB_BOXES = (YB_ROWS + BOX_ROWS - 1) / BOX_ROWS;
  static constexpr int YROWS = CH + YB_BOXES * BOX_ROWS;  // staged rows per chunk
  static constexpr int STAGE_Y = YROWS * LANES;     // float4 per stage
  static constexpr int STAGE_W = NC * R * CH;       // float2 slots per stage (W: the first half)
  static constexpr int CTAS_PER_SM = NC == 4 ? 2 : 3;  // the launch bounds' residency
  static_assert(2 * (CH - 1) + SW <= EWIN && EWIN <= STAGE_W, "envelope window of a chunk");
  static_assert(kPad >= SW + CH + 1, "staged rows stay inside the zero padding of y");
};
}  // namespace packed

template <int NC>
inline size_t pairsum_f32p_smem() {
  using namespace packed;
  using S = Shape<NC>;
  return 128 + (size_t)2 * S::STAGE_Y * sizeof(float4) + (size_t)2 * S::STAGE_W * sizeof(float2) +
         (size_t)2 * NK * S::NCT * sizeof(float);
}

__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long *b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *b, unsigned bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long *b) {
  asm volatile(
      "{\n .reg .b64 st;\n mbarrier.arrive.release.cta.shared::cta.b64 st, [%0];\n}" ::"r"(
          smem_u32(b))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for the phase of b with the given parity.  Returns false when the
// CTA's abort flag is up or the wait passes kWaitCycles (then it raises the
// flag and the error word).
__device__ __forceinline__ bool mbar_wait(unsigned long long *b, unsigned parity,
                                          volatile int *abort, int *err,
                                          long long limit = packed::kWaitCycles) {
  if (mbar_try_wait(b, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(b, parity)) {
    if (*abort) return false;
    if (clock64() - t0 > limit) {
      *abort = 1;
      atomicOr(err, 1);
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes,
                                         unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// 2-D TMA tile load (box from the tensor map) at element coordinates (x, y).
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ ulonglong2 lds_pair(const void *p) {
  return *reinterpret_cast<const ulonglong2 *>(p);
}

// Per-plan view of an FP32 pair-sum launch.  The tensor map comes first:
// TMA descriptors need 64-byte alignment.
struct PsDesc {  // aligned as CUtensorMap
  CUtensorMap ymap;      // y as rows of SSpad/2 float4; boxes of 512 B x 16 rows
  const float4 *y;       // pair-planar rows (kPad zero entries each side)
  const float2 *y0;      // y at k = 0 per sheet-sample
  const float *Ek;       // kappa envelope factor (recompute)
  const float *Ew;       // omega envelope by signed offset (recompute; w0 at ew_off)
  const float *W;        // W table (table storage)
  const long long *toff; // W-table offset per tile (table storage)
  const float *Pk, *ck;  // pure and pair factors
  float2 *C;             // coefficients out [ss][kk][kw]
  const int2 *order;     // super-tiles (kk, kws0) by decreasing cost (single-plan launch)
  // Shape groups (samples of several plans with one lattice, W recomputed):
  // per-sample pure and pair factors; NULL = Pk, ck for every sample.
  const float *const *pk_of;
  const float *const *ck_of;
  int nk, nw, SS, SSpad, rowstride, ntw, ew_off, table, G;
  // half = 1: at most 32 sheet-samples (16 lanes) with W recomputed; the two
  // half-warps then take two row pairs of a work item (a = 2i and 2i + 1),
  // reading 256-byte rows through a tensor map with 64-float boxes
  int half;
  // sep = 1: W recomputed in separable form, g(i, j) = a_i a_j b_k on the
  // pairs of k -- the omega factor a_w is in y, the kappa factor aK[row]
  // weights each row pair, b_k is in ck: the register blocks multiply y
  // rows alone and no envelope window is staged
  int sep;
  const float *aK;
  float cb, sb;          // cos / sin of the biphase
};

// Work unit {plan, kk, kws0, grp}: the 32-wide super-tile of row kk starting
// at kws0, for sample group grp of plan `plan`.
// Row-pair steps of a unit: kk/2 + 1 row pairs, two per step in half mode.
__host__ __device__ __forceinline__ int ps_rowsteps(int kk, int half) {
  return half ? (kk / 2 + 2) / 2 : kk / 2 + 1;
}
__host__ __device__ __forceinline__ int ps_nitems(int kk, int kws0, int half, int sw) {
  using namespace packed;
  return ps_rowsteps(kk, half) * ((kws0 + sw + CH - 1) / CH);
}
// The k-th unit of CTA c out of C (snake order over the cost-sorted units).
__device__ __forceinline__ int ps_unit_id(int k, int c, int C) {
  return k * C + ((k & 1) ? C - 1 - c : c);
}
// Unit u: units[u] in a batch launch; in a single-plan launch (units ==
// NULL) super-tile d0.order[u / G] for group u % G of plan d0.
__device__ __forceinline__ int4 ps_get_unit(int u, const PsDesc &d0,
                                            const int4 *__restrict__ units) {
  if (units) return units[u];
  const int2 t = d0.order[u / d0.G];
  return make_int4(0, t.x, t.y, u - (u / d0.G) * d0.G);
}

// One staged chunk for one compute warp: all register blocks of the chunk.
// RS: float4 per staged row (32, or 16 in half mode).
template <bool TABLE, int RS, bool SEPW = false>
__device__ __forceinline__ void ps_chunk(const float4 *__restrict__ pa,
                                         const float4 *__restrict__ pb,
                                         const float2 *__restrict__ pw,
                                         const float2 *__restrict__ pe, int i0, int kw0,
                                         f32x2 (&Txp)[packed::R], f32x2 (&Txm)[packed::R],
                                         f32x2 (&Ty)[packed::R]) {
  using namespace packed;
  // y_b rows by their offset m = v + U (NB - 1 - blk) from the lowest row any
  // block reads: every row keeps one name.
  ulonglong2 Bc[NV + U * (NB - 1)];
#pragma unroll
  for (int blk = 0; blk < NB; ++blk) {
    if (i0 + blk * U > kw0 + R - 1) break;
    ulonglong2 A[U];
#pragma unroll
    for (int uu = 0; uu < U; ++uu) A[uu] = lds_pair(pa + (blk * U + uu) * RS);
    const int m0 = U * (NB - 1 - blk);
#pragma unroll
    for (int v = (blk == 0 ? 0 : NV - U); v < NV; ++v) {
      const int vv = blk == 0 ? v : v - (NV - U);  // rows not loaded yet
      Bc[m0 + vv] = lds_pair(pb + (m0 + vv - U * (NB - 1)) * RS);
    }
    const ulonglong2 *B = Bc + m0;
    if constexpr (SEPW) {
      // separable form: the weights are in the rows, four packed FMAs per
      // product of two sheet-samples; omega outermost and the two updates
      // of Ty[r] in separate sweeps over the outputs, so that no FMA waits
      // on the one before it (every accumulator's terms keep their order)
#pragma unroll
      for (int uu = 0; uu < U; ++uu) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int v = r - uu + U - 1;
          Txp[r] = f2_fma(A[uu].x, B[v].x, Txp[r]);
          Txm[r] = f2_fma(A[uu].y, B[v].y, Txm[r]);
        }
#pragma unroll
        for (int r = 0; r < R; ++r) Ty[r] = f2_fma(A[uu].x, B[r - uu + U - 1].y, Ty[r]);
#pragma unroll
        for (int r = 0; r < R; ++r) Ty[r] = f2_fma(A[uu].y, B[r - uu + U - 1].x, Ty[r]);
      }
    } else if (TABLE) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const float4 w4 =
            *reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(pw) + r * CH + blk * U);
        const f32x2 w[U] = {f2_dup(w4.x), f2_dup(w4.y), f2_dup(w4.z), f2_dup(w4.w)};
#pragma unroll
        for (int uu = 0; uu < U; ++uu) {
          const int v = r - uu + U - 1;
          const f32x2 wpx = f2_mul(w[uu], A[uu].x), wpy = f2_mul(w[uu], A[uu].y);
          Txp[r] = f2_fma(wpx, B[v].x, Txp[r]);
          Txm[r] = f2_fma(wpy, B[v].y, Txm[r]);
          Ty[r] = f2_fma(wpx, B[v].y, Ty[r]);
          Ty[r] = f2_fma(wpy, B[v].x, Ty[r]);
        }
      }
    } else {
      // the block's NE = 14 weights: three 16-byte loads and one 8-byte load
      const float *pef = reinterpret_cast<const float *>(pe) + 8 * blk;
      float e[NE];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const float4 v4 = reinterpret_cast<const float4 *>(pef)[j];
        e[4 * j] = v4.x;
        e[4 * j + 1] = v4.y;
        e[4 * j + 2] = v4.z;
        e[4 * j + 3] = v4.w;
      }
      const float2 v2 = reinterpret_cast<const float2 *>(pef)[6];
      e[12] = v2.x;
      e[13] = v2.y;
#pragma unroll
      for (int r = 0; r < R; ++r) {
#pragma unroll
        for (int uu = 0; uu < U; ++uu) {
          const int v = r - uu + U - 1;
          const f32x2 w = f2_dup(e[2 * uu - r + R - 1]);
          const f32x2 wpx = f2_mul(w, A[uu].x), wpy = f2_mul(w, A[uu].y);
          Txp[r] = f2_fma(wpx, B[v].x, Txp[r]);
          Txm[r] = f2_fma(wpy, B[v].y, Txm[r]);
          Ty[r] = f2_fma(wpx, B[v].y, Ty[r]);
          Ty[r] = f2_fma(wpy, B[v].x, Ty[r]);
        }
      }
    }
  }
}

// The FP32 pair sum over one plan (d0, with descs = units = NULL) or any
// number of plans (descs[p] describes plan p, units[0..nunits) the work units
// sorted by decreasing cost).  MIXED = false compiles the full-group path
// alone (every descriptor has half = 0); MIXED = true also takes half-mode
// descriptors.
// FORM: kPsSeparable when every descriptor of the launch has W recomputed in
// separable form (the kernel holds those register blocks alone), else
// kPsAnyForm (each descriptor's form decided at run time).
constexpr int kPsAnyForm = 0, kPsSeparable = 2;

template <bool MIXED, int NCW, int FORM = kPsAnyForm>
__global__ void __launch_bounds__(packed::Shape<NCW>::NT, packed::Shape<NCW>::CTAS_PER_SM)
    k_pairsum_f32p(const __grid_constant__ PsDesc d0, const PsDesc *__restrict__ descs,
                   const int4 *__restrict__ units, int nunits, int *__restrict__ err) {
  using namespace packed;
  using S = Shape<NCW>;
  constexpr int NC = S::NC, NCT = S::NCT, SW = S::SW, YB_BOXES = S::YB_BOXES, YROWS = S::YROWS;
  constexpr int STAGE_Y = S::STAGE_Y, STAGE_W = S::STAGE_W;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned long long *full = reinterpret_cast<unsigned long long *>(smem_raw);  // [2]
  unsigned long long *empty = full + 2;                                         // [2]
  volatile int *abort = reinterpret_cast<volatile int *>(full + 4);
  float4 *sy = reinterpret_cast<float4 *>(smem_raw + 128);    // [2][STAGE_Y]
  float2 *sw = reinterpret_cast<float2 *>(sy + 2 * STAGE_Y);  // [2][STAGE_W] (W or envelope)
  float *kst = reinterpret_cast<float *>(sw + 2 * STAGE_W);   // [2 NK][NCT]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    mbar_init(&full[0], 32);
    mbar_init(&full[1], 32);
    mbar_init(&empty[0], NCT);
    mbar_init(&empty[1], NCT);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == NC) {
    // ---------------- producer ----------------
    unsigned q = 0;
    bool ok = true;
    for (int k = 0; ok; ++k) {
      const int u = ps_unit_id(k, blockIdx.x, gridDim.x);
      if (u >= nunits) break;
      const int4 un = ps_get_unit(u, d0, units);
      const PsDesc &d = descs ? descs[un.x] : d0;
      const int kk = un.y, kws0 = un.z, nch = (kws0 + SW + CH - 1) / CH;
      const int half = MIXED ? d.half : 0;
      const int nitems = ps_nitems(kk, kws0, half, SW), rs = d.rowstride;
      const bool tab = FORM == kPsAnyForm && d.table != 0;
      const bool sepf = FORM == kPsSeparable || d.sep != 0;
      const int x = un.w * LANES * 4;  // first float of the group in a row of y
      int a = 0, c = 0;
      for (int item = 0; item < nitems; ++item, ++q) {
        const int stage = q & 1;
        if (q >= 2 && !mbar_wait(&empty[stage], ((q >> 1) & 1) ^ 1, abort, err)) {
          ok = false;
          break;
        }
        const int i0 = c * CH;
        if (lane == 0) {
          // TABLE: the chunk's W rows of each tile whose rows reach it, one
          // contiguous 512-byte span per tile (the table is chunk-major)
          int ntile = 0;
          if (tab)
            for (int t = 0; t < NC; ++t) {
              const int k0 = kws0 + R * t;
              if (k0 < d.nw && c * CH < ((k0 + R + kTileU - 1) / kTileU) * kTileU) ++ntile;
            }
          const unsigned tx = YROWS * ROW_BYTES +
                              (tab ? ntile * R * CH * (unsigned)sizeof(float)
                                   : (sepf ? 0u : EWIN * (unsigned)sizeof(float)));
          mbar_expect_tx(&full[stage], tx);
          // one row pair (full rows), or two in half mode (half rows each; a
          // second row pair past the centre repeats the first and is
          // weighted 0 by the compute warps)
          for (int h = 0; h <= half; ++h) {
            const int ah = half ? min(2 * a + h, kk / 2) : a, bh = kk - ah;
            const int rw = half ? LANES / 2 : LANES;  // float4 per staged row
            float4 *dst = sy + stage * STAGE_Y + h * YROWS * (LANES / 2);
            tma_load_2d(dst, &d.ymap, x, ah * rs + kPad + i0, &full[stage]);
            const int jrow = bh * rs + kPad + kws0 - i0 - CH + 1;
#pragma unroll
            for (int j = 0; j < YB_BOXES; ++j)
              tma_load_2d(dst + (CH + BOX_ROWS * j) * rw, &d.ymap, x, jrow + BOX_ROWS * j,
                          &full[stage]);
          }
          if (!tab) {
            if (!sepf)
              bulk_g2s(sw + stage * STAGE_W, d.Ew + d.ew_off + 2 * i0 - kws0 - (SW - 1),
                       EWIN * sizeof(float), &full[stage]);
          } else {
            for (int t = 0; t < NC; ++t) {  // the tiles counted above
              const int k0 = kws0 + R * t;
              const int ncht = ((k0 + R + kTileU - 1) / kTileU) * kTileU / CH;
              if (k0 >= d.nw || c >= ncht) continue;
              const long long base = d.toff[kk * d.ntw + k0 / R];
              bulk_g2s(reinterpret_cast<float *>(sw + stage * STAGE_W) + t * R * CH,
                       d.W + base + ((long long)a * ncht + c) * R * CH,
                       R * CH * (unsigned)sizeof(float), &full[stage]);
            }
          }
        }
        mbar_arrive(&full[stage]);
        if (++c == nch) {
          c = 0;
          ++a;
        }
      }
    }
    if (!ok) {  // leave no bulk copy in flight: wait (bounded) for the last two stages
      for (unsigned j = (q >= 2 ? q - 2 : 0); j < q; ++j) {
        const long long t0 = clock64();
        while (!mbar_try_wait(&full[j & 1], (j >> 1) & 1) && clock64() - t0 < kWaitCycles) {
        }
      }
    }
    return;
  }

  // ---------------- compute warps ----------------
  float *kacc = kst + tid, *kcmp = kst + NK * NCT + tid;
  unsigned q = 0;
  for (int k = 0;; ++k) {
    const int u = ps_unit_id(k, blockIdx.x, gridDim.x);
    if (u >= nunits) break;
    const int4 un = ps_get_unit(u, d0, units);
    const PsDesc &d = descs ? descs[un.x] : d0;
    const int kk = un.y, kws0 = un.z, grp = un.w, nw = d.nw;
    const bool tab = FORM == kPsAnyForm && d.table != 0;
    const bool sepf = FORM == kPsSeparable || d.sep != 0;
    const int kw0 = kws0 + R * warp, nch = (kws0 + SW + CH - 1) / CH;
    const int half = MIXED ? d.half : 0;
    const int nitems = ps_nitems(kk, kws0, half, SW);
    const int hl = half ? lane >> 4 : 0;        // which row pair of a step this lane takes
    const int ln = half ? lane & 15 : lane;     // the lane's sample pair within the group
    const size_t SP = (size_t)d.SSpad / 2;  // float4 per lattice entry
    const bool tile_ok = kw0 < nw;
#pragma unroll
    for (int j = 0; j < NK; ++j) kacc[j * NCT] = kcmp[j * NCT] = 0.f;
    f32x2 Txp[R], Txm[R], Ty[R];
#pragma unroll
    for (int r = 0; r < R; ++r) Txp[r] = Txm[r] = Ty[r] = 0ull;
    int a = 0, c = 0;
    for (int item = 0; item < nitems; ++item, ++q) {
      const int stage = q & 1;
      if (!mbar_wait(&full[stage], (q >> 1) & 1, abort, err)) return;
      const int i0 = c * CH;
      if (tile_ok) {
        const float2 *pw = reinterpret_cast<const float2 *>(
            reinterpret_cast<const float *>(sw + stage * STAGE_W) + warp * R * CH);
        const float2 *pe = reinterpret_cast<const float2 *>(
            reinterpret_cast<const float *>(sw + stage * STAGE_W) + (SW - R) - R * warp);
        if (half) {
          const float4 *pa = sy + stage * STAGE_Y + hl * YROWS * (LANES / 2) + ln;
          const float4 *pb = pa + (CH + R * warp + CH - U) * (LANES / 2);
          if (sepf)
            ps_chunk<false, LANES / 2, true>(pa, pb, pw, pe, i0, kw0, Txp, Txm, Ty);
          else
            ps_chunk<false, LANES / 2>(pa, pb, pw, pe, i0, kw0, Txp, Txm, Ty);
        } else {
          const float4 *pa = sy + stage * STAGE_Y + lane;
          const float4 *pb = pa + (CH + R * warp + CH - U) * LANES;
          if (tab)
            ps_chunk<true, LANES>(pa, pb, pw, pe, i0, kw0, Txp, Txm, Ty);
          else if (sepf)
            ps_chunk<false, LANES, true>(pa, pb, pw, pe, i0, kw0, Txp, Txm, Ty);
          else
            ps_chunk<false, LANES>(pa, pb, pw, pe, i0, kw0, Txp, Txm, Ty);
        }
      }
      mbar_arrive(&empty[stage]);
      if (tile_ok && c == nch - 1) {  // row pair complete: centre-row halving and merge
        // Half mode: lanes 16-31 hand the odd row pair's terms to lanes 0-15,
        // which merge both row pairs in order -- the same sums, in the same
        // order, as the full mode, so a sample's result does not depend on
        // how many samples share its launch.
        const int ah = half ? 2 * a + hl : a;  // this lane's row pair
        const bool live = ah <= kk / 2;
        const int b = kk - (live ? ah : a);
        // the row pair's kappa weight: none for the table (in W), the
        // envelope at kk - 2a, or in separable form aK[a] aK[kk - a]
        // (the merge and the epilogue round every operation explicitly, so
        // that the kernel compiled for one weight form gives the bits of the
        // general one: a sample's result does not depend on the launch)
        auto rw = [&](int a_) {
          return sepf ? __fmul_rn(d.aK[a_], d.aK[kk - a_]) : d.Ek[kk - 2 * a_];
        };
        const float rowfac = tab ? 1.0f : (live ? rw(ah) : 0.0f);
        const bool odd_live = half && 2 * a + 1 <= kk / 2;
        const float rowfac_odd = odd_live ? rw(2 * a + 1) : 0.0f;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const float2 xp = f2_split(Txp[r]), xm = f2_split(Txm[r]), yy = f2_split(Ty[r]);
          float v[4] = {xp.x - xm.x, xp.y - xm.y, yy.x, yy.y};
          if (live && ah == b) {
            const int kw = kw0 + r;
            if ((kw & 1) == 0 && kw < nw) {
              const float4 h = d.y[((size_t)ah * d.rowstride + kPad + (kw >> 1)) * SP +
                                   (size_t)grp * LANES + ln];
              // the tile's offset in the table and its padded row length,
              // formed here (once per unit) rather than kept across the chunks
              const int my_L = ((kw0 + R + kTileU - 1) / kTileU) * kTileU;
              const float w0 =
                  tab ? d.W[d.toff[kk * d.ntw + kw0 / R] +
                            (((long long)ah * (my_L / CH) + ((kw >> 1) / CH)) * R + r) * CH +
                            ((kw >> 1) % CH)]
                      : (sepf ? 1.0f : d.Ew[d.ew_off]);
              const float t[4] = {__fsub_rn(__fmul_rn(h.x, h.x), __fmul_rn(h.z, h.z)),
                                  __fsub_rn(__fmul_rn(h.y, h.y), __fmul_rn(h.w, h.w)),
                                  __fmul_rn(__fmul_rn(2.f, h.x), h.z),
                                  __fmul_rn(__fmul_rn(2.f, h.y), h.w)};
#pragma unroll
              for (int j = 0; j < 4; ++j)
                v[j] = __fmul_rn(0.5f, __fadd_rn(v[j], __fmul_rn(w0, t[j])));
            } else {
#pragma unroll
              for (int j = 0; j < 4; ++j) v[j] *= 0.5f;
            }
          }
          float vo[4];  // the odd row pair (half mode, lanes 0-15)
#pragma unroll
          for (int j = 0; j < 4; ++j) vo[j] = half ? __shfl_down_sync(0xffffffffu, v[j], 16) : 0.f;
          if (hl == 0) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {  // Kahan: s += rowfac v with compensation
              float &s_ = kacc[(4 * r + j) * NCT], &cp = kcmp[(4 * r + j) * NCT];
              const float s0 = s_, yv = fmaf(rowfac, v[j], -cp);
              const float tt = s0 + yv;
              cp = (tt - s0) - yv;
              s_ = tt;
            }
            if (odd_live) {
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                float &s_ = kacc[(4 * r + j) * NCT], &cp = kcmp[(4 * r + j) * NCT];
                const float s0 = s_, yv = fmaf(rowfac_odd, vo[j], -cp);
                const float tt = s0 + yv;
                cp = (tt - s0) - yv;
                s_ = tt;
              }
            }
          }
          Txp[r] = Txm[r] = Ty[r] = 0ull;
        }
      }
      if (++c == nch) {
        c = 0;
        ++a;
      }
    }
    if (!tile_ok) continue;
    if (hl) continue;  // half mode: the sums are held by lanes 0-15
    const int ss0 = grp * 2 * LANES + 2 * ln;
    if (ss0 >= d.SS) continue;  // padding lanes
    const float *Pk = d.pk_of ? d.pk_of[ss0 >> 1] : d.Pk;
    const float *ck = d.ck_of ? d.ck_of[ss0 >> 1] : d.ck;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int kw = kw0 + r;
      if (kw >= nw) break;
      const int kidx = kk * nw + kw;
      const float4 yk4 =
          d.y[((size_t)kk * d.rowstride + kPad + kw) * SP + (size_t)grp * LANES + ln];
      const float cf = ck[kidx];  // the pair factor (the table holds the envelopes alone)
      const float P = Pk[kidx];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int ss = ss0 + h;
        if (ss >= d.SS) break;
        const float2 yk = (kidx == 0) ? d.y0[ss] : (h ? make_float2(yk4.y, yk4.w)
                                                       : make_float2(yk4.x, yk4.z));
        const float ar = kacc[(4 * r + h) * NCT] - kcmp[(4 * r + h) * NCT];
        const float ai = kacc[(4 * r + 2 + h) * NCT] - kcmp[(4 * r + 2 + h) * NCT];
        float2 out;
        out.x = fmaf(P, yk.x, __fmul_rn(cf, __fsub_rn(__fmul_rn(ar, d.cb), __fmul_rn(ai, d.sb))));
        out.y = fmaf(P, yk.y, __fmul_rn(cf, __fadd_rn(__fmul_rn(ar, d.sb), __fmul_rn(ai, d.cb))));
        d.C[((size_t)ss * d.nk + kk) * nw + kw] = out;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Difference pairs of mixed plans, FP32 (W recomputed): a second persistent
// launch after the sum pairs that adds, for k = (kk, kw), kw >= 1,
//   C^s_k += c_k e^{i beta} sum_{a=0..kk} Ek[|2a - kk|]
//            sum_{jw >= 1} Ew[kw + 2 jw] y^s_a[kw + jw] y^{-s}_{kk-a}[jw].
// The same pipeline as the sum pairs, with the Toeplitz window running the
// other way: per row pair (a, b = kk - a) -- all kk + 1 of them, the two
// parts being on different sheets -- the producer stages, per chunk of 16
// jw, the 16 rows jw of b from ys (the rows of y with the two sheets of each
// lane swapped and omega = 0 zeroed, so that the packed products pair sheet
// + of one part with sheet - of the other and jw = 0 contributes nothing)
// and the 47 rows kws0 + jw .. of a from y, plus the 64-entry window of the
// envelope of the signed difference d = kw + 2 jw starting at kws0 + 2 j0.
// A register block takes U = 4 values of jw (from b) and a window of 11 rows
// of a, of which 7 carry over to the next block.  Rows past the lattice read
// the zero padding of y.  Kahan merge per row pair as in the sum pairs; the
// epilogue adds the result to the coefficients the sum pairs wrote.
struct PsDiffDesc {  // aligned as CUtensorMap
  CUtensorMap amap;    // y: rows of SSpad/2 float4, boxes of 512 B x 16 rows
  CUtensorMap bmap;    // ys, the same shape
  const float *Ek;     // kappa envelope factor by |d|
  const float *Ewd;    // omega envelope of the signed difference, d >= 0
  const float *ck;     // pair factor c_k
  float2 *C;           // coefficients [ss][kk][kw], updated in place
  const int2 *order;   // super-tiles (kk, kws0) by decreasing difference cost
  int nk, nw, SS, SSpad, rowstride, G;
  float cb, sb;        // cos / sin of the biphase
};

__host__ __device__ __forceinline__ int psd_nch(int nw, int kws0) {
  return (nw - kws0 + packed::CH - 1) / packed::CH;
}

template <int RS>
__device__ __forceinline__ void ps_chunk_diff(const float4 *__restrict__ pb,
                                              const float4 *__restrict__ pa,
                                              const float *__restrict__ pe, int j0, int kw0,
                                              int nw, f32x2 (&Txp)[packed::R],
                                              f32x2 (&Txm)[packed::R], f32x2 (&Ty)[packed::R]) {
  using namespace packed;
  // rows of a by their offset m = U blk + v from the first row of the warp's
  // window: every row keeps one name
  ulonglong2 Ac[NV + U * (NB - 1)];
#pragma unroll
  for (int blk = 0; blk < NB; ++blk) {
    if (j0 + blk * U > nw - 1 - kw0) break;  // the rest reads zero padding only
    ulonglong2 Bv[U];
#pragma unroll
    for (int uu = 0; uu < U; ++uu) Bv[uu] = lds_pair(pb + (blk * U + uu) * RS);
#pragma unroll
    for (int v = (blk == 0 ? 0 : NV - U); v < NV; ++v)
      Ac[U * blk + v] = lds_pair(pa + (U * blk + v) * RS);
    const ulonglong2 *A = Ac + U * blk;
    const float *pef = pe + 8 * blk;  // weights d - (kw0 + 2 (j0 + U blk)) = r + 2 uu
    float e[NE];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float4 v4 = reinterpret_cast<const float4 *>(pef)[j];
      e[4 * j] = v4.x;
      e[4 * j + 1] = v4.y;
      e[4 * j + 2] = v4.z;
      e[4 * j + 3] = v4.w;
    }
    const float2 v2 = reinterpret_cast<const float2 *>(pef)[6];
    e[12] = v2.x;
    e[13] = v2.y;
#pragma unroll
    for (int r = 0; r < R; ++r) {
#pragma unroll
      for (int uu = 0; uu < U; ++uu) {
        const int v = r + uu;
        const f32x2 w = f2_dup(e[r + 2 * uu]);
        const f32x2 wpx = f2_mul(w, Bv[uu].x), wpy = f2_mul(w, Bv[uu].y);
        Txp[r] = f2_fma(wpx, A[v].x, Txp[r]);
        Txm[r] = f2_fma(wpy, A[v].y, Txm[r]);
        Ty[r] = f2_fma(wpx, A[v].y, Ty[r]);
        Ty[r] = f2_fma(wpy, A[v].x, Ty[r]);
      }
    }
  }
}

__global__ void __launch_bounds__(packed::Shape<4>::NT, 2) k_pairsum_f32d(
    const __grid_constant__ PsDiffDesc d, int nunits, int *__restrict__ err) {
  using namespace packed;
  using S = Shape<4>;
  constexpr int NC = S::NC, NCT = S::NCT, YB_BOXES = S::YB_BOXES, YROWS = S::YROWS;
  constexpr int STAGE_Y = S::STAGE_Y, STAGE_W = S::STAGE_W;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned long long *full = reinterpret_cast<unsigned long long *>(smem_raw);  // [2]
  unsigned long long *empty = full + 2;                                         // [2]
  volatile int *abort = reinterpret_cast<volatile int *>(full + 4);
  float4 *sy = reinterpret_cast<float4 *>(smem_raw + 128);    // [2][STAGE_Y]
  float2 *sw = reinterpret_cast<float2 *>(sy + 2 * STAGE_Y);  // [2][STAGE_W] (envelope)
  float *kst = reinterpret_cast<float *>(sw + 2 * STAGE_W);   // [2 NK][NCT]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    mbar_init(&full[0], 32);
    mbar_init(&full[1], 32);
    mbar_init(&empty[0], NCT);
    mbar_init(&empty[1], NCT);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int rs = d.rowstride;

  if (warp == NC) {
    // ---------------- producer ----------------
    unsigned q = 0;
    bool ok = true;
    for (int k = 0; ok; ++k) {
      const int u = ps_unit_id(k, blockIdx.x, gridDim.x);
      if (u >= nunits) break;
      const int2 t = d.order[u / d.G];
      const int grp = u - (u / d.G) * d.G;
      const int kk = t.x, kws0 = t.y, nch = psd_nch(d.nw, kws0);
      const int nitems = (kk + 1) * nch;
      const int x = grp * LANES * 4;  // first float of the group in a row of y
      int a = 0, c = 0;
      for (int item = 0; item < nitems; ++item, ++q) {
        const int stage = q & 1;
        if (q >= 2 && !mbar_wait(&empty[stage], ((q >> 1) & 1) ^ 1, abort, err)) {
          ok = false;
          break;
        }
        const int j0 = c * CH;
        if (lane == 0) {
          mbar_expect_tx(&full[stage], YROWS * ROW_BYTES + EWIN * (unsigned)sizeof(float));
          float4 *dst = sy + stage * STAGE_Y;
          // the 16 rows jw = j0 .. j0 + 15 of b = kk - a, from the swapped copy
          tma_load_2d(dst, &d.bmap, x, (kk - a) * rs + kPad + j0, &full[stage]);
          // the rows kws0 + j0 .. kws0 + j0 + 47 of a
#pragma unroll
          for (int j = 0; j < YB_BOXES; ++j)
            tma_load_2d(dst + (CH + BOX_ROWS * j) * LANES, &d.amap, x,
                        a * rs + kPad + kws0 + j0 + BOX_ROWS * j, &full[stage]);
          bulk_g2s(sw + stage * STAGE_W, d.Ewd + kws0 + 2 * j0, EWIN * sizeof(float),
                   &full[stage]);
        }
        mbar_arrive(&full[stage]);
        if (++c == nch) {
          c = 0;
          ++a;
        }
      }
    }
    if (!ok) {  // leave no bulk copy in flight: wait (bounded) for the last two stages
      for (unsigned j = (q >= 2 ? q - 2 : 0); j < q; ++j) {
        const long long t0 = clock64();
        while (!mbar_try_wait(&full[j & 1], (j >> 1) & 1) && clock64() - t0 < kWaitCycles) {
        }
      }
    }
    return;
  }

  // ---------------- compute warps ----------------
  float *kacc = kst + tid, *kcmp = kst + NK * NCT + tid;
  const size_t SP = (size_t)d.SSpad / 2;
  (void)SP;
  unsigned q = 0;
  for (int k = 0;; ++k) {
    const int u = ps_unit_id(k, blockIdx.x, gridDim.x);
    if (u >= nunits) break;
    const int2 t = d.order[u / d.G];
    const int grp = u - (u / d.G) * d.G;
    const int kk = t.x, kws0 = t.y, nw = d.nw;
    const int kw0 = kws0 + R * warp, nch = psd_nch(nw, kws0);
    const int nitems = (kk + 1) * nch;
    const bool tile_ok = kw0 < nw;
#pragma unroll
    for (int j = 0; j < NK; ++j) kacc[j * NCT] = kcmp[j * NCT] = 0.f;
    f32x2 Txp[R], Txm[R], Ty[R];
#pragma unroll
    for (int r = 0; r < R; ++r) Txp[r] = Txm[r] = Ty[r] = 0ull;
    int a = 0, c = 0;
    for (int item = 0; item < nitems; ++item, ++q) {
      const int stage = q & 1;
      if (!mbar_wait(&full[stage], (q >> 1) & 1, abort, err)) return;
      if (tile_ok) {
        const float4 *pb = sy + stage * STAGE_Y + lane;
        const float4 *pa = pb + (CH + R * warp) * LANES;
        const float *pe = reinterpret_cast<const float *>(sw + stage * STAGE_W) + R * warp;
        ps_chunk_diff<LANES>(pb, pa, pe, c * CH, kw0, nw, Txp, Txm, Ty);
      }
      mbar_arrive(&empty[stage]);
      if (tile_ok && c == nch - 1) {  // row pair complete: merge
        const int dk = 2 * a - kk;
        const float rowfac = d.Ek[dk < 0 ? -dk : dk];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const float2 xp = f2_split(Txp[r]), xm = f2_split(Txm[r]), yy = f2_split(Ty[r]);
          const float v[4] = {xp.x - xm.x, xp.y - xm.y, yy.x, yy.y};
#pragma unroll
          for (int j = 0; j < 4; ++j) {  // Kahan: s += rowfac v with compensation
            float &s_ = kacc[(4 * r + j) * NCT], &cp = kcmp[(4 * r + j) * NCT];
            const float s0 = s_, yv = fmaf(rowfac, v[j], -cp);
            const float tt = s0 + yv;
            cp = (tt - s0) - yv;
            s_ = tt;
          }
          Txp[r] = Txm[r] = Ty[r] = 0ull;
        }
      }
      if (++c == nch) {
        c = 0;
        ++a;
      }
    }
    if (!tile_ok) continue;
    const int ss0 = grp * 2 * LANES + 2 * lane;
    if (ss0 >= d.SS) continue;  // padding lanes
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int kw = kw0 + r;
      if (kw >= nw) break;
      if (kw == 0) continue;  // omega = 0 takes no difference pairs
      const int kidx = kk * nw + kw;
      const float cf = d.ck[kidx];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int ss = ss0 + h;
        if (ss >= d.SS) break;
        const float ar = kacc[(4 * r + h) * NCT] - kcmp[(4 * r + h) * NCT];
        const float ai = kacc[(4 * r + 2 + h) * NCT] - kcmp[(4 * r + 2 + h) * NCT];
        float2 &o = d.C[((size_t)ss * d.nk + kk) * nw + kw];
        float2 out = o;
        out.x += cf * (ar * d.cb - ai * d.sb);
        out.y += cf * (ar * d.sb + ai * d.cb);
        o = out;
      }
    }
  }
}

}  // namespace srm3
