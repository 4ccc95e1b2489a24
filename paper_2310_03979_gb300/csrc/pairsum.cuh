// pairsum.cuh - the pair sum that assembles the coefficients C^s_k (FFT form,
// Sec. 4.3): the plain FP64 form and the staged FP32 form.  Included by
// sample.cu only.
#pragma once

#include "srm3_internal.cuh"

namespace srm3 {

// ---------------------------------------------------------------------------
// a4 + a5, plain FP64 form: one thread per (k, sheet-sample), exact
// canonical half (centre row iw <= kw/2), W_ij = c_k Ek[|ik-jk|] Ew[iw-jw]
// rebuilt per pair:
//   A = sum_a Ek[kk-2a] sum_iw Ew[2iw-kw] y(a,iw) y(kk-a,kw-iw)
//   C = P_k y_k + c_k e^{i beta} A
__global__ void __launch_bounds__(256) k_pairsum_f64(
    int nk, int nw, int SS, int SSpad, int rowstride, const double2 *__restrict__ y,
    const double2 *__restrict__ y0, const double *__restrict__ Ek,
    const double *__restrict__ Ews, int ew_off, const double *__restrict__ Pk,
    const double *__restrict__ ck, double cb, double sb, double2 *__restrict__ C) {
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int ss = (int)(gid % SSpad);
  const long long k = gid / SSpad;
  if (k >= (long long)nk * nw || ss >= SS) return;
  const int kk = (int)(k / nw), kw = (int)(k - (long long)kk * nw);
  const double2 *yl = y + ss;
  double ar = 0.0, ai = 0.0;
  for (int a = 0; a <= kk / 2; ++a) {
    const int b = kk - a;
    const int lim = (a == b) ? kw / 2 : kw;
    const double2 *pa = yl + (size_t)(a * rowstride + kPad) * SSpad;
    const double2 *pb = yl + (size_t)(b * rowstride + kPad + kw) * SSpad;
    double rr = 0.0, ri = 0.0;
    for (int iw = 0; iw <= lim; ++iw) {
      double2 u = pa[(size_t)iw * SSpad];
      double2 v = pb[-(long long)iw * SSpad];
      double w = Ews[ew_off + 2 * iw - kw];
      double pr = u.x * v.x - u.y * v.y;
      double pi = u.x * v.y + u.y * v.x;
      rr = fma(w, pr, rr);
      ri = fma(w, pi, ri);
    }
    double f = Ek[kk - 2 * a];
    ar = fma(f, rr, ar);
    ai = fma(f, ri, ai);
  }
  double2 yk = (k == 0) ? y0[ss] : yl[((size_t)kk * rowstride + kPad + kw) * SSpad];
  double c = ck[k], P = Pk[k];
  double pr = c * (ar * cb - ai * sb), pim = c * (ar * sb + ai * cb);
  C[((size_t)ss * nk + kk) * nw + kw] = make_double2(P * yk.x + pr, P * yk.y + pim);
}


// ---------------------------------------------------------------------------
// a4 + a5, tiled FP32 form with shared-memory staging.  A CTA (4 warps)
// takes a super-tile of 32 outputs kws0..kws0+31 of lattice row kk for one
// group of 32 sheet-samples; warp w owns the 8-output tile kws0 + 8w and
// each lane one sheet-sample.  Per row pair (a, b = kk - a) a thread forms
//   T_r = sum_iw w(r, iw) y_a[iw] y_b[kw0 + r - iw],  r < 8,
// in 8-wide blocks of iw held in registers: 8 values of y_a and a window of
// 15 values of y_b serve all 64 (r, iw) products of a block.  The omega
// range [0, kws0 + 31] is walked in chunks of 32: the chunk's y_a rows, the
// y_b rows that the four tiles need (63) and, for the table path, the four
// tiles' W rows are copied global -> shared with 16-byte cp.async
// (zero-filled outside the lattice), double-buffered so that the copy of
// chunk t+1 overlaps the arithmetic on chunk t.  Every shared-memory
// operand of the inner loop is a compile-time offset from one base pointer
// per chunk.  Terms with iw > kw read zero padding; the centre row a = b
// runs the full range and is halved with its diagonal added back,
// T = (T_full + w y_{kw/2}^2) / 2.  The row partial T is merged into a
// Kahan-compensated accumulator once per row pair.
// TABLE: w(r, iw) from the W table (which holds c_k and the kappa factor).
// Otherwise w = Ew[2 iw - kw] from a shared copy of the envelope table
// (read as aligned float4 windows), rowfac = Ek[kk - 2a], and c_k is
// applied at the end.
namespace staged {
constexpr int R = kTileR, U = kTileU, ST = kWarpsPerCta, SW = ST * R, CH = 32;
constexpr int NB = CH / U;                    // blocks per chunk
constexpr int YB_ROWS = CH + SW - 1;
constexpr int STAGE_Y = (CH + YB_ROWS) * 32;  // float2 entries per stage
constexpr int STAGE_W = ST * R * CH;          // floats per stage
constexpr int EW = 2 * U + R - 2;             // envelope window per block (22)
constexpr int EW4 = (EW + 3) / 4;             // as float4 (6)
static_assert(STAGE_W == 2 * 128 * 4, "two W copies of 16 bytes per thread");
static_assert(YB_ROWS <= 8 * 8, "eight y_b rows per thread");
}  // namespace staged

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int n = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }

template <bool TABLE>
__global__ void __launch_bounds__(128, 3) k_pairsum_f32s(
    int nk, int nw, int SS, int SSpad, int rowstride, int G, const int2 *__restrict__ order,
    const long long *__restrict__ toff, int ntw, const float2 *__restrict__ y,
    const float2 *__restrict__ y0, const float *__restrict__ Ek,
    const float *__restrict__ Ews_g, int ew_off, int ew_len, const float *__restrict__ W,
    const float *__restrict__ Pk, const float *__restrict__ ck, float cb, float sb,
    float2 *__restrict__ C) {
  using namespace staged;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2 *sy = reinterpret_cast<float2 *>(smem_raw);        // [2][STAGE_Y]
  float *sw = reinterpret_cast<float *>(sy + 2 * STAGE_Y);  // [2][STAGE_W] (table)
  float *ews = sw;                                          // envelope copy (recompute)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (!TABLE) {
    for (int i = tid; i < ew_len; i += blockDim.x) ews[i] = Ews_g[i];
  }
  const int grp = blockIdx.x % G;
  const int2 tk = order[blockIdx.x / G];
  const int kk = tk.x, kws0 = tk.y;
  const int kw0 = kws0 + R * warp;  // this warp's tile
  const bool tile_ok = kw0 < nw;
  const int ss = grp * 32 + lane;
  const size_t SP = (size_t)SSpad;
  const int nrow = kk / 2 + 1;
  const int nch = (kws0 + SW + CH - 1) / CH;
  const int nitems = nrow * nch;

  // copy geometry: thread tid copies 16 bytes (two sheet-samples) at
  // column cpart of rows crow + 8 j
  const int cpart = tid & 15, crow = tid >> 4;
  const float2 *ysrc = y + (size_t)grp * 32 + cpart * 2;
  // W copies: tile cs0 and cs0 + 2 of the super-tile, row cr, float4 cc4
  const int cs0 = tid >> 6, cr = (tid >> 3) & 7, cc4 = tid & 7;
  auto tile_L = [&](int k0) { return ((k0 + R + U - 1) / U) * U; };
  auto tile_base = [&](int k0) -> long long {
    return (TABLE && k0 < nw) ? toff[kk * ntw + k0 / R] : -1;
  };
  const int cL0 = tile_L(kws0 + R * cs0), cL1 = tile_L(kws0 + R * (cs0 + 2));
  const long long cb0 = tile_base(kws0 + R * cs0), cb1 = tile_base(kws0 + R * (cs0 + 2));
  const int my_L = tile_L(kw0);
  const long long my_base = tile_base(kw0);

  auto issue = [&](int item, int stage) {
    if (item < nitems) {
      const int a = item / nch, c = item - a * nch;
      const int b = kk - a, i0 = c * CH;
      float2 *dya = sy + stage * STAGE_Y + crow * 32 + cpart * 2;
      float2 *dyb = dya + CH * 32;
      const float2 *ra = ysrc + (size_t)(a * rowstride + kPad) * SP;
      const float2 *rb = ysrc + (size_t)(b * rowstride + kPad) * SP;
#pragma unroll
      for (int j = 0; j < CH / 8; ++j) {
        const int iw = i0 + crow + 8 * j;
        const bool v = iw < nw;
        cp_async16(dya + j * 8 * 32, ra + (size_t)(v ? iw : 0) * SP, v);
      }
      const int jlo = kws0 - i0 - CH + 1 + crow;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (crow + 8 * j < YB_ROWS) {
          const int jw = jlo + 8 * j;
          const bool v = jw >= 0 && jw < nw;
          cp_async16(dyb + j * 8 * 32, rb + (size_t)(v ? jw : 0) * SP, v);
        }
      }
      if (TABLE) {
        float *dw = sw + stage * STAGE_W + (cs0 * R + cr) * CH + 4 * cc4;
        const int iw = i0 + 4 * cc4;
        const bool v0 = cb0 >= 0 && iw < cL0, v1 = cb1 >= 0 && iw < cL1;
        cp_async16(dw, v0 ? W + cb0 + ((long long)a * R + cr) * cL0 + iw : W, v0);
        cp_async16(dw + 2 * R * CH, v1 ? W + cb1 + ((long long)a * R + cr) * cL1 + iw : W, v1);
      }
    }
    cp_async_commit();
  };

  float2 acc[R], cmp[R], T[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    acc[r] = make_float2(0.f, 0.f);
    cmp[r] = make_float2(0.f, 0.f);
    T[r] = make_float2(0.f, 0.f);
  }

  issue(0, 0);
  issue(1, 1);
  int a = 0, c = 0;
  for (int t = 0; t < nitems; ++t) {
    const int stage = t & 1;
    const int i0 = c * CH;
    cp_async_wait1();
    __syncthreads();
    if (tile_ok) {
      const float2 *pa = sy + stage * STAGE_Y + lane;
      const float2 *pb = pa + (CH + R * warp + CH - U) * 32;
      const float *pw = sw + stage * STAGE_W + warp * R * CH;
      const float *pe = ews + ew_off + 2 * i0 - kw0 - (R - 1);
#pragma unroll
      for (int blk = 0; blk < NB; ++blk) {
        if (i0 + blk * U > kw0 + R - 1) break;
        float2 ya[U], yb[R + U - 1];
#pragma unroll
        for (int u = 0; u < U; ++u) ya[u] = pa[(blk * U + u) * 32];
#pragma unroll
        for (int v = 0; v < R + U - 1; ++v) yb[v] = pb[(v - blk * U) * 32];
        if (TABLE) {
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const float4 w0 = *reinterpret_cast<const float4 *>(pw + r * CH + blk * U);
            const float4 w1 = *reinterpret_cast<const float4 *>(pw + r * CH + blk * U + 4);
            const float w[U] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
            for (int u = 0; u < U; ++u) {
              const float2 p = ya[u], q = yb[r - u + U - 1];
              const float pr = fmaf(p.x, q.x, -p.y * q.y);
              const float pi = fmaf(p.x, q.y, p.y * q.x);
              T[r].x = fmaf(w[u], pr, T[r].x);
              T[r].y = fmaf(w[u], pi, T[r].y);
            }
          }
        } else {
          float e[4 * EW4];
#pragma unroll
          for (int q4 = 0; q4 < EW4; ++q4) {
            const float4 v4 = *reinterpret_cast<const float4 *>(pe + 2 * blk * U + 4 * q4);
            e[4 * q4] = v4.x;
            e[4 * q4 + 1] = v4.y;
            e[4 * q4 + 2] = v4.z;
            e[4 * q4 + 3] = v4.w;
          }
#pragma unroll
          for (int r = 0; r < R; ++r) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
              const float w = e[2 * u - r + R - 1];
              const float2 p = ya[u], q = yb[r - u + U - 1];
              const float pr = fmaf(p.x, q.x, -p.y * q.y);
              const float pi = fmaf(p.x, q.y, p.y * q.x);
              T[r].x = fmaf(w, pr, T[r].x);
              T[r].y = fmaf(w, pi, T[r].y);
            }
          }
        }
      }
      if (c == nch - 1) {  // row pair complete: centre-row halving and merge
        const int b = kk - a;
        if (a == b) {
          const float2 *ra = y + ss + (size_t)(a * rowstride + kPad) * SP;
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const int kw = kw0 + r;
            if ((kw & 1) == 0 && kw < nw) {
              const float2 h = ra[(size_t)(kw >> 1) * SP];
              const float w0 =
                  TABLE ? W[my_base + ((long long)a * R + r) * my_L + (kw >> 1)] : ews[ew_off];
              T[r].x = 0.5f * (T[r].x + w0 * (h.x * h.x - h.y * h.y));
              T[r].y = 0.5f * (T[r].y + w0 * (2.f * h.x * h.y));
            } else {
              T[r].x *= 0.5f;
              T[r].y *= 0.5f;
            }
          }
        }
        const float rowfac = TABLE ? 1.0f : Ek[kk - 2 * a];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          float yx = fmaf(rowfac, T[r].x, -cmp[r].x);
          float tx = acc[r].x + yx;
          cmp[r].x = (tx - acc[r].x) - yx;
          acc[r].x = tx;
          float yy = fmaf(rowfac, T[r].y, -cmp[r].y);
          float ty = acc[r].y + yy;
          cmp[r].y = (ty - acc[r].y) - yy;
          acc[r].y = ty;
          T[r] = make_float2(0.f, 0.f);
        }
      }
    }
    __syncthreads();
    issue(t + 2, stage);
    if (++c == nch) {
      c = 0;
      ++a;
    }
  }
  if (!tile_ok || ss >= SS) return;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int kw = kw0 + r;
    if (kw >= nw) break;
    const int k = kk * nw + kw;
    const float2 yk = (k == 0) ? y0[ss] : y[ss + ((size_t)kk * rowstride + kPad + kw) * SP];
    const float ar = acc[r].x - cmp[r].x, ai = acc[r].y - cmp[r].y;
    const float cf = TABLE ? 1.0f : ck[k];
    const float P = Pk[k];
    float2 out;
    out.x = fmaf(P, yk.x, cf * (ar * cb - ai * sb));
    out.y = fmaf(P, yk.y, cf * (ar * sb + ai * cb));
    C[((size_t)ss * nk + kk) * nw + kw] = out;
  }
}

}  // namespace srm3
