// sample.cu - per-sample work of the SRM3 sampler: Philox4x32-10 phases,
// the O(N^2) pair sum that assembles the coefficients C^s_k (FFT form,
// Sec. 4.3), and the hand-written 2-D inverse FFT to u(x,t).
#include <algorithm>
#include <cstring>

#include "srm3_internal.cuh"

namespace srm3 {

static int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of
// (hi, lo) = M * x on words 0 and 2, mixed with words 1 and 3 and the key;
// the key advances by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
    uint32_t hi0 = __umulhi(m0, c.x), lo0 = m0 * c.x;
    uint32_t hi1 = __umulhi(m1, c.z), lo1 = m1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

template <typename T>
struct Vec2;
template <>
struct Vec2<float> {
  using type = float2;
};
template <>
struct Vec2<double> {
  using type = double2;
};

// Unit phasor e^{i 2 pi (w + 1/2) 2^-32}.
__device__ __forceinline__ float2 phasor(uint32_t w, float) {
  float v = fmaf(__uint2float_rn(w), 0x1p-31f, 0x1p-32f);  // 2 (w + 1/2) 2^-32
  float s, c;
  sincospif(v, &s, &c);
  return make_float2(c, s);
}
__device__ __forceinline__ double2 phasor(uint32_t w, double) {
  double v = ((double)w + 0.5) * 0x1p-31;
  double s, c;
  sincospi(v, &s, &c);
  return make_double2(c, s);
}

// a3: phases.  Thread per (Philox counter, sample), sample index fastest.
// Counter c covers lattice entries e = 4c .. 4c+3 of e = (s nk + kk) nw + kw.
// Writes y^s_k = sqrt(q_k) z^s_k (0 where S = 0) into the padded layout
// y[kk][kPad + kw][ss], ss = 2 n + s, except that y at k = 0 goes to y0[ss]
// and the lattice slot of k = 0 holds 0 (it takes part in no pair).  With
// words != NULL writes the raw words[n][2][nk][nw] instead.
template <typename T>
__global__ void k_phases(int nk, int nw, int nsamp, SeedChunk seeds,
                         const T *__restrict__ sqq, typename Vec2<T>::type *__restrict__ y,
                         typename Vec2<T>::type *__restrict__ y0, int SSpad, int rowstride,
                         uint32_t *__restrict__ words) {
  using T2 = typename Vec2<T>::type;
  const long long nl = (long long)nk * nw;
  const long long nc = (2 * nl + 3) / 4;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= nc * nsamp) return;
  const int n = (int)(gid % nsamp);
  const long long c = gid / nsamp;
  const uint64_t seed = seeds.s[n];
  uint4 out = philox4x32_10(make_uint4((uint32_t)c, (uint32_t)(c >> 32), 0u, 0u),
                            make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  const uint32_t wv[4] = {out.x, out.y, out.z, out.w};
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    long long e = 4 * c + l;
    if (e >= 2 * nl) break;
    int s = e >= nl ? 1 : 0;
    long long r = e - s * nl;
    if (words) {
      words[((long long)n * 2 + s) * nl + r] = wv[l];
      continue;
    }
    int kk = (int)(r / nw), kw = (int)(r - (long long)kk * nw);
    T2 z = phasor(wv[l], T());
    T a = sqq[r];
    T2 v;
    v.x = a * z.x;
    v.y = a * z.y;
    int ss = 2 * n + s;
    if (r == 0) {
      y0[ss] = v;
      v.x = 0;
      v.y = 0;
    }
    y[((size_t)kk * rowstride + kPad + kw) * SSpad + ss] = v;
  }
}

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
// a4 + a5, tiled FP32 form.  A work unit is (tile, group): the tile is R = 8
// consecutive outputs kw0..kw0+7 of one lattice row kk, the group 32
// sheet-samples, one per lane.  Per row pair (a, b = kk - a) the thread
// forms T_r = sum_iw w(r, iw) y_a[iw] y_b[kw0 + r - iw] in U = 8 wide
// blocks of iw held in registers (a Toeplitz window of y_b serves all R
// outputs), then merges rowfac * T_r into a Kahan-compensated accumulator.
// Rows and blocks run over the full range iw in [0, kw0 + R - 1]; terms
// with iw > kw read the zero padding of y_b, and the centre row a = b is
// halved with its diagonal added back: T = (T_full + w y_{kw/2}^2) / 2.
// TABLE: w(r, iw) streamed from the W table (it already holds c_k and the
// kappa factor).  Otherwise w = Ew[2 iw - kw] from a shared-memory copy of
// the envelope table, rowfac = Ek[kk - 2a] and c_k is applied at the end.
template <bool TABLE>
__global__ void __launch_bounds__(128) k_pairsum_f32(
    int nk, int nw, int SS, int SSpad, int rowstride, int G, int nwork,
    const int2 *__restrict__ order, const long long *__restrict__ toff, int ntw,
    const float2 *__restrict__ y, const float2 *__restrict__ y0,
    const float *__restrict__ Ek, const float *__restrict__ Ews_g, int ew_off, int ew_len,
    const float *__restrict__ W, const float *__restrict__ Pk, const float *__restrict__ ck,
    float cb, float sb, float2 *__restrict__ C) {
  constexpr int R = kTileR, U = kTileU;
  extern __shared__ float ews[];
  if (!TABLE) {
    for (int i = threadIdx.x; i < ew_len; i += blockDim.x) ews[i] = Ews_g[i];
    __syncthreads();
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wu = blockIdx.x * kWarpsPerCta + warp;
  if (wu >= nwork) return;
  const int tile = wu / G, grp = wu - tile * G;
  const int2 tk = order[tile];
  const int kk = tk.x, kw0 = tk.y;
  const int ss = grp * 32 + lane;
  const float2 *yl = y + ss;
  const size_t SP = (size_t)SSpad;
  const int L = ((kw0 + R + U - 1) / U) * U;
  const float *Wt = TABLE ? W + toff[kk * ntw + kw0 / R] : nullptr;

  float2 acc[R], cmp[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    acc[r] = make_float2(0.f, 0.f);
    cmp[r] = make_float2(0.f, 0.f);
  }
  const int nrow = kk / 2 + 1;
  const int iw_last = kw0 + R - 1;
  for (int a = 0; a < nrow; ++a) {
    const int b = kk - a;
    const float2 *pa = yl + (size_t)(a * rowstride + kPad) * SP;
    const float2 *pb = yl + (size_t)(b * rowstride + kPad) * SP;
    const float *Wa = TABLE ? Wt + (size_t)a * R * L : nullptr;
    float2 T[R];
#pragma unroll
    for (int r = 0; r < R; ++r) T[r] = make_float2(0.f, 0.f);
    for (int iw0 = 0; iw0 <= iw_last; iw0 += U) {
      float2 ya[U], yb[R + U - 1];
#pragma unroll
      for (int u = 0; u < U; ++u) ya[u] = pa[(size_t)(iw0 + u) * SP];
      const int jlo = kw0 - iw0 - (U - 1);
#pragma unroll
      for (int v = 0; v < R + U - 1; ++v) yb[v] = pb[(long long)(jlo + v) * (long long)SP];
      if (TABLE) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const float4 w0 = *reinterpret_cast<const float4 *>(Wa + r * L + iw0);
          const float4 w1 = *reinterpret_cast<const float4 *>(Wa + r * L + iw0 + 4);
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
        float e[2 * U + R - 2];
        const int base = ew_off + 2 * iw0 - kw0 - (R - 1);
#pragma unroll
        for (int t = 0; t < 2 * U + R - 2; ++t) e[t] = ews[base + t];
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
    if (a == b) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int kw = kw0 + r;
        if ((kw & 1) == 0) {
          const float2 h = pa[(size_t)(kw >> 1) * SP];
          const float w0 = TABLE ? Wa[r * L + (kw >> 1)] : ews[ew_off];
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
      // Kahan merge of the row partial into the running sum
      float yx = fmaf(rowfac, T[r].x, -cmp[r].x);
      float tx = acc[r].x + yx;
      cmp[r].x = (tx - acc[r].x) - yx;
      acc[r].x = tx;
      float yy = fmaf(rowfac, T[r].y, -cmp[r].y);
      float ty = acc[r].y + yy;
      cmp[r].y = (ty - acc[r].y) - yy;
      acc[r].y = ty;
    }
  }
  if (ss >= SS) return;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int kw = kw0 + r;
    if (kw >= nw) break;
    const int k = kk * nw + kw;
    const float2 yk = (k == 0) ? y0[ss] : yl[((size_t)kk * rowstride + kPad + kw) * SP];
    const float ar = acc[r].x - cmp[r].x, ai = acc[r].y - cmp[r].y;
    const float cf = TABLE ? 1.0f : ck[k];
    const float P = Pk[k];
    float2 out;
    out.x = fmaf(P, yk.x, cf * (ar * cb - ai * sb));
    out.y = fmaf(P, yk.y, cf * (ar * sb + ai * cb));
    C[((size_t)ss * nk + kk) * nw + kw] = out;
  }
}

// ---------------------------------------------------------------------------
// a4 + a5, tiled FP32 form with shared-memory staging.  A CTA (4 warps)
// takes a super-tile of 32 outputs kws0..kws0+31 of lattice row kk for one
// group of 32 sheet-samples; warp w owns the 8-output tile kws0 + 8w and
// each lane one sheet-sample, with the same R x U register blocking as
// k_pairsum_f32.  For each row pair (a, kk - a) the omega range
// [0, kws0 + 31] is walked in chunks of CH = 32: the chunk's y_a rows, the
// y_b window that all four tiles need (CH + 31 rows) and, for the table
// path, the four tiles' W rows are copied global -> shared with 16-byte
// cp.async (zero-filled outside the lattice), double-buffered so that the
// copy of chunk t+1 overlaps the arithmetic on chunk t.
namespace staged {
constexpr int R = kTileR, U = kTileU, ST = kWarpsPerCta, SW = ST * R, CH = 32;
constexpr int YB_ROWS = CH + SW - 1;
constexpr int STAGE_Y = (CH + YB_ROWS) * 32;  // float2 entries per stage
constexpr int STAGE_W = ST * R * CH;          // floats per stage
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
  float2 *sy = reinterpret_cast<float2 *>(smem_raw);                 // [2][STAGE_Y]
  float *sw = reinterpret_cast<float *>(sy + 2 * STAGE_Y);           // [2][STAGE_W] (table)
  float *ews = TABLE ? nullptr : reinterpret_cast<float *>(sy + 2 * STAGE_Y);  // envelope
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
  const float2 *ybase = y + (size_t)grp * 32;  // lane 0 of the group
  const int nrow = kk / 2 + 1;
  const int nch = (kws0 + SW + CH - 1) / CH;
  const int nitems = nrow * nch;

  // W geometry (table path): this warp's tile, and the two tiles whose rows
  // this thread copies (q = tid and tid + 128 cover tiles tid/64 and +2).
  auto tile_L = [&](int k0) { return ((k0 + R + U - 1) / U) * U; };
  auto tile_base = [&](int k0) -> long long {
    return (TABLE && k0 < nw) ? toff[kk * ntw + k0 / R] : -1;
  };
  const int my_L = tile_L(kw0);
  const long long my_base = tile_base(kw0);
  const int cp_s0 = tid >> 6;
  const int cp_L0 = tile_L(kws0 + R * cp_s0), cp_L1 = tile_L(kws0 + R * (cp_s0 + 2));
  const long long cp_b0 = tile_base(kws0 + R * cp_s0), cp_b1 = tile_base(kws0 + R * (cp_s0 + 2));

  auto issue = [&](int item, int stage) {
    if (item < nitems) {
      const int a = item / nch, c = item - (item / nch) * nch;
      const int b = kk - a, i0 = c * CH;
      float2 *dya = sy + stage * STAGE_Y;
      float2 *dyb = dya + CH * 32;
      const float2 *ra = ybase + (size_t)(a * rowstride + kPad) * SP;
      const float2 *rb = ybase + (size_t)(b * rowstride + kPad) * SP;
      for (int q = tid; q < CH * 16; q += 128) {  // 16 x 16 B per 32-lane row
        const int row = q >> 4, part = q & 15;
        const int iw = i0 + row;
        const bool v = iw < nw;
        cp_async16(dya + row * 32 + part * 2, ra + (size_t)(v ? iw : 0) * SP + part * 2, v);
      }
      const int jlo = kws0 - i0 - CH + 1;
      for (int q = tid; q < YB_ROWS * 16; q += 128) {
        const int row = q >> 4, part = q & 15;
        const int jw = jlo + row;
        const bool v = jw >= 0 && jw < nw;
        cp_async16(dyb + row * 32 + part * 2, rb + (size_t)(v ? jw : 0) * SP + part * 2, v);
      }
      if (TABLE) {
        static_assert(ST * R * (CH / 4) == 256, "two W copies per thread");
        float *dw = sw + stage * STAGE_W;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int q = tid + 128 * j;
          const int s = q >> 6, rem = q & 63;
          const int r = rem >> 3, c4 = rem & 7;
          const int iw = i0 + 4 * c4;
          const long long wb = j ? cp_b1 : cp_b0;
          const int wl = j ? cp_L1 : cp_L0;
          const bool v = wb >= 0 && iw < wl;
          const float *src = v ? W + wb + ((long long)a * R + r) * wl + iw : W;
          cp_async16(dw + (s * R + r) * CH + 4 * c4, src, v);
        }
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
  for (int t = 0; t < nitems; ++t) {
    const int stage = t & 1;
    const int a = t / nch, c = t - (t / nch) * nch;
    const int i0 = c * CH;
    cp_async_wait1();
    __syncthreads();
    if (tile_ok) {
      const float2 *sya = sy + stage * STAGE_Y;
      const float2 *syb = sya + CH * 32;
      const float *swt = sw + stage * STAGE_W + warp * R * CH;
#pragma unroll 1
      for (int ib = 0; ib < CH; ib += U) {
        if (i0 + ib > kw0 + R - 1) break;
        float2 ya[U], yb[R + U - 1];
#pragma unroll
        for (int u = 0; u < U; ++u) ya[u] = sya[(ib + u) * 32 + lane];
        const int r0 = R * warp - ib + (CH - 1) - (U - 1);  // window row of v = 0
#pragma unroll
        for (int v = 0; v < R + U - 1; ++v) yb[v] = syb[(r0 + v) * 32 + lane];
        if (TABLE) {
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const float4 w0 = *reinterpret_cast<const float4 *>(swt + r * CH + ib);
            const float4 w1 = *reinterpret_cast<const float4 *>(swt + r * CH + ib + 4);
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
          float e[2 * U + R - 2];
          const int base = ew_off + 2 * (i0 + ib) - kw0 - (R - 1);
#pragma unroll
          for (int q = 0; q < 2 * U + R - 2; ++q) e[q] = ews[base + q];
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
          const float2 *pa = y + ss + (size_t)(a * rowstride + kPad) * SP;
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const int kw = kw0 + r;
            if ((kw & 1) == 0 && kw < nw) {
              const float2 h = pa[(size_t)(kw >> 1) * SP];
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

// ---------------------------------------------------------------------------
// a6: inverse transform.  u[mx][mt] = Re sum_kk e^{2 pi i kk mx / nx}
//   sum_m F[kk][m] e^{2 pi i m mt / nt}, F[kk][kw] = C^+_k,
//   F[kk][(nt - kw) mod nt] += C^-_k (FFT form, Sec. 4.3).
// Radix-2 decimation in time in shared memory, input in bit-reversed order,
// twiddles e^{+2 pi i j / nfft} from a table.
template <typename T2>
__device__ __forceinline__ T2 cmul(T2 a, T2 b) {
  T2 r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}

template <typename T2>
__device__ void fft_stages(T2 *buf, int ncols, int log2n, const T2 *__restrict__ tw,
                           int log2nfft) {
  const int n = 1 << log2n;
  const int halfn = n >> 1;
  const int total = ncols * halfn;
  for (int s = 1; s <= log2n; ++s) {
    const int half = 1 << (s - 1);
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      const int col = t >> (log2n - 1);
      const int bf = t & (halfn - 1);
      const int grp = bf >> (s - 1);
      const int j = bf & (half - 1);
      const int i0 = col * n + grp * 2 * half + j;
      const int i1 = i0 + half;
      const T2 w = tw[j << (log2nfft - s)];
      const T2 x0 = buf[i0];
      const T2 x1 = cmul(buf[i1], w);
      T2 o0, o1;
      o0.x = x0.x + x1.x;
      o0.y = x0.y + x1.y;
      o1.x = x0.x - x1.x;
      o1.y = x0.y - x1.y;
      buf[i0] = o0;
      buf[i1] = o1;
    }
    __syncthreads();
  }
}

__device__ __forceinline__ int brev(int m, int log2n) {
  return (int)(__brev((unsigned)m) >> (32 - log2n));
}

template <typename T2>
__global__ void k_fft_t(int nk, int nw, int nt, int log2nt, int log2nfft,
                        const T2 *__restrict__ C, const T2 *__restrict__ tw, T2 *__restrict__ H) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T2 *buf = reinterpret_cast<T2 *>(smem_raw);
  const int kk = blockIdx.x, n = blockIdx.y;
  for (int m = threadIdx.x; m < nt; m += blockDim.x) {
    buf[m].x = 0;
    buf[m].y = 0;
  }
  __syncthreads();
  const T2 *Cp = C + ((size_t)(2 * n) * nk + kk) * nw;
  const T2 *Cm = C + ((size_t)(2 * n + 1) * nk + kk) * nw;
  for (int kw = threadIdx.x; kw < nw; kw += blockDim.x) buf[brev(kw, log2nt)] = Cp[kw];
  __syncthreads();
  for (int kw = threadIdx.x; kw < nw; kw += blockDim.x) {
    const int m = kw == 0 ? 0 : nt - kw;
    const int pos = brev(m, log2nt);
    T2 v = buf[pos];
    const T2 c = Cm[kw];
    v.x += c.x;
    v.y += c.y;
    buf[pos] = v;
  }
  __syncthreads();
  fft_stages(buf, 1, log2nt, tw, log2nfft);
  T2 *Hrow = H + ((size_t)n * nk + kk) * nt;
  for (int m = threadIdx.x; m < nt; m += blockDim.x) Hrow[m] = buf[m];
}

template <typename T, typename T2>
__global__ void k_fft_x(int nk, int nx, int nt, int log2nx, int log2nfft, int TC,
                        const T2 *__restrict__ H, const T2 *__restrict__ tw, T *__restrict__ u) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T2 *buf = reinterpret_cast<T2 *>(smem_raw);
  const int mt0 = blockIdx.x * TC, n = blockIdx.y;
  for (int i = threadIdx.x; i < TC * nx; i += blockDim.x) {
    buf[i].x = 0;
    buf[i].y = 0;
  }
  __syncthreads();
  const T2 *Hn = H + (size_t)n * nk * nt + mt0;
  for (int idx = threadIdx.x; idx < nk * TC; idx += blockDim.x) {
    const int kk = idx / TC, c = idx - kk * TC;
    buf[c * nx + brev(kk, log2nx)] = Hn[(size_t)kk * nt + c];
  }
  __syncthreads();
  fft_stages(buf, TC, log2nx, tw, log2nfft);
  T *un = u + (size_t)n * nx * nt + mt0;
  for (int idx = threadIdx.x; idx < nx * TC; idx += blockDim.x) {
    const int mx = idx / TC, c = idx - mx * TC;
    un[(size_t)mx * nt + c] = buf[c * nx + mx].x;
  }
}

// ---------------------------------------------------------------------------
static size_t elem2(const srm3_plan *p) {
  return p->precision == SRM3_FP32 ? sizeof(float2) : sizeof(double2);
}

static int sspad_for(int chunk) { return ((2 * chunk + 31) / 32) * 32; }

int ensure_workspace(srm3_plan *p, int chunk) {
  if (p->ws_chunk >= chunk) return SRM3_OK;
  int cap = std::max(chunk, std::min(kMaxChunk, 64));
  for (void **q : {&p->y, &p->y0, &p->C, &p->H}) {
    if (*q) cudaFree(*q);
    *q = nullptr;
  }
  p->ws_chunk = 0;
  const size_t e2 = elem2(p);
  p->rowstride = p->nw + 2 * kPad;
  const int sp = sspad_for(cap);
  SRM3_CUDA(cudaMalloc(&p->y, (size_t)p->nk * p->rowstride * sp * e2));
  SRM3_CUDA(cudaMalloc(&p->y0, (size_t)sp * e2));
  SRM3_CUDA(cudaMalloc(&p->C, (size_t)2 * cap * p->nk * p->nw * e2));
  SRM3_CUDA(cudaMalloc(&p->H, (size_t)cap * p->nk * p->nt * e2));
  p->ws_chunk = cap;
  return SRM3_OK;
}

int run_phases(srm3_plan *p, const uint64_t *seeds, int n, uint32_t *words_out) {
  SeedChunk sc;
  std::memset(&sc, 0, sizeof(sc));
  std::memcpy(sc.s, seeds, sizeof(uint64_t) * n);
  const long long nl = (long long)p->nk * p->nw;
  const long long nc = (2 * nl + 3) / 4;
  const int blocks = cdiv(nc * n, 256);
  const int sp = sspad_for(n);
  if (!words_out) {
    SRM3_CUDA(cudaMemsetAsync(p->y, 0, (size_t)p->nk * p->rowstride * sp * elem2(p), p->stream));
  }
  if (p->precision == SRM3_FP32)
    k_phases<float><<<blocks, 256, 0, p->stream>>>(p->nk, p->nw, n, sc, (const float *)p->sqq,
                                                   (float2 *)p->y, (float2 *)p->y0, sp,
                                                   p->rowstride, words_out);
  else
    k_phases<double><<<blocks, 256, 0, p->stream>>>(p->nk, p->nw, n, sc, (const double *)p->sqq,
                                                    (double2 *)p->y, (double2 *)p->y0, sp,
                                                    p->rowstride, words_out);
  SRM3_CUDA(cudaGetLastError());
  return SRM3_OK;
}

int run_pairsum(srm3_plan *p, int n, void *C_out) {
  const int SS = 2 * n, sp = sspad_for(n);
  const float cbf = (float)std::cos(p->beta), sbf = (float)std::sin(p->beta);
  if (p->precision == SRM3_FP64) {
    const long long threads = (long long)p->nk * p->nw * sp;
    k_pairsum_f64<<<cdiv(threads, 256), 256, 0, p->stream>>>(
        p->nk, p->nw, SS, sp, p->rowstride, (const double2 *)p->y, (const double2 *)p->y0,
        (const double *)p->Ek, (const double *)p->Ews, p->ew_off, (const double *)p->Pk,
        (const double *)p->ck, std::cos(p->beta), std::sin(p->beta), (double2 *)C_out);
  } else if (p->staged) {
    using namespace staged;
    const int G = sp / 32;
    const int blocks = p->nsuper * G;
    const bool table = p->storage == SRM3_STORAGE_TABLE;
    const size_t smem = (size_t)2 * STAGE_Y * sizeof(float2) +
                        (table ? (size_t)2 * STAGE_W * sizeof(float)
                               : (size_t)p->ew_len * sizeof(float));
    if (table) {
      SRM3_CUDA(cudaFuncSetAttribute(k_pairsum_f32s<true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_pairsum_f32s<true><<<blocks, 32 * kWarpsPerCta, smem, p->stream>>>(
          p->nk, p->nw, SS, sp, p->rowstride, G, p->super_order, p->tile_off, p->ntw,
          (const float2 *)p->y, (const float2 *)p->y0, (const float *)p->Ek,
          (const float *)p->Ews, p->ew_off, p->ew_len, p->W, (const float *)p->Pk,
          (const float *)p->ck, cbf, sbf, (float2 *)C_out);
    } else {
      SRM3_CUDA(cudaFuncSetAttribute(k_pairsum_f32s<false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_pairsum_f32s<false><<<blocks, 32 * kWarpsPerCta, smem, p->stream>>>(
          p->nk, p->nw, SS, sp, p->rowstride, G, p->super_order, p->tile_off, p->ntw,
          (const float2 *)p->y, (const float2 *)p->y0, (const float *)p->Ek,
          (const float *)p->Ews, p->ew_off, p->ew_len, nullptr, (const float *)p->Pk,
          (const float *)p->ck, cbf, sbf, (float2 *)C_out);
    }
  } else {
    const int G = sp / 32;
    const int nwork = p->ntiles * G;
    const int blocks = cdiv(nwork, kWarpsPerCta);
    if (p->storage == SRM3_STORAGE_TABLE) {
      k_pairsum_f32<true><<<blocks, 32 * kWarpsPerCta, 0, p->stream>>>(
          p->nk, p->nw, SS, sp, p->rowstride, G, nwork, p->tile_order, p->tile_off, p->ntw,
          (const float2 *)p->y, (const float2 *)p->y0, (const float *)p->Ek,
          (const float *)p->Ews, p->ew_off, p->ew_len, p->W, (const float *)p->Pk,
          (const float *)p->ck, cbf, sbf, (float2 *)C_out);
    } else {
      const size_t smem = (size_t)p->ew_len * sizeof(float);
      if (smem > 48 * 1024)
        SRM3_CUDA(cudaFuncSetAttribute(k_pairsum_f32<false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_pairsum_f32<false><<<blocks, 32 * kWarpsPerCta, smem, p->stream>>>(
          p->nk, p->nw, SS, sp, p->rowstride, G, nwork, p->tile_order, p->tile_off, p->ntw,
          (const float2 *)p->y, (const float2 *)p->y0, (const float *)p->Ek,
          (const float *)p->Ews, p->ew_off, p->ew_len, nullptr, (const float *)p->Pk,
          (const float *)p->ck, cbf, sbf, (float2 *)C_out);
    }
  }
  SRM3_CUDA(cudaGetLastError());
  return SRM3_OK;
}

template <typename T, typename T2>
static int transform_impl(srm3_plan *p, const T2 *C, int n, T *out) {
  const int log2nfft = ilog2_exact(p->nfft);
  const size_t e2 = sizeof(T2);
  const size_t smem_t = (size_t)p->nt * e2;
  int TC = 16;
  while (TC > 1 && ((size_t)TC * p->nx * e2 > 96 * 1024 || TC > p->nt)) TC >>= 1;
  const size_t smem_x = (size_t)TC * p->nx * e2;
  const int lim = 200 * 1024;
  SRM3_CUDA(cudaFuncSetAttribute(k_fft_t<T2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  SRM3_CUDA(cudaFuncSetAttribute(k_fft_x<T, T2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  k_fft_t<T2><<<dim3(p->nk, n), 256, smem_t, p->stream>>>(p->nk, p->nw, p->nt, p->log2nt,
                                                          log2nfft, C, (const T2 *)p->tw,
                                                          (T2 *)p->H);
  SRM3_CUDA(cudaGetLastError());
  k_fft_x<T, T2><<<dim3(p->nt / TC, n), 256, smem_x, p->stream>>>(
      p->nk, p->nx, p->nt, p->log2nx, log2nfft, TC, (const T2 *)p->H, (const T2 *)p->tw, out);
  SRM3_CUDA(cudaGetLastError());
  return SRM3_OK;
}

int run_transform(srm3_plan *p, const void *C, int n, void *out) {
  if (p->precision == SRM3_FP32)
    return transform_impl<float, float2>(p, (const float2 *)C, n, (float *)out);
  return transform_impl<double, double2>(p, (const double2 *)C, n, (double *)out);
}

int stage_begin(srm3_plan *p, int stage, long long pair_terms, int *rec) {
  *rec = -1;
  if (!p->timing) return SRM3_OK;
  cudaEvent_t ev[2];
  for (int i = 0; i < 2; ++i) {
    if (!p->ev_pool.empty()) {
      ev[i] = p->ev_pool.back();
      p->ev_pool.pop_back();
    } else {
      SRM3_CUDA(cudaEventCreate(&ev[i]));
    }
  }
  SRM3_CUDA(cudaEventRecord(ev[0], p->stream));
  p->ev_recs.push_back({stage, ev[0], ev[1], pair_terms});
  *rec = (int)p->ev_recs.size() - 1;
  return SRM3_OK;
}

int stage_end(srm3_plan *p, int rec) {
  if (rec < 0) return SRM3_OK;
  SRM3_CUDA(cudaEventRecord(p->ev_recs[rec].b, p->stream));
  return SRM3_OK;
}

int collect_timings(srm3_plan *p) {
  SRM3_CUDA(cudaStreamSynchronize(p->stream));
  for (auto &r : p->ev_recs) {
    float ms = 0.f;
    SRM3_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
    p->t_stage_ms[r.stage] += ms;
    if (r.stage == 1) {
      p->t_pairsum_launches += 1;
      p->t_pair_terms += r.pair_terms;
    }
    p->ev_pool.push_back(r.a);
    p->ev_pool.push_back(r.b);
  }
  p->ev_recs.clear();
  return SRM3_OK;
}

// One chunk of samples through the three sampling stages.
static int run_chunk(srm3_plan *p, const uint64_t *seeds, int m, void *C, void *out) {
  int rc, rec;
  if ((rc = stage_begin(p, 0, 0, &rec))) return rc;
  if ((rc = run_phases(p, seeds, m, nullptr))) return rc;
  if ((rc = stage_end(p, rec))) return rc;
  if ((rc = stage_begin(p, 1, 2LL * m * p->pairs, &rec))) return rc;
  if ((rc = run_pairsum(p, m, C))) return rc;
  if ((rc = stage_end(p, rec))) return rc;
  if (!out) return SRM3_OK;
  if ((rc = stage_begin(p, 2, 0, &rec))) return rc;
  if ((rc = run_transform(p, C, m, out))) return rc;
  return stage_end(p, rec);
}

static int check_call(srm3_plan *p, const uint64_t *seeds, int n, const void *buf) {
  if (!p) return fail(SRM3_ERR_INVALID_ARG, "plan is NULL");
  if (n < 0) return fail(SRM3_ERR_INVALID_ARG, "n must be >= 0");
  if (n > 0 && (!seeds || !buf)) return fail(SRM3_ERR_INVALID_ARG, "seeds and buffer must be non-NULL");
  return SRM3_OK;
}

static size_t field_elems(const srm3_plan *p) { return (size_t)p->nx * p->nt; }
static size_t elem1(const srm3_plan *p) {
  return p->precision == SRM3_FP32 ? sizeof(float) : sizeof(double);
}

}  // namespace srm3

using namespace srm3;

SRM3_API int srm3_sample(srm3_plan *plan, const uint64_t *seeds, int n, void *out) {
  int rc = check_call(plan, seeds, n, out);
  if (rc || n == 0) return rc;
  const int chunk = std::min(n, kMaxChunk);
  rc = ensure_workspace(plan, chunk);
  if (rc) return rc;
  for (int s0 = 0; s0 < n; s0 += chunk) {
    const int m = std::min(chunk, n - s0);
    char *o = (char *)out + (size_t)s0 * field_elems(plan) * elem1(plan);
    if ((rc = run_chunk(plan, seeds + s0, m, plan->C, o))) return rc;
  }
  return SRM3_OK;
}

SRM3_API int srm3_sample_host(srm3_plan *plan, const uint64_t *seeds, int n, void *out_host) {
  int rc = check_call(plan, seeds, n, out_host);
  if (rc || n == 0) return rc;
  const int chunk = std::min(n, kMaxChunk);
  rc = ensure_workspace(plan, chunk);
  if (rc) return rc;
  const size_t bytes_per = field_elems(plan) * elem1(plan);
  void *dev = nullptr;
  SRM3_CUDA(cudaMallocAsync(&dev, (size_t)chunk * bytes_per, plan->stream));
  for (int s0 = 0; s0 < n && rc == SRM3_OK; s0 += chunk) {
    const int m = std::min(chunk, n - s0);
    if ((rc = run_chunk(plan, seeds + s0, m, plan->C, dev))) break;
    cudaError_t e = cudaMemcpyAsync((char *)out_host + (size_t)s0 * bytes_per, dev,
                                    (size_t)m * bytes_per, cudaMemcpyDeviceToHost, plan->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemcpyAsync(field to host)");
  }
  cudaFreeAsync(dev, plan->stream);
  if (rc) return rc;
  SRM3_CUDA(cudaStreamSynchronize(plan->stream));
  return SRM3_OK;
}

SRM3_API int srm3_phase_words(srm3_plan *plan, const uint64_t *seeds, int n, uint32_t *words) {
  int rc = check_call(plan, seeds, n, words);
  if (rc || n == 0) return rc;
  const size_t per = (size_t)2 * plan->nk * plan->nw;
  for (int s0 = 0; s0 < n; s0 += kMaxChunk) {
    const int m = std::min(kMaxChunk, n - s0);
    if ((rc = run_phases(plan, seeds + s0, m, words + (size_t)s0 * per))) return rc;
  }
  return SRM3_OK;
}

SRM3_API int srm3_coeffs(srm3_plan *plan, const uint64_t *seeds, int n, void *C) {
  int rc = check_call(plan, seeds, n, C);
  if (rc || n == 0) return rc;
  const int chunk = std::min(n, kMaxChunk);
  rc = ensure_workspace(plan, chunk);
  if (rc) return rc;
  const size_t per = (size_t)2 * plan->nk * plan->nw * elem2(plan);
  for (int s0 = 0; s0 < n; s0 += chunk) {
    const int m = std::min(chunk, n - s0);
    if ((rc = run_chunk(plan, seeds + s0, m, (char *)C + (size_t)s0 * per, nullptr))) return rc;
  }
  return SRM3_OK;
}

SRM3_API int srm3_field_from_coeffs(srm3_plan *plan, const void *C, int n, void *out) {
  if (!plan) return fail(SRM3_ERR_INVALID_ARG, "plan is NULL");
  if (n < 0 || (n > 0 && (!C || !out))) return fail(SRM3_ERR_INVALID_ARG, "bad C/out/n");
  if (n == 0) return SRM3_OK;
  const int chunk = std::min(n, kMaxChunk);
  int rc = ensure_workspace(plan, chunk);
  if (rc) return rc;
  const size_t perC = (size_t)2 * plan->nk * plan->nw * elem2(plan);
  const size_t perU = field_elems(plan) * elem1(plan);
  for (int s0 = 0; s0 < n; s0 += chunk) {
    const int m = std::min(chunk, n - s0);
    if ((rc = run_transform(plan, (const char *)C + (size_t)s0 * perC, m,
                            (char *)out + (size_t)s0 * perU)))
      return rc;
  }
  return SRM3_OK;
}

SRM3_API int srm3_enable_timing(srm3_plan *plan, int on) {
  if (!plan) return fail(SRM3_ERR_INVALID_ARG, "plan is NULL");
  plan->timing = on != 0;
  return SRM3_OK;
}

SRM3_API int srm3_get_timings(srm3_plan *plan, srm3_timings *t, int reset) {
  if (!plan || !t) return fail(SRM3_ERR_INVALID_ARG, "plan and t must be non-NULL");
  int rc = collect_timings(plan);
  if (rc) return rc;
  t->recursion_ms = plan->t_recursion_ms;
  t->recursion_fp32_ms = plan->t_rec32_ms;
  t->recursion_fp64_ms = plan->t_rec64_ms;
  t->recursion_passes_fp32 = plan->root_passes32;
  t->table_ms = plan->t_table_ms;
  t->phases_ms = plan->t_stage_ms[0];
  t->pairsum_ms = plan->t_stage_ms[1];
  t->transform_ms = plan->t_stage_ms[2];
  t->recursion_passes = plan->root_passes;
  t->pairsum_launches = plan->t_pairsum_launches;
  t->pair_terms = plan->t_pair_terms;
  if (reset) {
    plan->t_stage_ms[0] = plan->t_stage_ms[1] = plan->t_stage_ms[2] = 0.0;
    plan->t_pairsum_launches = 0;
    plan->t_pair_terms = 0;
  }
  return SRM3_OK;
}
