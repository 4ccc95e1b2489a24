// plan.cu - plan creation for the SRM3 sampler: lattice discretisation
// (Sec. 5), the pure-spectrum / partial-bicoherence recursion (Eq. pure)
// run level-parallel over the anti-diagonals of the lattice in FP64, the
// bracketing root search on eps, and the sampling tables (W table, tile
// order, FFT twiddles).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <cstdlib>
#include <mutex>
#include <numeric>
#include <unordered_map>

#include "recursion.cuh"
#include "srm3_internal.cuh"

namespace srm3 {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

int fail(int code, const std::string &msg) {
  g_last_error = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char *what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();  // clear a sticky launch error, if any
  return e == cudaErrorMemoryAllocation ? SRM3_ERR_OUT_OF_MEMORY : SRM3_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Discretisation: Kaimal S(omega) (Eq. kaimal_spectrum) times the normalised
// Lorentzian a/(pi (a^2 + kappa^2)), a = lam omega / (2 pi U); S := 0 where
// omega = 0 (Sec. 5).
__global__ void k_discretise_kaimal(int nk, int nw, double dk, double dw, double U,
                                    double z, double z0, double kvk, double lam,
                                    double *S) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nk * nw) return;
  int kk = idx / nw, kw = idx - kk * nw;
  double val = 0.0;
  if (kw > 0) {
    const double pi = 3.14159265358979323846;
    double kappa = kk * dk, omega = kw * dw;
    double ustar = kvk * U / log(z / z0);
    double kaimal = 0.5 * (200.0 / (2.0 * pi)) * ustar * ustar * (z / U) /
                    pow(1.0 + 50.0 * omega * z / (2.0 * pi * U), 5.0 / 3.0);
    double a = lam * omega / (2.0 * pi * U);
    val = kaimal * (a / (pi * (a * a + kappa * kappa)));
  }
  S[idx] = val;
}

// Squared envelope factors for the recursion: g^2 = EkSq[|ik-jk|] EwSq[|iw-jw|]
// (FP64, and an FP32 copy for the search passes).
__global__ void k_env_sq(int n, double sigma_n, double *out, float *out32) {
  int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= n) return;
  double a = d / sigma_n;
  double e = exp(-0.5 * a * a);
  out[d] = e * e;
  out32[d] = (float)(e * e);
}

// g^2 over (|ik - jk|, |iw - jw|) as one table, FP64 and FP32.
// Separable envelope: e^2 and e in FP32 per lattice point, and g^2 tables of
// ones (the envelope factors are carried by h = e^2 q and e_k^2).
__global__ void k_sep_tables(int nl, const double *__restrict__ e, double *e2, float *e32,
                             double *G2, float *G2_32) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nl) return;
  e2[i] = e[i] * e[i];
  e32[i] = (float)e[i];
  G2[i] = 1.0;
  G2_32[i] = 1.0f;
}

__global__ void k_g2(int nk, int nw, const double *__restrict__ EkSq,
                     const double *__restrict__ EwSq, double *G2, float *G2_32) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nk * nw) return;
  const int dk = i / nw, dw = i - dk * nw;
  const double v = EkSq[dk] * EwSq[dw];
  G2[i] = v;
  G2_32[i] = (float)v;
}

// The Gaussian envelope of the recursion in separable form.  On the pairs of
// a point, i + j = k, so with c = (n - 1)/2 per axis
//   (i - j)^2 = 2 (i - c)^2 + 2 (j - c)^2 - (k - 2c)^2
// and g^2(i, j) = exp(-(dk/s_k)^2 - (dw/s_w)^2) = a^2_i a^2_j b^2_k with
//   a^2_i = exp(-2 ((ik - ck)/s_k)^2 - 2 ((iw - cw)/s_w)^2),
//   b^2_k = exp(((kk - 2 ck)/s_k)^2 + ((kw - 2 cw)/s_w)^2).
// Centring at c keeps a^2 in [exp(-E/2), 1] and b^2 in [1, exp(E)], E =
// ((nk - 1)/s_k)^2 + ((nw - 1)/s_w)^2; every pair term stays a product of
// positive factors, so the sums keep their relative accuracy.
__global__ void k_gauss_sep(int nk, int nw, double sk, double sw, double *__restrict__ a2,
                            double *__restrict__ b2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nk * nw) return;
  const int ik = i / nw, iw = i - ik * nw;
  const double ck = 0.5 * (nk - 1), cw = 0.5 * (nw - 1);
  const double uk = (ik - ck) / sk, uw = (iw - cw) / sw;
  const double vk = (ik - 2.0 * ck) / sk, vw = (iw - 2.0 * cw) / sw;
  a2[i] = exp(-2.0 * (uk * uk + uw * uw));
  b2[i] = exp(vk * vk + vw * vw);
}


// dsb2[k] = w0 s0[k] + w1 s1[k] + w2 s2[k]: the slope in x of every point's
// sum_b2 from FP32 search planes (the derivative weights of the Lagrange
// polynomial through them).
__global__ void k_sb2_slope(long long n, const double *__restrict__ s0,
                            const double *__restrict__ s1, const double *__restrict__ s2,
                            double w0, double w1, double w2, double *__restrict__ dsb2) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dsb2[i] = fma(w0, s0[i], fma(w1, s1[i], w2 * s2[i]));
}

// The tables of an FP64 pass at x moved to x + dx to first order: sum_b2 +=
// dx dsb2 (clamped at 0), q = 1/(1 - sum_b2) (0 where S = 0, or where
// sum_b2 >= 1, which also sets *err); max_k sum_b2 into *maxb (bits of a
// double >= 0, zeroed before).
__global__ void k_sb2_shift(long long n, const double *__restrict__ S, double *__restrict__ sb2,
                            const double *__restrict__ dsb2, double dx, double *__restrict__ q,
                            unsigned long long *maxb, int *err) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (i < n && S[i] > 0.0) {  // S = 0: zero tables, as the pass left them
    v = fma(dx, dsb2[i], sb2[i]);
    v = v < 0.0 ? 0.0 : v;
    sb2[i] = v;
    if (v < 1.0) {
      q[i] = 1.0 / (1.0 - v);
    } else {
      q[i] = 0.0;
      atomicOr(err, 1);
    }
  }
  double m = v;  // warp maximum first: one atomic per warp
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0)
    atomicMax(maxb, (unsigned long long)__double_as_longlong(m));
}

// The tables at x from an FP64 pass at three values x_m around it: per
// point the quadratic through (x_m, sum_b2_m) taken at x (Lagrange weights
// w_m), clamped at 0, and q = 1/(1 - sum_b2) (0 where S = 0, or where
// sum_b2 >= 1, which also sets *err); into plane 0 of sum_b2 and into q;
// max_k sum_b2 into *maxb (bits of a double >= 0, zeroed before).
__global__ void k_sb2_interp3(long long n, const double *__restrict__ S, double *__restrict__ sb2,
                              double w0, double w1, double w2, double *__restrict__ q,
                              unsigned long long *maxb, int *err) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (i < n) {
    if (S[i] > 0.0) {
      v = fma(w0, sb2[i], fma(w1, sb2[n + i], w2 * sb2[2 * n + i]));
      v = v < 0.0 ? 0.0 : v;
      if (v < 1.0) {
        q[i] = 1.0 / (1.0 - v);
      } else {
        q[i] = 0.0;
        atomicOr(err, 1);
      }
    } else {
      q[i] = 0.0;
    }
    sb2[i] = v;
  }
  double m = v;  // warp maximum first: one atomic per warp
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0)
    atomicMax(maxb, (unsigned long long)__double_as_longlong(m));
}

// Reductions of plane 0 of sum_b2 and of S: max sum_b2, min (1 - sum_b2)
// over S > 0 and sum S, into scal[9], scal[10], scal[11].  k_reduce_part
// leaves one partial per CTA (kReduceCtas of them) and k_reduce_final
// combines them in CTA order, so that the sum does not depend on scheduling.
constexpr int kReduceCtas = 256;

__global__ void __launch_bounds__(256) k_reduce_part(long long n, const double *__restrict__ S,
                                                     const double *__restrict__ sb2,
                                                     double *__restrict__ part) {
  double mx = 0.0, mn = 1.0, sum = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double v = sb2[i], s = S[i];
    mx = fmax(mx, v);
    if (s > 0.0) mn = fmin(mn, 1.0 - v);
    sum += s;
  }
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    sum += __shfl_xor_sync(0xffffffffu, sum, o);
  }
  __shared__ double a[8], b[8], c[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { a[warp] = mx; b[warp] = mn; c[warp] = sum; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; ++w) { mx = fmax(mx, a[w]); mn = fmin(mn, b[w]); }
    sum = 0.0;
    for (int w = 0; w < 8; ++w) sum += c[w];
    part[3 * blockIdx.x] = mx;
    part[3 * blockIdx.x + 1] = mn;
    part[3 * blockIdx.x + 2] = sum;
  }
}

__global__ void k_reduce_final(int nparts, const double *__restrict__ part,
                               double *__restrict__ scal) {
  // one warp: lane l combines partials l, l + 32, ... in order, then a fixed
  // butterfly -- the same order on every run
  const int lane = threadIdx.x;
  double mx = 0.0, mn = 1.0, sum = 0.0;
  for (int j = lane; j < nparts; j += 32) {
    mx = fmax(mx, part[3 * j]);
    mn = fmin(mn, part[3 * j + 1]);
    sum += part[3 * j + 2];
  }
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    sum += __shfl_xor_sync(0xffffffffu, sum, o);
  }
  if (lane == 0) {
    scal[9] = mx;
    scal[10] = mn;
    scal[11] = sum;
  }
}

static int reduce_plane0(srm3_plan *p, cudaStream_t st) {
  const long long nl = (long long)p->nk * p->nw;
  if (!p->red_part) SRM3_CUDA(dev_alloc(&p->red_part, 3 * kReduceCtas * sizeof(double), st));
  const int ctas = (int)std::min<long long>(kReduceCtas, (nl + 255) / 256);
  k_reduce_part<<<ctas, 256, 0, st>>>(nl, p->S, p->sb2, p->red_part);
  k_reduce_final<<<1, 32, 0, st>>>(ctas, p->red_part, p->scal);
  p->n_launch += 2;
  return cudaGetLastError() == cudaSuccess ? SRM3_OK : fail(SRM3_ERR_CUDA, "plane reduction");
}

// ---------------------------------------------------------------------------
// Sampling tables.
template <typename T>
__global__ void k_sampling_tables(int n, double dkdw, double eps,
                                  const double *__restrict__ S,
                                  const double *__restrict__ qm,
                                  const double *__restrict__ sb2, T *sqq, T *Pk, T *ck) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double s = S[k];
  bool pos = s > 0.0;
  sqq[k] = (T)(pos ? sqrt(qm[k]) : 0.0);
  Pk[k] = (T)(pos ? 2.0 * sqrt(dkdw * s) * (1.0 - sb2[k]) : 0.0);
  ck[k] = (T)(pos ? 2.0 * eps * dkdw * sqrt(s) : 0.0);
}

// The separable form of the FP32 pair sum (Gaussian envelope): on the pairs
// of k, (i - j)^2 = 2 (i - c)^2 + 2 (j - c)^2 - (k - 2c)^2 per axis (c =
// (n - 1)/2), so g(i, j) = exp(-1/2 ((ik - jk)/sk)^2 - 1/2 ((iw - jw)/sw)^2)
// = a_i a_j b_k with a = exp(-((ik - ck)/sk)^2 - ((iw - cw)/sw)^2) and b =
// exp(1/2 ((kk - 2ck)/sk)^2 + 1/2 ((kw - 2cw)/sw)^2).  The pair sum then
// multiplies scaled phasor rows, sum (a_w y)_i (a_w y)_j per lattice row
// pair, weighted by aK[a] aK[kk - a] and at the end by c_k b_k; the pure term
// P_k y_k = (P_k / a_w) (a_w y)_k.  Factor ranges within [exp(-E/2), 1] and
// [1, exp(E)] (E <= 40), as the recursion's (k_gauss_sep).
__global__ void k_sep_sampling(int nk, int nw, double sk, double sw, const float *__restrict__ sqq,
                               const float *__restrict__ Pk, const float *__restrict__ ck,
                               float *__restrict__ sqq_s, float *__restrict__ Pk_s,
                               float *__restrict__ ck_s, float *__restrict__ aK) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nk * nw) return;
  const int kk = i / nw, kw = i - kk * nw;
  const double ck0 = 0.5 * (nk - 1), cw0 = 0.5 * (nw - 1);
  const double uw = (kw - cw0) / sw, vk = (kk - 2.0 * ck0) / sk, vw = (kw - 2.0 * cw0) / sw;
  const double aw = exp(-uw * uw), b = exp(0.5 * (vk * vk + vw * vw));
  sqq_s[i] = (float)((double)sqq[i] * aw);
  Pk_s[i] = (float)((double)Pk[i] / aw);
  ck_s[i] = (float)((double)ck[i] * b);
  if (kw == 0) {
    const double uk = (kk - ck0) / sk;
    aK[kk] = (float)exp(-uk * uk);
  }
}

template <typename T>
__global__ void k_env(int len, int off, double sigma_n, T *out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= len) return;
  double a = (double)(i - off) / sigma_n;
  out[i] = (T)exp(-0.5 * a * a);
}

// Twiddles of the radix-2 stages for every transform length up to n = 2^log2n,
// packed by stage: entry 2^(s-1) - 1 + j holds e^{+2 pi i m / n} with
// m = j 2^(log2n - s) (= e^{+2 pi i j / 2^s}), j < 2^(s-1), s = 1..log2n; the
// last entry is unused.
// Twiddles of the output transform: the pass-twiddle tables of lengths nx
// and nt / 2 (tx_twlen entries each: pass p >= 1 of the length-2^l transform
// holds w_{Ns R}^{k r} at k R + r), then e^{2 pi i m / nt}, m < nt / 2.
template <typename T2>
__global__ void k_tx_twiddles(int lx, int lm, T2 *tw) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int n1 = tx_twlen(lx), n2 = tx_twlen(lm), M = 1 << lm;
  if (e >= n1 + n2 + M) return;
  long long num = 0, den = 1;  // angle 2 pi num / den
  if (e >= n1 + n2) {
    num = e - n1 - n2;
    den = 2 * M;
  } else {
    const int l = e < n1 ? lx : lm;
    int q = e < n1 ? e : e - n1, ns = 1 << tx_lr(l, 0);
    for (int p = 1; p < tx_npass(l); ++p) {
      const int R = 1 << tx_lr(l, p);
      if (q < ns * R) {
        num = (long long)(q / R) * (q % R);
        den = (long long)ns * R;
        break;
      }
      q -= ns * R;
      ns *= R;
    }
  }
  double sn, cs;
  sincospi(2.0 * (double)num / (double)den, &sn, &cs);
  tw[e].x = cs;
  tw[e].y = sn;
}

template <typename T2>
__global__ void k_twiddles(int n, int log2n, T2 *tw) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  T2 v;
  v.x = 1;
  v.y = 0;
  if (idx < n - 1) {
    const int s = 32 - __clz(idx + 1);  // stage of this entry
    const int j = idx + 1 - (1 << (s - 1));
    const int m = j << (log2n - s);
    double sn, cs;
    sincospi(2.0 * (double)m / (double)n, &sn, &cs);
    v.x = cs;
    v.y = sn;
  }
  tw[idx] = v;
}

// W table, tile-major: for tile (kk, kw0), entry (a, r, iw) -- row pair
// a = 0..kk/2, output kw = kw0 + r, r < R, iw < L (L = kw0 + R rounded up to
// U) -- at ((a nch + iw / U) R + r) U + iw % U, nch = L / U: chunk-major, so
// the R rows of one omega chunk are one contiguous span the pair sum fetches
// with a single bulk copy.  W = Ek[kk-2a] Ew[2iw-kw] for iw <= kw < nw,
// else 0: the envelope of the pair alone, a function of the lattice shape --
// the spectrum's pair factor c_k multiplies each output at the end, so plans
// of one shape can share a table and the lanes of a batch.  Centre rows are stored in full (the kernel halves them).  W is
// real: the constant biphase is applied afterwards.  One CTA per tile, its
// threads writing the tile's float4 in storage order.
__global__ void __launch_bounds__(256) k_build_w(int t0, int nk, int nw, int ntw,
                                                 const long long *__restrict__ off,
                                                 const float *__restrict__ Ek,
                                                 const float *__restrict__ Ews, int ew_off,
                                                 float *__restrict__ W) {
  const int t = t0 + blockIdx.x;  // tiles of the plan's rows
  const int kk = t / ntw, tw = t - kk * ntw;
  const int kw0 = tw * kTileR;
  const int nrow = kk / 2 + 1;
  const int L = ((kw0 + kTileR + kTileU - 1) / kTileU) * kTileU;
  const int nch = L / kTileU;
  constexpr int V = kTileU / 4;  // float4 per chunk row
  float4 *dst = reinterpret_cast<float4 *>(W + off[t]);
  // float4 number f of the tile in storage order: (a nch + c, r, v)
  const int nf = nrow * nch * kTileR * V;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;
  for (int f = tid; f < nf; f += nth) {
    const int v = f % V, r = (f / V) % kTileR, ac = f / (V * kTileR);
    const int a = ac / nch, c = ac - a * nch;
    const int kw = kw0 + r, iw = c * kTileU + 4 * v;
    const float g = kw < nw ? Ek[kk - 2 * a] : 0.0f;
    const float *e = Ews + ew_off - kw;
    float4 w;
    w.x = (iw + 0 <= kw) ? g * e[2 * (iw + 0)] : 0.0f;
    w.y = (iw + 1 <= kw) ? g * e[2 * (iw + 1)] : 0.0f;
    w.z = (iw + 2 <= kw) ? g * e[2 * (iw + 2)] : 0.0f;
    w.w = (iw + 3 <= kw) ? g * e[2 * (iw + 3)] : 0.0f;
    dst[f] = w;
  }
}

// ---------------------------------------------------------------------------
static int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

struct PassResult {
  double max_sb2, min_pure, sumS;
  int err;
};

static thread_local cudaEvent_t t_ev[2] = {nullptr, nullptr};

static constexpr int kPlanes = 8;  // eps values per FP32 search pass
// eps values of the FP32 pass over the window around the coarse-lattice root
// (plans without the FFT form of the separable bulk)
static constexpr int kWindowPlanes = 4;
// largest exponent range of the separable Gaussian factors (k_gauss_sep)
static constexpr double kSepExpMax = 40.0;
// targets at least this loose may take the first-order table shift of
// find_eps, for steps up to kShiftMax of x
static constexpr double kShiftTol = 1e-10;
static constexpr double kShiftMax = 1e-5;
// tighter targets: one FP64 pass at x32 (1 + {-d, 0, d}), d = kInterpDel, and
// the tables interpolated to a root within kInterpReach x32 of x32
static constexpr double kInterpDel = 2e-6;
static constexpr double kInterpReach = 1e-5;
// pinned host scalars of a plan build (8 + 4 kPlanes doubles): [0, kPlanes)
// eps^2 dk dw per plane going in, [8, 8 + kPlanes) the planes' max sum_b2
// coming back ([9] the linear pass's max), kSumSlot the sum of S
static constexpr int kSumSlot = 8 + 4 * kPlanes - 1;

// The pinned host scalars of a plan build (above) and its error words
// ((kPlanes + 1) ints after them), one page-locked block per plan, kept for
// reuse when the plan is destroyed: page-locking costs ~0.1 ms, a tenth of
// the build of a small plan.
static constexpr size_t kPinErrOff = (8 + 4 * kPlanes) * sizeof(double);
static constexpr size_t kPinBytes = kPinErrOff + (kPlanes + 1) * sizeof(int);
static std::mutex g_pin_mu;
static std::vector<void *> g_pin_free;

static cudaError_t pinned_get(void **out) {
  {
    std::lock_guard<std::mutex> lock(g_pin_mu);
    if (!g_pin_free.empty()) {
      *out = g_pin_free.back();
      g_pin_free.pop_back();
      return cudaSuccess;
    }
  }
  return cudaMallocHost(out, kPinBytes);
}

static void pinned_put(void *p) {
  std::lock_guard<std::mutex> lock(g_pin_mu);
  g_pin_free.push_back(p);
}

// Index lists of the recursion pass, written on the device from small
// offset tables: the lattice points in level order (level d holds kk = lo
// .. hi, lo = max(0, d - nw + 1), hi = min(d, nk - 1)), and for bulk phase
// ph the points of its band of levels [D, min(2D, nlev)), D = ph BL, as
// pairs (kk, kw), (kk, kw + 1) along each lattice row: row kk of phase ph
// holds the pairs starting at kw = lo(kk), lo(kk) + 2, ... <= hi(kk).  A
// phase lists first, row by row, the pairs whose first point lies below
// level D + BL (the points of the fringe block that follows the phase),
// from entry seg[2 (ph - 1) nk + kk], then the others, from entry
// seg[(2 (ph - 1) + 1) nk + kk].
__global__ void k_level_points(int nk, int nw, int nlev, const int *__restrict__ lev_off,
                               int2 *__restrict__ pts) {
  const int d = blockIdx.x;
  if (d >= nlev) return;
  const int lo = max(0, d - nw + 1), hi = min(d, nk - 1);
  for (int kk = lo + threadIdx.x; kk <= hi; kk += blockDim.x)
    pts[lev_off[d] + kk - lo] = make_int2(kk, d - kk);
}

__global__ void k_bulk_pairs(int nk, int nw, int nlev, const int *__restrict__ seg,
                             int2 *__restrict__ pairs) {
  const int ph = 1 + blockIdx.y, kk = blockIdx.x;
  const int D = ph * kRecBL, dend = min(2 * D, nlev);
  const int lo = max(0, D - kk), hi = min(nw - 1, dend - 1 - kk);
  const int hu = min(hi, D + kRecBL - 1 - kk);  // last first point of the fringe block
  const int nu = hu >= lo ? (hu - lo) / 2 + 1 : 0;
  const int bu = seg[2 * (ph - 1) * nk + kk], bd = seg[(2 * (ph - 1) + 1) * nk + kk];
  for (int j = threadIdx.x; lo + 2 * j <= hi; j += blockDim.x)
    pairs[j < nu ? bu + j : bd + j - nu] = make_int2(kk, lo + 2 * j);
}

// Resident-block counts of the recursion kernels per device (they depend on
// the kernel and its shared memory only).
struct RecOccupancy {
  int nsm = 0, b64 = 0, b32 = 0, b64f = 0, b32f = 0;
};

template <bool SEP>
static int rec_occupancy_of(RecOccupancy &o) {
  int b64 = 0, b64f = 0, b32 = 0, b32f = 0;
  constexpr int sm = kRecSmem + kFringeSmem;
  SRM3_CUDA(cudaFuncSetAttribute(k_rec_pass<double, 1, SEP>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
  SRM3_CUDA(cudaFuncSetAttribute(k_rec_pass<float, kPlanes, SEP>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
  SRM3_CUDA(cudaFuncSetAttribute(k_rec_pass<float, kWindowPlanes, SEP>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
  SRM3_CUDA(cudaFuncSetAttribute(k_rec_pass<double, 3, SEP>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
  SRM3_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b64, k_rec_pass<double, 1, SEP>,
                                                          kRecThreads, sm));
  int b64x3 = 0;
  SRM3_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b64x3, k_rec_pass<double, 3, SEP>,
                                                          kRecThreads, sm));
  b64 = std::min(b64, b64x3);
  b64f = b64;
  SRM3_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b32, k_rec_pass<float, kPlanes, SEP>,
                                                          kRecThreads, sm));
  int b32w = 0;
  SRM3_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &b32w, k_rec_pass<float, kWindowPlanes, SEP>, kRecThreads, sm));
  b32 = std::min(b32, b32w);
  b32f = b32;
  o.b64 = std::min(o.b64, b64);
  o.b64f = std::min(o.b64f, b64f);
  o.b32 = std::min(o.b32, b32);
  o.b32f = std::min(o.b32f, b32f);
  return SRM3_OK;
}

// Resident CTAs per SM of every recursion kernel variant (the minimum over
// the plain and separable forms), per device.
static int rec_occupancy(int dev, RecOccupancy *out) {
  static std::mutex mu;
  static RecOccupancy cache[64];
  static bool have[64] = {};
  std::lock_guard<std::mutex> lock(mu);
  if (dev < 0 || dev >= 64) return fail(SRM3_ERR_NOT_SUPPORTED, "device ordinal beyond 64");
  if (!have[dev]) {
    RecOccupancy o;
    o.b64 = o.b64f = o.b32 = o.b32f = 1 << 30;
    SRM3_CUDA(cudaDeviceGetAttribute(&o.nsm, cudaDevAttrMultiProcessorCount, dev));
    int rc = rec_occupancy_of<false>(o);
    if (!rc) rc = rec_occupancy_of<true>(o);
    if (rc) return rc;
    cache[dev] = o;
    have[dev] = true;
  }
  *out = cache[dev];
  return SRM3_OK;
}

// Device state of the persistent recursion pass.
static int setup_recursion(srm3_plan *p, cudaStream_t st) {
  const int nk = p->nk, nw = p->nw;
  const int nlev = nk + nw - 1;
  // first point of each level, and the first bulk pair of each (phase, row)
  std::vector<int> lev_off(nlev + 1, 0);
  for (int d = 0; d < nlev; ++d)
    lev_off[d + 1] = lev_off[d] + std::min(d, nk - 1) - std::max(0, d - nw + 1) + 1;
  const int nph = std::max(0, (nlev - 1) / kRecBL);  // phases D = BL, 2 BL, ... < nlev
  std::vector<int> seg((size_t)2 * nph * nk + 1, 0);
  // pair_off[0 .. nph]: first pair of each phase (and the end); then
  // pair_off[nph + 1 + ph]: the first pair of phase ph past the fringe block
  std::vector<int> pair_off(2 * (nph + 1), 0);
  for (int ph = 1; ph <= nph; ++ph) {
    const int D = ph * kRecBL, dend = std::min(2 * D, nlev);
    for (int part = 0; part < 2; ++part)
      for (int kk = 0; kk < nk; ++kk) {
        const int lo = std::max(0, D - kk), hi = std::min(nw - 1, dend - 1 - kk);
        const int hu = std::min(hi, D + kRecBL - 1 - kk);
        const int nall = hi >= lo ? (hi - lo) / 2 + 1 : 0;
        const int nu = hu >= lo ? (hu - lo) / 2 + 1 : 0;
        const size_t i = (size_t)(2 * (ph - 1) + part) * nk + kk;
        seg[i + 1] = seg[i] + (part == 0 ? nu : nall - nu);
      }
    pair_off[nph + 1 + ph] = seg[(size_t)(2 * (ph - 1) + 1) * nk];
    pair_off[ph] = seg[(size_t)2 * ph * nk];
  }
  const int npairs = std::max(1, seg[(size_t)2 * nph * nk]);
  int *d_seg = nullptr;
  SRM3_CUDA(dev_alloc(&p->rec_items, sizeof(int2) * lev_off[nlev], st));
  SRM3_CUDA(dev_alloc(&p->rec_lev_off, sizeof(int) * (nlev + 1), st));
  SRM3_CUDA(dev_alloc(&p->rec_pairs, sizeof(int2) * npairs, st));
  SRM3_CUDA(dev_alloc(&p->rec_pair_off, sizeof(int) * pair_off.size(), st));
  SRM3_CUDA(dev_alloc(&d_seg, sizeof(int) * seg.size(), st));
  SRM3_CUDA(cudaMemcpyAsync(p->rec_lev_off, lev_off.data(), sizeof(int) * (nlev + 1),
                            cudaMemcpyHostToDevice, st));
  SRM3_CUDA(cudaMemcpyAsync(p->rec_pair_off, pair_off.data(), sizeof(int) * pair_off.size(),
                            cudaMemcpyHostToDevice, st));
  SRM3_CUDA(cudaMemcpyAsync(d_seg, seg.data(), sizeof(int) * seg.size(), cudaMemcpyHostToDevice,
                            st));
  k_level_points<<<nlev, 128, 0, st>>>(nk, nw, nlev, p->rec_lev_off, p->rec_items);
  if (nph > 0) k_bulk_pairs<<<dim3(nk, nph), 128, 0, st>>>(nk, nw, nlev, d_seg, p->rec_pairs);
  SRM3_CUDA(cudaGetLastError());
  p->n_launch += nph > 0 ? 2 : 1;
  SRM3_CUDA(dev_free(d_seg, st));
  // running bulk sums: up to 32 bytes per point (8 FP32 planes or 3 FP64)
  SRM3_CUDA(dev_alloc(&p->rec_partial, (size_t)nk * nw * 32, st));
  SRM3_CUDA(dev_alloc(&p->rec_max, kPlanes * sizeof(unsigned long long), st));
  // separable envelope: the FFT form of the bulk when its grids fit the
  // pass's shared memory (else the direct bulk, as for any envelope)
  if (p->sep) {
    int log2Lmax = 0;
    for (int D = kRecBL; D < nlev; D += kRecBL)
      log2Lmax = std::max(log2Lmax, ilog2_exact(kRecBL) + __builtin_ctz(D / kRecBL));
    const int L2max = 2 << log2Lmax;
    int log2Nc = 1;
    while ((1 << log2Nc) < nk + std::min(L2max, nk) - 1) ++log2Nc;
    const int cap = kRecSmem / (int)sizeof(double2);  // FP64 is the tighter case
    if (nlev > kRecBL && fft_row_len(1 << log2Nc) <= cap && fft_col_stride(L2max) <= cap) {
      const int ntw = std::max(1 << log2Nc, L2max);
      p->rec_fft = true;
      p->rec_log2Nc = log2Nc;
      SRM3_CUDA(dev_alloc(&p->rec_z, (size_t)L2max * ((size_t)1 << log2Nc) *
                                          std::max(kPlanes * sizeof(float2), sizeof(double2)), st));
      SRM3_CUDA(dev_alloc(&p->tw_rec32, ntw * sizeof(float2), st));
      SRM3_CUDA(dev_alloc(&p->tw_rec64, ntw * sizeof(double2), st));
      k_twiddles<float2><<<cdiv(ntw, 256), 256, 0, st>>>(ntw, ilog2_exact(ntw),
                                                         (float2 *)p->tw_rec32);
      k_twiddles<double2><<<cdiv(ntw, 256), 256, 0, st>>>(ntw, ilog2_exact(ntw),
                                                          (double2 *)p->tw_rec64);
      SRM3_CUDA(cudaGetLastError());
      p->n_launch += 2;
    }
  }
  // sum of S (the exact variance), once, read after the next synchronisation
  // of the stream (run_pass_multi); the plane-0 results of this reduction
  // are not used
  SRM3_CUDA(cudaMemsetAsync(p->sb2, 0, (size_t)nk * nw * sizeof(double), st));
  if (int rc0 = reduce_plane0(p, st)) return rc0;
  SRM3_CUDA(cudaMemcpyAsync(p->h_pinned + kSumSlot, p->scal + 11, sizeof(double),
                            cudaMemcpyDeviceToHost, st));
  p->sumS = -1.0;  // not read yet
  // barrier counter, two tickets per bulk phase (its points of the next
  // fringe block, then the others), and the fringe progress of every
  // lattice row
  p->rec_bar_tickets = 2 + 2 * ((nk + nw) / kRecBL + 1);
  p->rec_bar_words = p->rec_bar_tickets + nk;
  SRM3_CUDA(dev_alloc(&p->rec_bar, p->rec_bar_words * sizeof(unsigned int), st));
  SRM3_CUDA(cudaMemsetAsync(p->rec_bar, 0, p->rec_bar_words * sizeof(unsigned int), st));
  RecOccupancy occ;
  int rc = rec_occupancy(p->device, &occ);
  if (rc) return rc;
  const bool f = p->rec_fft;
  if ((f ? occ.b64f : occ.b64) < 1 || (f ? occ.b32f : occ.b32) < 1)
    return fail(SRM3_ERR_CUDA, "recursion kernel cannot be resident");
  const int nsm = occ.nsm;
  SRM3_CUDA(dev_alloc(&p->qm3, 3 * (size_t)nk * nw * sizeof(double), st));
  p->rec_grid64 = nsm;
  p->rec_grid32 = nsm;
  return SRM3_OK;
}

// One recursion pass at x_m = eps_m^2 for m < M planes: the FP64 pass
// (M = 1, writes qm; M = 3 writes qm3) or the FP32 search pass (M = kPlanes,
// or kWindowPlanes without the FFT form of the bulk; writes qm32).
static int start_w_table(srm3_plan *p, cudaStream_t st);

static int run_pass_multi(srm3_plan *p, cudaStream_t st, const double *x, int M, bool fp64,
                          PassResult *r) {
  for (int m = 0; m < M; ++m) p->h_pinned[m] = x[m] * p->dkdw;
  SRM3_CUDA(cudaMemcpyAsync(p->scal, p->h_pinned, M * sizeof(double), cudaMemcpyHostToDevice, st));
  SRM3_CUDA(cudaMemsetAsync(p->err, 0, (kPlanes + 1) * sizeof(int), st));
  SRM3_CUDA(cudaMemsetAsync(p->rec_bar, 0, p->rec_bar_words * sizeof(unsigned int), st));
  SRM3_CUDA(cudaMemsetAsync(p->rec_max, 0, kPlanes * sizeof(unsigned long long), st));
  RecArgs A;
  A.nk = p->nk;
  A.nw = p->nw;
  A.nlev = p->nk + p->nw - 1;
  A.nl = (long long)p->nk * p->nw;
  A.pts = p->rec_items;
  A.pt_off = p->rec_lev_off;
  A.pairs = p->rec_pairs;
  A.pair_off = p->rec_pair_off;
  A.pair_mid = p->rec_pair_off + (A.nlev - 1) / kRecBL + 1;
  A.tk_def = (p->nk + p->nw) / kRecBL + 1;
  A.S = p->S;
  if (fp64 && M != 1 && M != 3)
    return fail(SRM3_ERR_INVALID_ARG, "FP64 recursion pass takes one or three planes");
  if (fp64 && M == 3 && (p->rec_fft || p->mixed))
    return fail(SRM3_ERR_INVALID_ARG, "three-plane FP64 pass: direct bulk, sum pairs only");
  if (!fp64 && M != kPlanes && (M != kWindowPlanes || p->rec_fft))
    return fail(SRM3_ERR_INVALID_ARG, "FP32 recursion pass: 8 planes, or 4 with the direct bulk");
  const bool sepf = p->rec_sep;
  const bool x3 = fp64 && M == 3;
  if (x3 && sepf && !p->qo3) SRM3_CUDA(dev_alloc(&p->qo3, 3 * (size_t)p->nk * p->nw * sizeof(double), st));
  A.q = !fp64 ? (void *)p->qm32 : x3 ? (void *)p->qm3 : (sepf ? (void *)p->qh : (void *)p->qm);
  A.e2 = sepf ? (p->sep ? p->env_e2 : p->rs_a2) : nullptr;
  A.e2k = sepf ? (p->sep ? p->env_b2 : p->rs_b2) : nullptr;
  A.qout = (sepf && fp64) ? (x3 ? p->qo3 : p->qm) : nullptr;
  A.dsum = (p->mixed && fp64 && M == 1) ? p->Dsum : nullptr;
  A.acc = p->rec_partial;
  A.sb2 = p->sb2;
  A.G2 = fp64 ? (const void *)p->G2 : (const void *)p->G2_32;
  A.scal = p->scal;
  A.err = p->err;
  A.bar = p->rec_bar;
  A.row_done = p->rec_bar + p->rec_bar_tickets;
  A.abort = p->err + kPlanes;
  A.maxb = p->rec_max;
  A.zr = p->rec_fft ? p->rec_z : nullptr;
  A.twr = fp64 ? p->tw_rec64 : p->tw_rec32;
  A.log2Nc = p->rec_log2Nc;
  A.zcap = kRecSmem / (fp64 ? (int)sizeof(double2) : (int)sizeof(float2));
  // the fringe's state, and the FFT form's grids where it is used
  const int smem = kFringeSmem + (p->rec_fft ? kRecSmem : 0);
  void *args[] = {&A};
  SRM3_CUDA(cudaEventRecord(t_ev[0], st));
  const void *kern =
      x3 ? (sepf ? (const void *)k_rec_pass<double, 3, true>
                 : (const void *)k_rec_pass<double, 3, false>)
      : fp64 ? (sepf ? (const void *)k_rec_pass<double, 1, true>
                     : (const void *)k_rec_pass<double, 1, false>)
      : M == kWindowPlanes ? (sepf ? (const void *)k_rec_pass<float, kWindowPlanes, true>
                                   : (const void *)k_rec_pass<float, kWindowPlanes, false>)
             : (sepf ? (const void *)k_rec_pass<float, kPlanes, true>
                     : (const void *)k_rec_pass<float, kPlanes, false>);
  SRM3_CUDA(cudaLaunchCooperativeKernel(kern, fp64 ? p->rec_grid64 : p->rec_grid32, kRecThreads,
                                        args, smem, st));
  SRM3_CUDA(cudaGetLastError());
  p->n_launch += 1;
  if (fp64 && p->w_deferred) {  // the W table, on the room the pass leaves
    p->w_deferred = false;
    if (int rcw = start_w_table(p, p->w_stream)) return rcw;
  }
  SRM3_CUDA(cudaEventRecord(t_ev[1], st));
  SRM3_CUDA(cudaMemcpyAsync(p->h_pinned + 8, p->rec_max, M * sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, st));
  SRM3_CUDA(cudaMemcpyAsync(p->h_err, p->err, (kPlanes + 1) * sizeof(int), cudaMemcpyDeviceToHost,
                            st));
  SRM3_CUDA(cudaStreamSynchronize(st));
  if (p->sumS < 0.0) p->sumS = p->h_pinned[kSumSlot];  // copied by setup_recursion
  float ms = 0.f;
  SRM3_CUDA(cudaEventElapsedTime(&ms, t_ev[0], t_ev[1]));
  p->t_recursion_ms += ms;
  (fp64 ? p->t_rec64_ms : p->t_rec32_ms) += ms;
  if (p->h_err[kPlanes])
    return fail(SRM3_ERR_TIMEOUT, "recursion pass: grid barrier wait timed out");
  for (int m = 0; m < M; ++m) {
    r[m].max_sb2 = p->h_pinned[8 + m];  // the bits of a double, copied as such
    r[m].min_pure = 1.0 - r[m].max_sb2;
    r[m].sumS = p->sumS;
    r[m].err = p->h_err[m];
  }
  if (fp64)
    p->root_passes += 1;
  else
    p->root_passes32 += 1;
  return SRM3_OK;
}

static int run_pass(srm3_plan *p, cudaStream_t st, double x, bool fp64, PassResult *r) {
  return run_pass_multi(p, st, &x, 1, fp64, r);
}

// ---------------------------------------------------------------------------
// Mixed-sign interactions: Eq. pure as a fixed point.  With difference pairs
// S_p(k) depends on points of higher omega, so q = S/S_p solves
//   q_k = 1 / (1 - x dk dw [sum_{Pi(k)} g^2 q_i q_j + sum_{D(k)} g^2 q_i q_j]).
// The right side increases with q and with x, so iterations that start
// below the largest-S_p (smallest-q) solution rise to it monotonically: from
// q = 1, or from the converged q of a smaller x.  One iteration is the
// difference sums at the current q (k_rec_diff) followed by one level pass,
// which takes the sum pairs of every point from the values the pass has just
// formed at lower levels -- the Gauss-Seidel order of the plain recursion --
// and adds the difference sums before forming q_k.  The iterations stop when
// no q_k moves by more than kFpTol relative; they give up (the solve counts
// as failed, as above the target) after kFpMaxIters, and a pass that meets
// sum b_p^2 >= 1 fails at once.
constexpr double kFpTol = 4e-16;
constexpr int kFpMaxIters = 400;

__global__ void k_q_init(long long n, const double *__restrict__ S, double *__restrict__ q) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) q[i] = S[i] > 0.0 ? 1.0 : 0.0;
}

// max over S > 0 of |qn - qo| / qn into *out (the bits of a double >= 0)
__global__ void k_q_change(long long n, const double *__restrict__ S,
                           const double *__restrict__ qn, const double *__restrict__ qo,
                           unsigned long long *out) {
  double m = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    if (S[i] > 0.0 && qn[i] > 0.0) m = fmax(m, fabs(qn[i] - qo[i]) / qn[i]);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// Solve the fixed point at x from the iterate in p->qm; r: the last pass
// (r->err != 0: no solution was reached).
static int solve_mixed(srm3_plan *p, cudaStream_t st, double x, PassResult *r) {
  const long long nl = (long long)p->nk * p->nw;
  for (int it = 1; it <= kFpMaxIters; ++it) {
    k_rec_diff<<<cdiv(nl * 32, 256), 256, 0, st>>>(p->nk, p->nw, p->S, p->qm, p->EkSq, p->EwSq,
                                                    p->Dsum);
    SRM3_CUDA(cudaGetLastError());
    SRM3_CUDA(cudaMemcpyAsync(p->qprev, p->qm, nl * sizeof(double), cudaMemcpyDeviceToDevice, st));
    int rc = run_pass_multi(p, st, &x, 1, true, r);
    if (rc) return rc;
    p->fp_iters = it;
    if (r->err) return SRM3_OK;
    SRM3_CUDA(cudaMemsetAsync(p->fp_change, 0, sizeof(unsigned long long), st));
    k_q_change<<<std::min(cdiv(nl, 256), 1024), 256, 0, st>>>(nl, p->S, p->qm, p->qprev,
                                                               p->fp_change);
    SRM3_CUDA(cudaGetLastError());
    unsigned long long bits = 0;
    SRM3_CUDA(cudaMemcpyAsync(&bits, p->fp_change, sizeof(bits), cudaMemcpyDeviceToHost, st));
    SRM3_CUDA(cudaStreamSynchronize(st));
    double ch;
    std::memcpy(&ch, &bits, sizeof(ch));
    if (it >= 2 && ch <= kFpTol) return SRM3_OK;
  }
  r->err = 1;  // no convergence: treated as an infeasible x
  return SRM3_OK;
}

// One FP64 evaluation of max_k sum_b2 at x: a recursion pass, or for mixed
// plans a fixed-point solve started from the converged q of the largest x
// below the target seen so far (when x is above it), else from q = 1.
static int eval_fp64(srm3_plan *p, cudaStream_t st, double x, double target, PassResult *r) {
  if (!p->mixed) return run_pass_multi(p, st, &x, 1, true, r);
  const long long nl = (long long)p->nk * p->nw;
  if (p->qlo_x >= 0.0 && x >= p->qlo_x)
    SRM3_CUDA(cudaMemcpyAsync(p->qm, p->qlo, nl * sizeof(double), cudaMemcpyDeviceToDevice, st));
  else
    k_q_init<<<cdiv(nl, 256), 256, 0, st>>>(nl, p->S, p->qm);
  SRM3_CUDA(cudaGetLastError());
  int rc = solve_mixed(p, st, x, r);
  if (rc) return rc;
  if (!r->err && r->max_sb2 < target && x > p->qlo_x) {
    SRM3_CUDA(cudaMemcpyAsync(p->qlo, p->qm, nl * sizeof(double), cudaMemcpyDeviceToDevice, st));
    p->qlo_x = x;
  }
  return SRM3_OK;
}

// Bracketed FP64 root search on x = eps^2 for f(x) = max_k sum_b2(x) -
// target, which increases with x; a failed pass (some S_p <= 0) counts as
// above target.  Illinois regula falsi (bisection while the upper end is a
// failed pass) until |f| <= tol or the bracket is a few ulp wide.
struct Bracket {
  double xlo, flo, xhi, fhi;
  bool hi_failed;
};

static int illinois(srm3_plan *p, cudaStream_t st, double target, double tol, int max_it,
                    Bracket &b, double *xbest, PassResult *best, bool *tables_at_best) {
  int side = 0;
  PassResult r;
  double xlast = -1.0;
  for (int it = 0; it < max_it; ++it) {
    if (b.xhi - b.xlo <= 4.0 * 2.220446049250313e-16 * b.xhi) break;
    double x;
    if (b.hi_failed) {
      x = 0.5 * (b.xlo + b.xhi);
    } else {
      x = b.xhi - b.fhi * (b.xhi - b.xlo) / (b.fhi - b.flo);
      if (!(x > b.xlo && x < b.xhi)) x = 0.5 * (b.xlo + b.xhi);
    }
    int rc = eval_fp64(p, st, x, target, &r);
    if (rc) return rc;
    xlast = x;
    if (r.err) {
      b.xhi = x;
      b.hi_failed = true;
      side = 1;
      continue;
    }
    const double f = r.max_sb2 - target;
    *best = r;
    *xbest = x;
    if (std::fabs(f) <= tol) break;
    if (f < 0) {
      b.xlo = x;
      b.flo = f;
      if (side == -1 && !b.hi_failed) b.fhi *= 0.5;
      side = -1;
    } else {
      b.xhi = x;
      b.fhi = f;
      b.hi_failed = false;
      if (side == 1) b.flo *= 0.5;
      side = 1;
    }
  }
  *tables_at_best = (xlast == *xbest);
  return SRM3_OK;
}

// eps of a mixed plan: FP64 fixed-point solves only.  The slope at q = 1
// comes from one solve at a vanishing x (every q rounds to 1): L = sum_b2 /
// x, sum and difference pairs.  At x0 = target / max L the sum is at least
// the target (q >= 1), and at 0.9 (1 - target)^2 x0 it is below it (every q
// <= 1/(1 - target) below the root); Illinois regula falsi between them,
// each evaluation warm-started from the largest x found below the target.
static int find_eps_mixed(srm3_plan *p, cudaStream_t st, double target, double tol) {
  const long long nl = (long long)p->nk * p->nw;
  PassResult r;
  const double xt = 1e-20;
  p->qlo_x = -1.0;
  k_q_init<<<cdiv(nl, 256), 256, 0, st>>>(nl, p->S, p->qm);
  SRM3_CUDA(cudaGetLastError());
  int rc = solve_mixed(p, st, xt, &r);
  if (rc) return rc;
  const double Lmax = r.max_sb2 / xt;
  if (!(Lmax > 0.0))
    return fail(SRM3_ERR_BISECTION_FAILED, "no bispectral pairs: max_k sum_b2 is 0 for every eps");
  const double x0 = target / Lmax;
  Bracket b{0.0, -target, x0, 1.0, true};
  double xbest = -1.0;
  PassResult best{};
  const double xa = 0.9 * (1.0 - target) * (1.0 - target) * x0;
  if ((rc = eval_fp64(p, st, xa, target, &r))) return rc;
  if (!r.err && r.max_sb2 < target) {
    b.xlo = xa;
    b.flo = r.max_sb2 - target;
    xbest = xa;
    best = r;
  }
  if ((rc = eval_fp64(p, st, x0, target, &r))) return rc;
  if (!r.err) {
    b.fhi = r.max_sb2 - target;
    b.hi_failed = false;
    xbest = x0;
    best = r;
  }
  bool at_best = !r.err;
  if (r.err || std::fabs(r.max_sb2 - target) > tol) {
    rc = illinois(p, st, target, tol, 200, b, &xbest, &best, &at_best);
    if (rc) return rc;
  }
  if (xbest < 0.0) return fail(SRM3_ERR_BISECTION_FAILED, "eps search found no feasible point");
  if (!at_best) {
    if ((rc = eval_fp64(p, st, xbest, target, &best))) return rc;
    if (best.err) return fail(SRM3_ERR_BISECTION_FAILED, "eps search: final solve failed");
  }
  p->eps = std::sqrt(xbest);
  p->max_sb2 = best.max_sb2;
  p->min_pure = best.min_pure;
  p->variance = 4.0 * p->dkdw * best.sumS;
  return SRM3_OK;
}

// The tables of the last FP64 pass (sum_b2 plane 0, q) moved by dx in x to
// first order with the slopes in p->dsb2; r: the new max_k sum_b2 and
// whether some sum_b2 reached 1.
static int shift_tables(srm3_plan *p, cudaStream_t st, double dx, PassResult *r) {
  const long long nl = (long long)p->nk * p->nw;
  SRM3_CUDA(cudaMemsetAsync(p->rec_max, 0, sizeof(unsigned long long), st));
  SRM3_CUDA(cudaMemsetAsync(p->err, 0, sizeof(int), st));
  k_sb2_shift<<<cdiv(nl, 256), 256, 0, st>>>(nl, p->S, p->sb2, p->dsb2, dx, p->qm, p->rec_max,
                                             p->err);
  SRM3_CUDA(cudaGetLastError());
  SRM3_CUDA(cudaMemcpyAsync(p->h_pinned + 8, p->rec_max, sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, st));
  SRM3_CUDA(cudaMemcpyAsync(p->h_err, p->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  SRM3_CUDA(cudaStreamSynchronize(st));
  r->max_sb2 = p->h_pinned[8];  // the bits of a double, copied as such
  r->min_pure = 1.0 - r->max_sb2;
  r->err = p->h_err[0];
  return SRM3_OK;
}

// ---------------------------------------------------------------------------
// eps from max_k sum_b2 = target (plans without mixed interactions).
//
// FP32 stage.  Each FP32 pass evaluates f(x) = max_k sum_b2 - target at
// kPlanes values of x = eps^2 at once.  The root is bracketed in one of two
// ways:
//  * coarse start (lattices of at least kCoarsePoints points): the same
//    search on a coarser lattice -- every fk-th kappa and fw-th omega point
//    of this one, fk, fw powers of two keeping at least kCoarseMinDim points
//    per axis -- whose sums are the same quadrature of Eq. pure's pair
//    integral on a coarser grid, places the root within a few 1e-3; one pass
//    here over +-kCoarseWindow around it then brackets the root and samples
//    f finely enough around it for the steps below.  If that pass does not
//    bracket the root, the wide search follows, keeping its points.
//  * wide search: the linear pass (q == 1) bounds the root by target / max
//    L, as q >= 1 makes x L an under-estimate of sum_b2; the first pass
//    samples [(1 - target)^2 x0, x0] (x0 = target / Lmax, with margins), the
//    second zooms on the first pass's quadratic estimate, later ones (only
//    when the root was not inside) subdivide the bracket.
// Inverse quadratic interpolation through the bracket and its nearest
// feasible neighbour then gives x32, and the quadratic's slope at the root.
//
// FP64 stage: Newton steps from x32 with the FP32 slope, then secant steps
// on the FP64 values inside an FP64 bracket; Illinois if they leave it or
// stall.  Loose targets (FP32 plans) may instead move the tables of the
// first FP64 pass to the Newton root to first order (shift_tables).  The
// tables left in the plan are those of the final FP64 pass, or of that move.

static constexpr int kCoarseMinDim = 64;
static constexpr long long kCoarsePoints = 1LL << 16;
static constexpr double kCoarseWindow = 0.015;

struct Search32 {
  std::vector<std::pair<double, double>> pts;  // (x, f); f = +inf: failed pass
  int np = kPlanes;       // planes of the last pass
  double xs[kPlanes];
  PassResult r[kPlanes];  // the last pass
  double x0 = -1.0;       // target / Lmax once the wide search has run
};

// Lmax = max_k L_k, the small-x slope of sum_b2 (wide search).
static int linear_bound(srm3_plan *p, cudaStream_t st, double *Lmax) {
  if (p->sep) {
    // separable envelope: the slope at q = 1 from one FP32 pass at a
    // vanishing x (every q rounds to 1), L = sum_b2 / x
    const double xt = 1e-20;
    double xs0[kPlanes];
    PassResult r0[kPlanes];
    for (int m = 0; m < kPlanes; ++m) xs0[m] = xt;
    int rc0 = run_pass_multi(p, st, xs0, kPlanes, false, r0);
    if (rc0) return rc0;
    *Lmax = r0[0].max_sb2 / xt;
    return SRM3_OK;
  }
  const int nblk = cdiv(p->nw, kLinOut);
  const size_t smem = (size_t)3 * p->nw * sizeof(float);
  const long long nl = (long long)p->nk * p->nw;
  SRM3_CUDA(cudaFuncSetAttribute(k_rec_linear, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
  // the parts go to the FP32 search state, not yet in use (8 floats per point)
  static_assert(kLinParts <= kPlanes, "linear-pass parts fit the FP32 search state");
  k_rec_linear<<<p->nk * nblk * kLinParts, kLinOut, smem, st>>>(p->nk, p->nw, p->S, p->EkSq32,
                                                                 p->EwSq32, p->qm32);
  k_rec_linear_sum<<<cdiv(nl, 256), 256, 0, st>>>(nl, p->S, p->qm32, p->sb2, p->dkdw);
  SRM3_CUDA(cudaGetLastError());
  p->n_launch += 2;
  SRM3_CUDA(cudaMemsetAsync(p->qm32, 0, kLinParts * nl * sizeof(float), st));
  if (int rc1 = reduce_plane0(p, st)) return rc1;
  SRM3_CUDA(cudaMemcpyAsync(p->h_pinned + 9, p->scal + 9, sizeof(double),
                            cudaMemcpyDeviceToHost, st));
  SRM3_CUDA(cudaStreamSynchronize(st));
  *Lmax = p->h_pinned[9];
  return SRM3_OK;
}

// Index of the first point of s.pts (sorted) at or above the target, or
// pts.size() when every point is below it.
static size_t first_above(const Search32 &s) {
  size_t j = 0;
  while (j < s.pts.size() && s.pts[j].second < 0) ++j;
  return j;
}

static double quad_root(double xa, double fa, double xb, double fb, double xc, double fc) {
  return xa * fb * fc / ((fa - fb) * (fa - fc)) + xb * fa * fc / ((fb - fa) * (fb - fc)) +
         xc * fa * fb / ((fc - fa) * (fc - fb));
}

// The wide search, adding to the points s already holds; returns with a
// bracket whose upper end is feasible, or fails.
static int wide_search(srm3_plan *p, cudaStream_t st, double target, Search32 &s) {
  double Lmax = 0.0;
  int rc = linear_bound(p, st, &Lmax);
  if (rc) return rc;
  if (!(Lmax > 0.0))
    return fail(SRM3_ERR_BISECTION_FAILED, "no bispectral pairs: max_k sum_b2 is 0 for every eps");
  // at the root every sum_b2 <= target, so q <= 1/(1 - target) and x* lies
  // in [(1 - target)^2 x0, x0] (q >= 1 gives the upper end); the first pass
  // samples that range, with a margin for the FP32 Lmax.  Each later pass
  // centres its planes on the quadratic estimate of the passes so far,
  // half-width four times that estimate's distance from the secant root
  // (at least 2e-4 of it, at most half its distance to the bracket's ends),
  // until the root lies between two planes of one pass -- normally after
  // the second pass; a zoom that missed the root takes a third.
  const double x0 = target / Lmax;
  s.x0 = x0;
  double lo = 0.9 * (1.0 - target) * (1.0 - target) * x0, hi = 1.01 * x0;
  bool hi_known = false;
  double zoom_c = 0.0, zoom_w = 0.0;  // centre and half-width of the next zoom
  for (int pass = 0; pass < 12; ++pass) {
    const double lo_pass = lo, hi_pass = hi;  // the range the planes below cover
    s.np = kPlanes;
    for (int m = 0; m < kPlanes; ++m) {
      if (pass == 0)
        s.xs[m] = lo + (hi - lo) * m / (kPlanes - 1);
      else if (zoom_w > 0.0)
        s.xs[m] = zoom_c - zoom_w + 2.0 * zoom_w * m / (kPlanes - 1);
      else
        s.xs[m] = hi_known ? lo + (hi - lo) * (m + 1) / (kPlanes + 1)
                           : lo + (hi - lo) * (m + 1) / kPlanes;
    }
    rc = run_pass_multi(p, st, s.xs, kPlanes, false, s.r);
    if (rc) return rc;
    for (int m = 0; m < kPlanes; ++m)
      s.pts.push_back({s.xs[m], s.r[m].err ? INFINITY : s.r[m].max_sb2 - target});
    std::sort(s.pts.begin(), s.pts.end());
    const size_t j = first_above(s);
    if (j == s.pts.size()) {  // every point below target: move the range up
      lo = s.pts.back().first;
      hi = 2.0 * lo;
      hi_known = false;
      zoom_w = 0.0;
      continue;
    }
    lo = s.pts[j - 1].first;
    hi = s.pts[j].first;
    hi_known = true;
    // done when both ends of the bracket are planes of this pass (a zoom, or
    // a subdivision of the last bracket)
    const double h =
        pass == 0 ? 0.0 : (zoom_w > 0.0 ? 2.0 * zoom_w : hi_pass - lo_pass) / (kPlanes - 1);
    if (pass >= 1 && std::isfinite(s.pts[j].second) && hi - lo <= 1.01 * h) return SRM3_OK;
    zoom_w = 0.0;
    if (std::isfinite(s.pts[j].second) &&
        ((j + 1 < s.pts.size() && std::isfinite(s.pts[j + 1].second)) || j >= 2)) {
      // quadratic through the bracket and its feasible neighbour above, else
      // the one below
      const double xl = s.pts[j - 1].first, fl = s.pts[j - 1].second;
      const double xh = s.pts[j].first, fh = s.pts[j].second;
      const double xsec = xl - fl * (xh - xl) / (fh - fl);
      const bool above = j + 1 < s.pts.size() && std::isfinite(s.pts[j + 1].second);
      const double xq = above ? quad_root(xl, fl, xh, fh, s.pts[j + 1].first, s.pts[j + 1].second)
                              : quad_root(s.pts[j - 2].first, s.pts[j - 2].second, xl, fl, xh, fh);
      if (xq > xl && xq < xh) {
        zoom_c = xq;
        zoom_w = std::max(4.0 * std::fabs(xq - xsec), 2e-4 * xq);
        zoom_w = std::min(zoom_w, 0.5 * std::min(xq - xl, xh - xq));
      }
    }
  }
  if (!hi_known) return fail(SRM3_ERR_BISECTION_FAILED, "eps search: target not bracketed");
  return SRM3_OK;
}

// x32 from the points of s: inverse quadratic interpolation through the
// bracket and its nearest feasible neighbour (the secant root when that
// leaves the bracket); *slope = df/dx at the root (0 when unknown).
// Returns false when the bracket's upper end failed (no interpolation).
static bool root_fp32(const Search32 &s, double *x32, double *slope) {
  const size_t jb = first_above(s);
  *slope = 0.0;
  if (jb == 0 || jb == s.pts.size() || !std::isfinite(s.pts[jb].second)) {
    if (jb > 0 && jb < s.pts.size()) *x32 = 0.5 * (s.pts[jb - 1].first + s.pts[jb].first);
    return false;
  }
  const double xl = s.pts[jb - 1].first, fl = s.pts[jb - 1].second;
  const double xh = s.pts[jb].first, fh = s.pts[jb].second;
  const double xsec = xl - fl * (xh - xl) / (fh - fl);
  const bool above = jb + 1 < s.pts.size() && std::isfinite(s.pts[jb + 1].second);
  double x = xsec;
  if (above)
    x = quad_root(xl, fl, xh, fh, s.pts[jb + 1].first, s.pts[jb + 1].second);
  else if (jb >= 2)
    x = quad_root(s.pts[jb - 2].first, s.pts[jb - 2].second, xl, fl, xh, fh);
  if (!(x > xl && x < xh)) x = xsec;
  *x32 = x;
  *slope = (fh - fl) / (xh - xl);
  if (above) {
    // slope at the root of the quadratic through the three points
    const double xa = xl, fa = fl, xb = xh, fb = fh;
    const double xc = s.pts[jb + 1].first, fc = s.pts[jb + 1].second;
    const double dxdf = -xa * (fb + fc) / ((fa - fb) * (fa - fc)) -
                        xb * (fa + fc) / ((fb - fa) * (fb - fc)) -
                        xc * (fa + fb) / ((fc - fa) * (fc - fb));
    if (dxdf > 0.0) *slope = 1.0 / dxdf;
  }
  return true;
}

// S on the coarse lattice: every fk-th kappa and fw-th omega point.
__global__ void k_subsample(int nw, int fk, int fw, int nkc, int nwc, const double *__restrict__ S,
                            double *__restrict__ Sc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nkc * nwc) return;
  const int kc = i / nwc, wc = i - kc * nwc;
  Sc[i] = S[(size_t)kc * fk * nw + (size_t)wc * fw];
}

// The root of the FP32 search on the coarse lattice into *xc (-1: the
// lattice is too small for a coarse start).  The coarse plan borrows the
// plan's pinned host scalars; its device state is freed in stream order.
static int coarse_root(srm3_plan *p, cudaStream_t st, double target, double *xc) {
  *xc = -1.0;
  int fk = 1, fw = 1;
  while (p->nk / (2 * fk) >= kCoarseMinDim) fk *= 2;
  while (p->nw / (2 * fw) >= kCoarseMinDim) fw *= 2;
  if ((long long)p->nk * p->nw < kCoarsePoints || fk * fw < 4) return SRM3_OK;
  // the sum of S of this plan, copied to the shared pinned slot by
  // setup_recursion, is read before the coarse plan reuses the slot
  SRM3_CUDA(cudaStreamSynchronize(st));
  if (p->sumS < 0.0) p->sumS = p->h_pinned[kSumSlot];
  srm3_plan c;
  c.nk = p->nk / fk;
  c.nw = p->nw / fw;
  c.dk = p->dk * fk;
  c.dw = p->dw * fw;
  c.dkdw = c.dk * c.dw;
  c.precision = SRM3_FP32;
  c.device = p->device;
  c.rec_sep = p->rec_sep;
  c.sep = p->sep;
  c.sigma_g = p->sigma_g;
  c.h_pinned = p->h_pinned;
  c.h_err = p->h_err;
  struct Cleanup {
    srm3_plan *c;
    cudaStream_t st;
    ~Cleanup() {
      void *dev[] = {c->S,        c->sb2,       c->scal,    c->err,          c->qm32,
                     c->EkSq,     c->EkSq32,    c->EwSq,    c->EwSq32,       c->G2,
                     c->G2_32,    c->rs_a2,     c->rs_b2,   c->qm3,          c->rec_items,
                     c->rec_lev_off, c->rec_pairs, c->rec_pair_off, c->rec_partial,
                     c->rec_max,  c->rec_bar,   c->red_part, c->env_e2,      c->env_b2,
                     c->rec_z,    c->tw_rec32,  c->tw_rec64};
      for (void *d : dev)
        if (d) dev_free(d, st);
    }
  } cleanup{&c, st};
  const int nkc = c.nk, nwc = c.nw;
  const long long nlc = (long long)nkc * nwc;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  SRM3_CUDA(cudaEventCreate(&e0));
  SRM3_CUDA(cudaEventCreate(&e1));
  struct EvGuard {
    cudaEvent_t a, b;
    ~EvGuard() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } evg{e0, e1};
  SRM3_CUDA(cudaEventRecord(e0, st));
  SRM3_CUDA(dev_alloc(&c.S, nlc * sizeof(double), st));
  SRM3_CUDA(dev_alloc(&c.sb2, kPlanes * nlc * sizeof(double), st));
  SRM3_CUDA(dev_alloc(&c.scal, (8 + 4 * kPlanes) * sizeof(double), st));
  SRM3_CUDA(dev_alloc(&c.err, (kPlanes + 1) * sizeof(int), st));
  SRM3_CUDA(dev_alloc(&c.qm32, kPlanes * nlc * sizeof(float), st));
  SRM3_CUDA(cudaMemsetAsync(c.qm32, 0, kPlanes * nlc * sizeof(float), st));
  SRM3_CUDA(dev_alloc(&c.EkSq, nkc * sizeof(double), st));
  SRM3_CUDA(dev_alloc(&c.EkSq32, nkc * sizeof(float), st));
  SRM3_CUDA(dev_alloc(&c.EwSq, 2 * nwc * sizeof(double), st));
  SRM3_CUDA(dev_alloc(&c.EwSq32, 2 * nwc * sizeof(float), st));
  k_subsample<<<cdiv(nlc, 256), 256, 0, st>>>(p->nw, fk, fw, nkc, nwc, p->S, c.S);
  c.n_launch += 1;
  // the envelope's widths in the coarse lattice's index units: the same
  // function of frequency as on this lattice
  const double sk = p->sigma_g * p->nk / fk, sw = p->sigma_g * p->nw / fw;
  if (c.sep) {
    // separable kind: the factors a^2 and b^2 at the coarse points
    SRM3_CUDA(dev_alloc(&c.env_e2, nlc * sizeof(double), st));
    SRM3_CUDA(dev_alloc(&c.env_b2, nlc * sizeof(double), st));
    k_subsample<<<cdiv(nlc, 256), 256, 0, st>>>(p->nw, fk, fw, nkc, nwc, p->env_e2, c.env_e2);
    k_subsample<<<cdiv(nlc, 256), 256, 0, st>>>(p->nw, fk, fw, nkc, nwc, p->env_b2, c.env_b2);
    c.n_launch += 2;
  } else {
    k_env_sq<<<cdiv(nkc, 256), 256, 0, st>>>(nkc, sk, c.EkSq, c.EkSq32);
    k_env_sq<<<cdiv(2 * nwc, 256), 256, 0, st>>>(2 * nwc, sw, c.EwSq, c.EwSq32);
    c.n_launch += 2;
  }
  if (c.sep) {
    // no g^2 table: the separable recursion takes the pair factor from a^2
  } else if (c.rec_sep) {
    SRM3_CUDA(dev_alloc(&c.rs_a2, nlc * sizeof(double), st));
    SRM3_CUDA(dev_alloc(&c.rs_b2, nlc * sizeof(double), st));
    k_gauss_sep<<<cdiv(nlc, 256), 256, 0, st>>>(nkc, nwc, sk, sw, c.rs_a2, c.rs_b2);
  } else {
    SRM3_CUDA(dev_alloc(&c.G2, nlc * sizeof(double), st));
    SRM3_CUDA(dev_alloc(&c.G2_32, nlc * sizeof(float), st));
    k_g2<<<cdiv(nlc, 256), 256, 0, st>>>(nkc, nwc, c.EkSq, c.EwSq, c.G2, c.G2_32);
  }
  c.n_launch += c.sep ? 0 : 1;
  SRM3_CUDA(cudaGetLastError());
  int rc = setup_recursion(&c, st);
  if (rc) return rc;
  Search32 s;
  s.pts.push_back({0.0, -target});
  // a coarse lattice without pairs or without a root (its support can
  // differ from this lattice's) leaves the search to the wide form
  rc = wide_search(&c, st, target, s);
  if (rc && rc != SRM3_ERR_BISECTION_FAILED) return rc;
  double x = 0.0, slope = 0.0;
  const bool ok = !rc && root_fp32(s, &x, &slope);
  SRM3_CUDA(cudaEventRecord(e1, st));
  SRM3_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  SRM3_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  p->t_coarse_ms = ms;
  p->t_recursion_ms += c.t_recursion_ms;
  p->coarse_passes = c.root_passes32;
  p->coarse_launches = c.n_launch;
  p->coarse_fk = fk;
  p->coarse_fw = fw;
  if (ok) *xc = x;
  return SRM3_OK;
}

static int find_eps(srm3_plan *p, cudaStream_t st, double target, double tol) {
  int rc;
  Search32 s;
  s.pts.push_back({0.0, -target});
  p->coarse_start = false;
  {
    double xc = -1.0;
    rc = coarse_root(p, st, target, &xc);
    if (rc) return rc;
    if (xc > 0.0) {
      // four planes over the window (its spacing of 1 % still leaves x32
      // within ~1e-6 of the root, far inside the FP64 stage's reach), eight
      // for the FFT form of the separable bulk, which keeps exact passes
      s.np = p->rec_fft ? kPlanes : kWindowPlanes;
      for (int m = 0; m < s.np; ++m)
        s.xs[m] = xc * (1.0 + kCoarseWindow * (2.0 * m / (s.np - 1) - 1.0));
      rc = run_pass_multi(p, st, s.xs, s.np, false, s.r);
      if (rc) return rc;
      for (int m = 0; m < s.np; ++m)
        s.pts.push_back({s.xs[m], s.r[m].err ? INFINITY : s.r[m].max_sb2 - target});
      std::sort(s.pts.begin(), s.pts.end());
      const size_t j = first_above(s);
      p->coarse_start = j >= 2 && j < s.pts.size() && std::isfinite(s.pts[j].second);
    }
  }
  if (!p->coarse_start) {
    rc = wide_search(p, st, target, s);
    if (rc) return rc;
  }
  double x32 = 0.0, slope32 = 0.0;
  const bool hi_ok = root_fp32(s, &x32, &slope32);

  // Loose targets (FP32 plans, tol >= kShiftTol): the slope in x of every
  // point's sum_b2 at x32, the derivative of the quadratic through the three
  // planes of the last FP32 pass nearest x32 (two when only two are
  // feasible).  After the FP64 pass at x32 the Newton root x1 is typically
  // within 1e-7 x32; the tables are then moved there to first order,
  // sum_b2(x1) = sum_b2(x32) + (x1 - x32) dsb2 and q = 1/(1 - sum_b2),
  // instead of a second pass.  The error is the slope's (~1e-4 relative:
  // FP32 sums over planes a few 1e-3 apart, and the quadratic's remainder)
  // times the step plus the curvature term, ~1e-11 relative at a 1e-7 step,
  // far below the FP32 rounding of the tables these plans sample with; the
  // result is accepted only when its max_k sum_b2 meets the target within
  // tol.  The slopes need FP32 sums accurate relative to each point: not the
  // FFT form of the separable bulk, whose rounding is bounded relative to
  // the largest sums only (it keeps the second FP64 pass).
  bool shift_ok = false;
  if (tol >= kShiftTol && !p->rec_fft && hi_ok && slope32 > 0.0) {
    int m = -1;
    for (int i = 0; i + 1 < s.np && m < 0; ++i)
      if (s.xs[i] <= x32 && x32 <= s.xs[i + 1] && !s.r[i].err && !s.r[i + 1].err) m = i;
    if (m >= 0) {
      // the third plane: the nearer feasible neighbour of the pair
      int m3 = -1;
      const bool below = m >= 1 && !s.r[m - 1].err;
      const bool above = m + 2 < s.np && !s.r[m + 2].err;
      if (below && above)
        m3 = (x32 - s.xs[m - 1] <= s.xs[m + 2] - x32) ? m - 1 : m + 2;
      else if (below)
        m3 = m - 1;
      else if (above)
        m3 = m + 2;
      double w0, w1, w2 = 0.0;
      const double xa = s.xs[m], xb = s.xs[m + 1];
      if (m3 >= 0) {
        // derivative at x32 of the Lagrange quadratic through the three planes
        const double xc3 = s.xs[m3];
        w0 = ((x32 - xb) + (x32 - xc3)) / ((xa - xb) * (xa - xc3));
        w1 = ((x32 - xa) + (x32 - xc3)) / ((xb - xa) * (xb - xc3));
        w2 = ((x32 - xa) + (x32 - xb)) / ((xc3 - xa) * (xc3 - xb));
      } else {
        w1 = 1.0 / (xb - xa);
        w0 = -w1;
        m3 = m;
      }
      const long long nl = (long long)p->nk * p->nw;
      if (!p->dsb2) SRM3_CUDA(dev_alloc(&p->dsb2, nl * sizeof(double), st));
      k_sb2_slope<<<cdiv(nl, 256), 256, 0, st>>>(nl, p->sb2 + (size_t)m * nl,
                                                 p->sb2 + (size_t)(m + 1) * nl,
                                                 p->sb2 + (size_t)m3 * nl, w0, w1, w2, p->dsb2);
      SRM3_CUDA(cudaGetLastError());
      shift_ok = true;
    }
  }

  // FP64 stage: Newton steps from x32 with the FP32 slope, then secant steps
  // on the FP64 values, all inside an FP64 bracket; Illinois if they leave
  // it or stall.  The bracket's upper end is not yet evaluated in FP64: any
  // x above the root serves (the linear bound x0, else four times the FP32
  // bracket's upper end).
  const size_t jb = first_above(s);
  const double xup = s.x0 > 0.0 ? s.x0 : s.pts[std::min(jb, s.pts.size() - 1)].first;
  Bracket b{0.0, -target, 4.0 * xup, 1.0, true};
  double xbest = -1.0;
  PassResult best{};
  bool converged = false, at_best = false;
  double x = x32, xp = 0.0, fp = 0.0;
  bool have_prev = false;
  p->eps_shifted = false;
  p->eps_interp = false;
  // Tight targets (FP64 plans, direct bulk, sum pairs): one FP64 pass at the
  // three values x32 (1 + {-d, 0, d}); the root xr of the inverse quadratic
  // through the three (x, f), and every point's tables interpolated to it by
  // the quadratic through its three values -- an error of the order of the
  // third derivative times d^3 (~1e-17 relative), below the FP64 rounding of
  // the sums.  Accepted when the interpolated max meets the target within
  // tol; else the three values join the bracket and the steps below go on
  // from xr.
  auto note = [&](double xv, double f) {
    if (f < 0) {
      if (xv > b.xlo) {
        b.xlo = xv;
        b.flo = f;
      }
    } else if (b.hi_failed || xv < b.xhi) {
      b.xhi = xv;
      b.fhi = f;
      b.hi_failed = false;
    }
  };
  if (tol < kShiftTol && !p->rec_fft && !p->mixed && hi_ok) {
    double x3[3] = {x32 * (1.0 - kInterpDel), x32, x32 * (1.0 + kInterpDel)};
    PassResult r3[3];
    rc = run_pass_multi(p, st, x3, 3, true, r3);
    if (rc) return rc;
    bool ok3 = true;
    double f3[3];
    for (int m = 0; m < 3; ++m) {
      if (r3[m].err) {
        ok3 = false;
        b.xhi = std::min(b.xhi, x3[m]);
        b.hi_failed = true;
        continue;
      }
      f3[m] = r3[m].max_sb2 - target;
      note(x3[m], f3[m]);
    }
    if (ok3 && f3[2] > f3[0]) {
      slope32 = (f3[2] - f3[0]) / (x3[2] - x3[0]);
      const double xr = quad_root(x3[0], f3[0], x3[1], f3[1], x3[2], f3[2]);
      // the next point of the steps below in any case (beyond the reach, x32
      // was off: xr is an extrapolation, still the best estimate)
      if (xr > b.xlo && (b.hi_failed || xr < b.xhi)) x = xr;
      if (xr > b.xlo && (b.hi_failed || xr < b.xhi) && std::fabs(xr - x32) <= kInterpReach * x32) {
        const double w0 = (xr - x3[1]) * (xr - x3[2]) / ((x3[0] - x3[1]) * (x3[0] - x3[2]));
        const double w1 = (xr - x3[0]) * (xr - x3[2]) / ((x3[1] - x3[0]) * (x3[1] - x3[2]));
        const double w2 = (xr - x3[0]) * (xr - x3[1]) / ((x3[2] - x3[0]) * (x3[2] - x3[1]));
        const long long nl = (long long)p->nk * p->nw;
        SRM3_CUDA(cudaMemsetAsync(p->rec_max, 0, sizeof(unsigned long long), st));
        SRM3_CUDA(cudaMemsetAsync(p->err, 0, sizeof(int), st));
        k_sb2_interp3<<<cdiv(nl, 256), 256, 0, st>>>(nl, p->S, p->sb2, w0, w1, w2, p->qm,
                                                     p->rec_max, p->err);
        SRM3_CUDA(cudaGetLastError());
        SRM3_CUDA(cudaMemcpyAsync(p->h_pinned + 8, p->rec_max, sizeof(unsigned long long),
                                  cudaMemcpyDeviceToHost, st));
        SRM3_CUDA(cudaMemcpyAsync(p->h_err, p->err, sizeof(int), cudaMemcpyDeviceToHost, st));
        SRM3_CUDA(cudaStreamSynchronize(st));
        const double mx = p->h_pinned[8];  // the bits of a double, copied as such
        x = xr;
        if (!p->h_err[0] && std::fabs(mx - target) <= tol) {
          best.max_sb2 = mx;
          best.min_pure = 1.0 - mx;
          best.sumS = r3[1].sumS;
          best.err = 0;
          xbest = xr;
          converged = at_best = true;
          p->eps_interp = true;
        }
      }
    }
  }
  for (int it = 0; it < 6 && !converged; ++it) {
    PassResult q1;
    rc = run_pass(p, st, x, true, &q1);
    if (rc) return rc;
    if (q1.err) {
      b.xhi = std::min(b.xhi, x);
      b.hi_failed = true;
      at_best = false;
      break;
    }
    const double f = q1.max_sb2 - target;
    best = q1;
    xbest = x;
    at_best = true;
    if (f < 0) {
      if (x > b.xlo) {
        b.xlo = x;
        b.flo = f;
      }
    } else if (b.hi_failed || x < b.xhi) {
      b.xhi = x;
      b.fhi = f;
      b.hi_failed = false;
    }
    if (std::fabs(f) <= tol) {
      converged = true;
      break;
    }
    if (it == 0 && shift_ok) {
      const double x1 = x - f / slope32;
      if (x1 > b.xlo && (b.hi_failed || x1 < b.xhi) && std::fabs(x1 - x) <= kShiftMax * x) {
        PassResult q2;
        rc = shift_tables(p, st, x1 - x, &q2);
        if (rc) return rc;
        at_best = false;  // the tables have left x
        if (!q2.err && std::fabs(q2.max_sb2 - target) <= tol) {
          q2.sumS = q1.sumS;
          best = q2;
          xbest = x1;
          at_best = converged = true;
          p->eps_shifted = true;
          break;
        }
      }
    }
    const double s = (have_prev && f != fp) ? (f - fp) / (x - xp) : slope32;
    if (!(s > 0.0)) break;
    const double xn = x - f / s;
    if (!(xn > b.xlo && (b.hi_failed || xn < b.xhi))) break;
    xp = x;
    fp = f;
    have_prev = true;
    x = xn;
  }
  if (!converged) {
    rc = illinois(p, st, target, tol, 200, b, &xbest, &best, &at_best);
    if (rc) return rc;
  }
  if (xbest < 0.0) return fail(SRM3_ERR_BISECTION_FAILED, "eps search found no feasible point");
  if (!at_best) {
    PassResult q1;
    rc = run_pass(p, st, xbest, true, &q1);
    if (rc) return rc;
    if (q1.err) return fail(SRM3_ERR_BISECTION_FAILED, "eps search: final pass failed");
    best = q1;
  }
  p->eps = std::sqrt(xbest);
  p->max_sb2 = best.max_sb2;
  p->min_pure = best.min_pure;
  p->variance = 4.0 * p->dkdw * best.sumS;
  return SRM3_OK;
}


static long long tile_entries(int kk, int tw) {
  int kw0 = tw * kTileR;
  long long L = ((kw0 + kTileR + kTileU - 1) / kTileU) * kTileU;
  return (long long)(kk / 2 + 1) * kTileR * L;
}

// W table of an FP32 plan (tile offsets and the envelope tables ready),
// enqueued on st (allocation, build, CUDA events around it); finish_w_table
// waits for it and records its time and size.  The table depends on the
// lattice shape only, so a plan build runs it beside the recursion.
static int start_w_table(srm3_plan *p, cudaStream_t st) {
  if (p->W) return SRM3_OK;
  AllocOwner owner(p);
  cudaError_t e = dev_alloc(&p->W, (size_t)p->table_entries * sizeof(float), st);
  if (e != cudaSuccess) return cuda_fail(e, "dev_alloc(W table, st)");
  SRM3_CUDA(cudaEventCreate(&p->w_ev[0]));
  SRM3_CUDA(cudaEventCreate(&p->w_ev[1]));
  SRM3_CUDA(cudaEventRecord(p->w_ev[0], st));
  k_build_w<<<(p->row_hi - p->row_lo) * p->ntw, dim3(32, 8), 0, st>>>(
      p->row_lo * p->ntw, p->nk, p->nw, p->ntw, p->tile_off, (const float *)p->Ek,
      (const float *)p->Ews, p->ew_off, p->W);
  SRM3_CUDA(cudaGetLastError());
  SRM3_CUDA(cudaEventRecord(p->w_ev[1], st));
  return SRM3_OK;
}

static int finish_w_table(srm3_plan *p) {
  if (!p->w_ev[1]) return SRM3_OK;
  cudaError_t e = cudaEventSynchronize(p->w_ev[1]);
  float tms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&tms, p->w_ev[0], p->w_ev[1]);
  cudaEventDestroy(p->w_ev[0]);
  cudaEventDestroy(p->w_ev[1]);
  p->w_ev[0] = p->w_ev[1] = nullptr;
  if (e != cudaSuccess) return cuda_fail(e, "W table build");
  p->t_table_ms = tms;
  p->table_bytes = (double)p->table_entries * sizeof(float);
  return SRM3_OK;
}

int build_w_table(srm3_plan *p, cudaStream_t st) {
  int rc = start_w_table(p, st);
  return rc ? rc : finish_w_table(p);
}

// Tiles of the FP32 pair sum.  A plan restricted to lattice rows [row_lo,
// row_hi) (a shard of a k-sharded job) gets W-table space and work units for
// those rows only.
static int build_tiles(srm3_plan *p, cudaStream_t st, bool want_table, long long *table_entries) {
  const int nk = p->nk;
  p->ntw = cdiv(p->nw, kTileR);
  p->ntiles = nk * p->ntw;
  std::vector<long long> off(p->ntiles + 1, 0);
  for (int t = 0; t < p->ntiles; ++t) {
    const int kk = t / p->ntw, tw = t % p->ntw;
    const bool mine = kk >= p->row_lo && kk < p->row_hi;
    off[t + 1] = off[t] + (mine ? tile_entries(kk, tw) : 0);
  }
  // super-tiles of the FP32 pair sum, most expensive first, for both tile
  // shapes (32 and 16 outputs wide)
  int nsw = 0;
  for (int v = 0; v < 2; ++v) {
    const int sw = kTileR * (v == 0 ? 4 : 2);
    nsw = cdiv(p->nw, sw);
    p->nsuper[v] = (p->row_hi - p->row_lo) * nsw;
    std::vector<int2> sup(p->nsuper[v]);
    for (int i = 0; i < p->nsuper[v]; ++i)
      sup[i] = make_int2(p->row_lo + i / nsw, (i % nsw) * sw);
    std::stable_sort(sup.begin(), sup.end(), [&](int2 a, int2 b) {
      return (long long)(a.x / 2 + 1) * (a.y + sw) > (long long)(b.x / 2 + 1) * (b.y + sw);
    });
    SRM3_CUDA(dev_alloc(&p->super_order[v], sizeof(int2) * p->nsuper[v], st));
    SRM3_CUDA(cudaMemcpyAsync(p->super_order[v], sup.data(), sizeof(int2) * p->nsuper[v],
                              cudaMemcpyHostToDevice, st));
    p->super_host[v] = sup;
  }
  if (p->mixed) {  // the difference pass (32 wide): (kk + 1) row pairs x ceil((nw - kws0) / 16) chunks
    const int sw = kTileR * 4;
    nsw = cdiv(p->nw, sw);
    const int n = (p->row_hi - p->row_lo) * nsw;
    std::vector<int2> supd(n);
    for (int i = 0; i < n; ++i) supd[i] = make_int2(p->row_lo + i / nsw, (i % nsw) * sw);
    auto cost = [&](int2 t) { return (long long)(t.x + 1) * ((p->nw - t.y + 15) / 16); };
    std::stable_sort(supd.begin(), supd.end(),
                     [&](int2 a, int2 b) { return cost(a) > cost(b); });
    p->nsuper_d = n;
    SRM3_CUDA(dev_alloc(&p->super_order_d, sizeof(int2) * n, st));
    SRM3_CUDA(cudaMemcpyAsync(p->super_order_d, supd.data(), sizeof(int2) * n,
                              cudaMemcpyHostToDevice, st));
  }
  *table_entries = off[p->ntiles];
  (void)want_table;  // offsets are kept either way: the autotuner may build W later
  SRM3_CUDA(dev_alloc(&p->tile_off, sizeof(long long) * p->ntiles, st));
  SRM3_CUDA(cudaMemcpyAsync(p->tile_off, off.data(), sizeof(long long) * p->ntiles,
                            cudaMemcpyHostToDevice, st));
  SRM3_CUDA(cudaStreamSynchronize(st));
  return SRM3_OK;
}

int build_plan(srm3_plan *p, const srm3_spectrum *sp, const srm3_bispectrum *bs) {
  const int nk = p->nk, nw = p->nw;
  const size_t nl = (size_t)nk * nw;
  cudaStream_t st;
  SRM3_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  SRM3_CUDA(cudaEventCreate(&t_ev[0]));
  SRM3_CUDA(cudaEventCreate(&t_ev[1]));
  struct StreamGuard {
    cudaStream_t s;
    ~StreamGuard() {
      cudaStreamDestroy(s);
      cudaEventDestroy(t_ev[0]);
      cudaEventDestroy(t_ev[1]);
      t_ev[0] = t_ev[1] = nullptr;
    }
  } guard{st};

  {
    void *blk = nullptr;
    SRM3_CUDA(pinned_get(&blk));
    p->h_pinned = static_cast<double *>(blk);
    p->h_err = reinterpret_cast<int *>(static_cast<char *>(blk) + kPinErrOff);
  }
  SRM3_CUDA(dev_alloc(&p->S, nl * sizeof(double), st));
  SRM3_CUDA(dev_alloc(&p->qm, nl * sizeof(double), st));
  SRM3_CUDA(dev_alloc(&p->sb2, kPlanes * nl * sizeof(double), st));
  SRM3_CUDA(dev_alloc(&p->EkSq, nk * sizeof(double), st));
  // EwSq, EwSq32 hold 2 nw entries: the signed frequency difference of a
  // difference pair (kw + 2 jw) reaches 2 nw - 2
  SRM3_CUDA(dev_alloc(&p->EwSq, 2 * nw * sizeof(double), st));
  SRM3_CUDA(dev_alloc(&p->scal, (8 + 4 * kPlanes) * sizeof(double), st));
  SRM3_CUDA(dev_alloc(&p->err, (kPlanes + 1) * sizeof(int), st));
  SRM3_CUDA(cudaMemsetAsync(p->qm, 0, nl * sizeof(double), st));
  SRM3_CUDA(dev_alloc(&p->qm32, kPlanes * nl * sizeof(float), st));
  SRM3_CUDA(dev_alloc(&p->EkSq32, nk * sizeof(float), st));
  SRM3_CUDA(dev_alloc(&p->EwSq32, 2 * nw * sizeof(float), st));
  SRM3_CUDA(cudaMemsetAsync(p->qm32, 0, kPlanes * nl * sizeof(float), st));

  // a1: spectrum on the lattice
  if (sp->kind == SRM3_SPECTRUM_KAIMAL_LORENTZIAN) {
    k_discretise_kaimal<<<cdiv(nl, 256), 256, 0, st>>>(nk, nw, p->dk, p->dw, sp->U, sp->z,
                                                       sp->z0, sp->k_vk, sp->lam, p->S);
    SRM3_CUDA(cudaGetLastError());
  } else {
    SRM3_CUDA(cudaMemcpyAsync(p->S, sp->table, nl * sizeof(double), cudaMemcpyHostToDevice, st));
  }
  k_env_sq<<<cdiv(nk, 256), 256, 0, st>>>(nk, p->sigma_g * nk, p->EkSq, p->EkSq32);
  k_env_sq<<<cdiv(2 * nw, 256), 256, 0, st>>>(2 * nw, p->sigma_g * nw, p->EwSq, p->EwSq32);
  SRM3_CUDA(dev_alloc(&p->G2, nl * sizeof(double), st));
  SRM3_CUDA(dev_alloc(&p->G2_32, nl * sizeof(float), st));
  if (p->sep) {
    // separable envelope: the pair factor e_i^2 e_j^2 rides on h = e^2 q and
    // e_k^2 is applied when q_k is formed, so the g^2 table is all ones
    SRM3_CUDA(dev_alloc(&p->env_e, nl * sizeof(double), st));
    SRM3_CUDA(dev_alloc(&p->env_e2, nl * sizeof(double), st));
    SRM3_CUDA(dev_alloc(&p->env_e32, nl * sizeof(float), st));
    SRM3_CUDA(dev_alloc(&p->qh, nl * sizeof(double), st));
    SRM3_CUDA(cudaMemsetAsync(p->qh, 0, nl * sizeof(double), st));
    SRM3_CUDA(cudaMemcpyAsync(p->env_e, bs->env_table, nl * sizeof(double),
                              cudaMemcpyHostToDevice, st));
    k_sep_tables<<<cdiv(nl, 256), 256, 0, st>>>((int)nl, p->env_e, p->env_e2, p->env_e32,
                                                p->G2, p->G2_32);
    p->sep_b = bs->env_table_b != nullptr;
    if (p->sep_b) {
      SRM3_CUDA(dev_alloc(&p->env_b, nl * sizeof(double), st));
      SRM3_CUDA(dev_alloc(&p->env_b2, nl * sizeof(double), st));
      SRM3_CUDA(dev_alloc(&p->env_b32, nl * sizeof(float), st));
      SRM3_CUDA(cudaMemcpyAsync(p->env_b, bs->env_table_b, nl * sizeof(double),
                                cudaMemcpyHostToDevice, st));
      k_sep_tables<<<cdiv(nl, 256), 256, 0, st>>>((int)nl, p->env_b, p->env_b2, p->env_b32,
                                                  p->G2, p->G2_32);
    } else {
      p->env_b = p->env_e;
      p->env_b2 = p->env_e2;
      p->env_b32 = p->env_e32;
    }
  } else {
    k_g2<<<cdiv(nl, 256), 256, 0, st>>>(nk, nw, p->EkSq, p->EwSq, p->G2, p->G2_32);
    if (p->rec_sep) {
      // Gaussian envelope in separable form for the recursion (the sampling
      // path keeps W = c_k g(i, j))
      SRM3_CUDA(dev_alloc(&p->rs_a2, nl * sizeof(double), st));
      SRM3_CUDA(dev_alloc(&p->rs_b2, nl * sizeof(double), st));
      SRM3_CUDA(dev_alloc(&p->qh, nl * sizeof(double), st));
      SRM3_CUDA(cudaMemsetAsync(p->qh, 0, nl * sizeof(double), st));
      k_gauss_sep<<<cdiv(nl, 256), 256, 0, st>>>(nk, nw, p->sigma_g * nk, p->sigma_g * nw,
                                                 p->rs_a2, p->rs_b2);
    }
  }
  SRM3_CUDA(cudaGetLastError());

  // shape tables (envelope factors, twiddles), tiles, the storage choice
  // and the W table -- all functions of the lattice shape, ready before eps
  // is known: the W table (the O(N^2) FP32 pair sum only; separable
  // envelopes sample through the FFT self-convolution) is written on a
  // stream of its own while the recursion runs
  int rc = prepare_shape_tables(p, st);
  if (rc) return rc;
  cudaStream_t wst = nullptr;
  struct WStreamGuard {
    cudaStream_t *s;
    ~WStreamGuard() {
      if (*s) cudaStreamDestroy(*s);
    }
  } wguard{&wst};
  if (p->precision == SRM3_FP32 && !p->sep) {
    long long entries = 0;
    bool maybe_table = p->storage != SRM3_STORAGE_RECOMPUTE;
    rc = build_tiles(p, st, maybe_table, &entries);
    if (rc) return rc;
    p->table_entries = entries;
    const double bytes = (double)entries * sizeof(float);
    int tuned_nc = 4;
    const int tuned = tune_cache_lookup(nk, nw, &tuned_nc);
    if (tuned >= 0) p->ps_nc = tuned_nc;  // the tuned tile (results do not depend on it)
    if (p->storage == SRM3_STORAGE_TUNED)  // the autotuner's storage for this lattice
      p->storage = tuned >= 0 ? tuned : SRM3_STORAGE_AUTO;
    if (p->storage == SRM3_STORAGE_AUTO) {
      p->storage = bytes <= p->table_budget ? SRM3_STORAGE_TABLE : SRM3_STORAGE_RECOMPUTE;
    }
    if (p->mixed) p->storage = SRM3_STORAGE_RECOMPUTE;  // the table holds sum pairs only
    if (p->storage == SRM3_STORAGE_TABLE) {
      cudaEvent_t ready;
      SRM3_CUDA(cudaStreamCreateWithFlags(&wst, cudaStreamNonBlocking));
      SRM3_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
      SRM3_CUDA(cudaEventRecord(ready, st));  // envelope tables and tile offsets written
      SRM3_CUDA(cudaStreamWaitEvent(wst, ready, 0));
      cudaEventDestroy(ready);
      // launched beside the first FP64 recursion pass (run_pass_multi): that
      // pass leaves room on every SM (one CTA of 512 threads at 94
      // registers), the FP32 passes and the kernels before them do not
      p->w_stream = wst;
      p->w_deferred = true;
    } else {
      p->table_bytes = 0.0;
    }
  } else {
    p->storage = SRM3_STORAGE_RECOMPUTE;
    p->table_bytes = 0.0;
  }

  // a2: recursion, one graph node per anti-diagonal level
  rc = setup_recursion(p, st);
  if (rc) return rc;
  if (p->mixed) {
    SRM3_CUDA(dev_alloc(&p->Dsum, nl * sizeof(double), st));
    SRM3_CUDA(dev_alloc(&p->qprev, nl * sizeof(double), st));
    SRM3_CUDA(dev_alloc(&p->qlo, nl * sizeof(double), st));
    SRM3_CUDA(dev_alloc(&p->fp_change, sizeof(unsigned long long), st));
  }
  if (p->mixed && bs->target_max_sum_b2 > 0.0) {
    rc = find_eps_mixed(p, st, bs->target_max_sum_b2,
                        p->precision == SRM3_FP64 ? 1e-13 : 1e-9);
    if (rc) return rc;
  } else if (p->mixed) {
    PassResult r;
    p->qlo_x = -1.0;
    rc = eval_fp64(p, st, bs->eps * bs->eps, 2.0, &r);
    if (rc) return rc;
    if (r.err)
      return fail(SRM3_ERR_NONPOSITIVE_PURE,
                  p->fp_iters >= kFpMaxIters
                      ? "mixed interactions: the fixed point of Eq. pure was not reached"
                      : "sum_b2 >= 1 at some lattice point: the pure spectrum is not positive");
    p->eps = bs->eps;
    p->max_sb2 = r.max_sb2;
    p->min_pure = r.min_pure;
    p->variance = 4.0 * p->dkdw * r.sumS;
  } else if (bs->target_max_sum_b2 > 0.0) {
    // FP64 plans meet the target to 1e-13; for FP32 plans 1e-9 is far inside
    // what their fields can resolve (1e-4 sigma) and saves an FP64 pass
    rc = find_eps(p, st, bs->target_max_sum_b2, p->precision == SRM3_FP64 ? 1e-13 : 1e-9);
    if (rc) return rc;
  } else {
    PassResult r;
    rc = run_pass(p, st, bs->eps * bs->eps, true, &r);
    if (rc) return rc;
    if (r.err)
      return fail(SRM3_ERR_NONPOSITIVE_PURE,
                  "sum_b2 >= 1 at some lattice point: the pure spectrum is not positive");
    p->eps = bs->eps;
    p->max_sb2 = r.max_sb2;
    p->min_pure = r.min_pure;
    p->variance = 4.0 * p->dkdw * r.sumS;
  }

  if (p->w_deferred) {  // no FP64 pass ran: the W table now
    p->w_deferred = false;
    if ((rc = start_w_table(p, wst))) return rc;
  }
  // pair count: point (kk, kw) has floor(((kk + 1)(kw + 1) - 1) / 2) unordered
  // pairs (i, j != 0); per row, with c = kk + 1 and T = nw (nw + 1) / 2, the sum
  // over kw is (c T - nw - e) / 2, e the number of even c (kw + 1): nw for
  // even c, floor(nw / 2) for odd c
  long long pairs = 0;  // of the plan's rows
  const long long T = (long long)nw * (nw + 1) / 2;
  for (int kk = p->row_lo; kk < p->row_hi; ++kk) {
    const long long c = kk + 1, e = (c % 2 == 0) ? nw : nw / 2;
    pairs += (c * T - nw - e) / 2;
  }
  p->pairs = pairs;
  long long dpairs = 0;  // difference pairs of one sheet: (kk + 1) (nw - 1 - kw), kw >= 1
  if (p->mixed)
    for (int kk = p->row_lo; kk < p->row_hi; ++kk)
      dpairs += (long long)(kk + 1) * ((long long)(nw - 1) * (nw - 2) / 2);
  p->diffpairs = dpairs;

  rc = prepare_sampling_tables(p, st);
  if (rc) return rc;
  // the W table built beside the recursion (its own stream) is joined here
  if (p->w_ev[1]) {
    SRM3_CUDA(cudaStreamWaitEvent(st, p->w_ev[1], 0));
    if ((rc = finish_w_table(p))) return rc;
  }
  SRM3_CUDA(cudaStreamSynchronize(st));
  return SRM3_OK;
}

// The tables of the lattice shape: envelope factors by kappa and by signed
// omega offset (and of the signed difference for mixed plans), FFT
// twiddles, the self-convolution grid of separable plans.
int prepare_shape_tables(srm3_plan *p, cudaStream_t st) {
  const int nk = p->nk, nw = p->nw;
  const bool f32 = p->precision == SRM3_FP32;
  const size_t es = f32 ? sizeof(float) : sizeof(double);
  // signed envelope table Ews[ew_off + d] (terms outside the lattice meet
  // zero y, whatever their weight).  ew_off is
  // 3 mod 4, which puts the FP32 pair sum's 64-entry chunk windows of the
  // FP32 table (first d = 2 i0 - kws0 - (SW - 1), 1 mod 4) on 16-byte
  // boundaries; the table reaches d = 2 nw + 127, past the last window.
  p->ew_off = ((nw + 32 + 7) / 8) * 8 + 7;
  p->ew_len = p->ew_off + 2 * nw + 128;  // difference pairs reach d = 2 nw - 2
  if (p->sep) {  // zero-padded self-convolution grid
    p->log2cNk = 1;
    while ((1 << p->log2cNk) < 2 * nk - 1) ++p->log2cNk;
    p->log2cNw = 1;
    while ((1 << p->log2cNw) < 2 * nw - 1) ++p->log2cNw;
    p->cNk = 1 << p->log2cNk;
    p->cNw = 1 << p->log2cNw;
  }
  p->rowstride = nw + 2 * kPad;  // y row length, workspace or batch buffers
  SRM3_CUDA(dev_alloc(&p->Ek, nk * es, st));
  SRM3_CUDA(dev_alloc(&p->Ews, p->ew_len * es, st));
  const int tw_n = tx_twlen(p->log2nx) + tx_twlen(p->log2nt - 1) + p->nt / 2;
  SRM3_CUDA(dev_alloc(&p->tw, (size_t)tw_n * 2 * es, st));
  if (f32) {
    k_env<float><<<cdiv(nk, 256), 256, 0, st>>>(nk, 0, p->sigma_g * nk, (float *)p->Ek);
    k_env<float><<<cdiv(p->ew_len, 256), 256, 0, st>>>(p->ew_len, p->ew_off, p->sigma_g * nw,
                                                      (float *)p->Ews);
    SRM3_CUDA(dev_alloc(&p->ps_err, sizeof(int), st));
    SRM3_CUDA(cudaMemsetAsync(p->ps_err, 0, sizeof(int), st));
    if (p->mixed) {  // envelope of the signed difference d = kw + 2 jw, d from 0
      p->ewd_len = 2 * nw + 128;
      SRM3_CUDA(dev_alloc(&p->Ewd, p->ewd_len * sizeof(float), st));
      k_env<float><<<cdiv(p->ewd_len, 256), 256, 0, st>>>(p->ewd_len, 0, p->sigma_g * nw,
                                                         (float *)p->Ewd);
    }
    k_tx_twiddles<float2><<<cdiv(tw_n, 256), 256, 0, st>>>(p->log2nx, p->log2nt - 1,
                                                            (float2 *)p->tw);
    if (p->sep) {
      // pass twiddles of the self-convolution's lengths Nk, then Nw
      const int ntwc = tx_twlen(p->log2cNk) + tx_twlen(p->log2cNw) + (1 << p->log2cNw);
      SRM3_CUDA(dev_alloc(&p->tw_conv, (size_t)ntwc * sizeof(float2), st));
      k_tx_twiddles<float2><<<cdiv(ntwc, 256), 256, 0, st>>>(p->log2cNk, p->log2cNw,
                                                            (float2 *)p->tw_conv);
    }
  } else {
    k_env<double><<<cdiv(nk, 256), 256, 0, st>>>(nk, 0, p->sigma_g * nk, (double *)p->Ek);
    k_env<double><<<cdiv(p->ew_len, 256), 256, 0, st>>>(p->ew_len, p->ew_off,
                                                       p->sigma_g * nw, (double *)p->Ews);
    k_tx_twiddles<double2><<<cdiv(tw_n, 256), 256, 0, st>>>(p->log2nx, p->log2nt - 1,
                                                             (double2 *)p->tw);
    if (p->sep) {
      // pass twiddles of the self-convolution's lengths Nk, then Nw
      const int ntwc = tx_twlen(p->log2cNk) + tx_twlen(p->log2cNw) + (1 << p->log2cNw);
      SRM3_CUDA(dev_alloc(&p->tw_conv, (size_t)ntwc * sizeof(double2), st));
      k_tx_twiddles<double2><<<cdiv(ntwc, 256), 256, 0, st>>>(p->log2cNk, p->log2cNw,
                                                            (double2 *)p->tw_conv);
    }
  }
  SRM3_CUDA(cudaGetLastError());
  return SRM3_OK;
}

// The tables of the spectrum at the plan's eps: sqrt(q) masked by S > 0, the
// pure factor 2 sqrt(dk dw S)(1 - sum_b2) and the pair factor 2 eps dk dw
// sqrt(S).
int prepare_sampling_tables(srm3_plan *p, cudaStream_t st) {
  const size_t nl = (size_t)p->nk * p->nw;
  const bool f32 = p->precision == SRM3_FP32;
  const size_t es = f32 ? sizeof(float) : sizeof(double);
  SRM3_CUDA(dev_alloc(&p->sqq, nl * es, st));
  SRM3_CUDA(dev_alloc(&p->Pk, nl * es, st));
  SRM3_CUDA(dev_alloc(&p->ck, nl * es, st));
  if (f32) {
    k_sampling_tables<float><<<cdiv(nl, 256), 256, 0, st>>>(
        (int)nl, p->dkdw, p->eps, p->S, p->qm, p->sb2, (float *)p->sqq, (float *)p->Pk,
        (float *)p->ck);
    if (pairsum_sep_capable(p)) {
      SRM3_CUDA(dev_alloc(&p->sqq_s, nl * sizeof(float), st));
      SRM3_CUDA(dev_alloc(&p->Pk_s, nl * sizeof(float), st));
      SRM3_CUDA(dev_alloc(&p->ck_s, nl * sizeof(float), st));
      SRM3_CUDA(dev_alloc(&p->aK, p->nk * sizeof(float), st));
      k_sep_sampling<<<cdiv(nl, 256), 256, 0, st>>>(
          p->nk, p->nw, p->sigma_g * p->nk, p->sigma_g * p->nw, (const float *)p->sqq,
          (const float *)p->Pk, (const float *)p->ck, p->sqq_s, p->Pk_s, p->ck_s, p->aK);
    }
  }
  else
    k_sampling_tables<double><<<cdiv(nl, 256), 256, 0, st>>>(
        (int)nl, p->dkdw, p->eps, p->S, p->qm, p->sb2, (double *)p->sqq, (double *)p->Pk,
        (double *)p->ck);
  SRM3_CUDA(cudaGetLastError());
  return SRM3_OK;
}

// Freed plan memory the default pool keeps for reuse (a bridge-size plan
// with its W table is about 9.5 GB); beyond this it goes back to the device.
constexpr uint64_t kPoolKeepBytes = 32ull << 30;

namespace {
std::mutex g_alloc_mu;
std::unordered_map<void *, std::pair<srm3_plan *, size_t>> g_allocs;  // block -> owner, size
thread_local srm3_plan *g_alloc_owner = nullptr;
}  // namespace

AllocOwner::AllocOwner(srm3_plan *p) : prev(g_alloc_owner) { g_alloc_owner = p; }
AllocOwner::~AllocOwner() { g_alloc_owner = prev; }

cudaError_t dev_alloc(void **ptr, size_t bytes, cudaStream_t st) {
  static std::once_flag once[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 64)
    std::call_once(once[dev], [dev] {
      cudaMemPool_t pool;
      if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = kPoolKeepBytes;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
      }
    });
  e = cudaMallocAsync(ptr, bytes, st);
  if (e == cudaSuccess && g_alloc_owner) {
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    g_allocs[*ptr] = {g_alloc_owner, bytes};
    g_alloc_owner->dev_bytes += (double)bytes;
  }
  return e;
}

cudaError_t dev_free(void *ptr, cudaStream_t st) {
  {
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    auto it = g_allocs.find(ptr);
    if (it != g_allocs.end()) {
      it->second.first->dev_bytes -= (double)it->second.second;
      g_allocs.erase(it);
    }
  }
  return cudaFreeAsync(ptr, st);
}

void free_plan(srm3_plan *p) {
  for (auto &r : p->ev_recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : p->ev_pool) cudaEventDestroy(e);
  for (cudaEvent_t &e : p->w_ev)  // a W build the plan's failure left unjoined
    if (e) cudaEventDestroy(e);
  void *dev[] = {p->S,      p->qm,     p->sb2,       p->EkSq,       p->EwSq,   p->scal,
                 p->err,    p->sqq,    p->Pk,        p->ck,         p->Ek,     p->Ews,
                 p->tw,     p->tile_off, p->W,       p->y,      p->y0,
                 p->C,      p->H,      p->qm32,      p->EkSq32,     p->EwSq32, p->rec_items,
                 p->G2,     p->G2_32,  p->qm3,
                 p->rec_partial, p->super_order[0], p->super_order[1], p->rec_lev_off,
                 p->rec_bar, p->rec_max,
                 p->rec_pairs, p->rec_pair_off,
                 p->ps_err,  p->env_e,    p->env_e2,     p->env_e32, p->qh,
                 p->tw_conv, p->Zc, p->rec_z, p->tw_rec32, p->tw_rec64,
                 p->sep_b ? p->env_b : nullptr, p->sep_b ? p->env_b2 : nullptr,
                 p->sep_b ? (void *)p->env_b32 : nullptr,
                 p->Dsum, p->qprev, p->qlo, p->fp_change, p->Ewd, p->ys, p->super_order_d,
                 p->rs_a2, p->rs_b2, p->dsb2, p->red_part, p->sqq_s, p->Pk_s, p->ck_s, p->aK,
                 p->qo3};
  // no plan work may be in flight; the blocks go back to the pool
  cudaDeviceSynchronize();
  for (void *d : dev)
    if (d) dev_free(d, nullptr);
  if (p->h_pinned) pinned_put(p->h_pinned);  // h_err lies in the same block
}

}  // namespace srm3

using namespace srm3;

SRM3_API const char *srm3_last_error(void) { return g_last_error.c_str(); }

SRM3_API int srm3_plan_create(const srm3_spectrum *spectrum, const srm3_bispectrum *bispectrum,
                              const srm3_grid *grid, srm3_plan **out) {
  auto t0 = std::chrono::steady_clock::now();
  if (!out) return fail(SRM3_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!spectrum || !bispectrum || !grid)
    return fail(SRM3_ERR_INVALID_ARG, "spectrum, bispectrum and grid must be non-NULL");
  const srm3_grid &g = *grid;
  if (g.n_kappa < 1 || g.n_omega < 1 || g.n_kappa > 4096 || g.n_omega > 4096)
    return fail(SRM3_ERR_INVALID_ARG, "n_kappa and n_omega must be in [1, 4096]");
  if (!(g.kappa_u > 0.0) || !(g.omega_u > 0.0))
    return fail(SRM3_ERR_INVALID_ARG, "cutoffs must be positive");
  if (g.precision != SRM3_FP32 && g.precision != SRM3_FP64)
    return fail(SRM3_ERR_INVALID_ARG, "unknown precision");
  if (g.storage < SRM3_STORAGE_AUTO || g.storage > SRM3_STORAGE_TUNED)
    return fail(SRM3_ERR_INVALID_ARG, "unknown storage");
  if (g.precision == SRM3_FP64 && g.storage == SRM3_STORAGE_TABLE)
    return fail(SRM3_ERR_NOT_SUPPORTED, "the W table is FP32; FP64 plans recompute W");
  int lx = ilog2_exact(g.n_x), lt = ilog2_exact(g.n_t);
  if (lx < 1 || lt < 1 || g.n_x > kMaxFft || g.n_t > kMaxFft)
    return fail(SRM3_ERR_GRID_CONSTRAINT, "n_x and n_t must be powers of two in [2, 8192]");
  if (g.n_x < g.n_kappa || g.n_t < 2 * g.n_omega - 1)
    return fail(SRM3_ERR_GRID_CONSTRAINT, "need n_x >= n_kappa and n_t >= 2 n_omega - 1");
  if (spectrum->kind == SRM3_SPECTRUM_KAIMAL_LORENTZIAN) {
    if (!(spectrum->U > 0) || !(spectrum->z0 > 0) || !(spectrum->z > spectrum->z0) ||
        !(spectrum->lam > 0) || !(spectrum->k_vk > 0))
      return fail(SRM3_ERR_INVALID_ARG, "Kaimal parameters out of range");
  } else if (spectrum->kind == SRM3_SPECTRUM_TABLE) {
    if (!spectrum->table) return fail(SRM3_ERR_INVALID_ARG, "spectrum table is NULL");
    for (size_t i = 0; i < (size_t)g.n_kappa * g.n_omega; ++i)
      if (!(spectrum->table[i] >= 0.0) || !std::isfinite(spectrum->table[i]))
        return fail(SRM3_ERR_INVALID_ARG, "spectrum table must be finite and >= 0");
  } else {
    return fail(SRM3_ERR_INVALID_ARG, "unknown spectrum kind");
  }
  if (bispectrum->kind == SRM3_BISPECTRUM_GAUSS_ENVELOPE) {
    if (!(bispectrum->sigma_g > 0.0)) return fail(SRM3_ERR_INVALID_ARG, "sigma_g must be > 0");
  } else if (bispectrum->kind == SRM3_BISPECTRUM_SEPARABLE) {
    if (!bispectrum->env_table) return fail(SRM3_ERR_INVALID_ARG, "env_table is NULL");
    for (const double *t : {bispectrum->env_table, bispectrum->env_table_b}) {
      if (!t) continue;
      for (size_t i = 0; i < (size_t)g.n_kappa * g.n_omega; ++i)
        if (!(t[i] >= 0.0) || !std::isfinite(t[i]))
          return fail(SRM3_ERR_INVALID_ARG, "env_table and env_table_b must be finite and >= 0");
    }
  } else {
    return fail(SRM3_ERR_INVALID_ARG, "unknown bispectrum kind");
  }
  if (bispectrum->interactions != SRM3_INTERACTIONS_SUM &&
      bispectrum->interactions != SRM3_INTERACTIONS_MIXED)
    return fail(SRM3_ERR_INVALID_ARG, "unknown interactions");
  if (bispectrum->interactions == SRM3_INTERACTIONS_MIXED) {
    if (bispectrum->kind != SRM3_BISPECTRUM_GAUSS_ENVELOPE)
      return fail(SRM3_ERR_NOT_SUPPORTED, "mixed interactions take the Gaussian envelope only");
    if (g.storage == SRM3_STORAGE_TABLE)
      return fail(SRM3_ERR_NOT_SUPPORTED,
                  "mixed interactions recompute W (the W table holds sum pairs only)");
  }
  const bool all_rows = g.row_begin == 0 && g.row_end == 0;
  if (!all_rows && !(g.row_begin >= 0 && g.row_begin < g.row_end && g.row_end <= g.n_kappa))
    return fail(SRM3_ERR_INVALID_ARG, "rows must satisfy 0 <= row_begin < row_end <= n_kappa");
  if (!all_rows && bispectrum->kind == SRM3_BISPECTRUM_SEPARABLE)
    return fail(SRM3_ERR_NOT_SUPPORTED,
                "separable plans sample by an FFT over the whole lattice: no row range");
  const double tgt = bispectrum->target_max_sum_b2;
  if (!(tgt >= 0.0 && tgt < 1.0)) return fail(SRM3_ERR_INVALID_ARG, "target must be in [0, 1)");
  if (tgt == 0.0 && !(bispectrum->eps >= 0.0))
    return fail(SRM3_ERR_INVALID_ARG, "eps must be >= 0");

  srm3_plan *p = new (std::nothrow) srm3_plan();
  if (!p) return fail(SRM3_ERR_OUT_OF_MEMORY, "host allocation failed");
  p->nk = g.n_kappa;
  p->nw = g.n_omega;
  p->nx = g.n_x;
  p->nt = g.n_t;
  p->log2nx = lx;
  p->log2nt = lt;
  p->ku = g.kappa_u;
  p->wu = g.omega_u;
  p->dk = g.kappa_u / g.n_kappa;
  p->dw = g.omega_u / g.n_omega;
  p->dkdw = p->dk * p->dw;
  p->precision = g.precision;
  p->storage = g.storage;
  p->stream = (cudaStream_t)g.stream;
  p->sep = bispectrum->kind == SRM3_BISPECTRUM_SEPARABLE;
  p->mixed = bispectrum->interactions == SRM3_INTERACTIONS_MIXED;
  p->row_lo = all_rows ? 0 : g.row_begin;
  p->row_hi = all_rows ? g.n_kappa : g.row_end;
  p->sigma_g = p->sep ? 0.25 : bispectrum->sigma_g;
  {
    // the separable form of the Gaussian envelope needs the exponent range
    // E of its factors to fit the FP32 search passes (products down to
    // exp(-E), b^2 up to exp(E)); wider ranges (sigma_g below ~0.22) keep
    // the g^2 table
    const double sk = p->sigma_g * g.n_kappa, sw = p->sigma_g * g.n_omega;
    const double E = (g.n_kappa - 1) * (g.n_kappa - 1) / (sk * sk) +
                     (g.n_omega - 1) * (g.n_omega - 1) / (sw * sw);
    p->rec_sep = p->sep || (!p->mixed && E <= kSepExpMax);
  }
  p->beta = bispectrum->beta;
  p->table_budget = g.table_budget_bytes > 0 ? g.table_budget_bytes : 64.0 * (1ull << 30);
  cudaGetDevice(&p->device);
  int rc;
  {
    AllocOwner owner(p);
    rc = build_plan(p, spectrum, bispectrum);
  }
  if (rc) {
    free_plan(p);
    delete p;
    return rc;
  }
  p->plan_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out = p;
  return SRM3_OK;
}

SRM3_API void srm3_destroy(srm3_plan *plan) {
  if (!plan) return;
  free_plan(plan);
  delete plan;
}

SRM3_API int srm3_sync(srm3_plan *plan) {
  if (!plan) return fail(SRM3_ERR_INVALID_ARG, "plan is NULL");
  SRM3_CUDA(cudaStreamSynchronize(plan->stream));
  return check_pairsum_error(plan);
}

SRM3_API int srm3_set_stream(srm3_plan *plan, void *stream) {
  if (!plan) return fail(SRM3_ERR_INVALID_ARG, "plan is NULL");
  plan->stream = (cudaStream_t)stream;
  return SRM3_OK;
}

SRM3_API int srm3_plan_info(const srm3_plan *plan, srm3_info *info) {
  if (!plan || !info) return fail(SRM3_ERR_INVALID_ARG, "plan and info must be non-NULL");
  info->eps = plan->eps;
  info->max_sum_b2 = plan->max_sb2;
  info->min_pure_ratio = plan->min_pure;
  info->variance = plan->variance;
  info->table_bytes = plan->table_bytes;
  info->plan_ms = plan->plan_ms;
  info->pairs = plan->pairs;
  info->root_passes = plan->root_passes;
  info->root_passes_fp32 = plan->root_passes32;
  info->storage = plan->storage;
  info->precision = plan->precision;
  info->tile_r = kTileR;
  info->tile_width = kTileR * plan->ps_nc;
  info->recursion_flags = (plan->rec_sep ? SRM3_REC_SEPARABLE : 0) |
                          (plan->eps_shifted ? SRM3_REC_TABLES_MOVED : 0) |
                          (plan->eps_interp ? SRM3_REC_TABLES_INTERPOLATED : 0) |
                          (pairsum_sep_now(plan) ? SRM3_PAIRSUM_SEPARABLE : 0) |
                          (plan->coarse_start ? SRM3_REC_COARSE_START : 0);
  info->coarse_fk = plan->coarse_fk;
  info->coarse_fw = plan->coarse_fw;
  info->coarse_launches = plan->coarse_launches;
  info->coarse_passes = plan->coarse_passes;
  info->interactions = plan->mixed ? SRM3_INTERACTIONS_MIXED : SRM3_INTERACTIONS_SUM;
  info->fixed_point_iterations = plan->mixed ? plan->fp_iters : 0;
  info->diff_pairs = plan->diffpairs;
  info->device_bytes = plan->dev_bytes;
  return SRM3_OK;
}

// Exact third moment of u (Sec. 2, the third-order moment of the wave; the
// quadrant form of Sec. 4): with b_p(i,j) = eps g sqrt(dk dw q_i q_j) every
// factor of S_p cancels, and over both sheets
//   E[u^3] = 4 eps cos(beta) (dk dw)^2 sum_k sqrt(S_k)
//            sum_{Pi(k)} m_ij g_ij sqrt(S_i S_j),   m = 6 (i != j), 3 (i = j).
// One warp per lattice point, pairs enumerated as in the direct levels of the
// recursion (rows a <= kk/2, centre row iw <= kw/2, i = 0 skipped); FP64.
// part[k] = sqrt(S_k) times the point's pair sum.
// Mixed plans add their difference pairs (two distinct points: m = 6), g
// from the envelope of the signed frequency difference kw + 2 jw.
__global__ void k_moment3(int nk, int nw, const double *__restrict__ S,
                          const double *__restrict__ G2, const double *__restrict__ ea,
                          const double *__restrict__ eb, int mixed,
                          const double *__restrict__ EkSq, const double *__restrict__ EwSq,
                          double *__restrict__ part) {
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gw >= (long long)nk * nw) return;
  const int kk = (int)(gw / nw), kw = (int)(gw - (long long)kk * nw);
  double acc = 0.0;
  if (S[gw] > 0.0) {
    const int W = kw + 1, E = (kk / 2 + 1) * W;
    for (int e = lane; e < E; e += 32) {
      const int a = e / W, iw = e - a * W, b = kk - a, jw = kw - iw;
      const int lim = (a == b) ? kw / 2 : kw;
      if ((a == 0 && iw == 0) || iw > lim) continue;
      const size_t i = (size_t)a * nw + iw, j = (size_t)b * nw + jw;
      const double si = S[i], sj = S[j];
      if (!(si > 0.0) || !(sj > 0.0)) continue;
      const int dk = 2 * a - kk, dw = 2 * iw - kw;
      double g = sqrt(G2[(size_t)(dk < 0 ? -dk : dk) * nw + (dw < 0 ? -dw : dw)]);
      if (ea) g *= ea[i] * ea[j] * eb[gw];
      const double m = (i == j) ? 3.0 : 6.0;
      acc += m * g * sqrt(si * sj);
    }
    const int J = nw - 1 - kw;
    if (mixed && kw >= 1 && J >= 1) {
      const int E2 = (kk + 1) * J;
      for (int e = lane; e < E2; e += 32) {
        const int ia = e / J, jw = 1 + e - ia * J;
        const double si = S[(size_t)ia * nw + kw + jw], sj = S[(size_t)(kk - ia) * nw + jw];
        if (!(si > 0.0) || !(sj > 0.0)) continue;
        const int dk = 2 * ia - kk;
        const double g = sqrt(EkSq[dk < 0 ? -dk : dk] * EwSq[kw + 2 * jw]);
        acc += 6.0 * g * sqrt(si * sj);
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) part[gw] = acc * sqrt(S[gw] > 0.0 ? S[gw] : 0.0);
}

SRM3_API int srm3_plan_moments(const srm3_plan *plan, double *variance, double *third_moment) {
  if (!plan || !variance || !third_moment)
    return fail(SRM3_ERR_INVALID_ARG, "plan and outputs must be non-NULL");
  const long long nl = (long long)plan->nk * plan->nw;
  cudaStream_t st = plan->stream;
  double *part = nullptr;
  SRM3_CUDA(cudaMallocAsync(&part, nl * sizeof(double), st));
  const long long threads = nl * 32;
  k_moment3<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(
      plan->nk, plan->nw, plan->S, plan->G2, plan->sep ? plan->env_e : nullptr,
      plan->sep ? plan->env_b : nullptr, plan->mixed ? 1 : 0, plan->EkSq, plan->EwSq, part);
  cudaError_t e = cudaGetLastError();
  std::vector<double> h(nl);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h.data(), part, nl * sizeof(double), cudaMemcpyDeviceToHost, st);
  cudaError_t e2 = cudaFreeAsync(part, st);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "srm3_plan_moments");
  long double sum = 0.0L;
  for (long long k = 0; k < nl; ++k) sum += h[k];
  *variance = plan->variance;
  *third_moment = (double)(4.0L * plan->eps * std::cos(plan->beta) * plan->dkdw * plan->dkdw * sum);
  return SRM3_OK;
}

SRM3_API int srm3_plan_tables(const srm3_plan *plan, double *S, double *q, double *sum_b2) {
  if (!plan) return fail(SRM3_ERR_INVALID_ARG, "plan is NULL");
  const size_t nl = (size_t)plan->nk * plan->nw;
  SRM3_CUDA(cudaStreamSynchronize(plan->stream));
  std::vector<double> s(nl), qm(nl);
  SRM3_CUDA(cudaMemcpy(s.data(), plan->S, nl * sizeof(double), cudaMemcpyDeviceToHost));
  SRM3_CUDA(cudaMemcpy(qm.data(), plan->qm, nl * sizeof(double), cudaMemcpyDeviceToHost));
  if (S) std::memcpy(S, s.data(), nl * sizeof(double));
  if (q)
    for (size_t i = 0; i < nl; ++i) q[i] = s[i] > 0.0 ? qm[i] : 1.0;
  if (sum_b2) SRM3_CUDA(cudaMemcpy(sum_b2, plan->sb2, nl * sizeof(double), cudaMemcpyDeviceToHost));
  return SRM3_OK;
}

// ---------------------------------------------------------------------------
// Failure path of the grid barrier, without a fault: every CTA but 0 waits at
// a barrier CTA 0 never reaches, gives up after `polls` polls and raises the
// abort word, which the host reads (the context stays usable).
namespace srm3 {
__global__ void k_selftest_barrier(unsigned int *bar, int *abort, long long limit) {
  if (blockIdx.x == 0) return;  // the arrival nothing makes
  grid_barrier(bar, abort, gridDim.x, limit);
}

int selftest_barrier(long long polls, int *timed_out) {
  unsigned int *bar = nullptr;
  int *ab = nullptr;
  SRM3_CUDA(cudaMalloc(&bar, 64));
  SRM3_CUDA(cudaMalloc(&ab, sizeof(int)));
  cudaError_t e = cudaMemset(bar, 0, 64);
  if (e == cudaSuccess) e = cudaMemset(ab, 0, sizeof(int));
  void *args[] = {&bar, &ab, &polls};
  if (e == cudaSuccess)
    e = cudaLaunchCooperativeKernel((const void *)k_selftest_barrier, 2, 32, args, 0, 0);
  int h = 0;
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&h, ab, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(bar);
  cudaFree(ab);
  if (e != cudaSuccess) return cuda_fail(e, "grid barrier self-test");
  *timed_out = h;
  return SRM3_OK;
}
}  // namespace srm3
