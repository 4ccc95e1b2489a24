// plan.cu - plan creation for the SRM3 sampler: lattice discretisation
// (Sec. 5), the pure-spectrum / partial-bicoherence recursion (Eq. pure)
// run level-parallel over the anti-diagonals of the lattice in FP64, the
// bracketing root search on eps, and the sampling tables (W table, tile
// order, FFT twiddles).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>

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

// Squared envelope factors for the recursion: g^2 = EkSq[|ik-jk|] EwSq[|iw-jw|].
__global__ void k_env_sq(int n, double sigma_n, double *out) {
  int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= n) return;
  double a = d / sigma_n;
  double e = exp(-0.5 * a * a);
  out[d] = e * e;
}

// ---------------------------------------------------------------------------
// One anti-diagonal level d = kk + kw of the recursion.  Every part of a
// pair of Pi(k) lies on a lower level, so all points of a level are
// independent.  One CTA per point; warps take row pairs (a, kk - a),
// a <= kk/2, lanes take omega indices; canonical half: the centre row
// a = kk - a keeps iw <= kw/2; i = 0 is skipped.
//   sum_b2(k) = eps^2 dk dw sum_{Pi(k)} g^2 qm_i qm_j,  q_k = 1/(1 - sum_b2)
// (Eq. pure with b_p^2 = eps^2 g^2 dk dw q_i q_j for |B| = eps g sqrt(SSS)).
// LINEAR: q == 1 everywhere (masked by S > 0), all points in one launch;
// gives L_k = dk dw sum g^2, the small-eps slope used to bracket eps.
template <bool LINEAR>
__global__ void __launch_bounds__(256) k_rec_level(int nk, int nw, int d, int kk_lo,
                                                   const double *__restrict__ S,
                                                   double *__restrict__ qm,
                                                   double *__restrict__ sb2,
                                                   const double *__restrict__ EkSq,
                                                   const double *__restrict__ EwSq,
                                                   const double *__restrict__ scal,
                                                   int *__restrict__ err) {
  int kk, kw;
  if (LINEAR) {
    kk = blockIdx.x / nw;
    kw = blockIdx.x - kk * nw;
  } else {
    kk = kk_lo + blockIdx.x;
    kw = d - kk;
  }
  const int k = kk * nw + kw;
  if (!(S[k] > 0.0)) {
    if (threadIdx.x == 0) {
      sb2[k] = 0.0;
      if (!LINEAR) qm[k] = 0.0;
    }
    return;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  double acc = 0.0;
  const int nrow = kk / 2 + 1;
  for (int a = warp; a < nrow; a += nwarps) {
    const int b = kk - a;
    const int lim = (a == b) ? kw / 2 : kw;
    const double *qa = qm + (size_t)a * nw;
    const double *qb = qm + (size_t)b * nw;
    const double *Sa = S + (size_t)a * nw;
    const double *Sb = S + (size_t)b * nw;
    double racc = 0.0;
    for (int iw = lane; iw <= lim; iw += 32) {
      if (a == 0 && iw == 0) continue;
      double prod;
      if (LINEAR)
        prod = (Sa[iw] > 0.0 && Sb[kw - iw] > 0.0) ? 1.0 : 0.0;
      else
        prod = qa[iw] * qb[kw - iw];
      int dd = 2 * iw - kw;
      racc = fma(EwSq[dd < 0 ? -dd : dd], prod, racc);
    }
    acc = fma(EkSq[kk - 2 * a], racc, acc);
  }
  // block reduction
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double red[8];
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < nwarps; ++w) t += red[w];
    double s2 = scal[0] * t;
    sb2[k] = s2;
    if (!LINEAR) {
      if (s2 < 1.0) {
        qm[k] = 1.0 / (1.0 - s2);
      } else {
        qm[k] = 0.0;
        atomicOr(err, 1);
      }
    }
  }
}

// Reductions over the lattice: scal[1] = max sum_b2, scal[2] = min over
// S > 0 of (1 - sum_b2), scal[3] = sum S.
__global__ void k_reduce(int n, const double *__restrict__ S,
                         const double *__restrict__ sb2, double *__restrict__ scal) {
  double mx = 0.0, mn = 1.0, sum = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double v = sb2[i];
    mx = fmax(mx, v);
    if (S[i] > 0.0) mn = fmin(mn, 1.0 - v);
    sum += S[i];
  }
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    sum += __shfl_xor_sync(0xffffffffu, sum, o);
  }
  __shared__ double a[32], b[32], c[32];
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { a[warp] = mx; b[warp] = mn; c[warp] = sum; }
  __syncthreads();
  if (threadIdx.x == 0) {
    int nw = blockDim.x >> 5;
    for (int w = 1; w < nw; ++w) { mx = fmax(mx, a[w]); mn = fmin(mn, b[w]); }
    sum = 0.0;
    for (int w = 0; w < nw; ++w) sum += c[w];
    scal[1] = mx;
    scal[2] = mn;
    scal[3] = sum;
  }
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

template <typename T>
__global__ void k_env(int len, int off, double sigma_n, T *out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= len) return;
  double a = (double)(i - off) / sigma_n;
  out[i] = (T)exp(-0.5 * a * a);
}

template <typename T2>
__global__ void k_twiddles(int n, T2 *tw) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double s, c;
  sincospi(2.0 * (double)j / (double)n, &s, &c);
  T2 v;
  v.x = c;
  v.y = s;
  tw[j] = v;
}

// W table, tile-major: for tile (kk, kw0): rows a = 0..kk/2, then r < R,
// then iw < L (L = kw0 + R rounded up to U); W = c_k Ek[kk-2a] Ew[2iw-kw]
// for iw <= kw < nw, else 0.  Centre rows are stored in full (the kernel
// halves them).  W is real: the constant biphase is applied afterwards.
__global__ void k_build_w(int nk, int nw, int ntw, const long long *__restrict__ off,
                          const float *__restrict__ ck, const float *__restrict__ Ek,
                          const float *__restrict__ Ews, int ew_off, float *__restrict__ W) {
  const int t = blockIdx.x;
  const int kk = t / ntw, tw = t - kk * ntw;
  const int kw0 = tw * kTileR;
  const int nrow = kk / 2 + 1;
  const int L = ((kw0 + kTileR + kTileU - 1) / kTileU) * kTileU;
  const long long n = (long long)nrow * kTileR * L;
  float *dst = W + off[t];
  for (long long i = threadIdx.x; i < n; i += blockDim.x) {
    int iw = (int)(i % L);
    long long rest = i / L;
    int r = (int)(rest % kTileR);
    int a = (int)(rest / kTileR);
    int kw = kw0 + r;
    float v = 0.0f;
    if (kw < nw && iw <= kw) {
      v = ck[kk * nw + kw] * Ek[kk - 2 * a] * Ews[ew_off + 2 * iw - kw];
    }
    dst[i] = v;
  }
}

// ---------------------------------------------------------------------------
static int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

struct PassResult {
  double max_sb2, min_pure, sumS;
  int err;
};

static thread_local cudaEvent_t t_ev[2] = {nullptr, nullptr};

static int run_pass(srm3_plan *p, cudaStream_t st, double x, PassResult *r) {
  p->h_pinned[0] = x * p->dkdw;
  SRM3_CUDA(cudaMemcpyAsync(p->scal, p->h_pinned, sizeof(double), cudaMemcpyHostToDevice, st));
  SRM3_CUDA(cudaMemsetAsync(p->err, 0, sizeof(int), st));
  SRM3_CUDA(cudaEventRecord(t_ev[0], st));
  SRM3_CUDA(cudaGraphLaunch(p->rec_exec, st));
  SRM3_CUDA(cudaEventRecord(t_ev[1], st));
  SRM3_CUDA(cudaMemcpyAsync(p->h_pinned + 1, p->scal + 1, 3 * sizeof(double),
                            cudaMemcpyDeviceToHost, st));
  SRM3_CUDA(cudaMemcpyAsync(p->h_pinned + 4, p->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  SRM3_CUDA(cudaStreamSynchronize(st));
  float ms = 0.f;
  SRM3_CUDA(cudaEventElapsedTime(&ms, t_ev[0], t_ev[1]));
  p->t_recursion_ms += ms;
  r->max_sb2 = p->h_pinned[1];
  r->min_pure = p->h_pinned[2];
  r->sumS = p->h_pinned[3];
  int e;
  std::memcpy(&e, p->h_pinned + 4, sizeof(int));
  r->err = e;
  p->root_passes += 1;
  return SRM3_OK;
}

static int build_recursion_graph(srm3_plan *p, cudaStream_t st) {
  SRM3_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  const int nk = p->nk, nw = p->nw;
  for (int d = 0; d <= nk + nw - 2; ++d) {
    int lo = std::max(0, d - nw + 1), hi = std::min(d, nk - 1);
    k_rec_level<false><<<hi - lo + 1, 256, 0, st>>>(nk, nw, d, lo, p->S, p->qm, p->sb2,
                                                    p->EkSq, p->EwSq, p->scal, p->err);
  }
  k_reduce<<<1, 1024, 0, st>>>(nk * nw, p->S, p->sb2, p->scal);
  cudaGraph_t g;
  cudaError_t e = cudaStreamEndCapture(st, &g);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture(recursion)");
  p->rec_graph = g;
  SRM3_CUDA(cudaGraphInstantiate(&p->rec_exec, g, 0));
  return SRM3_OK;
}

// Root search on x = eps^2 for max_k sum_b2(x) = target.  f(x) = max sum_b2
// - target is increasing in x; a failed recursion (some S_p <= 0) counts as
// above target.  The bracket starts at [0, target / max L] (q >= 1 makes
// the linear estimate an upper bound) and shrinks by the Illinois variant
// of regula falsi, with bisection whenever the upper end is a failed pass.
static int find_eps(srm3_plan *p, cudaStream_t st, double target, double tol) {
  // linear pass for the bracket
  p->h_pinned[0] = p->dkdw;
  SRM3_CUDA(cudaMemcpyAsync(p->scal, p->h_pinned, sizeof(double), cudaMemcpyHostToDevice, st));
  k_rec_level<true><<<p->nk * p->nw, 256, 0, st>>>(p->nk, p->nw, 0, 0, p->S, p->qm, p->sb2,
                                                   p->EkSq, p->EwSq, p->scal, p->err);
  SRM3_CUDA(cudaGetLastError());
  k_reduce<<<1, 1024, 0, st>>>(p->nk * p->nw, p->S, p->sb2, p->scal);
  SRM3_CUDA(cudaMemcpyAsync(p->h_pinned + 1, p->scal + 1, sizeof(double),
                            cudaMemcpyDeviceToHost, st));
  SRM3_CUDA(cudaStreamSynchronize(st));
  double Lmax = p->h_pinned[1];
  if (!(Lmax > 0.0))
    return fail(SRM3_ERR_BISECTION_FAILED, "no bispectral pairs: max_k sum_b2 is 0 for every eps");

  double xlo = 0.0, flo = -target;
  double xhi = target / Lmax;
  PassResult r;
  int rc = run_pass(p, st, xhi, &r);
  if (rc) return rc;
  bool hi_failed = r.err != 0;
  double fhi = hi_failed ? 1.0 : r.max_sb2 - target;
  double xlast = xhi;
  bool last_ok = !hi_failed;
  if (!hi_failed && std::fabs(fhi) <= tol) {
    p->eps = std::sqrt(xhi);
    p->max_sb2 = r.max_sb2;
    p->min_pure = r.min_pure;
    p->variance = 4.0 * p->dkdw * r.sumS;
    return SRM3_OK;
  }
  int side = 0;
  PassResult best{};
  double xbest = -1.0;
  for (int it = 0; it < 200; ++it) {
    double x;
    if (hi_failed) {
      x = 0.5 * (xlo + xhi);
    } else {
      x = xhi - fhi * (xhi - xlo) / (fhi - flo);
      if (!(x > xlo && x < xhi)) x = 0.5 * (xlo + xhi);
    }
    rc = run_pass(p, st, x, &r);
    if (rc) return rc;
    xlast = x;
    if (r.err) {
      last_ok = false;
      xhi = x;
      hi_failed = true;
      side = 1;
    } else {
      last_ok = true;
      double f = r.max_sb2 - target;
      best = r;
      xbest = x;
      if (std::fabs(f) <= tol) break;
      if (f < 0) {
        xlo = x;
        flo = f;
        if (side == -1 && !hi_failed) fhi *= 0.5;
        side = -1;
      } else {
        xhi = x;
        fhi = f;
        hi_failed = false;
        if (side == 1) flo *= 0.5;
        side = 1;
      }
    }
    if (xhi - xlo <= 4.0 * 2.220446049250313e-16 * xhi) break;
  }
  if (xbest < 0.0)
    return fail(SRM3_ERR_BISECTION_FAILED, "eps search found no feasible point");
  if (!last_ok || xlast != xbest) {
    rc = run_pass(p, st, xbest, &r);
    if (rc) return rc;
    if (r.err) return fail(SRM3_ERR_BISECTION_FAILED, "eps search: final pass failed");
    best = r;
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

static int build_tiles(srm3_plan *p, cudaStream_t st, bool want_table, long long *table_entries) {
  const int nk = p->nk;
  p->ntw = cdiv(p->nw, kTileR);
  p->ntiles = nk * p->ntw;
  std::vector<long long> off(p->ntiles + 1, 0);
  std::vector<int> ids(p->ntiles);
  std::vector<long long> cost(p->ntiles);
  for (int t = 0; t < p->ntiles; ++t) {
    int kk = t / p->ntw, tw = t % p->ntw;
    cost[t] = tile_entries(kk, tw);
    off[t + 1] = off[t] + cost[t];
    ids[t] = t;
  }
  std::stable_sort(ids.begin(), ids.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<int2> order(p->ntiles);
  for (int i = 0; i < p->ntiles; ++i) {
    int t = ids[i];
    order[i] = make_int2(t / p->ntw, (t % p->ntw) * kTileR);
  }
  SRM3_CUDA(cudaMalloc(&p->tile_order, sizeof(int2) * p->ntiles));
  SRM3_CUDA(cudaMemcpyAsync(p->tile_order, order.data(), sizeof(int2) * p->ntiles,
                            cudaMemcpyHostToDevice, st));
  *table_entries = off[p->ntiles];
  if (want_table) {
    SRM3_CUDA(cudaMalloc(&p->tile_off, sizeof(long long) * p->ntiles));
    SRM3_CUDA(cudaMemcpyAsync(p->tile_off, off.data(), sizeof(long long) * p->ntiles,
                              cudaMemcpyHostToDevice, st));
  }
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

  SRM3_CUDA(cudaMallocHost(&p->h_pinned, 8 * sizeof(double)));
  SRM3_CUDA(cudaMalloc(&p->S, nl * sizeof(double)));
  SRM3_CUDA(cudaMalloc(&p->qm, nl * sizeof(double)));
  SRM3_CUDA(cudaMalloc(&p->sb2, nl * sizeof(double)));
  SRM3_CUDA(cudaMalloc(&p->EkSq, nk * sizeof(double)));
  SRM3_CUDA(cudaMalloc(&p->EwSq, nw * sizeof(double)));
  SRM3_CUDA(cudaMalloc(&p->scal, 8 * sizeof(double)));
  SRM3_CUDA(cudaMalloc(&p->err, sizeof(int)));
  SRM3_CUDA(cudaMemsetAsync(p->qm, 0, nl * sizeof(double), st));

  // a1: spectrum on the lattice
  if (sp->kind == SRM3_SPECTRUM_KAIMAL_LORENTZIAN) {
    k_discretise_kaimal<<<cdiv(nl, 256), 256, 0, st>>>(nk, nw, p->dk, p->dw, sp->U, sp->z,
                                                       sp->z0, sp->k_vk, sp->lam, p->S);
    SRM3_CUDA(cudaGetLastError());
  } else {
    SRM3_CUDA(cudaMemcpyAsync(p->S, sp->table, nl * sizeof(double), cudaMemcpyHostToDevice, st));
  }
  k_env_sq<<<cdiv(nk, 256), 256, 0, st>>>(nk, p->sigma_g * nk, p->EkSq);
  k_env_sq<<<cdiv(nw, 256), 256, 0, st>>>(nw, p->sigma_g * nw, p->EwSq);
  SRM3_CUDA(cudaGetLastError());

  // a2: recursion, one graph node per anti-diagonal level
  int rc = build_recursion_graph(p, st);
  if (rc) return rc;
  if (bs->target_max_sum_b2 > 0.0) {
    rc = find_eps(p, st, bs->target_max_sum_b2, 1e-13);
    if (rc) return rc;
  } else {
    PassResult r;
    rc = run_pass(p, st, bs->eps * bs->eps, &r);
    if (rc) return rc;
    if (r.err)
      return fail(SRM3_ERR_NONPOSITIVE_PURE,
                  "sum_b2 >= 1 at some lattice point: the pure spectrum is not positive");
    p->eps = bs->eps;
    p->max_sb2 = r.max_sb2;
    p->min_pure = r.min_pure;
    p->variance = 4.0 * p->dkdw * r.sumS;
  }

  // pair count
  long long pairs = 0;
  for (int kk = 0; kk < nk; ++kk)
    for (int kw = 0; kw < nw; ++kw) {
      if (kk == 0 && kw == 0) continue;
      long long m = (long long)(kk + 1) * (kw + 1) - 2;
      pairs += (m + 1) / 2;
    }
  p->pairs = pairs;

  rc = prepare_sampling_tables(p, st);
  if (rc) return rc;

  // tiles, storage choice and the W table
  if (p->precision == SRM3_FP32) {
    long long entries = 0;
    bool maybe_table = p->storage != SRM3_STORAGE_RECOMPUTE;
    rc = build_tiles(p, st, maybe_table, &entries);
    if (rc) return rc;
    double bytes = (double)entries * sizeof(float);
    if (p->storage == SRM3_STORAGE_AUTO) {
      p->storage = bytes <= p->table_budget ? SRM3_STORAGE_TABLE : SRM3_STORAGE_RECOMPUTE;
    }
    if (p->storage == SRM3_STORAGE_TABLE) {
      cudaError_t e = cudaMalloc(&p->W, (size_t)entries * sizeof(float));
      if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(W table)");
      SRM3_CUDA(cudaEventRecord(t_ev[0], st));
      k_build_w<<<p->ntiles, 256, 0, st>>>(nk, nw, p->ntw, p->tile_off, (const float *)p->ck,
                                            (const float *)p->Ek, (const float *)p->Ews,
                                            p->ew_off, p->W);
      SRM3_CUDA(cudaGetLastError());
      SRM3_CUDA(cudaEventRecord(t_ev[1], st));
      SRM3_CUDA(cudaEventSynchronize(t_ev[1]));
      float tms = 0.f;
      SRM3_CUDA(cudaEventElapsedTime(&tms, t_ev[0], t_ev[1]));
      p->t_table_ms = tms;
      p->table_bytes = bytes;
    } else {
      p->table_bytes = 0.0;
    }
  } else {
    p->storage = SRM3_STORAGE_RECOMPUTE;
    p->table_bytes = 0.0;
  }
  SRM3_CUDA(cudaStreamSynchronize(st));
  return SRM3_OK;
}

int prepare_sampling_tables(srm3_plan *p, cudaStream_t st) {
  const int nk = p->nk, nw = p->nw;
  const size_t nl = (size_t)nk * nw;
  const bool f32 = p->precision == SRM3_FP32;
  const size_t es = f32 ? sizeof(float) : sizeof(double);
  p->ew_off = nw + 32;
  p->ew_len = 2 * nw + 96 + kTileR + kTileU;
  p->nfft = std::max(p->nx, p->nt);
  SRM3_CUDA(cudaMalloc(&p->sqq, nl * es));
  SRM3_CUDA(cudaMalloc(&p->Pk, nl * es));
  SRM3_CUDA(cudaMalloc(&p->ck, nl * es));
  SRM3_CUDA(cudaMalloc(&p->Ek, nk * es));
  SRM3_CUDA(cudaMalloc(&p->Ews, p->ew_len * es));
  SRM3_CUDA(cudaMalloc(&p->tw, p->nfft * 2 * es));
  if (f32) {
    k_sampling_tables<float><<<cdiv(nl, 256), 256, 0, st>>>(
        (int)nl, p->dkdw, p->eps, p->S, p->qm, p->sb2, (float *)p->sqq, (float *)p->Pk,
        (float *)p->ck);
    k_env<float><<<cdiv(nk, 256), 256, 0, st>>>(nk, 0, p->sigma_g * nk, (float *)p->Ek);
    k_env<float><<<cdiv(p->ew_len, 256), 256, 0, st>>>(p->ew_len, p->ew_off, p->sigma_g * nw,
                                                      (float *)p->Ews);
    k_twiddles<float2><<<cdiv(p->nfft, 256), 256, 0, st>>>(p->nfft, (float2 *)p->tw);
  } else {
    k_sampling_tables<double><<<cdiv(nl, 256), 256, 0, st>>>(
        (int)nl, p->dkdw, p->eps, p->S, p->qm, p->sb2, (double *)p->sqq, (double *)p->Pk,
        (double *)p->ck);
    k_env<double><<<cdiv(nk, 256), 256, 0, st>>>(nk, 0, p->sigma_g * nk, (double *)p->Ek);
    k_env<double><<<cdiv(p->ew_len, 256), 256, 0, st>>>(p->ew_len, p->ew_off,
                                                       p->sigma_g * nw, (double *)p->Ews);
    k_twiddles<double2><<<cdiv(p->nfft, 256), 256, 0, st>>>(p->nfft, (double2 *)p->tw);
  }
  SRM3_CUDA(cudaGetLastError());
  SRM3_CUDA(cudaStreamSynchronize(st));
  return SRM3_OK;
}

void free_plan(srm3_plan *p) {
  for (auto &r : p->ev_recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : p->ev_pool) cudaEventDestroy(e);
  if (p->rec_exec) cudaGraphExecDestroy(p->rec_exec);
  if (p->rec_graph) cudaGraphDestroy(p->rec_graph);
  void *dev[] = {p->S,   p->qm, p->sb2, p->EkSq, p->EwSq,       p->scal,     p->err,
                 p->sqq, p->Pk, p->ck,  p->Ek,   p->Ews,        p->tw,       p->tile_order,
                 p->tile_off, p->W, p->y, p->y0, p->C,           p->H};
  for (void *d : dev)
    if (d) cudaFree(d);
  if (p->h_pinned) cudaFreeHost(p->h_pinned);
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
  if (g.storage < SRM3_STORAGE_AUTO || g.storage > SRM3_STORAGE_RECOMPUTE)
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
  if (bispectrum->kind != SRM3_BISPECTRUM_GAUSS_ENVELOPE)
    return fail(SRM3_ERR_INVALID_ARG, "unknown bispectrum kind");
  if (!(bispectrum->sigma_g > 0.0)) return fail(SRM3_ERR_INVALID_ARG, "sigma_g must be > 0");
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
  p->sigma_g = bispectrum->sigma_g;
  p->beta = bispectrum->beta;
  p->table_budget = g.table_budget_bytes > 0 ? g.table_budget_bytes : 64.0 * (1ull << 30);
  cudaGetDevice(&p->device);
  int rc = build_plan(p, spectrum, bispectrum);
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
  return SRM3_OK;
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
  info->storage = plan->storage;
  info->precision = plan->precision;
  info->tile_r = kTileR;
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
