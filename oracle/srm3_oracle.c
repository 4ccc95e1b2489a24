/*
 * srm3_oracle.c - plain FP64 CPU oracle for the third-order Spectral
 * Representation Method (SRM3) for one-dimensional stochastic waves u(x,t),
 * after Vandanapu & Shields, "Simulation of non-Gaussian wind field as a
 * 3rd-order stochastic wave" (arXiv 2310.03979).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * statement of what the GPU path computes.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg load it.  It shares no code,
 * header, table or constant with the CUDA library, and it includes nothing
 * from it.  Everything is IEEE FP64 (build with -ffp-contract=off).
 *
 * Model (one quadrant lattice per omega-sheet, sum interactions only):
 *   lattice   k = (kk, kw), 0 <= kk < Nk, 0 <= kw < Nw,
 *             kappa_k = kk*dk, omega_k = kw*dw, dk = kappa_u/Nk,
 *             dw = omega_u/Nw                           (Sec. 4.1)
 *   sheets    s = + (frequency +omega) and s = - (frequency -omega), each
 *             with its own independent phases            (Eq. quadrant_1d_wave)
 *   pairs     Pi(k) = unordered {i, j}, i + j = k componentwise, i != 0,
 *             j != 0, each counted once; enumerated as i <=_lex j.
 *   pure      S_p(k) = S(k) (1 - sum_{Pi(k)} b_p^2(i,j))   (Eq. pure, with
 *             b_p squared as in the 1-D form of Sec. 4 and in the FFT form)
 *   bicoh.    b_p^2(i,j) = |B(i,j)|^2 dk dw / (S_p(i) S_p(j) S(k))   (Sec. 4.1)
 *   biphase   beta = atan2(Im B, Re B)                       (Sec. 4.1)
 *   bispec.   |B(i,j)| = eps * g(i,j) * sqrt(S(i) S(j) S(k)),  B real times
 *             exp(i*beta) with a constant biphase beta.
 *   envelope  kind 0: g = exp(-1/2 ((ik-jk)/(sg*Nk))^2) * exp(-1/2 ((iw-jw)/(sg*Nw))^2)
 *             kind 1: g = e(i) e(j) e(k) for a caller table e (separable)
 *             kind 2: g = a(i) a(j) b(k) for caller tables a, b (separable;
 *             a = 1 gives envelopes of k alone, as in Sec. 5)
 *
 * Field (Eq. quadrant_1d_wave; FFT form of Sec. 4.3):
 *   u(x,t) = sum_s sum_k Re[ C^s_k exp(i(kappa_k x + s omega_k t)) ],
 *   C^s_k  = 2 sqrt(dk dw) [ sqrt(S_p(k)) e^{i phi^s_k}
 *            + sqrt(S(k)) sum_{Pi(k)} b_p(i,j) e^{i(phi^s_i + phi^s_j + beta)} ],
 *   on x = mx*dx, t = mt*dt, dk*dx = 2 pi / Nx, dw*dt = 2 pi / Nt (Sec. 4.3).
 *
 * Phases: phi^s_k = 2 pi (w + 1/2) 2^-32, where w is word (e & 3) of
 * Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11) at counter
 * (e >> 2) and key = seed, with e = (s*Nk + kk)*Nw + kw.
 *
 * Mixed-sign (difference) interactions, switched on by `mixed` (the pairs
 * of opposite-sign frequencies of the general form, Eq.
 * truncated_cosines_1d_wave, whose quadrant form Eq. quadrant_1d_wave
 * writes as the -w_i + w_j and +w_i - w_j cosines, and the signed sums
 * i_w + j_w = +-k_w of Eq. fft_2d_2_parts).  A point is a signed frequency
 * (kk, s kw); the difference pairs of k = (kk, s kw), kw >= 1, are
 *   i = (ia, s (kw + jw)) on sheet s,  j = (kk - ia, -s jw) on sheet -s,
 *   0 <= ia <= kk,  1 <= jw <= Nw - 1 - kw,
 * each unordered {i, j} once (the sheets tell i from j).  Pairs whose
 * frequencies cancel (iw = jw) would land on omega = 0 and are left out;
 * omega = 0 points take part in sum pairs of their own sheet only.  The
 * bispectrum is the same formula at the signed points: |B| = eps g(i,j)
 * sqrt(S_i S_j S_k), S and S_p at |omega| (both sheets share them), the
 * Gaussian envelope of the signed difference omega_i - omega_j (= s (kw +
 * 2 jw)), separable tables at |omega|.  With them S_p(k) depends on points
 * of higher |omega|, so Eq. pure becomes a fixed point: S_p is the largest
 * solution of S_p = S (1 - sum b_p^2(S_p)), reached by Gauss-Seidel sweeps
 * in lexicographic order from S_p = S (each sweep can only lower S_p, and
 * stays above every solution).  Sum interactions alone reach it in one
 * sweep: that is the recursion of the plain model.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_ERR_ARG (-1)
#define OR_ERR_NONPOSITIVE_PURE (-3)
#define OR_ERR_BISECTION (-4)

static const double OR_PI = 3.14159265358979323846264338327950288;

/* ------------------------------------------------------------------------ */
/* Spectrum: Kaimal (Eq. kaimal_spectrum) times a normalised Lorentzian
 * wavenumber density a / (pi (a^2 + kappa^2)) with a = lam*omega/(2 pi U);
 * u* = k_vk U / ln(z / z0) (Sec. 5).  S := 0 on the omega = 0 column, where
 * the Lorentzian degenerates to a delta. */
int or_kaimal_lorentzian(int nk, int nw, double kappa_u, double omega_u,
                         double U, double z, double z0, double k_vk,
                         double lam, double *S)
{
    if (nk <= 0 || nw <= 0 || !(U > 0) || !(z > z0) || !(z0 > 0) || !S)
        return OR_ERR_ARG;
    double dk = kappa_u / nk, dw = omega_u / nw;
    double ustar = k_vk * U / log(z / z0);
    for (int kk = 0; kk < nk; ++kk) {
        for (int kw = 0; kw < nw; ++kw) {
            double kappa = kk * dk, omega = kw * dw;
            double val = 0.0;
            if (kw > 0) {
                double kaimal = 0.5 * (200.0 / (2.0 * OR_PI)) * ustar * ustar
                              * (z / U)
                              / pow(1.0 + 50.0 * omega * z / (2.0 * OR_PI * U), 5.0 / 3.0);
                double a = lam * omega / (2.0 * OR_PI * U);
                double lorentz = a / (OR_PI * (a * a + kappa * kappa));
                val = kaimal * lorentz;
            }
            S[(size_t)kk * nw + kw] = val;
        }
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Bispectrum modulus |B(i,j)| for i + j = k (all three inside the lattice). */
typedef struct {
    int nk, nw;
    int env_kind;          /* 0 gaussian, 1 separable table, 2 separable pair */
    double sigma_g;
    const double *env_tab; /* kind 1: e[kk*nw + kw]; kind 2: a then b (2 nk nw) */
    double eps;
} or_bispec;

static double or_envelope(const or_bispec *B, int ik, int iw, int jk, int jw)
{
    if (B->env_kind == 0) {
        double ak = (double)(ik - jk) / (B->sigma_g * B->nk);
        double aw = (double)(iw - jw) / (B->sigma_g * B->nw);
        return exp(-0.5 * ak * ak) * exp(-0.5 * aw * aw);
    }
    /* kind 1: g = e(i) e(j) e(i+j); kind 2: g = a(i) a(j) b(i+j), which holds
     * envelopes that depend on i + j alone (a = 1), as the bispectrum of the
     * wind-field example of Sec. 5 does */
    int kk = ik + jk, kw = iw + jw;
    const double *a = B->env_tab;
    const double *b = B->env_kind == 2 ? B->env_tab + (size_t)B->nk * B->nw : B->env_tab;
    return a[(size_t)ik * B->nw + iw] * a[(size_t)jk * B->nw + jw]
         * b[(size_t)kk * B->nw + kw];
}

static double or_modB(const or_bispec *B, const double *S,
                      int ik, int iw, int jk, int jw)
{
    int nw = B->nw;
    double Si = S[(size_t)ik * nw + iw], Sj = S[(size_t)jk * nw + jw];
    double Sk = S[(size_t)(ik + jk) * nw + (iw + jw)];
    return B->eps * or_envelope(B, ik, iw, jk, jw) * sqrt(Si * Sj * Sk);
}

/* Canonical half of Pi(k): i = (ik, iw) with i <_lex j = k - i or i == j,
 * and i != 0.  Visits each unordered pair once. */
static int or_is_canonical(int kk, int kw, int ik, int iw)
{
    int jk = kk - ik, jw = kw - iw;
    if (ik == 0 && iw == 0) return 0;
    if (jk == 0 && jw == 0) return 0;
    if (ik < jk) return 1;
    if (ik == jk && iw <= jw) return 1;
    return 0;
}

/* b_p^2(i,j) per the partial bicoherence definition (Sec. 4.1). */
static double or_bp2(const or_bispec *B, const double *S, const double *Sp,
                     double dkdw, int ik, int iw, int jk, int jw)
{
    int nw = B->nw;
    double mb = or_modB(B, S, ik, iw, jk, jw);
    if (mb == 0.0) return 0.0;
    double Spi = Sp[(size_t)ik * nw + iw], Spj = Sp[(size_t)jk * nw + jw];
    double Sk = S[(size_t)(ik + jk) * nw + (iw + jw)];
    return mb * mb * dkdw / (Spi * Spj * Sk);
}

/* Envelope at signed points (ik, iw), (jk, jw) (omega indices signed):
 * the Gaussian of the signed differences, separable tables at |omega|. */
static double or_envelope_signed(const or_bispec *B, int ik, int iw, int jk, int jw)
{
    if (B->env_kind == 0) {
        double ak = (double)(ik - jk) / (B->sigma_g * B->nk);
        double aw = (double)(iw - jw) / (B->sigma_g * B->nw);
        return exp(-0.5 * ak * ak) * exp(-0.5 * aw * aw);
    }
    int kk = ik + jk, kw = abs(iw + jw);
    const double *a = B->env_tab;
    const double *b = B->env_kind == 2 ? B->env_tab + (size_t)B->nk * B->nw : B->env_tab;
    return a[(size_t)ik * B->nw + abs(iw)] * a[(size_t)jk * B->nw + abs(jw)]
         * b[(size_t)kk * B->nw + kw];
}

/* b_p^2 of the difference pair i = (ia, s (kw + jw)), j = (kk - ia, -s jw)
 * of k = (kk, s kw) (the sign s drops out: S, S_p at |omega|, the envelope
 * even in the signed difference). */
static double or_bp2_diff(const or_bispec *B, const double *S, const double *Sp,
                          double dkdw, int kk, int kw, int ia, int jw)
{
    int nw = B->nw, ib = kk - ia, iw = kw + jw;
    double Si = S[(size_t)ia * nw + iw], Sj = S[(size_t)ib * nw + jw];
    double Sk = S[(size_t)kk * nw + kw];
    double mb = B->eps * or_envelope_signed(B, ia, iw, ib, -jw) * sqrt(Si * Sj * Sk);
    if (mb == 0.0) return 0.0;
    double Spi = Sp[(size_t)ia * nw + iw], Spj = Sp[(size_t)ib * nw + jw];
    return mb * mb * dkdw / (Spi * Spj * Sk);
}

/* Pure-spectrum recursion (Eq. pure) at a given eps, in plain lexicographic
 * order (kk outer, kw inner): every part of a pair of Pi(k) precedes k.
 * Writes S_p and sum_b2[k] = sum_{Pi(k)} b_p^2.  Returns
 * OR_ERR_NONPOSITIVE_PURE at the first k with sum_b2 >= 1 (S_p <= 0). */
int or_recursion(int nk, int nw, double kappa_u, double omega_u,
                 const double *S, int env_kind, double sigma_g,
                 const double *env_tab, double eps,
                 double *Sp, double *sum_b2)
{
    if (nk <= 0 || nw <= 0 || !S || !Sp || !sum_b2) return OR_ERR_ARG;
    or_bispec B = {nk, nw, env_kind, sigma_g, env_tab, eps};
    double dkdw = (kappa_u / nk) * (omega_u / nw);
    for (int kk = 0; kk < nk; ++kk) {
        for (int kw = 0; kw < nw; ++kw) {
            size_t k = (size_t)kk * nw + kw;
            double acc = 0.0;
            if (S[k] > 0.0) {
                for (int ik = 0; ik <= kk; ++ik)
                    for (int iw = 0; iw <= kw; ++iw)
                        if (or_is_canonical(kk, kw, ik, iw))
                            acc += or_bp2(&B, S, Sp, dkdw, ik, iw, kk - ik, kw - iw);
            }
            sum_b2[k] = acc;
            Sp[k] = S[k] * (1.0 - acc);
            if (S[k] > 0.0 && !(acc < 1.0)) return OR_ERR_NONPOSITIVE_PURE;
        }
    }
    return OR_OK;
}

/* Eq. pure with sum and difference interactions (see the header): the
 * largest fixed point S_p = S (1 - sum_{Pi(k)} b_p^2 - sum_{D(k)} b_p^2),
 * by Gauss-Seidel sweeps over the lattice in lexicographic order, each
 * point from the current S_p of all others, starting at S_p = S.  Stops
 * after the first sweep in which no S_p(k) moves by more than tol S(k)
 * (and never before the second sweep); *sweeps receives the sweeps done.
 * Returns OR_ERR_NONPOSITIVE_PURE when some sum_b2 reaches 1 (the sweeps
 * have no positive fixed point to approach) and OR_ERR_BISECTION when
 * max_sweeps pass without convergence. */
int or_recursion_mixed(int nk, int nw, double kappa_u, double omega_u,
                       const double *S, int env_kind, double sigma_g,
                       const double *env_tab, double eps, double tol,
                       int max_sweeps, double *Sp, double *sum_b2, int *sweeps)
{
    if (nk <= 0 || nw <= 0 || !S || !Sp || !sum_b2 || max_sweeps < 2) return OR_ERR_ARG;
    or_bispec B = {nk, nw, env_kind, sigma_g, env_tab, eps};
    double dkdw = (kappa_u / nk) * (omega_u / nw);
    size_t nl = (size_t)nk * nw;
    for (size_t k = 0; k < nl; ++k) { Sp[k] = S[k]; sum_b2[k] = 0.0; }
    for (int sw = 1; sw <= max_sweeps; ++sw) {
        double moved = 0.0;
        for (int kk = 0; kk < nk; ++kk) {
            for (int kw = 0; kw < nw; ++kw) {
                size_t k = (size_t)kk * nw + kw;
                double acc = 0.0;
                if (S[k] > 0.0) {
                    for (int ik = 0; ik <= kk; ++ik)
                        for (int iw = 0; iw <= kw; ++iw)
                            if (or_is_canonical(kk, kw, ik, iw))
                                acc += or_bp2(&B, S, Sp, dkdw, ik, iw, kk - ik, kw - iw);
                    if (kw >= 1)
                        for (int ia = 0; ia <= kk; ++ia)
                            for (int jw = 1; jw <= nw - 1 - kw; ++jw)
                                acc += or_bp2_diff(&B, S, Sp, dkdw, kk, kw, ia, jw);
                }
                double sp = S[k] * (1.0 - acc);
                if (S[k] > 0.0 && !(acc < 1.0)) {
                    sum_b2[k] = acc;
                    Sp[k] = sp;
                    if (sweeps) *sweeps = sw;
                    return OR_ERR_NONPOSITIVE_PURE;
                }
                double d = fabs(sp - Sp[k]);
                if (S[k] > 0.0 && d > moved * S[k]) moved = d / S[k];
                sum_b2[k] = acc;
                Sp[k] = sp;
            }
        }
        if (sw >= 2 && moved <= tol) {
            if (sweeps) *sweeps = sw;
            return OR_OK;
        }
    }
    if (sweeps) *sweeps = max_sweeps;
    return OR_ERR_BISECTION;
}

/* The fixed-point tolerance and sweep limit of the bisection's evaluations
 * with difference interactions. */
#define OR_MIXED_TOL 1e-15
#define OR_MIXED_SWEEPS 100000

static double or_eval_max(int nk, int nw, double kappa_u, double omega_u,
                          const double *S, int env_kind, double sigma_g,
                          const double *env_tab, double eps, int mixed,
                          double *Sp, double *sum_b2)
{
    int rc = mixed ? or_recursion_mixed(nk, nw, kappa_u, omega_u, S, env_kind, sigma_g,
                                        env_tab, eps, OR_MIXED_TOL, OR_MIXED_SWEEPS, Sp,
                                        sum_b2, NULL)
                   : or_recursion(nk, nw, kappa_u, omega_u, S, env_kind, sigma_g,
                                  env_tab, eps, Sp, sum_b2);
    if (rc != OR_OK) return INFINITY;
    double m = 0.0;
    for (size_t k = 0; k < (size_t)nk * nw; ++k)
        if (sum_b2[k] > m) m = sum_b2[k];
    return m;
}

/* Plain bisection on eps so that max_k sum_b2(k) = target.  The bracket
 * [lo, hi] starts at [0, 1] and hi doubles until max sum_b2 >= target or
 * the recursion fails; a failed recursion counts as "above target".  Stops
 * when |max - target| <= tol, when the bracket is one ulp wide, or after
 * max_iter halvings.  On return Sp/sum_b2 hold the recursion at *eps_out. */
int or_bisect_eps(int nk, int nw, double kappa_u, double omega_u,
                  const double *S, int env_kind, double sigma_g,
                  const double *env_tab, int mixed, double target, double tol,
                  int max_iter, double *eps_out, double *max_out,
                  int *iters_out, double *Sp, double *sum_b2)
{
    if (!(target > 0.0 && target < 1.0) || !eps_out || !max_out) return OR_ERR_ARG;
    double lo = 0.0, hi = 1.0;
    int it = 0;
    double fhi = or_eval_max(nk, nw, kappa_u, omega_u, S, env_kind, sigma_g,
                             env_tab, hi, mixed, Sp, sum_b2);
    ++it;
    while (fhi < target) {
        if (fhi == 0.0 && hi > 1e300) return OR_ERR_BISECTION; /* no pairs */
        lo = hi;
        hi *= 2.0;
        fhi = or_eval_max(nk, nw, kappa_u, omega_u, S, env_kind, sigma_g,
                          env_tab, hi, mixed, Sp, sum_b2);
        ++it;
    }
    double mid = hi, fm = fhi;
    for (int n = 0; n < max_iter; ++n) {
        mid = 0.5 * (lo + hi);
        fm = or_eval_max(nk, nw, kappa_u, omega_u, S, env_kind, sigma_g,
                         env_tab, mid, mixed, Sp, sum_b2);
        ++it;
        if (fabs(fm - target) <= tol) break;
        if (fm < target) lo = mid; else hi = mid;
        if (hi - lo <= 2.220446049250313e-16 * hi) break;
    }
    if (!isfinite(fm)) {
        /* land on the feasible side of the bracket */
        mid = lo;
        fm = or_eval_max(nk, nw, kappa_u, omega_u, S, env_kind, sigma_g,
                         env_tab, mid, mixed, Sp, sum_b2);
        ++it;
    }
    *eps_out = mid;
    *max_out = fm;
    if (iters_out) *iters_out = it;
    return isfinite(fm) ? OR_OK : OR_ERR_BISECTION;
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64-bit
 * multiplications with a Weyl-sequence key schedule. */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                      uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)M0 * c0;
        uint64_t p1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += W0; k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Phase word for (seed, sheet s, kk, kw). */
static uint32_t or_phase_word(uint64_t seed, int nk, int nw, int s, int kk, int kw)
{
    uint64_t e = ((uint64_t)s * nk + kk) * nw + kw;
    uint64_t c = e >> 2;
    uint32_t ctr[4] = {(uint32_t)c, (uint32_t)(c >> 32), 0u, 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    or_philox4x32_10(ctr, key, out);
    return out[e & 3];
}

/* Phase words and angles for one sample: words[s][kk][kw] and
 * phi[s][kk][kw] = 2 pi (w + 1/2) 2^-32 in [0, 2 pi). */
void or_phases(int nk, int nw, uint64_t seed, uint32_t *words, double *phi)
{
    for (int s = 0; s < 2; ++s)
        for (int kk = 0; kk < nk; ++kk)
            for (int kw = 0; kw < nw; ++kw) {
                size_t e = ((size_t)s * nk + kk) * nw + kw;
                uint32_t w = or_phase_word(seed, nk, nw, s, kk, kw);
                if (words) words[e] = w;
                if (phi) phi[e] = 2.0 * OR_PI * (((double)w + 0.5) * 0x1p-32);
            }
}

/* ------------------------------------------------------------------------ */
/* Coefficients C^s_k (FFT form, Sec. 4.3) for one sample, from S, S_p and
 * the phases; with `mixed`, the difference pairs of the header too.  C[((s*nk + kk)*nw + kw)*2 + {0,1}] = (Re, Im).  The pair
 * exponential e^{i(phi_i + phi_j + beta)} is evaluated as the product of
 * the unit phasors.  OpenMP over k (each C_k is independent). */
int or_coeffs(int nk, int nw, double kappa_u, double omega_u,
              const double *S, const double *Sp, int env_kind, double sigma_g,
              const double *env_tab, int mixed, double eps, double beta, uint64_t seed,
              double *C)
{
    if (nk <= 0 || nw <= 0 || !S || !Sp || !C) return OR_ERR_ARG;
    size_t nl = (size_t)nk * nw;
    double *phi = (double *)malloc(2 * nl * sizeof(double));
    double *zr = (double *)malloc(2 * nl * sizeof(double));
    double *zi = (double *)malloc(2 * nl * sizeof(double));
    if (!phi || !zr || !zi) { free(phi); free(zr); free(zi); return OR_ERR_ARG; }
    or_phases(nk, nw, seed, NULL, phi);
    for (size_t e = 0; e < 2 * nl; ++e) { zr[e] = cos(phi[e]); zi[e] = sin(phi[e]); }
    or_bispec B = {nk, nw, env_kind, sigma_g, env_tab, eps};
    double dkdw = (kappa_u / nk) * (omega_u / nw);
    double cb = cos(beta), sb = sin(beta);
    long long ntot = (long long)nl;
#pragma omp parallel for schedule(dynamic, 16)
    for (long long kl = 0; kl < ntot; ++kl) {
        int kk = (int)(kl / nw), kw = (int)(kl % nw);
        size_t k = (size_t)kl;
        for (int s = 0; s < 2; ++s) {
            const double *Zr = zr + (size_t)s * nl, *Zi = zi + (size_t)s * nl;
            double pr = 0.0, pi = 0.0;
            if (S[k] > 0.0) {
                for (int ik = 0; ik <= kk; ++ik)
                    for (int iw = 0; iw <= kw; ++iw) {
                        if (!or_is_canonical(kk, kw, ik, iw)) continue;
                        int jk = kk - ik, jw = kw - iw;
                        double b2 = or_bp2(&B, S, Sp, dkdw, ik, iw, jk, jw);
                        if (b2 == 0.0) continue;
                        double b = sqrt(b2);
                        size_t a = (size_t)ik * nw + iw, c = (size_t)jk * nw + jw;
                        double xr = Zr[a] * Zr[c] - Zi[a] * Zi[c];
                        double xi = Zr[a] * Zi[c] + Zi[a] * Zr[c];
                        pr += b * (xr * cb - xi * sb);
                        pi += b * (xr * sb + xi * cb);
                    }
                /* difference pairs: i = (ia, kw + jw) on this sheet, j =
                 * (kk - ia, jw) on the other, phases phi^s_i + phi^{-s}_j */
                const double *Or = zr + (size_t)(1 - s) * nl, *Oi = zi + (size_t)(1 - s) * nl;
                if (mixed && kw >= 1)
                    for (int ia = 0; ia <= kk; ++ia)
                        for (int jw = 1; jw <= nw - 1 - kw; ++jw) {
                            double b2 = or_bp2_diff(&B, S, Sp, dkdw, kk, kw, ia, jw);
                            if (b2 == 0.0) continue;
                            double b = sqrt(b2);
                            size_t a = (size_t)ia * nw + (kw + jw), c = (size_t)(kk - ia) * nw + jw;
                            double xr = Zr[a] * Or[c] - Zi[a] * Oi[c];
                            double xi = Zr[a] * Oi[c] + Zi[a] * Or[c];
                            pr += b * (xr * cb - xi * sb);
                            pi += b * (xr * sb + xi * cb);
                        }
            }
            double amp_pure = sqrt(Sp[k] > 0.0 ? Sp[k] : 0.0);
            double amp_pair = sqrt(S[k]);
            double re = amp_pure * Zr[k] + amp_pair * pr;
            double im = amp_pure * Zi[k] + amp_pair * pi;
            double f = 2.0 * sqrt(dkdw);
            C[(((size_t)s * nl) + k) * 2 + 0] = f * re;
            C[(((size_t)s * nl) + k) * 2 + 1] = f * im;
        }
    }
    free(phi); free(zr); free(zi);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Field from coefficients by the direct double sum (no FFT), evaluated
 * separably: G[kk][mt] = sum_s sum_kw C^s[kk][kw] e^{i s 2pi kw mt / Nt},
 * then u[mx][mt] = Re sum_kk G[kk][mt] e^{i 2pi kk mx / Nx}.  The angle
 * index is reduced exactly in integers before cos/sin. */
int or_field_dft(int nk, int nw, int nx, int nt, const double *C, double *u)
{
    if (nk <= 0 || nw <= 0 || nx <= 0 || nt <= 0 || !C || !u) return OR_ERR_ARG;
    size_t nl = (size_t)nk * nw;
    double *gr = (double *)calloc((size_t)nk * nt, sizeof(double));
    double *gi = (double *)calloc((size_t)nk * nt, sizeof(double));
    if (!gr || !gi) { free(gr); free(gi); return OR_ERR_ARG; }
#pragma omp parallel for schedule(static)
    for (int mt = 0; mt < nt; ++mt) {
        for (int kk = 0; kk < nk; ++kk) {
            double ar = 0.0, ai = 0.0;
            for (int s = 0; s < 2; ++s) {
                for (int kw = 0; kw < nw; ++kw) {
                    long long r = ((long long)kw * mt) % nt;
                    if (s == 1) r = (nt - r) % nt;
                    double ang = 2.0 * OR_PI * (double)r / (double)nt;
                    double c = cos(ang), sn = sin(ang);
                    const double *Ck = C + (((size_t)s * nl) + (size_t)kk * nw + kw) * 2;
                    ar += Ck[0] * c - Ck[1] * sn;
                    ai += Ck[0] * sn + Ck[1] * c;
                }
            }
            gr[(size_t)kk * nt + mt] = ar;
            gi[(size_t)kk * nt + mt] = ai;
        }
    }
#pragma omp parallel for schedule(static)
    for (int mx = 0; mx < nx; ++mx) {
        for (int mt = 0; mt < nt; ++mt) {
            double acc = 0.0;
            for (int kk = 0; kk < nk; ++kk) {
                long long r = ((long long)kk * mx) % nx;
                double ang = 2.0 * OR_PI * (double)r / (double)nx;
                acc += gr[(size_t)kk * nt + mt] * cos(ang) - gi[(size_t)kk * nt + mt] * sin(ang);
            }
            u[(size_t)mx * nt + mt] = acc;
        }
    }
    free(gr); free(gi);
    return OR_OK;
}

/* Field at selected points from coefficients by the plain double sum
 * u = Re sum_s sum_k C^s_k e^{i(2pi kk mx/Nx + s 2pi kw mt/Nt)}. */
int or_field_points(int nk, int nw, int nx, int nt, const double *C,
                    int npts, const int *mx, const int *mt, double *u)
{
    if (nk <= 0 || nw <= 0 || npts < 0 || !C || (npts && (!mx || !mt || !u)))
        return OR_ERR_ARG;
    size_t nl = (size_t)nk * nw;
#pragma omp parallel for schedule(dynamic, 1)
    for (int p = 0; p < npts; ++p) {
        double acc = 0.0;
        for (int s = 0; s < 2; ++s)
            for (int kk = 0; kk < nk; ++kk)
                for (int kw = 0; kw < nw; ++kw) {
                    long long rx = ((long long)kk * mx[p]) % nx;
                    long long rt = ((long long)kw * mt[p]) % nt;
                    if (s == 1) rt = (nt - rt) % nt;
                    /* angle = 2 pi (rx/nx + rt/nt), reduced over the common period */
                    long long num = rx * (long long)nt + rt * (long long)nx;
                    long long den = (long long)nx * nt;
                    num %= den;
                    double ang = 2.0 * OR_PI * (double)num / (double)den;
                    const double *Ck = C + (((size_t)s * nl) + (size_t)kk * nw + kw) * 2;
                    acc += Ck[0] * cos(ang) - Ck[1] * sin(ang);
                }
        u[p] = acc;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Field at selected points by the literal cosine series of
 * Eq. quadrant_1d_wave (sum interactions, one sheet at a time; with
 * `mixed`, its two mixed cosines per pair, written at the frequencies of
 * their parts), with x = mx dx, t = mt dt.  Costs O(#pairs) per point:
 * tiny grids only. */
int or_field_series(int nk, int nw, double kappa_u, double omega_u,
                    int nx, int nt, const double *S, const double *Sp,
                    int env_kind, double sigma_g, const double *env_tab,
                    int mixed, double eps, double beta, uint64_t seed,
                    int npts, const int *mx, const int *mt, double *u)
{
    if (nk <= 0 || nw <= 0 || !S || !Sp || npts < 0) return OR_ERR_ARG;
    size_t nl = (size_t)nk * nw;
    double *phi = (double *)malloc(2 * nl * sizeof(double));
    if (!phi) return OR_ERR_ARG;
    or_phases(nk, nw, seed, NULL, phi);
    or_bispec B = {nk, nw, env_kind, sigma_g, env_tab, eps};
    double dk = kappa_u / nk, dw = omega_u / nw, dkdw = dk * dw;
    double dx = 2.0 * OR_PI / (nx * dk), dt = 2.0 * OR_PI / (nt * dw);
#pragma omp parallel for schedule(dynamic, 1)
    for (int p = 0; p < npts; ++p) {
        double x = mx[p] * dx, t = mt[p] * dt;
        double acc = 0.0;
        for (int s = 0; s < 2; ++s) {
            double sg = (s == 0) ? 1.0 : -1.0;
            const double *ph = phi + (size_t)s * nl;
            for (int kk = 0; kk < nk; ++kk)
                for (int kw = 0; kw < nw; ++kw) {
                    size_t k = (size_t)kk * nw + kw;
                    double theta = kk * dk * x + sg * (kw * dw) * t;
                    double sp = Sp[k] > 0.0 ? Sp[k] : 0.0;
                    acc += 2.0 * sqrt(sp * dkdw) * cos(theta + ph[k]);
                    if (!(S[k] > 0.0)) continue;
                    for (int ik = 0; ik <= kk; ++ik)
                        for (int iw = 0; iw <= kw; ++iw) {
                            if (!or_is_canonical(kk, kw, ik, iw)) continue;
                            int jk = kk - ik, jw = kw - iw;
                            double b2 = or_bp2(&B, S, Sp, dkdw, ik, iw, jk, jw);
                            if (b2 == 0.0) continue;
                            acc += 2.0 * sqrt(S[k] * dkdw) * sqrt(b2)
                                 * cos(theta + ph[(size_t)ik * nw + iw]
                                       + ph[(size_t)jk * nw + jw] + beta);
                        }
                    /* the mixed cosines: kappa_k x + s (omega_i - omega_j) t
                     * with phi^s_i + phi^{-s}_j, omega_i > omega_j */
                    const double *po = phi + (size_t)(1 - s) * nl;
                    if (mixed && kw >= 1)
                        for (int ia = 0; ia <= kk; ++ia)
                            for (int jw = 1; jw <= nw - 1 - kw; ++jw) {
                                double b2 = or_bp2_diff(&B, S, Sp, dkdw, kk, kw, ia, jw);
                                if (b2 == 0.0) continue;
                                double th = ia * dk * x + (kk - ia) * dk * x
                                          + sg * ((kw + jw) * dw) * t - sg * (jw * dw) * t;
                                acc += 2.0 * sqrt(S[k] * dkdw) * sqrt(b2)
                                     * cos(th + ph[(size_t)ia * nw + kw + jw]
                                           + po[(size_t)(kk - ia) * nw + jw] + beta);
                            }
                }
        }
        u[p] = acc;
    }
    free(phi);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Exact ensemble moments of the discrete series, obtained by averaging over
 * the independent uniform phases: only (pure_i, pure_j, pair_ij) triples
 * survive in E[u^3], with multiplicity 6 (i != j) or 3 (i == j), for sum
 * and (with `mixed`) difference pairs alike:
 *   var = sum_s sum_k |C-amplitudes|^2 / 2 = sum_s sum_k 2 S(k) dk dw,
 *   m3  = sum_s sum_k sum_{Pi(k)} m_ij (1/4) P_i P_j A_ij cos(beta),
 * with P = 2 sqrt(S_p dk dw) and A_ij = 2 sqrt(S(k) dk dw) b_p(i,j).
 * The variance is summed from the amplitudes (pure^2 + pair^2). */
int or_exact_moments(int nk, int nw, double kappa_u, double omega_u,
                     const double *S, const double *Sp, int env_kind,
                     double sigma_g, const double *env_tab, int mixed, double eps,
                     double beta, double *var, double *m3)
{
    if (nk <= 0 || nw <= 0 || !S || !Sp || !var || !m3) return OR_ERR_ARG;
    or_bispec B = {nk, nw, env_kind, sigma_g, env_tab, eps};
    double dkdw = (kappa_u / nk) * (omega_u / nw);
    double v = 0.0, t3 = 0.0;
    for (int kk = 0; kk < nk; ++kk)
        for (int kw = 0; kw < nw; ++kw) {
            size_t k = (size_t)kk * nw + kw;
            double sp = Sp[k] > 0.0 ? Sp[k] : 0.0;
            double pure2 = 4.0 * sp * dkdw;
            double pair2 = 0.0, tri = 0.0;
            if (S[k] > 0.0) {
                for (int ik = 0; ik <= kk; ++ik)
                    for (int iw = 0; iw <= kw; ++iw) {
                        if (!or_is_canonical(kk, kw, ik, iw)) continue;
                        int jk = kk - ik, jw = kw - iw;
                        double b2 = or_bp2(&B, S, Sp, dkdw, ik, iw, jk, jw);
                        if (b2 == 0.0) continue;
                        double A = 2.0 * sqrt(S[k] * dkdw) * sqrt(b2);
                        pair2 += A * A;
                        double Pi = 2.0 * sqrt(Sp[(size_t)ik * nw + iw] * dkdw);
                        double Pj = 2.0 * sqrt(Sp[(size_t)jk * nw + jw] * dkdw);
                        double mult = (ik == jk && iw == jw) ? 3.0 : 6.0;
                        tri += mult * 0.25 * Pi * Pj * A * cos(beta);
                    }
                /* difference pairs: two distinct points, multiplicity 6 */
                if (mixed && kw >= 1)
                    for (int ia = 0; ia <= kk; ++ia)
                        for (int jw = 1; jw <= nw - 1 - kw; ++jw) {
                            double b2 = or_bp2_diff(&B, S, Sp, dkdw, kk, kw, ia, jw);
                            if (b2 == 0.0) continue;
                            double A = 2.0 * sqrt(S[k] * dkdw) * sqrt(b2);
                            pair2 += A * A;
                            double Pi = 2.0 * sqrt(Sp[(size_t)ia * nw + kw + jw] * dkdw);
                            double Pj = 2.0 * sqrt(Sp[(size_t)(kk - ia) * nw + jw] * dkdw);
                            tri += 6.0 * 0.25 * Pi * Pj * A * cos(beta);
                        }
            }
            v += 2.0 * 0.5 * (pure2 + pair2); /* two sheets */
            t3 += 2.0 * tri;
        }
    *var = v;
    *m3 = t3;
    return OR_OK;
}

/* Number of threads the OpenMP regions use (1 without OpenMP). */
int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
