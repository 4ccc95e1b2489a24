/*
 * srm3.h - C ABI of the GB300 (sm_103a) sampler for third-order stochastic
 * waves u(x,t) by the bispectral Spectral Representation Method (SRM3) of
 * Vandanapu & Shields, arXiv 2310.03979.
 *
 * Model (Sec. 4.1-4.3 of the paper, with the readings stated below):
 *   lattice  k = (kk, kw), 0 <= kk < n_kappa, 0 <= kw < n_omega,
 *            kappa = kk*dk, omega = kw*dw, dk = kappa_u/n_kappa,
 *            dw = omega_u/n_omega (Sec. 4.1);
 *   sheets   s = + and s = -, one quadrant lattice each with independent
 *            phases (Eq. quadrant_1d_wave); pairs Pi(k) = unordered {i, j},
 *            i + j = k, i != 0, j != 0 (sum interactions within a sheet);
 *   pure     S_p(k) = S(k) (1 - sum_{Pi(k)} b_p^2)       (Eq. pure, b_p squared)
 *   bicoh.   b_p^2 = |B|^2 dk dw / (S_p(i) S_p(j) S(k))  (Sec. 4.1)
 *   field    u(x,t) = Re sum_s sum_k C^s_k e^{i(kappa x + s omega t)},
 *            C^s_k = 2 sqrt(dk dw) [sqrt(S_p) e^{i phi^s_k}
 *                    + sqrt(S) sum_{Pi(k)} b_p e^{i(phi^s_i + phi^s_j + beta)}]
 *            on x = mx dx, t = mt dt with dk dx = 2pi/n_x, dw dt = 2pi/n_t
 *            (FFT form and grid relations, Sec. 4.3).
 *   phases   phi^s_k = 2 pi (w + 1/2) 2^-32, w = word (e & 3) of
 *            Philox4x32-10 at counter (e >> 2, 0, 0, 0) (low word first) and
 *            key (seed lo, seed hi), e = (s n_kappa + kk) n_omega + kw,
 *            s = 0 for the + sheet and 1 for the - sheet.
 *
 * Errors: every int-returning call returns SRM3_OK (0) or a negative
 * SRM3_ERR_* code; srm3_last_error() returns a message for the calling
 * thread's last failure.  Calls that take a plan never free or replace a
 * caller buffer.  All device pointers are CUDA device addresses in the
 * current device's context; all host pointers are ordinary host memory.
 */
#ifndef SRM3_H
#define SRM3_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SRM3_OK 0
#define SRM3_ERR_INVALID_ARG (-1)      /* a NULL pointer, a size out of range */
#define SRM3_ERR_GRID_CONSTRAINT (-2)  /* n_x, n_t not powers of two >= the lattice */
#define SRM3_ERR_NONPOSITIVE_PURE (-3) /* sum b_p^2 >= 1 somewhere: S_p <= 0 */
#define SRM3_ERR_BISECTION_FAILED (-4) /* no eps reaches the target */
#define SRM3_ERR_OUT_OF_MEMORY (-5)
#define SRM3_ERR_CUDA (-6)             /* a CUDA runtime error; see srm3_last_error */
#define SRM3_ERR_TIMEOUT (-7)
#define SRM3_ERR_NOT_SUPPORTED (-8)

/* Power spectrum S(kappa, omega) on the lattice (Sec. 5). */
enum srm3_spectrum_kind {
    /* Kaimal S(omega) (Eq. kaimal_spectrum) with u* = k_vk U / ln(z/z0),
     * times a/(pi (a^2 + kappa^2)), a = lam omega / (2 pi U); S := 0 on the
     * omega = 0 column. */
    SRM3_SPECTRUM_KAIMAL_LORENTZIAN = 0,
    /* Caller table, host, row-major [n_kappa][n_omega], copied at create. */
    SRM3_SPECTRUM_TABLE = 1
};

typedef struct srm3_spectrum {
    int32_t kind;
    int32_t reserved;
    double U, z, z0, k_vk, lam; /* KAIMAL_LORENTZIAN parameters */
    const double *table;        /* TABLE: host, n_kappa*n_omega doubles, >= 0 */
} srm3_spectrum;

/* Bispectrum |B(i,j)| = eps g(i,j) sqrt(S(i) S(j) S(i+j)) with constant
 * biphase beta (Sec. 4, the bicoherence form of Eq. pure), and either
 *   GAUSS_ENVELOPE: g(i,j) = exp(-1/2 ((ik-jk)/(sigma_g n_kappa))^2)
 *                          * exp(-1/2 ((iw-jw)/(sigma_g n_omega))^2), or
 *   SEPARABLE:      g(i,j) = a(i) a(j) b(i+j), a from env_table and b from
 *                   env_table_b (b = a when env_table_b is NULL); a = 1 gives
 *                   envelopes of i + j alone, as in the wind-field example
 *                   of Sec. 5.
 * A separable g turns the pair sum of every lattice point into a
 * self-convolution: plans with it sample through a zero-padded 2-D FFT
 * instead of the O(N^2) pair sum (Sec. 4.3 FFT form; any storage setting is
 * ignored). */
enum srm3_bispectrum_kind {
    SRM3_BISPECTRUM_GAUSS_ENVELOPE = 0,
    SRM3_BISPECTRUM_SEPARABLE = 1
};

/* Which frequency pairs interact (the pair set of Eq. pure and of the
 * coefficients).
 *   SUM:   i + j = k within one sheet (the quadrant lattice of each sheet).
 *   MIXED: also the pairs of opposite-sign frequencies of the general form
 *          (Eq. truncated_cosines_1d_wave; the mixed cosines of Eq.
 *          quadrant_1d_wave; the signed sums of Eq. fft_2d_2_parts): for
 *          k = (kk, kw) on sheet s, kw >= 1, the pairs i = (ia, kw + jw) on
 *          sheet s and j = (kk - ia, jw) on the other sheet, 0 <= ia <= kk,
 *          1 <= jw <= n_omega - 1 - kw, with phases phi^s_i + phi^{-s}_j
 *          (pairs that would land on omega = 0 are left out; omega = 0
 *          points take sum pairs only).  The bispectrum is the same formula
 *          at the signed points: the Gaussian envelope of the signed
 *          frequency difference, kw + 2 jw here.  S_p then depends on points
 *          of higher omega, so Eq. pure is solved as a fixed point: the
 *          largest S_p with S_p = S (1 - sum b_p^2(S_p)), reached by
 *          iterations that start at S_p = S and can only lower it.  About
 *          twice the pair-terms of SUM.  GAUSS_ENVELOPE only; W is
 *          recomputed (STORAGE_TABLE is refused, AUTO and TUNED recompute);
 *          plans with it take no part in shape groups of a batch. */
enum srm3_interactions {
    SRM3_INTERACTIONS_SUM = 0,
    SRM3_INTERACTIONS_MIXED = 1
};

typedef struct srm3_bispectrum {
    int32_t kind;             /* enum srm3_bispectrum_kind */
    int32_t interactions;     /* enum srm3_interactions (0: SUM) */
    double target_max_sum_b2; /* in (0,1): eps found so that max_k sum b_p^2
                                 equals it to 1e-13; 0: use eps as given */
    double eps;               /* used when target_max_sum_b2 == 0; >= 0 */
    double sigma_g;           /* GAUSS_ENVELOPE: > 0; ignored otherwise */
    double beta;              /* biphase, radians */
    const double *env_table;  /* SEPARABLE: host, n_kappa*n_omega doubles
                                 a[kk*n_omega + kw], finite and >= 0; read
                                 during srm3_plan_create only (the caller
                                 keeps ownership); ignored otherwise */
    const double *env_table_b;/* SEPARABLE: b in the same layout and rules,
                                 or NULL for b = a; ignored otherwise */
} srm3_bispectrum;

enum srm3_precision {
    SRM3_FP32 = 0, /* tiled FP32 pair sum with compensated merge, FP32 FFT */
    SRM3_FP64 = 1  /* plain FP64 pair sum (one warp per k and sheet-sample), FP64 FFT */
};
enum srm3_storage {
    SRM3_STORAGE_AUTO = 0,     /* table if it fits the budget, else recompute */
    SRM3_STORAGE_TABLE = 1,    /* W streamed from an HBM table (FP32 only) */
    SRM3_STORAGE_RECOMPUTE = 2, /* W rebuilt from envelope factors in-kernel */
    SRM3_STORAGE_TUNED = 3      /* the storage srm3_autotune chose for this lattice
                                   shape in this process, else as AUTO */
};

typedef struct srm3_grid {
    int32_t n_kappa, n_omega; /* lattice, >= 1 each */
    double kappa_u, omega_u;  /* cutoffs, > 0 */
    int32_t n_x, n_t;         /* output grid: powers of two, n_x >= n_kappa,
                                 n_t >= 2 n_omega - 1, each <= 8192 */
    int32_t precision;        /* enum srm3_precision */
    int32_t storage;          /* enum srm3_storage */
    void *stream;             /* cudaStream_t for all plan work; NULL = default */
    double table_budget_bytes;/* AUTO: largest W table allowed (0 = 64 GiB) */
    /* Lattice rows [row_begin, row_end) whose coefficients the plan computes
     * (0, 0 = all rows): one shard of a job that splits the W table and the
     * pair sum by rows of kappa across devices -- the distributed storage of
     * the bispectrum the paper proposes for domains past one node's memory
     * (Sec. 4.3).  The recursion still covers the whole lattice (every row's
     * S_p is needed); the W table, the work units and srm3_info.pairs cover
     * the plan's rows only.  Such a plan gives coefficients (srm3_coeffs
     * writes its rows of C and leaves the others untouched), not fields:
     * srm3_sample and srm3_sample_host refuse it with NOT_SUPPORTED, and so
     * does srm3_batch_create; gather every shard's rows, then call
     * srm3_field_from_coeffs.  Not for SEPARABLE plans (their pair sum is an
     * FFT over the whole lattice). */
    int32_t row_begin, row_end;
} srm3_grid;

typedef struct srm3_plan srm3_plan;

/* Build a plan: discretise S on the lattice, run the pure-spectrum recursion
 * over the anti-diagonals of the lattice in FP64 (Eq. pure), find eps by a
 * bracketing root search on max_k sum b_p^2 when a target is given, and,
 * for STORAGE_TABLE, write the W table to HBM.  The plan owns all of its
 * device memory.  Synchronous: returns when the plan is ready.  On error
 * *out stays NULL.  Errors: INVALID_ARG, GRID_CONSTRAINT, NONPOSITIVE_PURE
 * (an explicit eps drives some S_p <= 0), BISECTION_FAILED, OUT_OF_MEMORY,
 * CUDA. */
int srm3_plan_create(const srm3_spectrum *spectrum,
                     const srm3_bispectrum *bispectrum, const srm3_grid *grid,
                     srm3_plan **out);

/* Draw n samples: Philox phases per seed, the coefficients C^s_k by the
 * pair sum (FFT form, Sec. 4.3), then the 2-D inverse transform to
 * u[n][n_x][n_t].  seeds: host array of n seeds.  out: device buffer of
 * n*n_x*n_t floats (FP32 plan) or doubles (FP64 plan), row-major
 * [sample][mx][mt].  Asynchronous on the plan's stream; launch errors
 * return at once, execution errors surface at srm3_sync.  The same
 * (plan, seed) gives bit-identical output whatever n or the other seeds.
 * n == 0 is a no-op.  Not thread-safe per plan (workspace is shared). */
int srm3_sample(srm3_plan *plan, const uint64_t *seeds, int n, void *out);

/* As srm3_sample with a HOST output buffer: copies the seeds in and the
 * field out (n*n_x*n_t elements) inside the call; returns after the copy. */
int srm3_sample_host(srm3_plan *plan, const uint64_t *seeds, int n, void *out_host);

/* Free the plan and its device memory.  NULL is a no-op.  The caller must
 * not have plan work in flight (call srm3_sync first). */
void srm3_destroy(srm3_plan *plan);

/* Wait for the plan's stream; returns the first asynchronous error. */
int srm3_sync(srm3_plan *plan);

/* Re-target the plan's stream (cudaStream_t). */
int srm3_set_stream(srm3_plan *plan, void *stream);

/* Message for the calling thread's last error ("" if none). */
const char *srm3_last_error(void);

typedef struct srm3_info {
    double eps;              /* bispectrum scale in use */
    double max_sum_b2;       /* max_k sum_{Pi(k)} b_p^2 at eps */
    double min_pure_ratio;   /* min over S>0 of S_p/S = 1 - sum b_p^2 */
    double variance;         /* exact ensemble variance sum_s sum_k 2 S dk dw */
    double table_bytes;      /* bytes of the W table (0 when recomputed) */
    double plan_ms;          /* wall time of srm3_plan_create */
    int64_t pairs;           /* sum_k |Pi(k)| over the plan's rows */
    int32_t root_passes;     /* FP64 recursion passes of the build */
    int32_t storage;         /* storage actually chosen */
    int32_t precision;
    int32_t tile_r;          /* outputs per thread along omega (FP32 path) */
    int32_t root_passes_fp32;/* FP32 recursion passes used to locate eps */
    int32_t interactions;    /* enum srm3_interactions */
    int32_t fixed_point_iterations; /* MIXED: iterations of the final solve */
    int64_t diff_pairs;      /* MIXED: difference pairs of one sheet, sum over k
                                of (kk + 1)(n_omega - 1 - kw), kw >= 1; else 0.
                                Pair-terms per sample: 2 (pairs + diff_pairs) */
    double device_bytes;     /* device memory the plan holds now: lattice and
                                sampling tables, recursion state, W table and
                                the sampling workspace (which grows with the
                                largest n sampled, up to 128 per chunk);
                                batch buffers are the batch's */
    int32_t tile_width;      /* FP32 pair-sum work unit: 32 or 16 outputs (the
                                autotuner's choice for the lattice shape, else
                                32); the results do not depend on it */
    int32_t recursion_flags; /* bit 0 (SRM3_REC_SEPARABLE): the recursion ran in
                                separable form, g^2(i,j) = a_i^2 a_j^2 b_k^2 on the
                                pairs of k (the separable kind, or the Gaussian
                                envelope split on i + j = k, Sec. 4.1 Eq. pure);
                                bit 1 (SRM3_REC_TABLES_MOVED): the tables are those
                                of the FP64 pass at the FP32 root estimate, moved to
                                the final eps to first order (FP32 plans);
                                bit 2 (SRM3_PAIRSUM_SEPARABLE): the FP32 pair sum
                                runs in separable form, g = a_i a_j b_k with the
                                omega factor folded into the phasor rows (W
                                recomputed, Gaussian envelope, Sec. 4.3);
                                bit 3 (SRM3_REC_COARSE_START): the eps search
                                started from the root of the same search on a
                                coarser lattice (coarse_fk, coarse_fw below) and
                                one FP32 pass on this lattice bracketed it (no
                                linear bound on this lattice);
                                bit 4 (SRM3_REC_TABLES_INTERPOLATED): the tables
                                are those of one FP64 pass at three eps^2 values
                                x32 (1 +- 2e-6) around the FP32 root, taken per
                                point at the final eps^2 by the quadratic through
                                the three (FP64 plans) */
    int32_t coarse_fk, coarse_fw; /* the coarse lattice of the eps search takes
                                every coarse_fk-th kappa and coarse_fw-th omega
                                point of this one (1, 1: no coarse search; plans
                                with a target, sum interactions and at least
                                65536 points, either envelope kind) */
    int32_t coarse_launches;  /* kernels the coarse search launched */
    int32_t coarse_passes;    /* its FP32 recursion passes */
} srm3_info;

#define SRM3_REC_SEPARABLE 1
#define SRM3_REC_TABLES_MOVED 2
#define SRM3_PAIRSUM_SEPARABLE 4
#define SRM3_REC_COARSE_START 8
#define SRM3_REC_TABLES_INTERPOLATED 16

int srm3_plan_info(const srm3_plan *plan, srm3_info *info);

/* Exact ensemble moments of u at any (x, t): the variance
 * sum_s sum_k 2 S_k dk dw and the third moment
 * E[u^3] = 4 eps cos(beta) (dk dw)^2 sum_k sqrt(S_k) sum_{Pi(k)} m g sqrt(S_i S_j)
 * (m = 6 for i != j, 3 for i = j; Sec. 2 moments of the quadrant form of
 * Sec. 4; MIXED plans add their difference pairs with m = 6), the pair sum
 * taken on the GPU in FP64.  Synchronous on the plan's
 * stream; allocates nk*nw doubles (stream-ordered) for the duration. */
int srm3_plan_moments(const srm3_plan *plan, double *variance, double *third_moment);

/* Failure path of the bounded waits, exercised on the current device without
 * a fault: a cooperative launch whose CTA 0 never reaches a grid barrier (the
 * recursion's barrier, polling limit 2^14) and a wait on an mbarrier that
 * nothing arrives at (the FP32 pair sum's wait, limit 2e7 cycles).  Each
 * wait gives up, raises its error word and returns; *barrier_timed_out and
 * *wait_timed_out receive those words (1 when the timeout fired).  Takes about
 * 20 ms; synchronous; the device stays usable. */
int srm3_selftest_timeouts(int *barrier_timed_out, int *wait_timed_out);

/* Copy the plan's FP64 tables to host arrays of n_kappa*n_omega doubles
 * (any may be NULL): S, q = S/S_p (1 where S = 0), sum_b2. */
int srm3_plan_tables(const srm3_plan *plan, double *S, double *q, double *sum_b2);

/* Philox phase words for n seeds: device buffer words[n][2][n_kappa][n_omega]
 * (uint32), exactly the words behind the phases of srm3_sample.  Async. */
int srm3_phase_words(srm3_plan *plan, const uint64_t *seeds, int n, uint32_t *words);

/* Coefficients C^s_k for n seeds before the transform: device buffer
 * C[n][2][n_kappa][n_omega] of interleaved (re, im) floats or doubles per
 * the plan's precision.  Async. */
int srm3_coeffs(srm3_plan *plan, const uint64_t *seeds, int n, void *C);

/* The transform stage alone: u = Re sum_s sum_k C^s_k e^{i(...)} for n
 * coefficient sets laid out as srm3_coeffs writes them (device), into a
 * device buffer u[n][n_x][n_t].  Async. */
int srm3_field_from_coeffs(srm3_plan *plan, const void *C, int n, void *out);

/* Capacity of the fixed scratch behind srm3_field_from_coeffs_noalloc:
 * 16 MiB per device.  The array is part of the library's device code, so
 * these 16 MiB are held on every device where any srm3 kernel has been
 * loaded, whether or not the no-allocation entry point is ever called, and
 * stay held until the process exits. */
#define SRM3_NOALLOC_SCRATCH_BYTES (16u << 20)

/* srm3_field_from_coeffs that allocates no device memory.  The paper has no
 * counterpart: this is a library service, not part of the method.
 *
 * Who needs it: a caller that may not allocate device memory while it
 * computes fields.  Two common cases:
 *  - a process whose device memory is already held by another allocator
 *    (for instance a framework's caching allocator that reserved most of
 *    HBM), where a fresh cudaMalloc can fail in the middle of a request;
 *  - a latency-bound serving loop: cudaMalloc and cudaFree can synchronise
 *    the device and stall other streams, which shows up as tail latency.
 * srm3_field_from_coeffs grows the plan's workspace with cudaMalloc on first
 * use (and when n grows); this entry point never calls cudaMalloc,
 * cudaMallocAsync, cudaFree or any other allocating routine.  It neither
 * uses nor grows the plan's workspace.
 *
 * Arguments, layouts and result are those of srm3_field_from_coeffs: C is a
 * device buffer C[n][2][n_kappa][n_omega] of interleaved (re, im) values in
 * the plan's precision; out is a device buffer u[n][n_x][n_t].  The launch
 * sequence is the one srm3_field_from_coeffs runs, with the scratch in
 * place of the workspace, and each set is transformed independently of the
 * others, so the values are bit-identical to srm3_field_from_coeffs.
 * Asynchronous on the plan's stream.
 *
 * Scratch: the intermediate of the two FFT stages, n_x * n_omega complex
 * values per coefficient set (8 bytes each in FP32, 16 in FP64), lives in a
 * fixed array of SRM3_NOALLOC_SCRATCH_BYTES that the library defines in
 * device memory, one per device.  Sets are transformed in groups that fit.
 * Nothing in it needs to start at zero: the first stage writes every entry
 * that the second stage reads.
 *
 * Set-up: the first call on each device looks up the array's address
 * (cudaGetSymbolAddress, with the plan's device current), which can load
 * the library's device code onto that device; later calls reuse the cached
 * address.  Make that first call before any stream capture begins.  The
 * cached address lives as long as the process: after a cudaDeviceReset (or
 * any other reset of the device's primary context) it is stale, so do not
 * call this entry point on a device that has been reset.  The plan's device
 * is made current for the call and the previous current device is restored
 * before return.
 *
 * Concurrency: the array is shared by every plan and stream on a device.
 * Calls whose work overlaps on one device (on different streams, or from
 * host threads that do not order their calls) race on it and produce wrong
 * fields.  Calls issued one after another on the same stream are safe.
 *
 * Errors: SRM3_ERR_INVALID_ARG for a NULL plan, n < 0, NULL buffers with
 * n > 0, or a plan whose one coefficient set needs more scratch than
 * SRM3_NOALLOC_SCRATCH_BYTES (n_x * n_omega * 8 bytes in FP32, * 16 in FP64);
 * SRM3_ERR_CUDA when the address lookup or a launch fails.  The message is
 * in srm3_last_error(). */
int srm3_field_from_coeffs_noalloc(srm3_plan *plan, const void *C, int n, void *out);

/* Stage timings from CUDA events recorded on the plan's stream.  The
 * recursion and W-table figures cover the last plan build (always
 * recorded); the sampling stages accumulate over srm3_sample /
 * srm3_sample_host / srm3_coeffs calls made while timing is enabled. */
typedef struct srm3_timings {
    double recursion_ms;   /* sum over all recursion passes of the build */
    double table_ms;       /* W-table build */
    double phases_ms;      /* Philox phase kernels */
    double pairsum_ms;     /* pair-sum kernels (the dominant stage) */
    double transform_ms;   /* both FFT stages */
    int32_t recursion_passes;
    int32_t pairsum_launches;
    int64_t pair_terms;    /* pair-terms issued by the timed pair-sum launches */
    double recursion_fp32_ms;  /* part of recursion_ms spent in FP32 search passes */
    double recursion_fp64_ms;  /* part of recursion_ms spent in FP64 passes */
    int32_t recursion_passes_fp32;
    int32_t recursion_passes_coarse; /* FP32 passes of the coarse eps search */
    double coarse_ms;      /* the coarse eps search, its tables included (its
                              passes are also part of recursion_ms) */
} srm3_timings;

/* on != 0: bracket every sampling-stage launch with CUDA events. */
int srm3_enable_timing(srm3_plan *plan, int on);

/* Wait for the plan's stream, then report the timings; reset != 0 clears
 * the sampling-stage sums afterwards. */
int srm3_get_timings(srm3_plan *plan, srm3_timings *t, int reset);

/* ---- Autotuning (FP32 plans) ---------------------------------------------
 * The FP32 pair sum can read W from the stored table or rebuild it from the
 * envelope factors, and its work unit can be 32 outputs wide (four compute
 * warps) or 16 (two: less idle work in the last chunks of every row pair,
 * which matters on short rows); which is fastest depends on the lattice and
 * the number of samples.  srm3_autotune times one pair-sum launch of every
 * (storage, tile) on this plan for n samples (the phases of seeds 1..n, in
 * the plan's workspace), keeps the fastest -- building the W table when a
 * table form wins and the plan has none (if it fits the plan's table
 * budget), freeing it when recomputation wins -- and records the choice for
 * the plan's (n_kappa, n_omega) in this process: plans created later with
 * that lattice take the tile (the coefficients do not depend on it), and
 * those created with SRM3_STORAGE_TUNED the storage too.  Synchronous.
 * Errors: INVALID_ARG (n outside 1..128), NOT_SUPPORTED (FP64 plan, mixed
 * or separable plan), OUT_OF_MEMORY, CUDA. */
typedef struct srm3_tune_result {
    double table_ms;      /* fastest launch with the stored table; < 0: not tried */
    double recompute_ms;  /* fastest launch with W rebuilt in the kernel */
    int32_t storage;      /* the choice: SRM3_STORAGE_TABLE or SRM3_STORAGE_RECOMPUTE */
    int32_t samples;      /* n */
    int32_t tile_width;   /* the choice of tile: 32 or 16 outputs per work unit */
    int32_t reserved;
    double table_ms_w32, table_ms_w16;         /* each (storage, tile) timed; < 0: */
    double recompute_ms_w32, recompute_ms_w16; /* not tried */
} srm3_tune_result;
int srm3_autotune(srm3_plan *plan, int n, srm3_tune_result *result);

/* Set the FP32 pair sum's work unit of this plan to 32 or 16 outputs (what
 * srm3_autotune would choose, set by hand).  The coefficients are the same
 * bit for bit either way: each output's sums and their order do not depend
 * on the unit.  Takes effect at the next sampling call or batch creation.
 * Errors: INVALID_ARG (width not 16 or 32), NOT_SUPPORTED (FP64 or
 * separable plan). */
int srm3_set_tile_width(srm3_plan *plan, int width);

/* ---- Batches of plans ------------------------------------------------------
 * One sampling job over m plans with uneven lattices and sample counts: the
 * phases of every plan, ONE persistent pair-sum launch over the work units
 * of all FP32 plans (cost-sorted across plans, in the tile width of the
 * plans that carry most of the pair-terms; FP64 plans get their own plain
 * launches), then the transforms, all on one stream.  FP32 plans of the plain pair set that share a lattice shape
 * (n_kappa, n_omega, n_x, n_t, cutoffs, envelope width, biphase), a storage
 * (W recomputed, or a stored W table: the table holds the pair envelopes
 * alone, a function of the shape) and a tile width form a shape group: their
 * samples share the lanes of the pair sum -- the weights depend only on the
 * shape, each sample keeps its own pure and pair factors -- so many spectra
 * with one or a few samples each still fill the kernel; a group uses buffers
 * of the batch, not the plans' workspaces, and the first plan's weights.  srm3_batch_create checks the plans
 * (one device, no plan twice), allocates the group buffers and sizes the
 * other plans' workspaces for their counts, and puts the descriptors and
 * the unit list on the device (at most 4096 samples per shape group).  counts[i] in 1..128;
 * outs[i]: device buffer u[counts[i]][n_x][n_t] in plan i's precision;
 * stream: cudaStream_t, NULL = a stream of the batch's own.  While the batch
 * exists the workspaces of the plans outside shape groups belong to it: they
 * may not grow (srm3_sample with more samples than the batch gave such a
 * plan fails with NOT_SUPPORTED), and sampling from such a plan while a
 * batch run may be in flight races.  The
 * plans must outlive the batch.  Errors: INVALID_ARG, NOT_SUPPORTED,
 * OUT_OF_MEMORY, CUDA. */
typedef struct srm3_batch srm3_batch;
int srm3_batch_create(srm3_plan *const *plans, const int32_t *counts, void *const *outs, int m,
                      void *stream, srm3_batch **out);

/* Run the batch for seeds[sum of counts] (host; plan 0's seeds first, then
 * plan 1's, ...), read before the call returns; they are copied into a
 * device buffer that the phase kernels read.  The batch's own buffers are
 * stream-ordered allocations on its stream: creating or destroying a batch
 * does not wait for work on other streams.  After srm3_batch_capture the
 * launch sequence is the captured graph.  Asynchronous on the batch stream.
 * A sample's field is bit-identical to srm3_sample of the same plan and seed. */
int srm3_batch_run(srm3_batch *b, const uint64_t *seeds);

/* Capture the batch's launch sequence (phases, pair sums, transforms) into a
 * CUDA graph by stream capture on the batch stream, and replay that graph in
 * later srm3_batch_run calls.  Nothing is allocated during the capture. */
int srm3_batch_capture(srm3_batch *b);

/* Wait for the batch stream; returns the first asynchronous error. */
int srm3_batch_sync(srm3_batch *b);

/* Pair-terms of one run: sum over plans of 2 |Pi| counts[i]. */
int64_t srm3_batch_pair_terms(const srm3_batch *b);

/* Device memory the batch allocated for itself (released by
 * srm3_batch_destroy): per shape group with T samples in all, at most m of
 * them from one plan, on an n_kappa x n_omega lattice with n_t-point rows,
 * y + y0 = (n_kappa (n_omega + 128) + 1) P 8 bytes (P = 2 T sheet-samples
 * rounded up to a multiple of 64), C = 2 T n_kappa n_omega 8, H = m n_kappa
 * n_t 8 and 16 T of factor pointers; plus 8 bytes of seed per sample, the
 * plan descriptors and 16 bytes per work unit.  Plans outside shape groups
 * sample on their own workspace, which their srm3_info.device_bytes counts;
 * the caller's output buffers are not included. */
int64_t srm3_batch_device_bytes(const srm3_batch *b);

/* Cap the batch's FP32 pair-sum launch at max_ctas CTAs (0: as many as are
 * resident, the default).  The launch is persistent and otherwise fills
 * every SM; a cap leaves room for work on other streams to run beside it
 * (a serving loop keeps short requests moving this way).  Set it before
 * srm3_batch_capture for graph replays. */
int srm3_batch_set_max_ctas(srm3_batch *b, int max_ctas);

/* on != 0: record CUDA events around the batch's FP32 pair-sum launch in
 * later runs (set it before srm3_batch_capture for graph replays: the
 * events become event-record nodes of the graph). */
int srm3_batch_enable_timing(srm3_batch *b, int on);

/* Duration of the pair-sum launch of the last run, in ms (waits for it);
 * 0 when timing is off or the batch has no FP32 plan. */
int srm3_batch_pairsum_ms(srm3_batch *b, double *ms);

/* Free the batch (not its plans).  NULL is a no-op.  No run may be in flight. */
void srm3_batch_destroy(srm3_batch *b);

/* ---------------------------------------------------------------------------
 * Ensemble statistics of sampled fields (Sec. 6: sample mean, variance and
 * skewness of the simulated waves against their targets, and the empirical
 * PDF and CDF).  A running accumulator on the device, fed with any number of
 * sampled batches (srm3_sample output, or any device array), read at the end:
 *   power sums  sum (u - shift)^p, p = 1..4, in FP64 (FP32 input is summed
 *               in FP32 over runs of 16 values, then in FP64);
 *   histogram   nbins equal bins over [lo, hi): bin floor((u - lo) *
 *               (nbins / (hi - lo))), evaluated in the input's precision
 *               with each operation rounded once; values below lo and at or
 *               above hi (or NaN) are counted apart.
 * Deterministic: the same values given in the same calls give bit-identical
 * sums and counts on a given device.  Calls on one accumulator must not run
 * concurrently (one stream, or ordered streams).
 * ------------------------------------------------------------------------- */
#define SRM3_STATS_MAX_BINS 16384

typedef struct srm3_stats srm3_stats;

typedef struct srm3_stats_result {
    double count;          /* values accumulated */
    double power_sum[4];   /* sum (u - shift)^p, p = 1..4 */
    double mean;           /* shift + power_sum[0] / count */
    double variance;       /* population central moments from the power sums */
    double skewness;       /* c3 / c2^1.5 (0 when c2 = 0) */
    double kurtosis;       /* c4 / c2^2 (0 when c2 = 0) */
    uint64_t below, above; /* values outside [lo, hi) */
} srm3_stats_result;

/* New accumulator on the current device (zeroed).  1 <= nbins <=
 * SRM3_STATS_MAX_BINS, finite lo < hi, finite shift (a value near the mean
 * keeps the power sums well conditioned; 0 for zero-mean waves). */
int srm3_stats_create(int32_t nbins, double lo, double hi, double shift, srm3_stats **out);

/* Add count values of the device array u (16-byte aligned; float when
 * precision == SRM3_FP32, double when SRM3_FP64).  Asynchronous on stream
 * (a cudaStream_t; NULL = the legacy default stream).  count == 0 is a
 * no-op. */
int srm3_stats_add(srm3_stats *s, const void *u, int32_t precision, int64_t count, void *stream);

/* Wait for stream and read the running results; hist (host, nbins entries,
 * may be NULL) receives the bin counts. */
int srm3_stats_read(srm3_stats *s, void *stream, srm3_stats_result *r, uint64_t *hist);

/* Zero the accumulator (asynchronous on stream). */
int srm3_stats_reset(srm3_stats *s, void *stream);

/* Free the accumulator.  NULL is a no-op.  No call may be in flight. */
void srm3_stats_destroy(srm3_stats *s);

#ifdef __cplusplus
}
#endif

#endif /* SRM3_H */
