// srm3_internal.cuh - plan object, error plumbing and shared device helpers of
// the SRM3 sampler.  Not part of the public ABI (include/srm3.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "srm3.h"

#define SRM3_API extern "C" __attribute__((visibility("default")))

namespace srm3 {

// The complex pair type of a precision.
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

// Tile shape of the FP32 pair sum: R outputs along omega per thread; the W
// table rows of a tile are padded to a multiple of kTileU (the pair sum's
// omega chunk) and stored chunk-major: entry (a, r, iw) of a tile at
// ((a nch + iw / kTileU) kTileR + r) kTileU + iw % kTileU, nch = L / kTileU,
// so that the kTileR rows of one chunk are one contiguous 512-byte span.
// The y rows carry
// kPad zero entries on both sides: every row the FP32 pair sum stages lies
// within omega index [-31, nw + 30], so its copies need no bounds checks.
constexpr int kTileR = 8;
constexpr int kTileU = 16;
constexpr int kPad = 64;
constexpr int kMaxChunk = 128;     // samples per internal launch chunk
constexpr int kWarpsPerCta = 4;    // FP32 pair-sum CTA: 4 warps = 4 work units
constexpr int kMaxFft = 8192;

struct SeedChunk {
  uint64_t s[kMaxChunk];
};

void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);
// Device memory of plans and their workspaces: stream-ordered allocations
// from the device's default memory pool, whose release threshold is raised
// on first use (to 32 GB) so that freed memory stays in the pool -- building
// and freeing plans back to back then maps no pages.  dev_free returns a
// block to the pool in the order of stream st.
cudaError_t dev_alloc(void **ptr, size_t bytes, cudaStream_t st);
template <typename T>
cudaError_t dev_alloc(T **ptr, size_t bytes, cudaStream_t st) {
  return dev_alloc(reinterpret_cast<void **>(ptr), bytes, st);
}
cudaError_t dev_free(void *ptr, cudaStream_t st);
// Device memory held by a plan: blocks from dev_alloc made while an
// AllocOwner of the plan is in scope (on this thread) are charged to its
// dev_bytes, and dev_free of such a block gives the bytes back.
struct AllocOwner {
  explicit AllocOwner(srm3_plan *p);
  ~AllocOwner();
  srm3_plan *prev;
};
// Grid-barrier timeout self-test (plan.cu): *timed_out = the abort word.
int selftest_barrier(long long polls, int *timed_out);

#define SRM3_CUDA(call)                                 \
  do {                                                  \
    cudaError_t e__ = (call);                           \
    if (e__ != cudaSuccess) return cuda_fail(e__, #call); \
  } while (0)

}  // namespace srm3

struct srm3_plan {
  // lattice and grid
  int nk = 0, nw = 0, nx = 0, nt = 0;
  int log2nx = 0, log2nt = 0;
  double ku = 0, wu = 0, dk = 0, dw = 0, dkdw = 0;
  int row_lo = 0, row_hi = 0;  // lattice rows whose coefficients the plan computes
  double dev_bytes = 0.0;       // device memory the plan holds (see AllocOwner)
  int precision = SRM3_FP32;
  int storage = SRM3_STORAGE_RECOMPUTE;
  cudaStream_t stream = nullptr;
  int device = 0;

  // model
  double sigma_g = 0.25, beta = 0.0;
  // separable envelope g(i,j) = e(i) e(j) e(i+j): the recursion keeps
  // h = e^2 q for its pair sums (G2 = 1) and sampling is an FFT convolution
  bool sep = false;
  double *env_e = nullptr, *env_e2 = nullptr;  // a and a^2 per lattice point
  float *env_e32 = nullptr;                     // a in FP32
  // b and b^2 (g = a(i) a(j) b(i+j)); the a tables when b = a
  double *env_b = nullptr, *env_b2 = nullptr;
  float *env_b32 = nullptr;
  bool sep_b = false;                           // b has tables of its own
  double *qh = nullptr;                         // h = e^2 q of the FP64 passes
  // the recursion in separable form: the separable kind, or the Gaussian
  // envelope split on i + j = k (a^2 per point in rs_a2, b^2 in rs_b2)
  bool rec_sep = false;
  double *rs_a2 = nullptr, *rs_b2 = nullptr;
  // FFT self-convolution grid of the separable pair sum (powers of two,
  // cNk >= 2 nk - 1, cNw >= 2 nw - 1), its twiddles e^{+2 pi i j / ntwc},
  // and the workspace of zc_ss sheet-samples (complex, plan precision)
  int cNk = 0, cNw = 0, log2cNk = 0, log2cNw = 0;
  void *tw_conv = nullptr;
  void *Zc = nullptr;
  long long zc_ss = 0;
  // mixed-sign interactions: opposite-sheet pairs as well; Eq. pure then
  // a fixed point solved by iterations of (difference sums at the previous
  // iterate, level pass)
  bool mixed = false;
  int64_t diffpairs = 0;          // difference pairs of one sheet
  int fp_iters = 0;               // iterations of the last fixed-point solve
  double *Dsum = nullptr;         // difference-pair sums per point [nk*nw]
  double *dsb2 = nullptr;         // d sum_b2 / dx per point from two FP32 search planes
  double *red_part = nullptr;     // per-CTA partials of the plane reduction
  bool eps_shifted = false;       // the final tables are an FP64 pass moved to eps to first order
  bool eps_interp = false;        // ... or interpolated to eps from an FP64 pass at three eps values
  double *qo3 = nullptr;          // q of the three-plane FP64 pass, separable form ([3][nl])
  // eps search from the root on a coarser lattice (every coarse_fk-th kappa,
  // coarse_fw-th omega point): its kernels, passes and time; coarse_start
  // when one pass on this lattice then bracketed the root
  bool coarse_start = false;
  int coarse_fk = 1, coarse_fw = 1, coarse_launches = 0, coarse_passes = 0;
  double t_coarse_ms = 0.0;
  int n_launch = 0;               // recursion-stage kernels launched (counted where launched)
  double *qprev = nullptr;        // previous iterate of q
  double *qlo = nullptr;          // converged q at qlo_x (warm start of the search)
  double qlo_x = -1.0;
  unsigned long long *fp_change = nullptr;  // max relative change of q (bits)
  void *Ewd = nullptr;            // FP32 envelope of the difference d >= 0, [ewd_len]
  int ewd_len = 0;
  void *ys = nullptr;             // FP32: y with the two sheets of each lane swapped
  int nsuper_d = 0;
  int2 *super_order_d = nullptr;  // super-tiles by decreasing difference-pair cost
  double eps = 0.0, max_sb2 = 0.0, min_pure = 1.0, variance = 0.0;
  double plan_ms = 0.0, table_bytes = 0.0, table_budget = 0.0;
  int root_passes = 0;    // FP64 recursion passes
  int root_passes32 = 0;  // FP32 recursion passes (eps search)
  int64_t pairs = 0;

  // FP64 plan tables [nk*nw]
  double *S = nullptr;    // spectrum on the lattice
  double *qm = nullptr;   // q = S/S_p where S > 0, else 0
  double *sb2 = nullptr;  // sum_{Pi(k)} b_p^2
  double *EkSq = nullptr; // squared envelope factor along kappa, |d| < nk
  double *EwSq = nullptr; // squared envelope factor along omega, |d| < nw
  double *scal = nullptr; // device scalars: [0] eps^2 dk dw, [1] max sb2,
                          // [2] min (1 - sb2) over S > 0, [3] sum S
  int *err = nullptr;     // device error word
  float *qm32 = nullptr;  // FP32 recursion state for the eps search passes
  float *EkSq32 = nullptr, *EwSq32 = nullptr;
  double *qm3 = nullptr;  // three-plane FP64 recursion state [k][3] (eps search)
  double *G2 = nullptr;   // g^2 table [nk][nw] over (|ik-jk|, |iw-jw|), FP64
  float *G2_32 = nullptr; // the same in FP32 (search passes)
  int2 *rec_items = nullptr;         // (kk, row chunk) work items of all levels
  double *rec_partial = nullptr;     // per-level chunk sums [point slot][chunk]
  int maxch = 0;

  // per-precision sampling tables (float or double by precision)
  void *sqq = nullptr;    // sqrt(q) masked by S > 0, [nk*nw]
  void *Pk = nullptr;     // pure factor 2 sqrt(dk dw S) (1 - sb2), [nk*nw]
  void *ck = nullptr;     // pair factor 2 eps dk dw sqrt(S), [nk*nw]
  // the FP32 pair sum in separable form (Gaussian envelope, W recomputed):
  // g(i, j) = a_i a_j b_k on the pairs of k, the omega factor a_w folded
  // into y (sqq_s = sqrt(q) a_w), the kappa factor a_k per lattice row
  // (aK, applied per row pair), b_k into the pair factor (ck_s = ck b_k) and
  // 1/a_w into the pure factor (Pk_s = Pk / a_w); FP32, [nk*nw] (aK [nk])
  float *sqq_s = nullptr, *Pk_s = nullptr, *ck_s = nullptr, *aK = nullptr;
  void *Ek = nullptr;     // envelope factor along kappa, |d| < nk
  void *Ews = nullptr;    // envelope factor along omega, signed d, offset ew_off
  int ew_off = 0, ew_len = 0;
  void *tw = nullptr;     // output-transform twiddles: pass tables of lengths nx and
                          // nt / 2, then e^{2 pi i m / nt}, m < nt / 2

  // FP32 tiled pair sum: tiles (kk, kw0) in decreasing-cost order
  int ntw = 0, ntiles = 0;
  long long table_entries = 0;    // floats of the W table (built or not)
  int ps_ctas[2] = {0, 0};        // resident CTAs of the persistent FP32 pair sum, per tile shape
  int ps_nc = 4;                  // compute warps of the FP32 pair-sum tile: 4 (32 wide) or 2 (16)
  int *ps_err = nullptr;          // its error word (bounded waits that ran out)
  // super-tiles of the FP32 pair sum by decreasing cost, per tile shape
  // (index 0: 32 wide, 4 compute warps; 1: 16 wide, 2 compute warps), on the
  // device and on the host (batch unit lists)
  int nsuper[2] = {0, 0};
  int2 *super_order[2] = {nullptr, nullptr};
  std::vector<int2> super_host[2];
  long long *tile_off = nullptr;  // W-table offset per tile id (kk*ntw + tw)
  float *W = nullptr;             // W table (STORAGE_TABLE): the pair envelopes of the shape
  cudaEvent_t w_ev[2] = {nullptr, nullptr};  // around its build while it runs
  // the W build's stream during plan creation, and whether the build is still
  // to be launched (it starts right after the first FP64 recursion pass, beside it)
  cudaStream_t w_stream = nullptr;
  bool w_deferred = false;

  // sampling workspace
  int ws_chunk = 0;
  int batch_refs = 0;             // batches holding this workspace (it may not grow)
  void *y = nullptr, *y0 = nullptr, *C = nullptr, *H = nullptr;
  int rowstride = 0;

  // stage timing (CUDA events on the plan stream)
  bool timing = false;
  struct EvRec {
    int stage;  // 0 phases, 1 pairsum, 2 transform
    cudaEvent_t a, b;
    long long pair_terms;
  };
  std::vector<EvRec> ev_recs;
  std::vector<cudaEvent_t> ev_pool;
  double t_recursion_ms = 0.0, t_table_ms = 0.0;
  double t_rec32_ms = 0.0, t_rec64_ms = 0.0;
  double t_stage_ms[3] = {0.0, 0.0, 0.0};
  int t_pairsum_launches = 0;
  long long t_pair_terms = 0;

  // recursion graph (one pass = every anti-diagonal level + reductions)
  // persistent recursion pass
  int *rec_lev_off = nullptr;        // first item of each level
  int2 *rec_pairs = nullptr;         // bulk point pairs of every phase
  int *rec_pair_off = nullptr;       // first pair of each bulk phase
  unsigned int *rec_bar = nullptr;   // grid barrier counter and bulk-phase tickets
  int rec_bar_words = 0, rec_bar_tickets = 0;
  unsigned long long *rec_max = nullptr;  // per-plane max sum_b2 of a pass (bits)
  double sumS = 0.0;                      // sum of S over the lattice
  // separable envelope: the bulk of a pass as an online FFT self-convolution
  // (rec_fft), its product grid (room for kPlanes FP32 planes or one FP64
  // plane of 2 Lmax x Nc complex values) and packed twiddles in both
  // precisions
  bool rec_fft = false;
  int rec_log2Nc = 0;
  void *rec_z = nullptr, *tw_rec32 = nullptr, *tw_rec64 = nullptr;
  int maxpts = 0, rec_grid64 = 0, rec_grid32 = 0;
  double *h_pinned = nullptr;  // pinned host scalars
  int *h_err = nullptr;        // pinned host error words
};

namespace srm3 {
// plan.cu
int build_plan(srm3_plan *p, const srm3_spectrum *sp, const srm3_bispectrum *bs);
void free_plan(srm3_plan *p);
// sample.cu
int ensure_workspace(srm3_plan *p, int chunk);
int run_phases(srm3_plan *p, const uint64_t *seeds, int n, uint32_t *words_out);
int run_pairsum(srm3_plan *p, int n, void *C_out);
int run_transform(srm3_plan *p, const void *C, int n, void *out);
// The two FFT stages for n coefficient sets on stream st with the x-stage
// columns in H (n * transform_elems(p) complex values in the plan's
// precision), which the caller supplies: the plan workspace, a batch buffer
// or fixed scratch.
int transform_on(srm3_plan *p, cudaStream_t st, const void *C, int n, void *out, void *H);
// Complex values of the transform's intermediate per coefficient set: the
// x-stage output G[nx][nw].
inline size_t transform_elems(const srm3_plan *p) { return (size_t)p->nx * p->nw; }
int prepare_shape_tables(srm3_plan *p, cudaStream_t st);
int prepare_sampling_tables(srm3_plan *p, cudaStream_t st);
int stage_begin(srm3_plan *p, int stage, long long pair_terms, int *rec);
int stage_end(srm3_plan *p, int rec);
int collect_timings(srm3_plan *p);
int check_pairsum_error(srm3_plan *p);
int sspad_for(int chunk);
// The separable pair sum (FFT self-convolution, conv.cu) of n samples whose
// phasor rows y / y0 are laid out for sspad_for(n), on stream st.
int conv_pairsum_on(srm3_plan *p, cudaStream_t st, int n, const void *y, const void *y0,
                    void *C_out);
int build_w_table(srm3_plan *p, cudaStream_t st);
// autotuner choices per lattice shape (process-wide): storage (or -1 when
// the shape was never tuned) and the pair-sum tile's compute warps
int tune_cache_lookup(int nk, int nw, int *nc = nullptr);
void tune_cache_store(int nk, int nw, int storage, int nc);
// tile-shape index of nc compute warps (4 -> 0, 2 -> 1)
inline int tile_index(int nc) { return nc == 4 ? 0 : 1; }
}  // namespace srm3

static inline int ilog2_exact(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return ((1 << l) == v) ? l : -1;
}

// The FP32 pair sum may take the separable form (plan tables sqq_s, Pk_s,
// ck_s, aK): a Gaussian envelope whose factors' exponent range fits (the
// recursion's separable form), sum interactions only; it does take it while
// the plan's W is recomputed.
inline bool pairsum_sep_capable(const srm3_plan *p) {
  return p->precision == SRM3_FP32 && p->rec_sep && !p->sep && !p->mixed;
}
inline bool pairsum_sep_now(const srm3_plan *p) {
  return pairsum_sep_capable(p) && p->sqq_s && p->storage == SRM3_STORAGE_RECOMPUTE;
}
