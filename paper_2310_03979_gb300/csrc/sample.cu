// sample.cu - per-sample work of the SRM3 sampler: Philox4x32-10 phases,
// the O(N^2) pair sum that assembles the coefficients C^s_k (FFT form,
// Sec. 4.3), and the hand-written 2-D inverse FFT to u(x,t).
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <type_traits>

#include <cudaTypedefs.h>  // PFN_cuTensorMapEncodeTiled

#include "fft.cuh"
#include "pairsum.cuh"
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
// y[kk][kPad + kw][ss], ss = ss_off + 2 n + s, except that y at k = 0 goes to y0[ss]
// and the lattice slot of k = 0 holds 0 (it takes part in no pair).  With
// words != NULL writes the raw words[n][2][nk][nw] instead.  FP32 mixed
// plans (ys != NULL) also get ys, the same rows with the two sheets of each
// sample swapped in its lane ({x-, x+, y-, y+}) and the omega = 0 column
// zero: the partners of the difference pairs, which never sit at omega = 0.
template <typename T>
__global__ void k_phases(int nk, int nw, int nsamp, SeedChunk seeds,
                         const uint64_t *__restrict__ dseeds, int ss_off,
                         const T *__restrict__ sqq, typename Vec2<T>::type *__restrict__ y,
                         typename Vec2<T>::type *__restrict__ y0, int SSpad, int rowstride,
                         uint32_t *__restrict__ words, float *__restrict__ ys) {
  using T2 = typename Vec2<T>::type;
  const long long nl = (long long)nk * nw;
  const long long nc = (2 * nl + 3) / 4;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= nc * nsamp) return;
  const int n = (int)(gid % nsamp);
  const long long c = gid / nsamp;
  const uint64_t seed = dseeds ? dseeds[n] : seeds.s[n];
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
    int ss = ss_off + 2 * n + s;
    if (r == 0) {
      y0[ss] = v;
      v.x = 0;
      v.y = 0;
    }
    const size_t row = (size_t)kk * rowstride + kPad + kw;
    if constexpr (sizeof(T) == sizeof(float)) {
      // FP32: pair-planar {x_{2l}, x_{2l+1}, y_{2l}, y_{2l+1}} per sample pair l
      float *yf = reinterpret_cast<float *>(y) + (row * (SSpad / 2) + (ss >> 1)) * 4 + (ss & 1);
      yf[0] = v.x;
      yf[2] = v.y;
      if (ys) {
        float *sf = ys + (row * (SSpad / 2) + (ss >> 1)) * 4 + (1 - (ss & 1));
        sf[0] = kw == 0 ? 0.0f : (float)v.x;
        sf[2] = kw == 0 ? 0.0f : (float)v.y;
      }
    } else {
      y[row * SSpad + ss] = v;
    }
  }
}

// ---------------------------------------------------------------------------
static size_t elem2(const srm3_plan *p) {
  return p->precision == SRM3_FP32 ? sizeof(float2) : sizeof(double2);
}

// sheet-samples per lattice entry, padded to whole 64-wide groups of the
// FP32 pair sum
int sspad_for(int chunk) { return ((2 * chunk + 63) / 64) * 64; }

int ensure_workspace(srm3_plan *p, int chunk) {
  if (p->ws_chunk >= chunk) return SRM3_OK;
  AllocOwner owner(p);
  if (p->batch_refs > 0)
    return fail(SRM3_ERR_NOT_SUPPORTED,
                "the plan's workspace belongs to a batch and cannot grow while the batch exists");
  int cap = std::max(chunk, std::min(kMaxChunk, 64));
  for (void **q : {&p->y, &p->y0, &p->C, &p->H, &p->ys}) {
    if (*q) dev_free(*q, p->stream);
    *q = nullptr;
  }
  p->ws_chunk = 0;
  const size_t e2 = elem2(p);
  p->rowstride = p->nw + 2 * kPad;
  const int sp = sspad_for(cap);
  SRM3_CUDA(dev_alloc(&p->y, (size_t)p->nk * p->rowstride * sp * e2, p->stream));
  SRM3_CUDA(dev_alloc(&p->y0, (size_t)sp * e2, p->stream));
  SRM3_CUDA(dev_alloc(&p->C, (size_t)2 * cap * p->nk * p->nw * e2, p->stream));
  SRM3_CUDA(dev_alloc(&p->H, (size_t)cap * transform_elems(p) * e2, p->stream));
  if (p->mixed && p->precision == SRM3_FP32)
    SRM3_CUDA(dev_alloc(&p->ys, (size_t)p->nk * p->rowstride * sp * e2, p->stream));
  if (p->sep) {  // the self-convolution grid's n_kappa rows, every sheet-sample of a chunk
    if (p->Zc) dev_free(p->Zc, p->stream);
    p->Zc = nullptr;
    SRM3_CUDA(dev_alloc(&p->Zc, (size_t)2 * cap * p->nk * p->cNw * e2, p->stream));
    p->zc_ss = 2LL * cap;
  }
  // stream-ordered blocks: usable from any stream (batches) once this passes
  SRM3_CUDA(cudaStreamSynchronize(p->stream));
  p->ws_chunk = cap;
  return SRM3_OK;
}

// Phases of n samples of plan p on stream st into y / y0 laid out for sp
// sheet-samples per lattice entry, from sheet-sample ss_off on; seeds from
// the host array `seeds` (passed by value) or, when dseeds != NULL, from
// device memory.  The zero padding of y is the caller's.
static int phases_into(srm3_plan *p, cudaStream_t st, const uint64_t *seeds,
                       const uint64_t *dseeds, int n, void *y, void *y0, int sp, int ss_off,
                       uint32_t *words_out) {
  SeedChunk sc;
  std::memset(&sc, 0, sizeof(sc));
  if (!dseeds && seeds) std::memcpy(sc.s, seeds, sizeof(uint64_t) * n);
  const long long nl = (long long)p->nk * p->nw;
  const long long nc = (2 * nl + 3) / 4;
  const int blocks = cdiv(nc * n, 256);
  // the swapped copy of the mixed FP32 pair sum (plan workspace only)
  float *ys = (p->mixed && p->precision == SRM3_FP32 && y == p->y) ? (float *)p->ys : nullptr;
  // the separable pair sum takes the rows with the omega factor folded in
  // (not the raw Philox words, which do not depend on the table)
  const float *sq32 = pairsum_sep_now(p) ? p->sqq_s : (const float *)p->sqq;
  if (p->precision == SRM3_FP32)
    k_phases<float><<<blocks, 256, 0, st>>>(p->nk, p->nw, n, sc, dseeds, ss_off, sq32,
                                            (float2 *)y, (float2 *)y0, sp, p->rowstride,
                                            words_out, ys);
  else
    k_phases<double><<<blocks, 256, 0, st>>>(p->nk, p->nw, n, sc, dseeds, ss_off,
                                             (const double *)p->sqq, (double2 *)y,
                                             (double2 *)y0, sp, p->rowstride, words_out,
                                             nullptr);
  SRM3_CUDA(cudaGetLastError());
  return SRM3_OK;
}

// Phases of n samples into the plan's own workspace (zeroed first).
static int phases_on(srm3_plan *p, cudaStream_t st, const uint64_t *seeds,
                     const uint64_t *dseeds, int n, uint32_t *words_out) {
  const int sp = sspad_for(n);
  if (!words_out) {
    SRM3_CUDA(cudaMemsetAsync(p->y, 0, (size_t)p->nk * p->rowstride * sp * elem2(p), st));
    if (p->ys)
      SRM3_CUDA(cudaMemsetAsync(p->ys, 0, (size_t)p->nk * p->rowstride * sp * elem2(p), st));
  }
  return phases_into(p, st, seeds, dseeds, n, p->y, p->y0, sp, 0, words_out);
}

int run_phases(srm3_plan *p, const uint64_t *seeds, int n, uint32_t *words_out) {
  return phases_on(p, p->stream, seeds, nullptr, n, words_out);
}

// Descriptor of plan p for an FP32 pair-sum launch over n samples whose
// phasor rows are in p->y (laid out for n) and whose coefficients go to C_out.
static int fill_pairsum_desc_into(srm3_plan *p, int n, void *y, void *y0, void *C_out,
                                  PsDesc *d);
int fill_pairsum_desc(srm3_plan *p, int n, void *C_out, PsDesc *d) {
  return fill_pairsum_desc_into(p, n, p->y, p->y0, C_out, d);
}

// The driver's tensor-map encoder, looked up once.
static int tensor_map_encoder(PFN_cuTensorMapEncodeTiled_v12000 *out) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult qr;
    SRM3_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                               cudaEnableDefault, &qr));
    if (qr != cudaDriverEntryPointSuccess || !fn)
      return fail(SRM3_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }
  *out = encode;
  return SRM3_OK;
}

// The same for phasor rows y / y0 of n samples laid out for sspad_for(n).
static int fill_pairsum_desc_into(srm3_plan *p, int n, void *y, void *y0, void *C_out,
                                  PsDesc *d) {
  PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (int rc = tensor_map_encoder(&encode)) return rc;
  const int sp = sspad_for(n);
  std::memset(static_cast<void *>(d), 0, sizeof(*d));
  const bool table = p->storage == SRM3_STORAGE_TABLE;
  // at most 32 sheet-samples with W recomputed: half-group mode (two row
  // pairs per work item, one on each half-warp)
  const bool half = !table && 2 * n <= packed::LANES;
  // 2-D tensor map over y: rows of sp / 2 float4 (the sample pairs of one
  // lattice entry), boxes of one 64-sample group (512 bytes), or of its first
  // 32 sheet-samples (256 bytes) in half mode, x 16 rows
  const cuuint64_t dims[2] = {(cuuint64_t)sp * 2, (cuuint64_t)p->nk * p->rowstride};
  const cuuint64_t strides[1] = {(cuuint64_t)sp * 2 * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)packed::LANES * (half ? 2 : 4),
                             (cuuint32_t)packed::BOX_ROWS};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode(&d->ymap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, y, dims, strides,
                            box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    return fail(SRM3_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  d->y = (const float4 *)y;
  d->y0 = (const float2 *)y0;
  d->Ek = (const float *)p->Ek;
  d->Ew = (const float *)p->Ews;
  d->W = table ? p->W : nullptr;
  d->toff = table ? p->tile_off : nullptr;
  const bool sepf = pairsum_sep_now(p);
  d->Pk = sepf ? p->Pk_s : (const float *)p->Pk;
  d->ck = sepf ? p->ck_s : (const float *)p->ck;
  d->sep = sepf ? 1 : 0;
  d->aK = sepf ? p->aK : nullptr;
  d->C = (float2 *)C_out;
  d->order = p->super_order[tile_index(p->ps_nc)];
  d->nk = p->nk;
  d->nw = p->nw;
  d->SS = 2 * n;
  d->SSpad = sp;
  d->rowstride = p->rowstride;
  d->ntw = p->ntw;
  d->ew_off = p->ew_off;
  d->table = table ? 1 : 0;
  d->G = sp / (2 * packed::LANES);
  d->half = half ? 1 : 0;
  d->cb = (float)std::cos(p->beta);
  d->sb = (float)std::sin(p->beta);
  return SRM3_OK;
}

// One FP32 pair-sum launch on stream st: plan d0 alone (descs == NULL) or the
// batch descs/units, with the tile of nc compute warps (4 or 2); the grid is
// the resident CTA count (persistent kernel).  nunits == 0 only prepares
// (attributes, resident CTA count).
template <int NC>
static int launch_pairsum_f32_nc(srm3_plan *p, cudaStream_t st, const PsDesc &d0,
                                 const PsDesc *descs, const int4 *units, int nunits, int max_ctas,
                                 bool mixed, int form) {
  const size_t smem = pairsum_f32p_smem<NC>();
  constexpr int NT = packed::Shape<NC>::NT;
  // every instantiation: the general form and the separable form alone
  const void *kf[4] = {(const void *)k_pairsum_f32p<false, NC>,
                       (const void *)k_pairsum_f32p<true, NC>,
                       (const void *)k_pairsum_f32p<false, NC, kPsSeparable>,
                       (const void *)k_pairsum_f32p<true, NC, kPsSeparable>};
  for (const void *f : kf) {
    SRM3_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    SRM3_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  }
  int &ctas = p->ps_ctas[tile_index(NC)];
  if (ctas == 0) {  // resident CTAs of the persistent kernel (both forms)
    int nsm = 0, per_sm = 1 << 30;
    SRM3_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->device));
    for (const void *f : kf) {
      int n = 0;
      SRM3_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, NT, smem));
      per_sm = std::min(per_sm, n);
    }
    if (per_sm < 1) return fail(SRM3_ERR_NOT_SUPPORTED, "FP32 pair sum does not fit on an SM");
    ctas = nsm * per_sm;
  }
  int grid = std::min(nunits, ctas);
  if (max_ctas > 0) grid = std::min(grid, max_ctas);
  if (grid == 0) return SRM3_OK;
  if (form == kPsSeparable && mixed)
    k_pairsum_f32p<true, NC, kPsSeparable><<<grid, NT, smem, st>>>(d0, descs, units, nunits,
                                                                   p->ps_err);
  else if (form == kPsSeparable)
    k_pairsum_f32p<false, NC, kPsSeparable><<<grid, NT, smem, st>>>(d0, descs, units, nunits,
                                                                    p->ps_err);
  else if (mixed)
    k_pairsum_f32p<true, NC><<<grid, NT, smem, st>>>(d0, descs, units, nunits, p->ps_err);
  else
    k_pairsum_f32p<false, NC><<<grid, NT, smem, st>>>(d0, descs, units, nunits, p->ps_err);
  SRM3_CUDA(cudaGetLastError());
  return SRM3_OK;
}

// The instantiation for a descriptor's weight form: the separable form has
// one of its own (its register blocks alone: 166 registers and no spills
// against 168 and spills, 6 % faster on the bridge lattice); the stored
// table and the weighted recompute form take the general kernel (compiled
// for the table alone it spilled more and ran 0.3 % slower).
static int ps_form_of(const PsDesc &d) {
  return !d.table && d.sep ? kPsSeparable : kPsAnyForm;
}

// form: kPsSeparable when every descriptor of the launch has the separable
// weight form, else kPsAnyForm; -1: that of d0 for a single-plan launch
// (descs == NULL).
int launch_pairsum_f32(srm3_plan *p, cudaStream_t st, const PsDesc &d0, const PsDesc *descs,
                       const int4 *units, int nunits, int max_ctas, bool mixed, int nc,
                       int form = -1) {
  if (form < 0) form = descs ? kPsAnyForm : ps_form_of(d0);
  if (nc == 2)
    return launch_pairsum_f32_nc<2>(p, st, d0, descs, units, nunits, max_ctas, mixed, form);
  return launch_pairsum_f32_nc<4>(p, st, d0, descs, units, nunits, max_ctas, mixed, form);
}

// The difference-pair launch of a mixed FP32 plan over n samples whose rows
// are in the plan workspace (y and its swapped copy ys, laid out for
// sspad_for(n)), adding to the coefficients C_out that the sum pairs wrote.
static int launch_pairsum_f32_diff(srm3_plan *p, cudaStream_t st, int n, void *C_out) {
  PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (int rc = tensor_map_encoder(&encode)) return rc;
  const int sp = sspad_for(n);
  PsDiffDesc d;
  std::memset(static_cast<void *>(&d), 0, sizeof(d));
  const cuuint64_t dims[2] = {(cuuint64_t)sp * 2, (cuuint64_t)p->nk * p->rowstride};
  const cuuint64_t strides[1] = {(cuuint64_t)sp * 2 * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)packed::LANES * 4, (cuuint32_t)packed::BOX_ROWS};
  const cuuint32_t estr[2] = {1, 1};
  for (int m = 0; m < 2; ++m) {
    const CUresult r = encode(m == 0 ? &d.amap : &d.bmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                              m == 0 ? p->y : p->ys, dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
      return fail(SRM3_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  }
  d.Ek = (const float *)p->Ek;
  d.Ewd = (const float *)p->Ewd;
  d.ck = (const float *)p->ck;
  d.C = (float2 *)C_out;
  d.order = p->super_order_d;
  d.nk = p->nk;
  d.nw = p->nw;
  d.SS = 2 * n;
  d.SSpad = sp;
  d.rowstride = p->rowstride;
  d.G = sp / (2 * packed::LANES);
  d.cb = (float)std::cos(p->beta);
  d.sb = (float)std::sin(p->beta);
  const size_t smem = pairsum_f32p_smem<4>();
  SRM3_CUDA(cudaFuncSetAttribute(k_pairsum_f32d, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
  SRM3_CUDA(cudaFuncSetAttribute(k_pairsum_f32d, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 100));
  int nsm = 0, per_sm = 0;
  SRM3_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->device));
  SRM3_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pairsum_f32d,
                                                          packed::Shape<4>::NT,
                                                          smem));
  if (per_sm < 1) return fail(SRM3_ERR_NOT_SUPPORTED, "difference pair sum does not fit on an SM");
  const int nunits = p->nsuper_d * d.G;
  const int grid = std::min(nunits, nsm * per_sm);
  if (grid == 0) return SRM3_OK;
  k_pairsum_f32d<<<grid, packed::Shape<4>::NT, smem, st>>>(d, nunits, p->ps_err);
  SRM3_CUDA(cudaGetLastError());
  return SRM3_OK;
}

static int pairsum_f64_on(srm3_plan *p, cudaStream_t st, int n, void *C_out) {
  const int SS = 2 * n, sp = sspad_for(n);
  const long long threads = (long long)p->nk * p->nw * SS * 32;  // a warp per (k, sheet-sample)
  k_pairsum_f64<<<cdiv(threads, 256), 256, 0, st>>>(
      p->nk, p->nw, SS, sp, p->rowstride, (const double2 *)p->y, (const double2 *)p->y0,
      (const double *)p->Ek, (const double *)p->Ews, p->ew_off, (const double *)p->Pk,
      (const double *)p->ck, std::cos(p->beta), std::sin(p->beta), (double2 *)C_out,
      p->mixed ? 1 : 0, p->row_lo, p->row_hi);
  SRM3_CUDA(cudaGetLastError());
  return SRM3_OK;
}

int run_pairsum(srm3_plan *p, int n, void *C_out) {
  if (p->sep) return conv_pairsum_on(p, p->stream, n, p->y, p->y0, C_out);
  if (p->precision == SRM3_FP64) return pairsum_f64_on(p, p->stream, n, C_out);
  PsDesc d;
  int rc = fill_pairsum_desc(p, n, C_out, &d);
  if (rc) return rc;
  rc = launch_pairsum_f32(p, p->stream, d, nullptr, nullptr,
                          p->nsuper[tile_index(p->ps_nc)] * d.G, 0, d.half != 0, p->ps_nc);
  if (rc || !p->mixed) return rc;
  return launch_pairsum_f32_diff(p, p->stream, n, C_out);
}

int run_transform(srm3_plan *p, const void *C, int n, void *out) {
  return transform_on(p, p->stream, C, n, out, p->H);
}

int check_pairsum_error(srm3_plan *p) {
  if (!p->ps_err) return SRM3_OK;
  int h = 0;
  SRM3_CUDA(cudaMemcpy(&h, p->ps_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) return fail(SRM3_ERR_TIMEOUT, "FP32 pair sum: a pipeline wait ran out of time");
  return SRM3_OK;
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
  if ((rc = stage_begin(p, 1, 2LL * m * (p->pairs + p->diffpairs), &rec))) return rc;
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

// Autotuner choices per lattice shape, process-wide: (storage, compute warps).
static std::mutex g_tune_mu;
static std::map<std::pair<int, int>, std::pair<int, int>> g_tune;

int tune_cache_lookup(int nk, int nw, int *nc) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tune.find({nk, nw});
  if (it == g_tune.end()) return -1;
  if (nc) *nc = it->second.second;
  return it->second.first;
}

void tune_cache_store(int nk, int nw, int storage, int nc) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune[{nk, nw}] = {storage, nc};
}

}  // namespace srm3

// A sampling job over several plans (see srm3_batch_create).  FP32 plans
// with W recomputed and the same lattice shape form one shape group: their
// samples share the lanes of the pair sum (the weights depend only on the
// shape; each sample brings its own pure and pair factors) and batch-owned
// buffers.  Other plans (stored W table, FP64) run on their own workspace.
struct srm3_batch {
  struct Group {
    std::vector<int> members;     // plan indices of the batch
    std::vector<int> sample_off;  // per member: first sample within the group
    int total = 0, sp = 0, nmax = 0;
    void *y = nullptr, *y0 = nullptr, *C = nullptr, *H = nullptr;
    size_t ybytes = 0;
    const float **pk_of = nullptr, **ck_of = nullptr;  // device, [total]
  };
  std::vector<srm3_plan *> plans;
  std::vector<int> counts, seed_off, group_of;  // group_of[i]: group index or -1
  std::vector<void *> outs;
  std::vector<Group> groups;
  int total = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  uint64_t *dseeds = nullptr;     // device seeds the phase kernels read
  std::vector<uint64_t> hseeds;   // pageable staging copy (read before run returns)
  srm3::PsDesc *ddesc = nullptr;  // per group and per FP32 table plan
  // work units of all of them, by decreasing cost, per tile shape (index 0:
  // 32 wide, 1: 16 wide -- each descriptor's plan's tile), one after the
  // other in dunits: one persistent launch per tile shape present
  int4 *dunits = nullptr;
  int nunits = 0;                 // both shapes
  int nunits_v[2] = {0, 0};
  bool mixed_v[2] = {false, false};  // some descriptor of the shape takes the half-group mode
  int ps_form = 0;                   // the weight form common to every descriptor (kPsAnyForm: none)
  srm3_plan *lead = nullptr;      // first FP32 plan: CTA count and error word of the launch
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long pair_terms = 0;
  bool holds_refs = false;        // the plans' batch_refs were raised
  bool timing = false;            // events around the pair-sum launch
  bool capturing = false;         // inside srm3_batch_capture
  int max_ctas = 0;               // cap on the pair sum's CTAs (0: all resident)
  cudaEvent_t ps_ev[2] = {nullptr, nullptr};
  long long dev_bytes = 0;        // device memory the batch allocated itself
};

using namespace srm3;

// The launch sequence of one batch run on the batch stream.
static int batch_launch(srm3_batch *b) {
  int rc;
  for (auto &g : b->groups) {
    SRM3_CUDA(cudaMemsetAsync(g.y, 0, g.ybytes, b->stream));
    for (size_t m = 0; m < g.members.size(); ++m) {
      const int i = g.members[m];
      if ((rc = phases_into(b->plans[i], b->stream, nullptr, b->dseeds + b->seed_off[i],
                            b->counts[i], g.y, g.y0, g.sp, 2 * g.sample_off[m], nullptr)))
        return rc;
    }
  }
  for (size_t i = 0; i < b->plans.size(); ++i)
    if (b->group_of[i] < 0 &&
        (rc = phases_on(b->plans[i], b->stream, nullptr, b->dseeds + b->seed_off[i],
                        b->counts[i], nullptr)))
      return rc;
  if (b->nunits > 0) {
    PsDesc none;
    std::memset(static_cast<void *>(&none), 0, sizeof(none));
    // in a capture the events must be external nodes of the graph
    const unsigned evf = b->capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    if (b->timing) SRM3_CUDA(cudaEventRecordWithFlags(b->ps_ev[0], b->stream, evf));
    for (int v = 0, off = 0; v < 2; off += b->nunits_v[v], ++v)
      if (b->nunits_v[v] > 0 &&
          (rc = launch_pairsum_f32(b->lead, b->stream, none, b->ddesc, b->dunits + off,
                                   b->nunits_v[v], b->max_ctas, b->mixed_v[v], v == 0 ? 4 : 2,
                                   b->ps_form)))
        return rc;
    if (b->timing) SRM3_CUDA(cudaEventRecordWithFlags(b->ps_ev[1], b->stream, evf));
  }
  for (size_t i = 0; i < b->plans.size(); ++i) {
    srm3_plan *p = b->plans[i];
    if (p->mixed && p->precision == SRM3_FP32) {  // its difference pairs, after its sum pairs
      if ((rc = launch_pairsum_f32_diff(p, b->stream, b->counts[i], p->C))) return rc;
    } else if (p->sep) {
      if ((rc = conv_pairsum_on(p, b->stream, b->counts[i], p->y, p->y0, p->C))) return rc;
    } else if (p->precision == SRM3_FP64 &&
               (rc = pairsum_f64_on(p, b->stream, b->counts[i], p->C))) {
      return rc;
    }
  }
  for (auto &g : b->groups)
    for (size_t m = 0; m < g.members.size(); ++m) {
      const int i = g.members[m];
      srm3_plan *p = b->plans[i];
      const char *C = (const char *)g.C + (size_t)2 * g.sample_off[m] * p->nk * p->nw *
                                              sizeof(float2);
      if ((rc = transform_on(p, b->stream, C, b->counts[i], b->outs[i], g.H))) return rc;
    }
  for (size_t i = 0; i < b->plans.size(); ++i)
    if (b->group_of[i] < 0 &&
        (rc = transform_on(b->plans[i], b->stream, b->plans[i]->C, b->counts[i], b->outs[i],
                           b->plans[i]->H)))
      return rc;
  return SRM3_OK;
}

// Device buffers of a batch are stream-ordered allocations on its stream, so
// that creating and freeing batches never waits for work on other streams.
static void batch_free(srm3_batch *b) {
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->holds_refs)
    for (size_t i = 0; i < b->plans.size(); ++i)
      if (b->group_of[i] < 0) --b->plans[i]->batch_refs;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (cudaEvent_t e : b->ps_ev)
    if (e) cudaEventDestroy(e);
  for (auto &g : b->groups)
    for (void *q : {g.y, g.y0, g.C, g.H, (void *)g.pk_of, (void *)g.ck_of})
      if (q) cudaFreeAsync(q, b->stream);
  for (void *q : {(void *)b->dseeds, (void *)b->ddesc, (void *)b->dunits})
    if (q) cudaFreeAsync(q, b->stream);
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

// A plan restricted to a range of lattice rows computes only those rows'
// coefficients: fields need the gathered coefficients of every shard
// (srm3_field_from_coeffs).
static int check_all_rows(const srm3_plan *p) {
  if (p->row_lo != 0 || p->row_hi != p->nk)
    return fail(SRM3_ERR_NOT_SUPPORTED,
                "the plan computes the coefficients of rows " + std::to_string(p->row_lo) + ".." +
                    std::to_string(p->row_hi - 1) + " only: gather every shard's rows and "
                    "call srm3_field_from_coeffs");
  return SRM3_OK;
}

SRM3_API int srm3_sample(srm3_plan *plan, const uint64_t *seeds, int n, void *out) {
  int rc = check_call(plan, seeds, n, out);
  if (rc || n == 0) return rc;
  if ((rc = check_all_rows(plan))) return rc;
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
  if ((rc = check_all_rows(plan))) return rc;
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
  return check_pairsum_error(plan);
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
  t->recursion_passes_coarse = plan->coarse_passes;
  t->coarse_ms = plan->t_coarse_ms;
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

SRM3_API int srm3_set_tile_width(srm3_plan *plan, int width) {
  if (!plan) return fail(SRM3_ERR_INVALID_ARG, "plan is NULL");
  if (width != 16 && width != 32) return fail(SRM3_ERR_INVALID_ARG, "width must be 16 or 32");
  if (plan->precision != SRM3_FP32 || plan->sep)
    return fail(SRM3_ERR_NOT_SUPPORTED, "tile shapes apply to FP32 plans of the O(N^2) pair sum");
  plan->ps_nc = width / kTileR;
  return SRM3_OK;
}

SRM3_API int srm3_autotune(srm3_plan *plan, int n, srm3_tune_result *res) {
  if (!plan || !res) return fail(SRM3_ERR_INVALID_ARG, "plan and result must be non-NULL");
  if (n < 1 || n > kMaxChunk) return fail(SRM3_ERR_INVALID_ARG, "n must be in 1..128");
  if (plan->precision != SRM3_FP32 || plan->sep)
    return fail(SRM3_ERR_NOT_SUPPORTED,
                "autotuning applies to FP32 plans of the O(N^2) pair sum only");
  if (plan->mixed)
    return fail(SRM3_ERR_NOT_SUPPORTED,
                "mixed plans recompute W: there is no storage to choose");
  int rc = ensure_workspace(plan, n);
  if (rc) return rc;
  std::vector<uint64_t> seeds(n);
  for (int j = 0; j < n; ++j) seeds[j] = (uint64_t)j + 1;
  if ((rc = run_phases(plan, seeds.data(), n, nullptr))) return rc;
  const bool can_table = (double)plan->table_entries * sizeof(float) <= plan->table_budget;
  if (can_table && !plan->W) {
    if ((rc = build_w_table(plan, plan->stream))) return rc;
  }
  cudaEvent_t ev[2];
  SRM3_CUDA(cudaEventCreate(&ev[0]));
  SRM3_CUDA(cudaEventCreate(&ev[1]));
  auto time_one = [&](int storage, int nc, double *ms) -> int {
    plan->storage = storage;
    plan->ps_nc = nc;
    PsDesc d;
    int r = fill_pairsum_desc(plan, n, plan->C, &d);
    if (r) return r;
    const int nunits = plan->nsuper[tile_index(nc)] * d.G;
    if ((r = launch_pairsum_f32(plan, plan->stream, d, nullptr, nullptr, nunits, 0, d.half != 0,
                                nc)))
      return r;
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      SRM3_CUDA(cudaEventRecord(ev[0], plan->stream));
      if ((r = launch_pairsum_f32(plan, plan->stream, d, nullptr, nullptr, nunits, 0,
                                  d.half != 0, nc)))
        return r;
      SRM3_CUDA(cudaEventRecord(ev[1], plan->stream));
      SRM3_CUDA(cudaEventSynchronize(ev[1]));
      float t = 0.f;
      SRM3_CUDA(cudaEventElapsedTime(&t, ev[0], ev[1]));
      best = std::min(best, t);
    }
    *ms = best;
    return SRM3_OK;
  };
  // every (storage, tile) the plan can take: the stored table when it exists,
  // W recomputed; 32- and 16-wide tiles
  double t[2][2] = {{-1.0, -1.0}, {-1.0, -1.0}};  // [storage: table, recompute][tile]
  for (int v = 0; v < 2 && !rc; ++v) {
    const int nc = v == 0 ? 4 : 2;
    if (plan->W) rc = time_one(SRM3_STORAGE_TABLE, nc, &t[0][v]);
    if (!rc) rc = time_one(SRM3_STORAGE_RECOMPUTE, nc, &t[1][v]);
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  if (rc) return rc;
  // the default (W recomputed, 32 wide) unless another form is faster by at
  // least kTuneMargin: single-launch timings jitter by a few per cent, and a
  // batch runs one launch per tile width and groups plans by storage
  constexpr double kTuneMargin = 0.03;
  int bs = 1, bv = 0;
  for (int st = 0; st < 2; ++st)
    for (int v = 0; v < 2; ++v)
      if (t[st][v] >= 0.0 && t[st][v] < t[bs][bv] * (1.0 - kTuneMargin)) {
        bs = st;
        bv = v;
      }
  const int choice = bs == 0 ? SRM3_STORAGE_TABLE : SRM3_STORAGE_RECOMPUTE;
  const int nc = bv == 0 ? 4 : 2;
  plan->storage = choice;
  plan->ps_nc = nc;
  if (choice == SRM3_STORAGE_RECOMPUTE && plan->W) {
    SRM3_CUDA(cudaStreamSynchronize(plan->stream));
    SRM3_CUDA(dev_free(plan->W, plan->stream));
    plan->W = nullptr;
    plan->table_bytes = 0.0;
  }
  tune_cache_store(plan->nk, plan->nw, choice, nc);
  res->table_ms = std::min(t[0][0] < 0 ? 1e30 : t[0][0], t[0][1] < 0 ? 1e30 : t[0][1]);
  if (res->table_ms >= 1e30) res->table_ms = -1.0;
  res->recompute_ms = std::min(t[1][0], t[1][1]);
  res->storage = choice;
  res->samples = n;
  res->tile_width = kTileR * nc;
  res->table_ms_w32 = t[0][0];
  res->table_ms_w16 = t[0][1];
  res->recompute_ms_w32 = t[1][0];
  res->recompute_ms_w16 = t[1][1];
  SRM3_CUDA(cudaStreamSynchronize(plan->stream));
  return check_pairsum_error(plan);
}

SRM3_API int srm3_batch_create(srm3_plan *const *plans, const int32_t *counts,
                               void *const *outs, int m, void *stream, srm3_batch **out) {
  if (!out) return fail(SRM3_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (m < 1 || !plans || !counts || !outs)
    return fail(SRM3_ERR_INVALID_ARG, "need m >= 1 plans, counts and outputs");
  int dev = -1;
  for (int i = 0; i < m; ++i) {
    if (!plans[i] || !outs[i])
      return fail(SRM3_ERR_INVALID_ARG, "NULL plan or output in the batch");
    if (counts[i] < 1 || counts[i] > kMaxChunk)
      return fail(SRM3_ERR_INVALID_ARG, "batch sample counts must be in 1..128");
    if (dev < 0) dev = plans[i]->device;
    if (plans[i]->device != dev)
      return fail(SRM3_ERR_NOT_SUPPORTED, "the plans of a batch must be on one device");
    if (plans[i]->row_lo != 0 || plans[i]->row_hi != plans[i]->nk)
      return fail(SRM3_ERR_NOT_SUPPORTED, "a batch takes plans of the whole lattice only");
    for (int j = 0; j < i; ++j)
      if (plans[j] == plans[i])
        return fail(SRM3_ERR_INVALID_ARG,
                    "a plan appears twice in the batch (it has one workspace)");
  }
  srm3_batch *b = new srm3_batch();
  auto bail = [&](int rc) {
    batch_free(b);
    return rc;
  };
  int rc;
  if (stream) {
    b->stream = (cudaStream_t)stream;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaStreamCreateWithFlags"));
    b->own_stream = true;
  }
  std::vector<PsDesc> descs;
  std::vector<std::pair<long long, int4>> units[2];  // per tile shape
  // one tile width for the whole batch -- the width of the plans that carry
  // most of its pair-terms (results do not depend on it): one persistent
  // launch, no tail of a second
  long long terms_v[2] = {0, 0};
  for (int i = 0; i < m; ++i)
    if (plans[i]->precision == SRM3_FP32 && !plans[i]->sep)
      terms_v[tile_index(plans[i]->ps_nc)] += (plans[i]->pairs + plans[i]->diffpairs) * counts[i];
  const int batch_nc = terms_v[1] > terms_v[0] ? 2 : 4;
  auto add_units = [&](srm3_plan *p, int j, const PsDesc &d) {
    const int v = tile_index(batch_nc);
    b->mixed_v[v] = b->mixed_v[v] || d.half != 0;
    for (const int2 &t : p->super_host[v]) {
      const long long cost = ps_nitems(t.x, t.y, d.half, kTileR * batch_nc);
      for (int g = 0; g < d.G; ++g) units[v].push_back({cost, make_int4(j, t.x, t.y, g)});
    }
  };
  // plans of one shape group share the lead plan's weights (envelope windows
  // or its W table of pair envelopes) and its tile; each sample keeps its
  // own spectrum's factors
  auto same_shape = [](const srm3_plan *a, const srm3_plan *c) {
    return a->nk == c->nk && a->nw == c->nw && a->nx == c->nx && a->nt == c->nt &&
           a->ku == c->ku && a->wu == c->wu && a->sigma_g == c->sigma_g && a->beta == c->beta &&
           a->storage == c->storage;
  };
  for (int i = 0; i < m; ++i) {
    srm3_plan *p = plans[i];
    b->plans.push_back(p);
    b->counts.push_back(counts[i]);
    b->outs.push_back(outs[i]);
    b->seed_off.push_back(b->total);
    b->total += counts[i];
    b->pair_terms += 2LL * (p->pairs + p->diffpairs) * counts[i];
    int gi = -1;
    if (p->precision == SRM3_FP32 && !p->sep && !p->mixed &&
        (p->storage == SRM3_STORAGE_RECOMPUTE || (p->storage == SRM3_STORAGE_TABLE && p->W))) {
      for (size_t g = 0; g < b->groups.size() && gi < 0; ++g)
        if (same_shape(b->plans[b->groups[g].members[0]], p)) gi = (int)g;
      if (gi < 0) {
        gi = (int)b->groups.size();
        b->groups.emplace_back();
      }
      auto &g = b->groups[gi];
      g.members.push_back(i);
      g.sample_off.push_back(g.total);
      g.total += counts[i];
      g.nmax = std::max(g.nmax, counts[i]);
    } else if ((rc = ensure_workspace(p, counts[i]))) {
      return bail(rc);
    }
    b->group_of.push_back(gi);
    if (p->precision == SRM3_FP32 && !p->sep && !b->lead) b->lead = p;
  }
  cudaError_t e;
  for (auto &g : b->groups) {  // batch-owned buffers of each shape group
    srm3_plan *p = b->plans[g.members[0]];
    if (g.total > 4096) return bail(fail(SRM3_ERR_INVALID_ARG,
                                         "more than 4096 samples of one lattice shape"));
    g.sp = sspad_for(g.total);
    g.ybytes = (size_t)p->nk * p->rowstride * g.sp * sizeof(float2);
    const size_t cb = (size_t)2 * g.total * p->nk * p->nw * sizeof(float2);
    const size_t hb = (size_t)g.nmax * transform_elems(p) * sizeof(float2);
    cudaStream_t st = b->stream;
    b->dev_bytes += (long long)(g.ybytes + (size_t)g.sp * sizeof(float2) + cb + hb +
                                2 * sizeof(float *) * g.total);
    if ((e = cudaMallocAsync(&g.y, g.ybytes, st)) != cudaSuccess ||
        (e = cudaMallocAsync(&g.y0, (size_t)g.sp * sizeof(float2), st)) != cudaSuccess ||
        (e = cudaMallocAsync(&g.C, cb, st)) != cudaSuccess ||
        (e = cudaMallocAsync(&g.H, hb, st)) != cudaSuccess ||
        (e = cudaMallocAsync((void **)&g.pk_of, sizeof(float *) * g.total, st)) != cudaSuccess ||
        (e = cudaMallocAsync((void **)&g.ck_of, sizeof(float *) * g.total, st)) != cudaSuccess)
      return bail(cuda_fail(e, "cudaMallocAsync(batch shape group)"));
    std::vector<const float *> pk(g.total), ck(g.total);
    for (size_t mm = 0; mm < g.members.size(); ++mm) {
      srm3_plan *q = b->plans[g.members[mm]];
      const bool sepf = pairsum_sep_now(q);  // as the group's descriptor (same shape and storage)
      for (int j = 0; j < b->counts[g.members[mm]]; ++j) {
        pk[g.sample_off[mm] + j] = sepf ? q->Pk_s : (const float *)q->Pk;
        ck[g.sample_off[mm] + j] = sepf ? q->ck_s : (const float *)q->ck;
      }
    }
    if ((e = cudaMemcpyAsync(g.pk_of, pk.data(), sizeof(float *) * g.total,
                             cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(g.ck_of, ck.data(), sizeof(float *) * g.total,
                             cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      return bail(cuda_fail(e, "cudaMemcpy(batch factor tables)"));
    PsDesc d;
    if ((rc = fill_pairsum_desc_into(p, g.total, g.y, g.y0, g.C, &d))) return bail(rc);
    d.pk_of = g.pk_of;
    d.ck_of = g.ck_of;
    const int j = (int)descs.size();
    descs.push_back(d);
    add_units(p, j, d);
  }
  for (int i = 0; i < m; ++i) {  // FP32 plans with a stored W table, on their workspace
    srm3_plan *p = b->plans[i];
    if (b->group_of[i] >= 0 || p->precision != SRM3_FP32 || p->sep) continue;
    PsDesc d;
    if ((rc = fill_pairsum_desc(p, counts[i], p->C, &d))) return bail(rc);
    const int j = (int)descs.size();
    descs.push_back(d);
    add_units(p, j, d);
  }
  std::vector<int4> u;
  for (int v = 0; v < 2; ++v) {
    std::stable_sort(units[v].begin(), units[v].end(),
                     [](const std::pair<long long, int4> &x, const std::pair<long long, int4> &y) {
                       return x.first > y.first;
                     });
    b->nunits_v[v] = (int)units[v].size();
    for (const auto &un : units[v]) u.push_back(un.second);
  }
  b->nunits = (int)u.size();
  if (!descs.empty()) {
    b->dev_bytes += (long long)(sizeof(PsDesc) * descs.size() + sizeof(int4) * u.size());
    b->ps_form = ps_form_of(descs[0]);
    for (const PsDesc &dd : descs)
      if (ps_form_of(dd) != b->ps_form) b->ps_form = kPsAnyForm;
    e = cudaMallocAsync(&b->ddesc, sizeof(PsDesc) * descs.size(), b->stream);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaMallocAsync(batch descriptors)"));
    e = cudaMemcpyAsync(b->ddesc, descs.data(), sizeof(PsDesc) * descs.size(),
                        cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaMemcpyAsync(batch descriptors)"));
    e = cudaMallocAsync(&b->dunits, sizeof(int4) * u.size(), b->stream);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaMallocAsync(batch units)"));
    e = cudaMemcpyAsync(b->dunits, u.data(), sizeof(int4) * u.size(), cudaMemcpyHostToDevice,
                        b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaMemcpyAsync(batch units)"));
    // kernel attributes and resident CTA count, set before any capture
    PsDesc none;
    std::memset(static_cast<void *>(&none), 0, sizeof(none));
    for (int v = 0; v < 2; ++v)
      if ((rc = launch_pairsum_f32(b->lead, b->stream, none, b->ddesc, b->dunits, 0, 0,
                                   b->mixed_v[v], v == 0 ? 4 : 2, b->ps_form)))
        return bail(rc);
  }
  b->dev_bytes += (long long)(sizeof(uint64_t) * b->total);
  e = cudaMallocAsync(&b->dseeds, sizeof(uint64_t) * b->total, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bail(cuda_fail(e, "cudaMallocAsync(batch seeds)"));
  b->hseeds.resize(b->total);
  for (int i = 0; i < m; ++i)  // plans whose own workspace the batch uses
    if (b->group_of[i] < 0) ++b->plans[i]->batch_refs;
  b->holds_refs = true;
  *out = b;
  return SRM3_OK;
}

SRM3_API int srm3_batch_run(srm3_batch *b, const uint64_t *seeds) {
  if (!b || !seeds) return fail(SRM3_ERR_INVALID_ARG, "batch and seeds must be non-NULL");
  // from pageable memory the copy has read the host buffer when it returns
  std::memcpy(b->hseeds.data(), seeds, sizeof(uint64_t) * b->total);
  SRM3_CUDA(cudaMemcpyAsync(b->dseeds, b->hseeds.data(), sizeof(uint64_t) * b->total,
                            cudaMemcpyHostToDevice, b->stream));
  if (b->exec) {
    SRM3_CUDA(cudaGraphLaunch(b->exec, b->stream));
    return SRM3_OK;
  }
  return batch_launch(b);
}

SRM3_API int srm3_batch_capture(srm3_batch *b) {
  if (!b) return fail(SRM3_ERR_INVALID_ARG, "batch is NULL");
  SRM3_CUDA(cudaStreamSynchronize(b->stream));
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  if (b->graph) {
    cudaGraphDestroy(b->graph);
    b->graph = nullptr;
  }
  SRM3_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  b->capturing = true;
  const int rc = batch_launch(b);
  b->capturing = false;
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(b->stream, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  b->graph = g;
  SRM3_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
  return SRM3_OK;
}

SRM3_API int srm3_batch_sync(srm3_batch *b) {
  if (!b) return fail(SRM3_ERR_INVALID_ARG, "batch is NULL");
  SRM3_CUDA(cudaStreamSynchronize(b->stream));
  return b->lead ? check_pairsum_error(b->lead) : SRM3_OK;
}

SRM3_API int64_t srm3_batch_pair_terms(const srm3_batch *b) { return b ? b->pair_terms : 0; }

SRM3_API int64_t srm3_batch_device_bytes(const srm3_batch *b) { return b ? b->dev_bytes : 0; }

SRM3_API int srm3_batch_set_max_ctas(srm3_batch *b, int max_ctas) {
  if (!b || max_ctas < 0) return fail(SRM3_ERR_INVALID_ARG, "batch is NULL or max_ctas < 0");
  b->max_ctas = max_ctas;
  return SRM3_OK;
}

SRM3_API int srm3_batch_enable_timing(srm3_batch *b, int on) {
  if (!b) return fail(SRM3_ERR_INVALID_ARG, "batch is NULL");
  if (on && !b->ps_ev[0]) {
    SRM3_CUDA(cudaEventCreate(&b->ps_ev[0]));
    SRM3_CUDA(cudaEventCreate(&b->ps_ev[1]));
  }
  b->timing = on != 0 && b->nunits > 0;
  return SRM3_OK;
}

SRM3_API int srm3_batch_pairsum_ms(srm3_batch *b, double *ms) {
  if (!b || !ms) return fail(SRM3_ERR_INVALID_ARG, "batch and ms must be non-NULL");
  *ms = 0.0;
  if (!b->timing) return SRM3_OK;
  SRM3_CUDA(cudaEventSynchronize(b->ps_ev[1]));
  float t = 0.f;
  SRM3_CUDA(cudaEventElapsedTime(&t, b->ps_ev[0], b->ps_ev[1]));
  *ms = t;
  return SRM3_OK;
}

SRM3_API void srm3_batch_destroy(srm3_batch *b) {
  if (b) batch_free(b);
}

// ---------------------------------------------------------------------------
// Failure path of the bounded mbarrier wait of the FP32 pair sum, without a
// fault: one thread waits on an mbarrier (count 1) that nothing arrives at,
// gives up after `cycles` clock cycles and raises the error word.
namespace srm3 {
__global__ void k_selftest_mbar(int *err, long long limit) {
  __shared__ unsigned long long b;
  __shared__ int ab;
  if (threadIdx.x == 0) {
    mbar_init(&b, 1);
    ab = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait(&b, 0, &ab, err, limit);
}
}  // namespace srm3

SRM3_API int srm3_selftest_timeouts(int *barrier_timed_out, int *wait_timed_out) {
  if (!barrier_timed_out || !wait_timed_out)
    return fail(SRM3_ERR_INVALID_ARG, "outputs must be non-NULL");
  // about 10 ms of waiting each: 2^14 polls of an L2 word, 2e7 clock cycles
  int rc = selftest_barrier(1ll << 14, barrier_timed_out);
  if (rc) return rc;
  int *er = nullptr;
  SRM3_CUDA(cudaMalloc(&er, sizeof(int)));
  cudaError_t e = cudaMemset(er, 0, sizeof(int));
  if (e == cudaSuccess) {
    k_selftest_mbar<<<1, 32>>>(er, 20000000ll);
    e = cudaGetLastError();
  }
  int h = 0;
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&h, er, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(er);
  if (e != cudaSuccess) return cuda_fail(e, "mbarrier wait self-test");
  *wait_timed_out = h;
  return SRM3_OK;
}
