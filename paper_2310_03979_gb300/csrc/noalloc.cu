// noalloc.cu - srm3_field_from_coeffs_noalloc: the transform stage with its
// intermediate held in a fixed device array of the library instead of plan
// workspace, for callers that may not allocate device memory.  The paper has
// no counterpart; the launch sequence is that of srm3_field_from_coeffs.
#include <algorithm>
#include <mutex>

#include "srm3_internal.cuh"

namespace {

constexpr size_t kScratchBytes = SRM3_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

}  // namespace

// The x-stage columns of one group of coefficient sets, [set][mx][kw]
// complex.  Never read before the x stage of the same call has written it.
static __device__ __align__(256) unsigned char srm3_noalloc_scratch[kScratchBytes];

namespace srm3 {
namespace {

std::mutex g_scratch_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of srm3_noalloc_scratch on `dev`, which is the current
// device.  Looked up once per device, then cached for the life of the
// process: a cudaDeviceReset (or any reset of the device's primary context)
// unloads the module, and the cached address is then stale.
int scratch_address(int dev, void **addr) {
  if (dev < 0 || dev >= kMaxDevices)
    return fail(SRM3_ERR_NOT_SUPPORTED, "srm3_field_from_coeffs_noalloc: device ordinal " +
                                            std::to_string(dev) + " is beyond the " +
                                            std::to_string(kMaxDevices) + " it caches");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void *a = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&a, srm3_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(srm3_noalloc_scratch)");
    g_scratch_addr[dev] = a;
  }
  *addr = g_scratch_addr[dev];
  return SRM3_OK;
}

// Makes `dev` current for the lifetime of the guard and restores the
// caller's device afterwards.
struct DeviceGuard {
  int prev = -1;
  bool switched = false;
  int enter(int dev) {
    SRM3_CUDA(cudaGetDevice(&prev));
    if (prev != dev) {
      SRM3_CUDA(cudaSetDevice(dev));
      switched = true;
    }
    return SRM3_OK;
  }
  ~DeviceGuard() {
    if (switched) cudaSetDevice(prev);
  }
};

// The transform of n sets in groups whose x-stage columns fit the scratch, by
// the launch sequence of srm3_field_from_coeffs (transform_on) with the
// scratch in place of the plan workspace.
int field_noalloc(srm3_plan *p, const void *C, int n, void *out, void *scratch) {
  const size_t e2 = p->precision == SRM3_FP32 ? sizeof(float2) : sizeof(double2);
  const size_t e1 = p->precision == SRM3_FP32 ? sizeof(float) : sizeof(double);
  const size_t perH = transform_elems(p) * e2;
  const size_t perC = (size_t)2 * p->nk * p->nw * e2;
  const size_t perU = (size_t)p->nx * p->nt * e1;
  // gridDim.y carries the set index: at most 65535 sets per launch.
  const int group = (int)std::min<size_t>(kScratchBytes / perH, 65535);
  for (int s0 = 0; s0 < n; s0 += group) {
    const int m = std::min(group, n - s0);
    const int rc = transform_on(p, p->stream, (const char *)C + (size_t)s0 * perC, m,
                                (char *)out + (size_t)s0 * perU, scratch);
    if (rc) return rc;
  }
  return SRM3_OK;
}

}  // namespace
}  // namespace srm3

using namespace srm3;

SRM3_API int srm3_field_from_coeffs_noalloc(srm3_plan *plan, const void *C, int n, void *out) {
  if (!plan) return fail(SRM3_ERR_INVALID_ARG, "plan is NULL");
  if (n < 0 || (n > 0 && (!C || !out))) return fail(SRM3_ERR_INVALID_ARG, "bad C/out/n");
  const size_t e2 = plan->precision == SRM3_FP32 ? sizeof(float2) : sizeof(double2);
  const size_t perH = transform_elems(plan) * e2;
  if (perH > kScratchBytes)
    return fail(SRM3_ERR_INVALID_ARG,
                "srm3_field_from_coeffs_noalloc: one coefficient set needs " +
                    std::to_string(perH) + " bytes of scratch (n_x * n_omega complex values), "
                    "more than the SRM3_NOALLOC_SCRATCH_BYTES = " +
                    std::to_string(kScratchBytes) + " it has; use srm3_field_from_coeffs");
  if (n == 0) return SRM3_OK;
  DeviceGuard guard;
  int rc = guard.enter(plan->device);
  if (rc) return rc;
  void *scratch = nullptr;
  if ((rc = scratch_address(plan->device, &scratch))) return rc;
  return field_noalloc(plan, C, n, out, scratch);
}
