// Edge corrections E x without any allocation.
//
// mbs_apply_operator(plan, MBS_OP_E, ...) keeps the corrections in the plan's
// FFT buffer and stages host data through buffers it allocates on first use.
// Callers that must not trigger a device allocation when they call (a process
// whose device memory is handed out entirely by another framework's caching
// allocator, or a fixed memory budget) use this entry point instead: the
// correction scratch is a fixed array in this file, sized for grids of up to
// kNoAllocMaxVoxels voxels, the plan's buffers are not touched, and only device
// pointers are accepted.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/mbs.h"
#include "mbs_internal.h"

namespace {

constexpr long long kNoAllocMaxVoxels = 1ll << 21;  // 2,097,152 complex64 voxels = 16 MiB

// Shared by every call on a device; each GPU that loads the library holds it
// until the process exits.
static __device__ __align__(256) float2 g_corr_scratch[kNoAllocMaxVoxels];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float2* g_addr[kMaxDevices] = {};

thread_local std::string g_noalloc_err;

mbs_status nfail(mbs_status s, const std::string& m) {
  g_noalloc_err = m;
  return s;
}

// The device a pointer's memory lives on, or -1 for host (or unknown) memory.
int device_of(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) ? at.device : -1;
}

// Device address of the scratch on the current device `dev` (looked up once).
float2* scratch_on(int dev, cudaError_t* err) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_corr_scratch);
    if (e != cudaSuccess) {
      cudaGetLastError();
      *err = e;
      return nullptr;
    }
    g_addr[dev] = (float2*)p;
  }
  return g_addr[dev];
}

}  // namespace

namespace mbs {
bool noalloc_prepare_current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return false;
  }
  cudaError_t e = cudaSuccess;
  return scratch_on(dev, &e) != nullptr;
}
}  // namespace mbs

extern "C" {

const char* mbs_noalloc_last_error(void) { return g_noalloc_err.c_str(); }

mbs_status mbs_apply_edge_corrections_noalloc(const mbs_plan* plan, const void* x, void* out) {
  g_noalloc_err.clear();
  mbs::CorrView v;
  if (!plan || !x || !out || !mbs_plan_corr_view(plan, &v)) return nfail(MBS_EINVAL, "null argument");
  if (x == out) return nfail(MBS_EINVAL, "x and out must not alias");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return nfail(MBS_ECUDA, "no usable current device");
  }
  if (dev != v.device)
    return nfail(MBS_EINVAL, "the current device (" + std::to_string(dev) + ") is not the plan's device (" +
                                 std::to_string(v.device) + ")");
  const int dx = device_of(x), dout = device_of(out);
  if (dx < 0 || dout < 0)
    return nfail(MBS_EINVAL, "x and out must be device pointers (host data would need a staging allocation)");
  if (dx != v.device || dout != v.device) return nfail(MBS_EINVAL, "x and out must be on the plan's device");
  if (v.nvox > kNoAllocMaxVoxels)
    return nfail(MBS_EINVAL, "grid of " + std::to_string(v.nvox) + " voxels exceeds the " +
                                 std::to_string(kNoAllocMaxVoxels) + "-voxel scratch of this entry point");
  // normally found when the plan was created on this device
  cudaError_t le = cudaSuccess;
  float2* scratch = scratch_on(dev, &le);
  if (!scratch) return nfail(MBS_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(le));
  float2* o = (float2*)out;
  cudaError_t e = mbs::launch_zero(o, v.nvox, v.stream);
  if (!e && v.has_shell) {
    // Every boundary-layer voxel of the scratch is written (not added) by the
    // first corrected axis whose layers hold it, before any axis adds to it or
    // the final kernel reads it, so what an earlier call left there is never
    // read and nothing needs clearing. No solver state is passed (null): these
    // kernels never leave early.
    mbs::CorrArgs c = {};
    c.F = (const float2*)x;
    c.C = scratch;
    c.cW = v.cW;
    c.c = v.c;
    c.tc = v.tc;
    c.tb = v.tb;
    c.g = v.g;
    c.state = nullptr;
    for (int d = 0; d < 3 && !e; d++) {
      if (v.g.ax[d].a <= 0) continue;
      c.axis = d;
      e = mbs::launch_corr(c, v.stream);
    }
    if (!e) {
      mbs::ShellArgs s = {};
      s.C = scratch;
      s.out = o;
      s.tb = v.tb;
      s.g = v.g;
      s.state = nullptr;
      s.mode = mbs::SHELL_SET_E;
      e = mbs::launch_shell(s, 152 * 8, v.stream);
    }
  }
  if (!e) e = cudaStreamSynchronize(v.stream);
  if (e) return nfail(MBS_ECUDA, std::string("edge corrections: ") + cudaGetErrorString(e));
  return MBS_OK;
}

}  // extern "C"
