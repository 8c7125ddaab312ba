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

bool on_device(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

const char* mbs_noalloc_last_error(void) { return g_noalloc_err.c_str(); }

mbs_status mbs_apply_edge_corrections_noalloc(const mbs_plan* plan, const void* x, void* out) {
  g_noalloc_err.clear();
  mbs::CorrView v;
  if (!plan || !x || !out || !mbs_plan_corr_view(plan, &v)) return nfail(MBS_EINVAL, "null argument");
  if (x == out) return nfail(MBS_EINVAL, "x and out must not alias");
  if (!on_device(x) || !on_device(out))
    return nfail(MBS_EINVAL, "x and out must be device pointers (host data would need a staging allocation)");
  if (v.nvox > kNoAllocMaxVoxels)
    return nfail(MBS_EINVAL, "grid of " + std::to_string(v.nvox) + " voxels exceeds the " +
                                 std::to_string(kNoAllocMaxVoxels) + "-voxel scratch of this entry point");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return nfail(MBS_ECUDA, "no usable current device");
  float2* scratch = nullptr;
  {
    // once per device, with that device current: the device address of the array
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_corr_scratch);
      if (e != cudaSuccess) return nfail(MBS_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_addr[dev] = (float2*)p;
    }
    scratch = g_addr[dev];
  }
  float2* o = (float2*)out;
  cudaError_t e = mbs::launch_zero(o, v.nvox, v.stream);
  if (!e && v.has_shell) {
    // every boundary-layer voxel of the scratch is written by the first axis
    // that covers it before it is read, so nothing needs clearing
    mbs::CorrArgs c = {};
    c.F = (const float2*)x;
    c.C = scratch;
    c.cW = v.cW;
    c.c = v.c;
    c.tc = v.tc;
    c.tb = v.tb;
    c.g = v.g;
    c.state = v.free_state;
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
      s.state = v.free_state;
      s.mode = mbs::SHELL_SET_E;
      e = mbs::launch_shell(s, 152 * 8, v.stream);
    }
  }
  if (!e) e = cudaStreamSynchronize(v.stream);
  if (e) return nfail(MBS_ECUDA, std::string("edge corrections: ") + cudaGetErrorString(e));
  return MBS_OK;
}

}  // extern "C"
