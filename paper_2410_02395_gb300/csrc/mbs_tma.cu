// TMA-fed strided passes (mbs_tma.cuh): instantiations, tensor maps and
// launchers.
#include <mutex>
#include <unordered_map>

#include "mbs_tma.cuh"

namespace mbs {

// Edge lengths with TMA-fed kernels (a box is at most 256 along an axis: the
// 320 tile is two boxes of 160).
#define MBS_TMA_SIZES(X) X(32) X(64) X(128) X(256) X(320)

bool tma_len_supported(int n) {
  switch (n) {
#define MBS_TMA_HAS(n) case n:
    MBS_TMA_SIZES(MBS_TMA_HAS)
#undef MBS_TMA_HAS
    return true;
    default:
      return false;
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// Tensor map over the FFT buffer (dims N2, N1, N0 of 8-byte elements) with the
// tile box of a pass along `axis` for edge n: {32, n, 1} or {32, 1, n}.
bool make_tma_map(CUtensorMap* tm, void* K, const GridDesc& g, int axis, int n) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || !tma_len_supported(n)) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)g.N2, (cuuint64_t)g.N1, (cuuint64_t)g.N0};
  const cuuint64_t strides[2] = {(cuuint64_t)g.N2 * 8, (cuuint64_t)g.N1 * g.N2 * 8};
  if (strides[0] % 16 || strides[1] % 16 || ((uintptr_t)K % 16)) return false;
  const cuuint32_t bl = (cuuint32_t)tma_box_len(n);
  const cuuint32_t box[3] = {32, axis == 1 ? bl : 1u, axis == 0 ? bl : 1u};
  const cuuint32_t es[3] = {1, 1, 1};
  const CUresult r = fn(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, K, dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Persistent grid: as many CTAs as fit on the device at once (cached per
// kernel), or `cap` per SM when the plan's tuner chose fewer.
template <class Kern>
static int persistent_blocks(Kern kernel, int threads, size_t smem, int ntiles, int cap) {
  static std::mutex mu;
  static std::unordered_map<const void*, int> cache;
  int per_sm = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find((const void*)kernel);
    if (it != cache.end()) {
      per_sm = it->second;
    } else {
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess) per_sm = 1;
      cache[(const void*)kernel] = per_sm;
    }
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (per_sm < 1) per_sm = 1;
  if (cap > 0 && cap < per_sm) per_sm = cap;
  const int b = per_sm * (sms > 0 ? sms : 1);
  return ntiles < b ? ntiles : b;
}

template <int N>
static cudaError_t run_tma(int kind, int axis, bool inv, const PassArgs& a, const CUtensorMap& tm, cudaStream_t st) {
  const size_t smem = (size_t)2 * N * 32 * sizeof(float2);
  const int threads = 32 * warps_for(N);
  const int gx = (int)((a.g.N2 + 31) / 32);
  const int ny = (int)(axis == 0 ? a.g.N1 : a.g.N0);
  const int ntiles = gx * ny * a.nsub;
  if (ntiles == 0) return cudaSuccess;
  cudaError_t e;
#define MBS_TMA_LAUNCH(KER)                                      \
  e = set_smem(KER, smem);                                       \
  if (e) return e;                                               \
  KER<<<persistent_blocks(KER, threads, smem, ntiles, a.tma_ctas), threads, smem, st>>>(a, tm);
  if (kind == 3) {  // axis-0 pass: forward, multiplier, inverse
    if (axis != 0) return cudaErrorInvalidValue;
    MBS_TMA_LAUNCH((k_mid_tma<N>))
  } else {
    if (axis != 1) return cudaErrorInvalidValue;
    if (inv) {
      MBS_TMA_LAUNCH((k_strided_tma<N, 1, true>))
    } else {
      MBS_TMA_LAUNCH((k_strided_tma<N, 1, false>))
    }
  }
#undef MBS_TMA_LAUNCH
  return cudaGetLastError();
}

// Resident CTAs per SM of the TMA-fed pass for edge n (0: no such kernel).
int tma_max_ctas(int n, int kind) {
  int per_sm = 0;
  const int threads = 32 * warps_for(n);
#define MBS_TMA_OCC(N)                                                                                        \
  case N: {                                                                                                    \
    const size_t smem = (size_t)2 * N * 32 * sizeof(float2);                                                   \
    if (kind == 3) {                                                                                           \
      if (set_smem(k_mid_tma<N>, smem) ||                                                                     \
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mid_tma<N>, threads, smem) != cudaSuccess)  \
        per_sm = 0;                                                                                            \
    } else {                                                                                                   \
      if (set_smem(k_strided_tma<N, 1, false>, smem) ||                                                        \
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_strided_tma<N, 1, false>, threads, smem) !=  \
              cudaSuccess)                                                                                     \
        per_sm = 0;                                                                                            \
    }                                                                                                          \
    break;                                                                                                     \
  }
  switch (n) {
    MBS_TMA_SIZES(MBS_TMA_OCC)
    default:
      break;
  }
#undef MBS_TMA_OCC
  cudaGetLastError();
  return per_sm;
}

cudaError_t launch_strided_tma(int n, int axis, bool inv, const PassArgs& a, const CUtensorMap& tm, cudaStream_t st) {
  switch (n) {
#define MBS_TMA_CASE(n) \
  case n:               \
    return run_tma<n>(2, axis, inv, a, tm, st);
    MBS_TMA_SIZES(MBS_TMA_CASE)
#undef MBS_TMA_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_mid_tma(int n, const PassArgs& a, const CUtensorMap& tm, cudaStream_t st) {
  if (a.mode != MID_PROP && a.mode != MID_LSYM) return cudaErrorInvalidValue;
  switch (n) {
#define MBS_TMA_MID_CASE(n) \
  case n:                   \
    return run_tma<n>(3, 0, false, a, tm, st);
    MBS_TMA_SIZES(MBS_TMA_MID_CASE)
#undef MBS_TMA_MID_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace mbs
