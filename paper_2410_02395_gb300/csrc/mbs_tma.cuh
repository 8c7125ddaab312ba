// Strided FFT passes fed by the Tensor Memory Accelerator: the axis-1 pass and
// the axis-0 pass (forward transform, k-space multiplier, inverse transform).
//
// A tile is 32 consecutive axis-2 positions x one subdomain's n positions
// along the pass axis (one i0, or one i1). It is one box of the 3-D tensor map
// over the FFT buffer (dims N2, N1, N0; 8-byte elements), or two boxes of n/2
// when n is above 256 (a box is at most 256 long along an axis), so one or two
// cp.async.bulk.tensor copies bring the whole tile into shared memory as [n][32]
// (row e = element e of the 32 pencils; positions past N2 read as zeros).
// Persistent CTAs walk the tiles with two buffers: the copy of the next tile
// is in flight while the current one is transformed in place; the last radix
// stage stores straight to global memory. Every wait on an mbarrier is bounded
// and taken by one thread, which publishes the outcome to the whole CTA through
// shared memory before a barrier, so all threads leave together. Past the limit
// (PassArgs::tma_wait, in SM clock cycles; 0 -> about 2 s) the kernel marks the
// solver state (MBS_ETIMEOUT, done), waits with the full bound for the copies it
// still has in flight (this tile's and the next one's), so no copy writes the
// shared memory of a CTA that has left, and returns.
#pragma once
#include <cuda.h>

#include "mbs_passes.cuh"

namespace mbs {

constexpr long long kTmaWaitCycles = 4000000000ll;  // about 2 s at the GB300 clock

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounds below this poll with the non-blocking test_wait: try_wait may suspend
// the thread for a hardware-chosen time, which could outlast a short bound.
constexpr long long kTmaPollBelow = 100000;
// Wait for the phase of the given parity, giving up after `limit` SM clock cycles.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, long long limit) {
  const long long t0 = clock64();
  if (limit < kTmaPollBelow) {
    while (!mbar_test_wait(bar, parity))
      if (clock64() - t0 > limit) return false;
    return true;
  }
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(tm)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// Tile t of a pass along AXIS (1 or 0): axis-2 block ib, the other axis's index
// y (i0 for AXIS 1, i1 for AXIS 0), subdomain slot js of the launch's group.
struct TmaTile {
  int ib, y, js;
};
__device__ __forceinline__ TmaTile tma_tile(int t, int gx, int ny) {
  TmaTile r;
  r.ib = t % gx;
  const int q = t / gx;
  r.y = q % ny;
  r.js = q / ny;
  return r;
}

// Box length along the pass axis for edge n: n, or n/2 above 256.
__host__ __device__ constexpr int tma_box_len(int n) { return n > 256 ? n / 2 : n; }

template <int N, int AXIS>
__device__ __forceinline__ void tma_issue(const PassArgs& a, const CUtensorMap* tm, const TmaTile& tl, float2* buf,
                                          uint64_t* bar, unsigned bytes) {
  constexpr int BL = tma_box_len(N);
  static_assert(N % BL == 0 && N / BL <= 2, "one or two boxes per tile");
  const int j = a.subs[tl.js];
  mbar_expect_tx(bar, bytes);
#pragma unroll
  for (int h = 0; h < N / BL; h++) {
    if (AXIS == 1)
      tma_load_3d(buf + h * BL * 32, tm, tl.ib * 32, a.g.ax[1].off[j] + h * BL, tl.y, bar);
    else
      tma_load_3d(buf + h * BL * 32, tm, tl.ib * 32, tl.y, a.g.ax[0].off[j] + h * BL, bar);
  }
}

__device__ __forceinline__ void tma_fail(const PassArgs& a) {
  if (a.state) {
    DevState* s = const_cast<DevState*>(a.state);
    atomicCAS(&s->status, 0, (int)MBS_ETIMEOUT);
    s->done = 1;
  }
}

// The persistent loop shared by the axis-1 and axis-0 kernels; body(buf, tile)
// transforms one tile that sits in buf ([N][32]).
template <int N, int AXIS, class Body>
__device__ __forceinline__ void tma_tiles(const PassArgs& a, const CUtensorMap* tm, float2* dyn, uint64_t* bar,
                                          int* ok, Body body) {
  const int tid = threadIdx.x;
  const int gx = (int)((a.g.N2 + 31) / 32);
  const int ny = (int)(AXIS == 1 ? a.g.N0 : a.g.N1);
  const int ntiles = gx * ny * a.nsub;
  constexpr unsigned kBytes = N * 32 * sizeof(float2);
  const long long limit = a.tma_wait > 0 ? a.tma_wait : kTmaWaitCycles;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_proxy_async();
  }
  __syncthreads();
  int t = blockIdx.x;
  if (t < ntiles && tid == 0) tma_issue<N, AXIS>(a, tm, tma_tile(t, gx, ny), dyn, &bar[0], kBytes);
  for (int k = 0; t < ntiles; k++, t += gridDim.x) {
    const int b = k & 1;
    const int tn = t + gridDim.x;
    if (tid == 0) {
      if (tn < ntiles) tma_issue<N, AXIS>(a, tm, tma_tile(tn, gx, ny), dyn + (b ^ 1) * N * 32, &bar[b ^ 1], kBytes);
      const bool got = mbar_wait(&bar[b], (k >> 1) & 1, limit);
      if (!got) {
        tma_fail(a);
        // drain with the full bound: no copy may land after the CTA has left
        mbar_wait(&bar[b], (k >> 1) & 1, kTmaWaitCycles);
        if (tn < ntiles) mbar_wait(&bar[b ^ 1], ((k + 1) >> 1) & 1, kTmaWaitCycles);
      }
      *ok = got ? 1 : 0;
    }
    __syncthreads();  // every thread sees the same outcome of the wait
    if (!*ok) return;
    body(reinterpret_cast<float2(*)[32]>(dyn + b * N * 32), tma_tile(t, gx, ny));
    fence_proxy_async();  // this tile's generic-proxy accesses before the buffer's next copy
    __syncthreads();
  }
}

// Resident CTAs per SM asked of the register allocator: 32 warps per SM, or as
// many CTAs as two [N][32] buffers each leave room for in shared memory.
constexpr int tma_min_blocks(int n) {
  const int by_warps = 32 / warps_for(n) > 1 ? 32 / warps_for(n) : 1;
  const int by_smem = (200 * 1024) / (n * 32 * 8 * 2);
  const int m = by_warps < by_smem ? by_warps : by_smem;
  return m > 1 ? m : 1;
}

template <int N, int AXIS, bool INV>
__global__ void __launch_bounds__(32 * warps_for(N), tma_min_blocks(N)) k_strided_tma(const __grid_constant__ PassArgs a,
                                                                      const __grid_constant__ CUtensorMap tm) {
  constexpr int W = warps_for(N);
  extern __shared__ __align__(1024) float2 dyn[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int ok;
  if (a.state && a.state->done) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float2* K = a.K;
  tma_tiles<N, AXIS>(a, &tm, dyn, bar, &ok, [&](float2 (*sm)[32], const TmaTile& tl) {
    const int j = a.subs[tl.js];
    const long long i2 = (long long)tl.ib * 32 + lane;
    bool valid = i2 < a.g.N2;
    if (valid && a.active)
      valid = AXIS == 1 ? sub_active(a.active, a.g, a.tb.sub[0][tl.y], j, a.tb.sub[2][i2])
                        : sub_active(a.active, a.g, j, a.tb.sub[1][tl.y], a.tb.sub[2][i2]);
    long long base, stride;
    if (AXIS == 1) {
      base = (long long)tl.y * a.g.N1 * a.g.N2 + (long long)a.g.ax[1].off[j] * a.g.N2 + i2;
      stride = a.g.N2;
    } else {
      base = (long long)a.g.ax[0].off[j] * a.g.N1 * a.g.N2 + (long long)tl.y * a.g.N2 + i2;
      stride = a.g.N1 * a.g.N2;
    }
    if (valid) valid = grid_range_ok(a.g, base, base + (long long)(N - 1) * stride, BC_TMA);
    if (!__any_sync(0xffffffffu, valid)) return;  // no pencil of this tile is active: nothing to store
    auto sld = [&](int e) { return sm[e][lane]; };
    auto gst = [&](int e, float2 v) {
      if (valid) K[base + e * stride] = v;
    };
    fft_run<N, W, INV, false, 0, 1, true, false>(warp, lane, sm, a.tw, sld, gst);
  });
}

// Axis-0 pass fed by TMA: forward transform, the k-space multiplier of
// k_mid_turn (the propagator 1/(c(k0^2 - |p|^2) + 1) or the symbol of L, scaled
// by 1/(n0 n1 n2)) and the inverse transform of each tile, the last stage
// storing straight to global memory.
template <int N>
__global__ void __launch_bounds__(32 * warps_for(N), tma_min_blocks(N)) k_mid_tma(const __grid_constant__ PassArgs a,
                                                                 const __grid_constant__ CUtensorMap tm) {
  constexpr int W = warps_for(N);
  extern __shared__ __align__(1024) float2 dyn[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int ok;
  if (a.state && a.state->done) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float2* K = a.K;
  const float2 c = a.c, ck0 = a.ck0;
  const bool prop = a.mode == MID_PROP;
  // c is purely imaginary (Eq. c_scale2), so Re c(k0^2 - |p|^2) = Re(c k0^2) for every p
  const float dx = ck0.x, ex = dx + 1.f;
  tma_tiles<N, 0>(a, &tm, dyn, bar, &ok, [&](float2 (*sm)[32], const TmaTile& tl) {
    const int j = a.subs[tl.js];
    const int off0 = a.g.ax[0].off[j];
    const long long i1 = tl.y;
    const long long i2 = (long long)tl.ib * 32 + lane;
    bool valid = i2 < a.g.N2;
    const long long i2c = valid ? i2 : 0;
    if (valid && a.active) valid = sub_active(a.active, a.g, j, a.tb.sub[1][i1], a.tb.sub[2][i2c]);
    const long long base = (long long)off0 * a.g.N1 * a.g.N2 + i1 * a.g.N2 + i2;
    const long long stride = a.g.N1 * a.g.N2;
    if (valid) valid = grid_range_ok(a.g, base, base + (long long)(N - 1) * stride, BC_TMA);
    if (!__any_sync(0xffffffffu, valid)) return;  // no pencil of this tile is active: nothing to store
    const float pl = a.tb.p2[1][i1] + a.tb.p2[2][i2c];
    const float sc = a.tb.invn[0][off0] * a.tb.invn[1][i1] * a.tb.invn[2][i2c];
    const float* p20 = a.tb.p2[0] + off0;
    auto sld = [&](int e) { return sm[e][lane]; };
    auto gst = [&](int e, float2 v) {
      if (valid) K[base + e * stride] = v;
    };
    auto mul = [&](int e, float2 v) {
      const float p2 = __ldg(p20 + e) + pl;
      const float dy = fmaf(-c.y, p2, ck0.y);  // Im c(k0^2 - |p|^2)
      if (prop) {
        const float inv = sc * __frcp_rn(fmaf(ex, ex, dy * dy));
        return cmul(v, make_float2(ex * inv, -dy * inv));
      }
      return cmul(v, make_float2(dx * sc, dy * sc));
    };
    fft_fwd_mul_inv<N, W, true, false>(warp, lane, sm, a.tw, sld, gst, mul);
  });
}

}  // namespace mbs
