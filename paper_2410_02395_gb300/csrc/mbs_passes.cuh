// FFT pass kernels of one MBS iteration (Eq. wavesim_iter, Sec. 3.1).
//
//   rows_first  axis-2 forward transform; fuses u = B x + y - E x (medium,
//               source and edge corrections of V, Sec. 3.1 steps 3-5) into the
//               coalesced staged load.
//   strided     axis-1 forward / inverse transform (global loads straight into
//               the first radix stage, global stores from the last); the
//               TMA-fed form of this pass is in mbs_tma.cuh, the Bluestein
//               forms of all four passes in mbs_bluestein.cuh.
//   mid         axis-0 forward transform, k-space multiplier, axis-0 inverse
//               transform in one pass; the multiplier is the propagator
//               1/(c(k0^2 - |p|^2) + 1) (or the symbol of L), both scaled by
//               1/(n0 n1 n2) so the inverse transforms need no extra pass.
//   rows_last   axis-2 inverse transform; fuses e = x - w, the medium factor,
//               the Richardson update x <- x - alpha (I - V)(x - w) and the FP64
//               residual sum on voxels away from the subdomain edges.
//
// All transforms are per subdomain: a pass along axis d launches one grid per
// distinct subdomain size along d; grid.z (or .y) selects the subdomain.
#pragma once
#include <mutex>
#include <type_traits>
#include <unordered_map>

#include <cuda_bf16.h>

#include "mbs_fft.cuh"
#include "mbs_internal.h"
#include "mbs_reduce.cuh"

namespace mbs {

// Asynchronous 8-byte global -> shared copies (completed by cp_async_wait_all).
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Resident CTAs per SM asked of the register allocator: 32 warps per SM, i.e.
// at most 64 registers per thread (the tiles of that many CTAs fit in 228 KB).
// Edges of 17-20 warps (272 < n <= 320) ask for two CTAs per SM (40 warps, at
// most 48-56 registers): a few registers spill, but one CTA's loads overlap the
// other's transform; on the 1280^3 workload (320^3 subdomains) every pass got
// faster, 63.7 -> 52.7 ms per iteration (one CTA per SM had 78-96 registers).
__host__ __device__ constexpr int fft_min_blocks(int n) {
  return 32 / warps_for(n) > 1 ? 32 / warps_for(n) : (warps_for(n) <= 20 ? 2 : 1);
}

template <int N>
__device__ __forceinline__ float2 (*tile_of(float2* dyn))[kPad] {
  return reinterpret_cast<float2 (*)[kPad]>(dyn);
}

// ---------------------------------------------------------------------------
// Row tiles: 32 consecutive grid rows (i0, i1) x one axis-2 subdomain segment.
// Per-row data is set up by the first warp; the staged global traffic is
// issued in chunks of CH independent loads per thread (memory-level
// parallelism), then consumed.
// ---------------------------------------------------------------------------
// x <- x + d with x = hi + lo (lo two bfloat16): TwoSum of hi and (d + lo), the
// rounding error kept in lo, so that thousands of small updates do not lose
// the bits FP32 alone would drop.
__device__ __forceinline__ float two_sum(float a, float b, float& err) {
  const float s = a + b, bb = s - a;
  err = (a - (s - bb)) + (b - bb);
  return s;
}
__device__ __forceinline__ float2 acc_update(float2 hi, unsigned& lo, float2 d) {
  const __nv_bfloat162 l = *reinterpret_cast<const __nv_bfloat162*>(&lo);
  const float2 lf = __bfloat1622float2(l);
  float ex, ey;
  const float2 s = make_float2(two_sum(hi.x, d.x + lf.x, ex), two_sum(hi.y, d.y + lf.y, ey));
  const __nv_bfloat162 nl = __floats2bfloat162_rn(ex, ey);
  lo = *reinterpret_cast<const unsigned*>(&nl);
  return s;
}

// A row tile: 32 consecutive grid rows rho = i0*N1 + i1 from rho0, one axis-2
// segment starting at off2. Row r starts at (rho0 + r) * N2 + off2; its flags
// are bits of three 32-bit masks built by the first warp with ballots:
// valid (inside the grid), layer (i0 or i1 inside an axis-0/1 boundary layer)
// and src (inside the source box's rows).
struct RowTile {
  long long base0;  // rho0 * N2 + off2
  long long N2;
  unsigned valid, layer, src;
  __device__ __forceinline__ long long base(int r) const { return base0 + (long long)r * N2; }
  __device__ __forceinline__ bool ok(int r) const { return (valid >> r) & 1u; }
  __device__ __forceinline__ bool lay(int r) const { return (layer >> r) & 1u; }
  __device__ __forceinline__ bool in_src(int r) const { return (src >> r) & 1u; }
};

// A CTA's coordinates in the grid of one plan's launch: the block itself in a
// single-plan launch, or the plan-local block of a batched launch (several
// plans' passes of the same edge in one grid, grid.z selecting the plan).
struct Blk {
  unsigned x, y, z, nx, ny;
};
__device__ __forceinline__ Blk blk_here() { return Blk{blockIdx.x, blockIdx.y, blockIdx.z, gridDim.x, gridDim.y}; }

// Rows of inactive subdomains (subdomain activation) count as outside the grid.
__device__ __forceinline__ RowTile setup_rows(unsigned* masks, const PassArgs& a, int off2, int j2, unsigned bx) {
  const int tid = threadIdx.x;
  const long long rho0 = (long long)bx * 32;
  if (tid < 32) {
    const long long rows = a.g.N0 * a.g.N1;
    const long long rho = rho0 + tid;
    bool v = false, l = false, sr = false;
    if (rho < rows) {
      const long long i0 = rho / a.g.N1, i1 = rho - i0 * a.g.N1;
      v = sub_active(a.active, a.g, a.tb.sub[0][i0], a.tb.sub[1][i1], j2) &&
          grid_range_ok(a.g, rho * a.g.N2, rho * a.g.N2 + a.g.N2 - 1, BC_ROWS);  // the row's voxels
      l = a.tb.shell[0][i0] | a.tb.shell[1][i1];
      sr = a.S && i0 >= a.sbox[0] && i0 < a.sbox[1] && i1 >= a.sbox[2] && i1 < a.sbox[3];
    }
    const unsigned mv = __ballot_sync(0xffffffffu, v), ml = __ballot_sync(0xffffffffu, l),
                   ms = __ballot_sync(0xffffffffu, sr);
    if (tid == 0) {
      masks[0] = mv;
      masks[1] = ml;
      masks[2] = ms;
    }
  }
  __syncthreads();
  RowTile t;
  t.N2 = a.g.N2;
  t.base0 = rho0 * a.g.N2 + off2;
  t.valid = masks[0];
  t.layer = masks[1];
  t.src = masks[2];
  return t;
}

// Element e of an axis-2 segment of length N lies in a boundary layer of that axis.
template <int N>
__device__ __forceinline__ bool in_layer2(const PassArgs& a, int e) {
  return a.g.ax[2].a > 0 && (e < a.g.t || e >= N - a.g.t);
}

// Element (r, e) of a row tile (32 rows x N) handled by thread tid at step k.
// When NT divides 32 N and N divides NT (NT = 2N for every N >= 64 that is a
// multiple of 16), each thread keeps one element index e and walks rows
// r, r + NT/N, ...; the rows stay below 32 for k < 32 N / NT.
// Staged voxels per thread and chunk in the row passes: CH loads of each
// array in flight per thread. Edges above 256 run two CTAs per SM with at most
// 48 registers, where the first pass (x, B and E x staged) spills less with a
// chunk of 4: on the 1280^3 workload it went from 11.4 to 10.7 ms, while the
// last pass (only the FFT buffer staged) went from 12.5 to 14.3 ms and keeps 8.
__host__ __device__ constexpr int row_chunk(int pert, int ch) { return pert < ch ? pert : ch; }

template <int N, int NT>
struct TileMap {
  static constexpr bool fixed = (NT % N) == 0 && ((32 * N) % NT) == 0;
  __device__ __forceinline__ static bool at(int tid, int k, int& r, int& e) {
    if constexpr (fixed) {
      r = tid / N + k * (NT / N);
      e = tid % N;
      return r < 32;
    } else {
      const int idx = tid + k * NT;
      r = idx / N;
      e = idx - r * N;
      return idx < 32 * N;
    }
  }
};

// ---------------------------------------------------------------------------
// Axis-2 forward pass with the fused medium/source/correction prologue:
// u = B x + y - E x (FIRST_ITER) or u = x (FIRST_PLAIN), then the transform.
// ---------------------------------------------------------------------------
// TC: compile-time truncation width of the fused axis-2 corrections (0: runtime t).
template <int N, int TC>
__device__ __forceinline__ void rows_first_body(const PassArgs& a, const Blk& bk) {
  constexpr int W = warps_for(N);
  constexpr int NT = 32 * W;
  constexpr int PERT = (32 * N + NT - 1) / NT;
  constexpr int CH = row_chunk(PERT, N > 256 ? 4 : 8);
  extern __shared__ float2 dyn[];
  float2 (*sm)[kPad] = tile_of<N>(dyn);
  __shared__ unsigned masks[3];
  if (a.state && a.state->done) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int j2 = a.subs[bk.y];
  const int off2 = a.g.ax[2].off[j2];
  const RowTile rt = setup_rows(masks, a, off2, j2, bk.x);
  if (rt.valid == 0u) return;  // every row of the tile inside inactive subdomains
  const bool iter = a.mode == FIRST_ITER;
  // The tile's 32 rows x N elements lie within 32 * N2 <= 2^18 voxels of its
  // origin, so in-tile offsets are 32-bit.
  const float2* __restrict__ Xt = a.X + rt.base0;
  const float2* __restrict__ Bt = a.B + rt.base0;
  float2* Kt = a.K + rt.base0;
  const unsigned n2 = (unsigned)a.g.N2;
  // Axis-2 edge corrections of x on this segment (Sec. 3.1 steps 1-5) need the
  // segment's own first/last t voxels and the neighbours' adjacent t voxels of
  // every row: fetched asynchronously into shared memory while the tile loads.
  const bool e2 = iter && a.fuse_e2 && a.g.ax[2].a > 0;
  const int t = TC > 0 ? TC : a.g.t;
  const AxisDesc& ax2 = a.g.ax[2];
  const int L = ax2.left[j2], R = ax2.right[j2];
  // xe[k][r] (pitch 33): k < t own first t, < 2t own last t, < 3t left's last t,
  // < 4t right's first t of row r. c is purely imaginary and W real, so cW = i w
  // with w = Im(cW) real: wsm[m] = w at column - row = m - (t - 1).
  float2* xe = dyn + N * kPad;
  float* wsm = reinterpret_cast<float*>(xe + 4 * t * kPad);
  if (e2) {
    for (int idx = tid; idx < 32 * 4 * t; idx += NT) {
      const int r = idx / (4 * t), k = idx - r * 4 * t;  // consecutive threads: one row's values
      long long pos = -1;
      if (rt.ok(r)) {
        if (k < t) pos = off2 + k;
        else if (k < 2 * t) pos = off2 + N - t + (k - t);
        else if (k < 3 * t) pos = L >= 0 ? ax2.off[L] + ax2.n[L] - t + (k - 2 * t) : -1;
        else pos = R >= 0 ? ax2.off[R] + (k - 3 * t) : -1;
      }
      if (pos >= 0) cp_async8(xe + k * kPad + r, Xt + ((long long)r * n2 + (pos - off2)));
      else xe[k * kPad + r] = make_float2(0.f, 0.f);
    }
    cp_async_commit();
    if (tid < 2 * t - 1) {
      const int m = tid, aa = m < t - 1 ? t - 1 - m : 0, bb = aa + m - (t - 1);
      wsm[m] = a.cW[aa * t + bb].y;
    }
  }
  // Tiles with all 32 rows inside the grid and none in the source box (almost
  // all) take a loop without those per-voxel tests.
  auto load = [&](auto full_tile) {
    constexpr bool FULL = decltype(full_tile)::value;
    if constexpr (FULL && N > 256) {
      if (iter) {
        // Edges above 256 (two CTAs per SM, at most 48 registers): x goes straight
        // into the tile by cp.async, which holds no registers while the copies
        // fly, so B and the E x of the layer rows can be staged 8 per thread;
        // each thread then combines the voxels it copied itself, which needs no
        // barrier. 320^3: 0.195 -> 0.186 ms per first pass (at 128, where more
        // registers are free, the register-staged loop below was faster).
        constexpr int CHB = row_chunk(PERT, 8);
        for (int k = 0; k < PERT; k++) {
          int r, e;
          if (TileMap<N, NT>::at(tid, k, r, e)) cp_async8(&sm[e][r], Xt + ((unsigned)r * n2 + (unsigned)e));
        }
        cp_async_commit();
        for (int k0 = 0; k0 < PERT; k0 += CHB) {
          float2 bv[CHB], cv[CHB];
#pragma unroll
          for (int c = 0; c < CHB; c++) {
            int r, e;
            bv[c] = cv[c] = make_float2(0.f, 0.f);
            if (TileMap<N, NT>::at(tid, k0 + c, r, e)) {
              const unsigned o = (unsigned)r * n2 + (unsigned)e;
              bv[c] = __ldg(Bt + o);
              if (rt.lay(r) || (!a.fuse_e2 && in_layer2<N>(a, e))) cv[c] = Kt[o];  // E x from the correction kernels
            }
          }
          if (k0 == 0) cp_async_wait_all();
#pragma unroll
          for (int c = 0; c < CHB; c++) {
            int r, e;
            if (TileMap<N, NT>::at(tid, k0 + c, r, e)) sm[e][r] = csub(cmul(bv[c], sm[e][r]), cv[c]);
          }
        }
        return;
      }
    }
    for (int k0 = 0; k0 < PERT; k0 += CH) {
      float2 xv[CH], bv[CH], cv[CH];
#pragma unroll
      for (int c = 0; c < CH; c++) {
        int r, e;
        const bool ok = TileMap<N, NT>::at(tid, k0 + c, r, e);
        xv[c] = bv[c] = cv[c] = make_float2(0.f, 0.f);
        if (ok && (FULL || rt.ok(r))) {
          const unsigned o = (unsigned)r * n2 + (unsigned)e;
          xv[c] = __ldg(Xt + o);
          if (iter) {
            bv[c] = __ldg(Bt + o);
            if (rt.lay(r) || (!a.fuse_e2 && in_layer2<N>(a, e))) cv[c] = Kt[o];  // E x from the correction kernels
          }
        }
      }
#pragma unroll
      for (int c = 0; c < CH; c++) {
        int r, e;
        if (TileMap<N, NT>::at(tid, k0 + c, r, e)) {
          float2 u = xv[c];
          if (iter && (FULL || rt.ok(r))) {
            u = csub(cmul(bv[c], xv[c]), cv[c]);
            if (!FULL) {
              const long long i2 = off2 + e;
              if (rt.in_src(r) && i2 >= a.sbox[4] && i2 < a.sbox[5]) u = cadd(u, cmul(a.mc, a.S[rt.base(r) + e]));
            }
          }
          sm[e][r] = u;
        }
      }
    }
  };
  const bool full_tile = rt.valid == 0xffffffffu && rt.src == 0u;
  if (full_tile)
    load(std::true_type{});
  else
    load(std::false_type{});
  if (e2) {
    // Warp w corrects tile elements q(k) for k = w, w + W, ... < 2t, lane = row:
    //   first t: u -= sum_b cW[b][q]  (x_left[n_l-t+b] - x[n-t+b])
    //   last t:  u -= sum_b cW[aa][b] (x_right[b]      - x[b])
    // with cW = i w: sum_b cW d_b = i v, v = sum_b w_b d_b.
    cp_async_wait_all();
    __syncthreads();
    for (int k = warp; k < 2 * t; k += W) {
      const int q = k < t ? k : N - t + (k - t);
      if (k >= t && q < t) continue;  // also in the first range (N < 2t): done there
      const float2* xr = xe + lane;
      float vx = 0.f, vy = 0.f;
      if constexpr (TC > 0) {
        if (q < TC) {
#pragma unroll
          for (int b = 0; b < TC; b++) {
            const float w = wsm[q - b + TC - 1];
            const float2 d = csub(xr[(2 * TC + b) * kPad], xr[(TC + b) * kPad]);
            vx = fmaf(w, d.x, vx);
            vy = fmaf(w, d.y, vy);
          }
        }
        if (q >= N - TC) {
          const int aa = q - (N - TC);
#pragma unroll
          for (int b = 0; b < TC; b++) {
            const float w = wsm[b - aa + TC - 1];
            const float2 d = csub(xr[(3 * TC + b) * kPad], xr[b * kPad]);
            vx = fmaf(w, d.x, vx);
            vy = fmaf(w, d.y, vy);
          }
        }
      } else {
        if (q < t) {
          for (int b = 0; b < t; b++) {
            const float w = wsm[q - b + t - 1];
            const float2 d = csub(xr[(2 * t + b) * kPad], xr[(t + b) * kPad]);
            vx = fmaf(w, d.x, vx);
            vy = fmaf(w, d.y, vy);
          }
        }
        if (q >= N - t) {
          const int aa = q - (N - t);
          for (int b = 0; b < t; b++) {
            const float w = wsm[b - aa + t - 1];
            const float2 d = csub(xr[(3 * t + b) * kPad], xr[b * kPad]);
            vx = fmaf(w, d.x, vx);
            vy = fmaf(w, d.y, vy);
          }
        }
      }
      float2 u = sm[q][lane];
      u.x += vy;  // u -= i v
      u.y -= vx;
      sm[q][lane] = u;
    }
  }
  if constexpr (N > 1) {
    __syncthreads();
    auto sld = [&](int e) { return sm[e][lane]; };
    auto sst = [&](int e, float2 v) { sm[e][lane] = v; };
    fft_run<N, W, false, false, 0, 1, true, true>(warp, lane, sm, a.tw, sld, sst);
  }
  __syncthreads();
  for (int k0 = 0; k0 < PERT; k0++) {
    int r, e;
    if (TileMap<N, NT>::at(tid, k0, r, e) && rt.ok(r)) Kt[(unsigned)r * n2 + (unsigned)e] = sm[e][r];
  }
}

// Row tiles of one plan's pass: (N0 N1 + 31) / 32 along x, the subdomain slots along y.
__device__ __forceinline__ unsigned row_blocks(const PassArgs& a) { return (unsigned)((a.g.N0 * a.g.N1 + 31) / 32); }

template <int N, int TC>
__global__ void __launch_bounds__(32 * warps_for(N), fft_min_blocks(N)) k_rows_first(const __grid_constant__ PassArgs a) {
  rows_first_body<N, TC>(a, blk_here());
}

// Batched form: plan blockIdx.z of `d`; blocks past that plan's extent leave at once.
template <int N, int TC>
__global__ void __launch_bounds__(32 * warps_for(N), fft_min_blocks(N)) k_rows_first_batch(const PassArgs* __restrict__ d) {
  __shared__ PassArgs a;
  const PassArgs& ga = d[blockIdx.z];
  const unsigned nx = row_blocks(ga), ny = (unsigned)ga.nsub;
  if (blockIdx.x >= nx || blockIdx.y >= ny) return;
  stage_args(&a, &ga);
  rows_first_body<N, TC>(a, Blk{blockIdx.x, blockIdx.y, 0u, nx, ny});
}

// ---------------------------------------------------------------------------
// Axis-2 inverse pass with the fused update epilogue (Eq. wavesim_iter):
// e = x - w; away from the boundary layers r = B e, x <- x - alpha r and the
// FP64 |r|^2; on the layers e is stored for the correction step.
// ---------------------------------------------------------------------------
template <int N, bool RES>
__device__ __forceinline__ void rows_last_body(const PassArgs& a, const Blk& bk) {
  constexpr int W = warps_for(N);
  constexpr int NT = 32 * W;
  constexpr int PERT = (32 * N + NT - 1) / NT;
  constexpr int CH = row_chunk(PERT, RES ? 4 : 8);  // fewer staged voxels when x is staged too
  extern __shared__ float2 dyn[];
  float2 (*sm)[kPad] = tile_of<N>(dyn);
  __shared__ unsigned masks[3];
  __shared__ double red[32];
  if (a.state && a.state->done) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int j2 = a.subs[bk.y];
  const int off2 = a.g.ax[2].off[j2];
  const RowTile rt = setup_rows(masks, a, off2, j2, bk.x);
  // |r|^2 of this thread's (at most N/W) voxels in FP32, then FP64 across threads
  // and blocks: GB300's FP64 rate is too low for a per-voxel FP64 accumulation.
  float acc = 0.f;
  if (rt.valid != 0u) {  // else every row lies in inactive subdomains: only the partial (zero) is stored
    float2* K = a.K;
    for (int k0 = 0; k0 < PERT; k0 += CH) {
      float2 kv[CH];
#pragma unroll
      for (int c = 0; c < CH; c++) {
        int r, e;
        kv[c] = make_float2(0.f, 0.f);
        if (TileMap<N, NT>::at(tid, k0 + c, r, e) && rt.ok(r)) kv[c] = K[rt.base(r) + e];
      }
#pragma unroll
      for (int c = 0; c < CH; c++) {
        int r, e;
        if (TileMap<N, NT>::at(tid, k0 + c, r, e)) sm[e][r] = kv[c];
      }
    }
    if constexpr (N > 1) {
      __syncthreads();
      auto sld = [&](int e) { return sm[e][lane]; };
      auto sst = [&](int e, float2 v) { sm[e][lane] = v; };
      fft_run<N, W, true, false, 0, 1, true, true>(warp, lane, sm, a.tw, sld, sst);
    }
    __syncthreads();
    const int mode = a.mode;
    const float2* X = a.X;
    const float2* __restrict__ B = a.B;
    const bool need_x = mode != LAST_PLAIN;
    const bool need_b = mode != LAST_PLAIN;
    constexpr int CR = RES ? CH : 1;  // the residual form also stages x (high and low words)
    for (int k0 = 0; k0 < PERT; k0 += CH) {
      float2 xv[CH], bv[CH], sv[CR];
      unsigned lv[CR];
#pragma unroll
      for (int c = 0; c < CH; c++) {
        int r, e;
        const bool ok = TileMap<N, NT>::at(tid, k0 + c, r, e);
        xv[c] = make_float2(0.f, 0.f);
        bv[c] = make_float2(0.f, 0.f);
        if constexpr (RES) {
          sv[c] = make_float2(0.f, 0.f);
          lv[c] = 0u;
        }
        if (ok) {
          if (rt.ok(r)) {
            const long long gi = rt.base(r) + e;
            if (need_x) xv[c] = X[gi];
            if (need_b) bv[c] = __ldg(B + gi);
            if constexpr (RES) {
              sv[c] = a.Xs[gi];
              lv[c] = a.Xlo[gi];
            }
          }
        }
      }
#pragma unroll
      for (int c = 0; c < CH; c++) {
        int r, e;
        if (!TileMap<N, NT>::at(tid, k0 + c, r, e) || !rt.ok(r)) continue;
        const long long gi = rt.base(r) + e;
        const float2 w = sm[e][r];
        if (mode == LAST_PLAIN) {
          a.Xout[gi] = w;
        } else if (mode == LAST_AOUT) {
          a.Xout[gi] = cadd(w, cmul(make_float2(1.f - bv[c].x, -bv[c].y), xv[c]));
        } else if (RES) {
          if constexpr (RES) {
            // residual form: xv = r'_n, e = r' - w, r'_{n+1} = r' - alpha (I - V) e,
            // x_{n+1} = x_n - alpha r'_n; |r'_n|^2 of every voxel is summed here
            acc = fmaf(xv[c].x, xv[c].x, fmaf(xv[c].y, xv[c].y, acc));
            a.Xs[gi] = acc_update(sv[c], lv[c], make_float2(-a.alpha * xv[c].x, -a.alpha * xv[c].y));
            a.Xlo[gi] = lv[c];
            const float2 ee = csub(xv[c], w);
            if (rt.lay(r) || in_layer2<N>(a, e)) {
              a.E[gi] = ee;  // r' on the layers is finished by the layer update
            } else {
              const float2 rr = cmul(bv[c], ee);
              a.Xout[gi] = make_float2(fmaf(-a.alpha, rr.x, xv[c].x), fmaf(-a.alpha, rr.y, xv[c].y));
            }
          }
        } else {
          const float2 ee = csub(xv[c], w);
          if (rt.lay(r) || in_layer2<N>(a, e)) {
            a.E[gi] = ee;  // finished by the layer update once all of e is known
          } else {
            const float2 rr = cmul(bv[c], ee);
            acc = fmaf(rr.x, rr.x, fmaf(rr.y, rr.y, acc));
            a.Xout[gi] = (mode == LAST_ITER) ? make_float2(fmaf(-a.alpha, rr.x, xv[c].x), fmaf(-a.alpha, rr.y, xv[c].y))
                                             : make_float2(-rr.x, -rr.y);
          }
        }
      }
    }
  }
  if (a.partials) {
    const double s = block_sum((double)acc, red);
    finish_block_at(Finish{a.partials, a.slot0, a.n_total, a.fin, a.hist}, s, red, bk.x + bk.nx * bk.y,
                    bk.nx * bk.ny);
  }
}

template <int N, bool RES>
__global__ void __launch_bounds__(32 * warps_for(N), fft_min_blocks(N)) k_rows_last(const __grid_constant__ PassArgs a) {
  rows_last_body<N, RES>(a, blk_here());
}

template <int N, bool RES>
__global__ void __launch_bounds__(32 * warps_for(N), fft_min_blocks(N)) k_rows_last_batch(const PassArgs* __restrict__ d) {
  __shared__ PassArgs a;
  const PassArgs& ga = d[blockIdx.z];
  const unsigned nx = row_blocks(ga), ny = (unsigned)ga.nsub;
  if (blockIdx.x >= nx || blockIdx.y >= ny) return;
  stage_args(&a, &ga);
  rows_last_body<N, RES>(a, Blk{blockIdx.x, blockIdx.y, 0u, nx, ny});
}

// ---------------------------------------------------------------------------
// Axis-1 / axis-0 transform of a tile of 32 consecutive axis-2 positions.
// ---------------------------------------------------------------------------
// bk: x the block of 32 axis-2 positions, y the index along the other axis
// (i0 for AXIS 1, i1 for AXIS 0), z the subdomain slot.
template <int N, int AXIS, bool INV>
__device__ __forceinline__ void strided_body(const PassArgs& a, const Blk& bk) {
  constexpr int W = warps_for(N);
  extern __shared__ float2 dyn[];
  float2 (*sm)[kPad] = tile_of<N>(dyn);
  if (a.state && a.state->done) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = a.subs[bk.z];
  const long long i2 = (long long)bk.x * 32 + lane;
  bool valid = i2 < a.g.N2;
  if (valid && a.active)
    valid = AXIS == 1 ? sub_active(a.active, a.g, a.tb.sub[0][bk.y], j, a.tb.sub[2][i2])
                      : sub_active(a.active, a.g, j, a.tb.sub[1][bk.y], a.tb.sub[2][i2]);
  long long base, stride;
  if (AXIS == 1) {
    base = (long long)bk.y * a.g.N1 * a.g.N2 + (long long)a.g.ax[1].off[j] * a.g.N2 + i2;
    stride = a.g.N2;
  } else {
    base = (long long)a.g.ax[0].off[j] * a.g.N1 * a.g.N2 + (long long)bk.y * a.g.N2 + i2;
    stride = a.g.N1 * a.g.N2;
  }
  if (valid) valid = grid_range_ok(a.g, base, base + (long long)(N - 1) * stride, BC_STRIDED);
  if (!__any_sync(0xffffffffu, valid)) return;  // the same 32 pencils in every warp
  float2* K = a.K;
  auto gld = [&](int e) { return valid ? K[base + e * stride] : make_float2(0.f, 0.f); };
  auto gst = [&](int e, float2 v) {
    if (valid) K[base + e * stride] = v;
  };
  if constexpr (N > 1) fft_run<N, W, INV, false, 0, 1, false, false>(warp, lane, sm, a.tw, gld, gst);
}

template <int N, int AXIS, bool INV>
__global__ void __launch_bounds__(32 * warps_for(N), fft_min_blocks(N)) k_strided(const __grid_constant__ PassArgs a) {
  strided_body<N, AXIS, INV>(a, blk_here());
}

// Batched form: grid.y folds (index along the other axis, subdomain slot).
template <int N, int AXIS, bool INV>
__global__ void __launch_bounds__(32 * warps_for(N), fft_min_blocks(N)) k_strided_batch(const PassArgs* __restrict__ d) {
  __shared__ PassArgs a;
  const PassArgs& ga = d[blockIdx.z];
  const unsigned gx = (unsigned)((ga.g.N2 + 31) / 32), ny = (unsigned)(AXIS == 1 ? ga.g.N0 : ga.g.N1);
  if (blockIdx.x >= gx || blockIdx.y >= ny * (unsigned)ga.nsub) return;
  stage_args(&a, &ga);
  strided_body<N, AXIS, INV>(a, Blk{blockIdx.x, blockIdx.y % ny, blockIdx.y / ny, gx, ny});
}

// ---------------------------------------------------------------------------
// Axis-0 pass: forward transform, multiplier, inverse transform.
// ---------------------------------------------------------------------------
struct MidPencil {
  long long base, stride;
  bool valid;
  float pl;     // p1^2 + p2^2 of this pencil
  float sc;     // 1 / (n0 n1 n2)
  const float* p20;
};

// bk: x the block of 32 axis-2 positions, y the index i1, z the subdomain slot.
__device__ __forceinline__ MidPencil mid_pencil(const PassArgs& a, const Blk& bk) {
  MidPencil m;
  const int lane = threadIdx.x & 31;
  const int j = a.subs[bk.z];
  const int off0 = a.g.ax[0].off[j];
  const long long i1 = bk.y;
  const long long i2 = (long long)bk.x * 32 + lane;
  m.valid = i2 < a.g.N2;
  const long long i2c = m.valid ? i2 : 0;
  if (m.valid && a.active) m.valid = sub_active(a.active, a.g, j, a.tb.sub[1][i1], a.tb.sub[2][i2c]);
  m.base = (long long)off0 * a.g.N1 * a.g.N2 + i1 * a.g.N2 + i2;
  m.stride = a.g.N1 * a.g.N2;
  if (m.valid)
    m.valid = grid_range_ok(a.g, m.base, m.base + (long long)(a.g.ax[0].n[j] - 1) * m.stride, BC_MID);
  m.pl = a.tb.p2[1][i1] + a.tb.p2[2][i2c];
  m.sc = a.tb.invn[0][off0] * a.tb.invn[1][i1] * a.tb.invn[2][i2c];
  m.p20 = a.tb.p2[0] + off0;
  return m;
}

// Propagator (L + I)^-1 = 1/(c(k0^2 - |p|^2) + 1) (Sec. 2) or the symbol of L,
// c(k0^2 - |p|^2) (Eq. L-convolution), times 1/(n0 n1 n2).
template <int N>
__device__ __forceinline__ void mid_turn_body(const PassArgs& a, const Blk& bk) {
  constexpr int W = warps_for(N);
  extern __shared__ float2 dyn[];
  float2 (*sm)[kPad] = tile_of<N>(dyn);
  if (a.state && a.state->done) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const MidPencil m = mid_pencil(a, bk);
  if (!__any_sync(0xffffffffu, m.valid)) return;  // the same 32 pencils in every warp
  const float2 c = a.c, ck0 = a.ck0;
  float2* K = a.K;
  auto gld = [&](int e) { return m.valid ? K[m.base + e * m.stride] : make_float2(0.f, 0.f); };
  auto gst = [&](int e, float2 v) {
    if (m.valid) K[m.base + e * m.stride] = v;
  };
  const bool prop = a.mode == MID_PROP;
  // c is purely imaginary (Eq. c_scale2), so Re c(k0^2 - |p|^2) = Re(c k0^2) for every p
  const float dx = ck0.x, ex = dx + 1.f;
  auto mul = [&](int e, float2 v) {
    const float p2 = __ldg(m.p20 + e) + m.pl;
    const float dy = fmaf(-c.y, p2, ck0.y);  // Im c(k0^2 - |p|^2)
    if (prop) {
      const float inv = m.sc * __frcp_rn(fmaf(ex, ex, dy * dy));
      return cmul(v, make_float2(ex * inv, -dy * inv));
    }
    return cmul(v, make_float2(dx * m.sc, dy * m.sc));
  };
  if constexpr (N == 1) {
    if (m.valid) K[m.base] = mul(0, K[m.base]);
  } else {
    fft_fwd_mul_inv<N, W, false, false>(warp, lane, sm, a.tw, gld, gst, mul);
  }
}

template <int N, int MIN_BLOCKS>
__global__ void __launch_bounds__(32 * warps_for(N), MIN_BLOCKS) k_mid_turn(const __grid_constant__ PassArgs a) {
  mid_turn_body<N>(a, blk_here());
}

template <int N, int MIN_BLOCKS>
__global__ void __launch_bounds__(32 * warps_for(N), MIN_BLOCKS) k_mid_turn_batch(const PassArgs* __restrict__ d) {
  __shared__ PassArgs a;
  const PassArgs& ga = d[blockIdx.z];
  const unsigned gx = (unsigned)((ga.g.N2 + 31) / 32), ny = (unsigned)ga.g.N1;
  if (blockIdx.x >= gx || blockIdx.y >= ny * (unsigned)ga.nsub) return;
  stage_args(&a, &ga);
  mid_turn_body<N>(a, Blk{blockIdx.x, blockIdx.y % ny, blockIdx.y / ny, gx, ny});
}

// Forward-only (MID_FWD) or scaled inverse-only (MID_INV) axis-0 transform.
template <int N>
__global__ void __launch_bounds__(32 * warps_for(N), fft_min_blocks(N)) k_mid_plain(const __grid_constant__ PassArgs a) {
  constexpr int W = warps_for(N);
  extern __shared__ float2 dyn[];
  float2 (*sm)[kPad] = tile_of<N>(dyn);
  if (a.state && a.state->done) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const MidPencil m = mid_pencil(a, blk_here());
  float2* K = a.K;
  auto gst = [&](int e, float2 v) {
    if (m.valid) K[m.base + e * m.stride] = v;
  };
  if (a.mode == MID_FWD) {
    auto gld = [&](int e) { return m.valid ? K[m.base + e * m.stride] : make_float2(0.f, 0.f); };
    if constexpr (N > 1) fft_run<N, W, false, false, 0, 1, false, false>(warp, lane, sm, a.tw, gld, gst);
  } else {
    auto gls = [&](int e) { return m.valid ? cscale(K[m.base + e * m.stride], m.sc) : make_float2(0.f, 0.f); };
    if constexpr (N > 1) {
      fft_run<N, W, true, false, 0, 1, false, false>(warp, lane, sm, a.tw, gls, gst);
    } else {
      if (m.valid) K[m.base] = gls(0);
    }
  }
}

// ---------------------------------------------------------------------------
// Launch helpers for one size.
// ---------------------------------------------------------------------------
inline size_t tile_bytes(int n) { return (size_t)n * kPad * sizeof(float2); }

// Resident CTAs per SM asked of the register allocator for the axis-0 pass
// (forward + multiplier + inverse): as many as the other passes. At n = 128 this
// spills a few registers but runs 4 % faster than 3 CTAs per SM without spills
// (measured on the 256^3 workload).
constexpr int mid_min_blocks(int n) { return fft_min_blocks(n); }

// Per kernel (keyed by its address): above 48 KB, the dynamic shared-memory
// opt-in for the largest size requested so far. The L1/shared split is left to
// the CUDA driver: these kernels read twiddles, tables and B through L1.
struct KernelAttrs {
  std::mutex mu;
  std::unordered_map<const void*, size_t> smem;     // opted-in dynamic bytes
};
inline KernelAttrs& kernel_attrs() {
  static KernelAttrs k;
  return k;
}

template <class K>
inline cudaError_t set_smem(K kernel, size_t bytes) {
  KernelAttrs& ka = kernel_attrs();
  std::lock_guard<std::mutex> lk(ka.mu);
  const void* key = (const void*)kernel;
  auto it = ka.smem.find(key);
  if (it != ka.smem.end() && it->second >= bytes) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  if (bytes > 48 * 1024)
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) ka.smem[key] = bytes;
  return e;
}

template <int N>
cudaError_t run_size(int kind, int axis, bool inv, const PassArgs& a, int nrow_blocks, cudaStream_t st) {
  const size_t sm = tile_bytes(N);
  const dim3 blk(32 * warps_for(N));
  cudaError_t e = cudaSuccess;
  const unsigned gx = (unsigned)((a.g.N2 + 31) / 32);
  switch (kind) {
    case 0: {
      // tile, then the axis-2 edge values [4t][33] and the 2t-1 Toeplitz weights (floats)
      const size_t edge = a.g.ax[2].a > 0 ? ((size_t)4 * a.g.t * kPad + a.g.t) * sizeof(float2) : 0;
      const size_t smax = sm + ((size_t)4 * kMaxT * kPad + kMaxT) * sizeof(float2);
      if (a.g.t == 8) {
        e = set_smem(k_rows_first<N, 8>, smax);
        if (e) return e;
        k_rows_first<N, 8><<<dim3(nrow_blocks, a.nsub), blk, sm + edge, st>>>(a);
      } else {
        e = set_smem(k_rows_first<N, 0>, smax);
        if (e) return e;
        k_rows_first<N, 0><<<dim3(nrow_blocks, a.nsub), blk, sm + edge, st>>>(a);
      }
      break;
    }
    case 1: {
      if (a.mode == LAST_RES) {
        e = set_smem(k_rows_last<N, true>, sm);
        if (e) return e;
        k_rows_last<N, true><<<dim3(nrow_blocks, a.nsub), blk, sm, st>>>(a);
      } else {
        e = set_smem(k_rows_last<N, false>, sm);
        if (e) return e;
        k_rows_last<N, false><<<dim3(nrow_blocks, a.nsub), blk, sm, st>>>(a);
      }
      break;
    }
    case 2: {
      if (axis == 1) {
        if (inv) {
          e = set_smem(k_strided<N, 1, true>, sm);
          if (e) return e;
          k_strided<N, 1, true><<<dim3(gx, (unsigned)a.g.N0, a.nsub), blk, sm, st>>>(a);
        } else {
          e = set_smem(k_strided<N, 1, false>, sm);
          if (e) return e;
          k_strided<N, 1, false><<<dim3(gx, (unsigned)a.g.N0, a.nsub), blk, sm, st>>>(a);
        }
      } else {
        if (inv) {
          e = set_smem(k_strided<N, 0, true>, sm);
          if (e) return e;
          k_strided<N, 0, true><<<dim3(gx, (unsigned)a.g.N1, a.nsub), blk, sm, st>>>(a);
        } else {
          e = set_smem(k_strided<N, 0, false>, sm);
          if (e) return e;
          k_strided<N, 0, false><<<dim3(gx, (unsigned)a.g.N1, a.nsub), blk, sm, st>>>(a);
        }
      }
      break;
    }
    case 3: {
      const dim3 grd(gx, (unsigned)a.g.N1, a.nsub);
      if (a.mode == MID_PROP || a.mode == MID_LSYM) {
        e = set_smem(k_mid_turn<N, mid_min_blocks(N)>, sm);
        if (e) return e;
        k_mid_turn<N, mid_min_blocks(N)><<<grd, blk, sm, st>>>(a);
      } else {
        e = set_smem(k_mid_plain<N>, sm);
        if (e) return e;
        k_mid_plain<N><<<grd, blk, sm, st>>>(a);
      }
      break;
    }
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Batched passes (several plans' passes of one edge in one launch, plan
// blockIdx.z of d, grid sized for the largest plan): compiled for edges up to
// kBatchMaxN. kind 0 first pass (tc: 8 for the t = 8 form of the fused axis-2
// corrections), 1 last pass, 2 axis-1 pass, 3 axis-0 pass (forward, propagator,
// inverse). smem: the largest dynamic shared memory of the plans.
constexpr int kBatchMaxN = 128;

template <int N>
cudaError_t run_size_batch(int kind, bool inv, int tc, const PassArgs* d, dim3 grid, size_t smem, cudaStream_t st) {
  if constexpr (N > kBatchMaxN) {
    return cudaErrorInvalidValue;
  } else {
    const dim3 blk(32 * warps_for(N));
    cudaError_t e = cudaSuccess;
    switch (kind) {
      case 0:
        if (tc == 8) {
          e = set_smem(k_rows_first_batch<N, 8>, smem);
          if (e) return e;
          k_rows_first_batch<N, 8><<<grid, blk, smem, st>>>(d);
        } else {
          e = set_smem(k_rows_first_batch<N, 0>, smem);
          if (e) return e;
          k_rows_first_batch<N, 0><<<grid, blk, smem, st>>>(d);
        }
        break;
      case 1:
        e = set_smem(k_rows_last_batch<N, false>, smem);
        if (e) return e;
        k_rows_last_batch<N, false><<<grid, blk, smem, st>>>(d);
        break;
      case 2:
        if (inv) {
          e = set_smem(k_strided_batch<N, 1, true>, smem);
          if (e) return e;
          k_strided_batch<N, 1, true><<<grid, blk, smem, st>>>(d);
        } else {
          e = set_smem(k_strided_batch<N, 1, false>, smem);
          if (e) return e;
          k_strided_batch<N, 1, false><<<grid, blk, smem, st>>>(d);
        }
        break;
      case 3:
        e = set_smem(k_mid_turn_batch<N, mid_min_blocks(N)>, smem);
        if (e) return e;
        k_mid_turn_batch<N, mid_min_blocks(N)><<<grid, blk, smem, st>>>(d);
        break;
      default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
}

}  // namespace mbs

// One case of a size-group switch (mbs_fft_group.cuh): launch the pass kernel
// for edge n and report its launch status through *err.
#define MBS_CASE(n) \
  case n:           \
    *err = mbs::run_size<n>(kind, axis, inv, a, nrb, st); \
    return true;
#define MBS_CASE_BATCH(n) \
  case n:                 \
    *err = mbs::run_size_batch<n>(kind, inv, tc, d, grid, smem, st); \
    return true;
