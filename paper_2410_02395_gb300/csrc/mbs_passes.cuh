// FFT pass kernels of one MBS iteration (Eq. wavesim_iter, Sec. 3.1).
//
//   rows_first  axis-2 forward transform; fuses u = B x + y - E x (medium,
//               source and edge corrections of V, Sec. 3.1 steps 3-5) into the
//               coalesced staged load.
//   strided     axis-1 forward / inverse transform (global loads straight into
//               the first radix stage, global stores from the last).
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
#include "mbs_fft.cuh"
#include "mbs_internal.h"

namespace mbs {

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < nw; i++) s += red[i];
  }
  return s;
}

template <int N>
__device__ __forceinline__ float2 (*tile_of(float2* dyn))[kPad] {
  return reinterpret_cast<float2 (*)[kPad]>(dyn);
}

// ---------------------------------------------------------------------------
// Axis-2 forward pass with the fused medium/source/correction prologue.
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(32 * warps_for(N)) k_rows_first(const __grid_constant__ PassArgs a) {
  constexpr int W = warps_for(N);
  extern __shared__ float2 dyn[];
  float2 (*sm)[kPad] = tile_of<N>(dyn);
  __shared__ long long rbase[32];
  __shared__ int rflag[32];
  if (a.state && a.state->done) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int j2 = a.subs[blockIdx.y];
  const int off2 = a.g.ax[2].off[j2];
  const long long rows = a.g.N0 * a.g.N1;
  if (tid < 32) {
    const long long rho = (long long)blockIdx.x * 32 + tid;
    int f = 0;
    long long base = 0;
    if (rho < rows) {
      const long long i0 = rho / a.g.N1, i1 = rho - i0 * a.g.N1;
      base = rho * a.g.N2 + off2;
      f = 1;
      if (a.tb.shell[0][i0] | a.tb.shell[1][i1]) f |= 2;
      if (a.S && i0 >= a.sbox[0] && i0 < a.sbox[1] && i1 >= a.sbox[2] && i1 < a.sbox[3]) f |= 4;
    }
    rbase[tid] = base;
    rflag[tid] = f;
  }
  __syncthreads();
  const bool iter = a.mode == FIRST_ITER;
  for (int idx = tid; idx < 32 * N; idx += 32 * W) {
    const int r = idx / N, e = idx - r * N;
    const int f = rflag[r];
    float2 u = make_float2(0.f, 0.f);
    if (f & 1) {
      const long long gi = rbase[r] + e;
      const float2 x = a.X[gi];
      if (iter) {
        u = cmul(a.B[gi], x);
        if ((f & 2) || a.tb.shell[2][off2 + e]) u = csub(u, a.K[gi]);
        if (f & 4) {
          const int i2 = off2 + e;
          if (i2 >= a.sbox[4] && i2 < a.sbox[5]) u = cadd(u, cmul(a.mc, a.S[gi]));
        }
      } else {
        u = x;
      }
    }
    sm[e][r] = u;
  }
  if constexpr (N > 1) {
    __syncthreads();
    auto sld = [&](int e) { return sm[e][lane]; };
    auto sst = [&](int e, float2 v) { sm[e][lane] = v; };
    fft_run<N, W, false, false, 0, 1, true, true>(warp, lane, sm, a.tw, sld, sst);
  }
  __syncthreads();
  for (int idx = tid; idx < 32 * N; idx += 32 * W) {
    const int r = idx / N, e = idx - r * N;
    if (rflag[r] & 1) a.K[rbase[r] + e] = sm[e][r];
  }
}

// ---------------------------------------------------------------------------
// Axis-2 inverse pass with the fused update epilogue.
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(32 * warps_for(N)) k_rows_last(const __grid_constant__ PassArgs a) {
  constexpr int W = warps_for(N);
  extern __shared__ float2 dyn[];
  float2 (*sm)[kPad] = tile_of<N>(dyn);
  __shared__ long long rbase[32];
  __shared__ int rflag[32];
  __shared__ double red[32];
  if (a.state && a.state->done) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int j2 = a.subs[blockIdx.y];
  const int off2 = a.g.ax[2].off[j2];
  const long long rows = a.g.N0 * a.g.N1;
  if (tid < 32) {
    const long long rho = (long long)blockIdx.x * 32 + tid;
    int f = 0;
    long long base = 0;
    if (rho < rows) {
      const long long i0 = rho / a.g.N1, i1 = rho - i0 * a.g.N1;
      base = rho * a.g.N2 + off2;
      f = 1;
      if (a.tb.shell[0][i0] | a.tb.shell[1][i1]) f |= 2;
    }
    rbase[tid] = base;
    rflag[tid] = f;
  }
  __syncthreads();
  for (int idx = tid; idx < 32 * N; idx += 32 * W) {
    const int r = idx / N, e = idx - r * N;
    sm[e][r] = (rflag[r] & 1) ? a.K[rbase[r] + e] : make_float2(0.f, 0.f);
  }
  if constexpr (N > 1) {
    __syncthreads();
    auto sld = [&](int e) { return sm[e][lane]; };
    auto sst = [&](int e, float2 v) { sm[e][lane] = v; };
    fft_run<N, W, true, false, 0, 1, true, true>(warp, lane, sm, a.tw, sld, sst);
  }
  __syncthreads();
  double acc = 0.0;
  const int mode = a.mode;
  for (int idx = tid; idx < 32 * N; idx += 32 * W) {
    const int r = idx / N, e = idx - r * N;
    const int f = rflag[r];
    if (!(f & 1)) continue;
    const long long gi = rbase[r] + e;
    const float2 w = sm[e][r];
    if (mode == LAST_PLAIN) {
      a.Xout[gi] = w;
    } else if (mode == LAST_AOUT) {
      const float2 b = a.B[gi];
      a.Xout[gi] = cadd(w, cmul(make_float2(1.f - b.x, -b.y), a.X[gi]));
    } else {
      const float2 x = a.X[gi];
      const float2 ee = csub(x, w);
      if ((f & 2) || a.tb.shell[2][off2 + e]) {
        a.K[gi] = ee;  // finished by the shell kernel once all of e is known
      } else {
        const float2 rr = cmul(a.B[gi], ee);
        acc += (double)rr.x * rr.x + (double)rr.y * rr.y;
        a.Xout[gi] = (mode == LAST_ITER) ? make_float2(fmaf(-a.alpha, rr.x, x.x), fmaf(-a.alpha, rr.y, x.y))
                                         : make_float2(-rr.x, -rr.y);
      }
    }
  }
  if (a.partials) {
    const double s = block_sum(acc, red);
    if (tid == 0) a.partials[blockIdx.x + (long long)gridDim.x * blockIdx.y] = s;
  }
}

// ---------------------------------------------------------------------------
// Axis-1 / axis-0 transform of a tile of 32 consecutive axis-2 positions.
// ---------------------------------------------------------------------------
template <int N, int AXIS, bool INV>
__global__ void __launch_bounds__(32 * warps_for(N)) k_strided(const __grid_constant__ PassArgs a) {
  constexpr int W = warps_for(N);
  extern __shared__ float2 dyn[];
  float2 (*sm)[kPad] = tile_of<N>(dyn);
  if (a.state && a.state->done) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = a.subs[blockIdx.z];
  const long long i2 = (long long)blockIdx.x * 32 + lane;
  const bool valid = i2 < a.g.N2;
  long long base, stride;
  if (AXIS == 1) {
    base = (long long)blockIdx.y * a.g.N1 * a.g.N2 + (long long)a.g.ax[1].off[j] * a.g.N2 + i2;
    stride = a.g.N2;
  } else {
    base = (long long)a.g.ax[0].off[j] * a.g.N1 * a.g.N2 + (long long)blockIdx.y * a.g.N2 + i2;
    stride = a.g.N1 * a.g.N2;
  }
  float2* K = a.K;
  auto gld = [&](int e) { return valid ? K[base + e * stride] : make_float2(0.f, 0.f); };
  auto gst = [&](int e, float2 v) {
    if (valid) K[base + e * stride] = v;
  };
  if constexpr (N > 1) fft_run<N, W, INV, false, 0, 1, false, false>(warp, lane, sm, a.tw, gld, gst);
}

// ---------------------------------------------------------------------------
// Axis-0 pass: forward transform, multiplier, inverse transform.
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(32 * warps_for(N)) k_mid(const __grid_constant__ PassArgs a) {
  constexpr int W = warps_for(N);
  extern __shared__ float2 dyn[];
  float2 (*sm)[kPad] = tile_of<N>(dyn);
  if (a.state && a.state->done) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = a.subs[blockIdx.z];
  const int off0 = a.g.ax[0].off[j];
  const long long i1 = blockIdx.y;
  const long long i2 = (long long)blockIdx.x * 32 + lane;
  const bool valid = i2 < a.g.N2;
  const long long i2c = valid ? i2 : 0;
  const long long base = (long long)off0 * a.g.N1 * a.g.N2 + i1 * a.g.N2 + i2;
  const long long stride = a.g.N1 * a.g.N2;
  const float pl = a.tb.p2[1][i1] + a.tb.p2[2][i2c];
  const float sc = a.tb.invn[0][off0] * a.tb.invn[1][i1] * a.tb.invn[2][i2c];
  const float* p20 = a.tb.p2[0] + off0;
  const float2 c = a.c, ck0 = a.ck0;
  float2* K = a.K;
  auto gld = [&](int e) { return valid ? K[base + e * stride] : make_float2(0.f, 0.f); };
  auto gst = [&](int e, float2 v) {
    if (valid) K[base + e * stride] = v;
  };
  const int mode = a.mode;
  auto mul_prop = [&](int e, float2 v) {
    const float p2 = __ldg(p20 + e) + pl;
    // den = c (k0^2 - |p|^2) + 1
    const float dx = fmaf(-c.x, p2, ck0.x + 1.f), dy = fmaf(-c.y, p2, ck0.y);
    const float inv = sc / fmaf(dx, dx, dy * dy);
    return cmul(v, make_float2(dx * inv, -dy * inv));
  };
  auto mul_lsym = [&](int e, float2 v) {
    const float p2 = __ldg(p20 + e) + pl;
    return cmul(v, make_float2(fmaf(-c.x, p2, ck0.x) * sc, fmaf(-c.y, p2, ck0.y) * sc));
  };
  if constexpr (N == 1) {
    if (valid) {
      float2 v = K[base];
      if (mode == MID_PROP) v = mul_prop(0, v);
      else if (mode == MID_LSYM) v = mul_lsym(0, v);
      else if (mode == MID_INV) v = cscale(v, sc);
      K[base] = v;
    }
  } else {
    if (mode == MID_PROP) {
      fft_fwd_mul_inv<N, W, false, false>(warp, lane, sm, a.tw, gld, gst, mul_prop);
    } else if (mode == MID_LSYM) {
      fft_fwd_mul_inv<N, W, false, false>(warp, lane, sm, a.tw, gld, gst, mul_lsym);
    } else if (mode == MID_FWD) {
      fft_run<N, W, false, false, 0, 1, false, false>(warp, lane, sm, a.tw, gld, gst);
    } else {
      auto gls = [&](int e) { return cscale(gld(e), sc); };
      fft_run<N, W, true, false, 0, 1, false, false>(warp, lane, sm, a.tw, gls, gst);
    }
  }
}

// ---------------------------------------------------------------------------
// Launch helpers for one size.
// ---------------------------------------------------------------------------
inline size_t tile_bytes(int n) { return (size_t)n * kPad * sizeof(float2); }

// Opt in to more than 48 KB of dynamic shared memory once per kernel.
template <class K>
inline cudaError_t set_smem(K kernel, size_t bytes) {
  static bool done = false;
  if (bytes <= 48 * 1024 || done) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) done = true;
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
      e = set_smem(k_rows_first<N>, sm);
      if (e) return e;
      k_rows_first<N><<<dim3(nrow_blocks, a.nsub), blk, sm, st>>>(a);
      break;
    }
    case 1: {
      e = set_smem(k_rows_last<N>, sm);
      if (e) return e;
      k_rows_last<N><<<dim3(nrow_blocks, a.nsub), blk, sm, st>>>(a);
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
      e = set_smem(k_mid<N>, sm);
      if (e) return e;
      k_mid<N><<<dim3(gx, (unsigned)a.g.N1, a.nsub), blk, sm, st>>>(a);
      break;
    }
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace mbs

// Size-group translation units define
//   bool mbs_fft_group_<k>(int n, int kind, int axis, bool inv, const PassArgs&, int, cudaStream_t, cudaError_t*)
#define MBS_CASE(n) \
  case n:           \
    *err = mbs::run_size<n>(kind, axis, inv, a, nrb, st); \
    return true;
