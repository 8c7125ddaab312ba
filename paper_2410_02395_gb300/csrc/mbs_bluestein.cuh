// Pass kernels for subdomain edges n with a prime factor above 7 (n <= 256):
// the length-n DFT by Bluestein's chirp-z algorithm on a compiled M-point FFT
// (M >= 2n - 1). With c[m] = exp(-i pi m^2 / n), nk = (n^2 + k^2 - (k - n)^2) / 2
// turns the DFT into a circular convolution:
//   X[k] = c[k] sum_m (x[m] c[m]) conj(c[k - m]),
// done as IFFT_M(FFT_M(a) * FFT_M(b)) with a = x c zero-padded to M and
// b[m] = conj(c[|m|]) for |m| < n (indices mod M). The inverse transform is
// the same with conj(c). The tables (chirp c, the spectra FFT_M(b) / M of both
// directions) are computed in FP64 on the host.
//
// The kernels do the work of k_rows_first / k_rows_last / k_strided /
// k_mid_turn for such an edge, with a run-time n and the tile of M rows; the
// fused axis-2 corrections of k_rows_first are not done here (the plan then
// computes E_2 x with the correction kernels into the FFT buffer).
#pragma once
#include "mbs_passes.cuh"

namespace mbs {

// Rows 0..n-1 of the tile hold 32 pencils (lane = pencil); on return they hold
// their length-n DFT (INV: exponent +, unnormalised).
template <int M, int W, bool INV>
__device__ __forceinline__ void bluestein_run(int warp, int lane, float2 (*sm)[kPad], const float2* __restrict__ tw,
                                              const float2* __restrict__ chirp, const float2* __restrict__ bhat,
                                              int n) {
  for (int m = warp; m < M; m += W) {
    float2 v = make_float2(0.f, 0.f);
    if (m < n) {
      const float2 c = __ldg(chirp + m);
      v = INV ? cmulc(sm[m][lane], c) : cmul(sm[m][lane], c);
    }
    sm[m][lane] = v;
  }
  auto sld = [&](int e) { return sm[e][lane]; };
  auto sst = [&](int e, float2 v) { sm[e][lane] = v; };
  __syncthreads();
  fft_run<M, W, false, false, 0, 1, true, true>(warp, lane, sm, tw, sld, sst);
  __syncthreads();
  const float2* __restrict__ bh = bhat + (INV ? M : 0);
  for (int m = warp; m < M; m += W) sm[m][lane] = cmul(sm[m][lane], __ldg(bh + m));
  __syncthreads();
  fft_run<M, W, true, false, 0, 1, true, true>(warp, lane, sm, tw, sld, sst);
  __syncthreads();
  for (int k = warp; k < n; k += W) {
    const float2 c = __ldg(chirp + k);
    sm[k][lane] = INV ? cmulc(sm[k][lane], c) : cmul(sm[k][lane], c);
  }
}

__device__ __forceinline__ bool in_layer2_n(const PassArgs& a, int e, int n) {
  return a.g.ax[2].a > 0 && (e < a.g.t || e >= n - a.g.t);
}

// Axis-2 forward pass: u = B x + y - E x (FIRST_ITER; E x, all axes, is in K on
// the boundary layers) or u = x (FIRST_PLAIN), then the transform into K.
template <int M>
__global__ void __launch_bounds__(32 * warps_for(M), fft_min_blocks(M)) k_rows_first_bl(const __grid_constant__ PassArgs a) {
  constexpr int W = warps_for(M);
  constexpr int NT = 32 * W;
  extern __shared__ float2 dyn[];
  float2 (*sm)[kPad] = tile_of<M>(dyn);
  __shared__ unsigned masks[3];
  if (a.state && a.state->done) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = a.bl_n;
  const int off2 = a.g.ax[2].off[a.subs[blockIdx.y]];
  const RowTile rt = setup_rows(masks, a, off2, a.subs[blockIdx.y], blockIdx.x);
  const bool iter = a.mode == FIRST_ITER;
  for (int idx = tid; idx < 32 * n; idx += NT) {
    const int r = idx / n, e = idx - r * n;
    float2 u = make_float2(0.f, 0.f);
    if (rt.ok(r)) {
      const long long gi = rt.base(r) + e;
      const float2 xv = __ldg(a.X + gi);
      u = xv;
      if (iter) {
        u = cmul(__ldg(a.B + gi), xv);
        if (rt.lay(r) || in_layer2_n(a, e, n)) u = csub(u, a.K[gi]);
        const long long i2 = off2 + e;
        if (rt.in_src(r) && i2 >= a.sbox[4] && i2 < a.sbox[5]) u = cadd(u, cmul(a.mc, a.S[gi]));
      }
    }
    sm[e][r] = u;
  }
  __syncthreads();
  bluestein_run<M, W, false>(warp, lane, sm, a.tw, a.bl_chirp, a.bl_bhat, n);
  __syncthreads();
  for (int idx = tid; idx < 32 * n; idx += NT) {
    const int r = idx / n, e = idx - r * n;
    if (rt.ok(r)) a.K[rt.base(r) + e] = sm[e][r];
  }
}

// One voxel of the axis-2 inverse pass's epilogue (the modes of k_rows_last).
template <bool RES>
__device__ __forceinline__ void rows_last_voxel(const PassArgs& a, int mode, long long gi, float2 w, bool lay,
                                                float& acc) {
  if (mode == LAST_PLAIN) {
    a.Xout[gi] = w;
    return;
  }
  const float2 xv = a.X[gi];
  const float2 bv = __ldg(a.B + gi);
  if (mode == LAST_AOUT) {
    a.Xout[gi] = cadd(w, cmul(make_float2(1.f - bv.x, -bv.y), xv));
    return;
  }
  const float2 ee = csub(xv, w);
  if constexpr (RES) {
    // residual form: xv = r'_n; x_{n+1} = x_n - alpha r'_n; r'_{n+1} = r'_n - alpha (I - V) e
    acc = fmaf(xv.x, xv.x, fmaf(xv.y, xv.y, acc));
    unsigned lo = a.Xlo[gi];
    a.Xs[gi] = acc_update(a.Xs[gi], lo, make_float2(-a.alpha * xv.x, -a.alpha * xv.y));
    a.Xlo[gi] = lo;
    if (lay) {
      a.E[gi] = ee;
    } else {
      const float2 rr = cmul(bv, ee);
      a.Xout[gi] = make_float2(fmaf(-a.alpha, rr.x, xv.x), fmaf(-a.alpha, rr.y, xv.y));
    }
  } else {
    if (lay) {
      a.E[gi] = ee;
    } else {
      const float2 rr = cmul(bv, ee);
      acc = fmaf(rr.x, rr.x, fmaf(rr.y, rr.y, acc));
      a.Xout[gi] = (mode == LAST_ITER) ? make_float2(fmaf(-a.alpha, rr.x, xv.x), fmaf(-a.alpha, rr.y, xv.y))
                                       : make_float2(-rr.x, -rr.y);
    }
  }
}

// Axis-2 inverse pass with the update epilogue.
template <int M, bool RES>
__global__ void __launch_bounds__(32 * warps_for(M), fft_min_blocks(M)) k_rows_last_bl(const __grid_constant__ PassArgs a) {
  constexpr int W = warps_for(M);
  constexpr int NT = 32 * W;
  extern __shared__ float2 dyn[];
  float2 (*sm)[kPad] = tile_of<M>(dyn);
  __shared__ unsigned masks[3];
  __shared__ double red[32];
  if (a.state && a.state->done) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = a.bl_n;
  const int off2 = a.g.ax[2].off[a.subs[blockIdx.y]];
  const RowTile rt = setup_rows(masks, a, off2, a.subs[blockIdx.y], blockIdx.x);
  for (int idx = tid; idx < 32 * n; idx += NT) {
    const int r = idx / n, e = idx - r * n;
    sm[e][r] = rt.ok(r) ? a.K[rt.base(r) + e] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  bluestein_run<M, W, true>(warp, lane, sm, a.tw, a.bl_chirp, a.bl_bhat, n);
  __syncthreads();
  float acc = 0.f;
  const int mode = a.mode;
  for (int idx = tid; idx < 32 * n; idx += NT) {
    const int r = idx / n, e = idx - r * n;
    if (rt.ok(r))
      rows_last_voxel<RES>(a, mode, rt.base(r) + e, sm[e][r], rt.lay(r) || in_layer2_n(a, e, n), acc);
  }
  if (a.partials) {
    const double s = block_sum((double)acc, red);
    finish_block(Finish{a.partials, a.slot0, a.n_total, a.fin, a.hist}, s, red);
  }
}

// Axis-1 / axis-0 transform of 32 consecutive axis-2 positions.
template <int M, int AXIS, bool INV>
__global__ void __launch_bounds__(32 * warps_for(M), fft_min_blocks(M)) k_strided_bl(const __grid_constant__ PassArgs a) {
  constexpr int W = warps_for(M);
  extern __shared__ float2 dyn[];
  float2 (*sm)[kPad] = tile_of<M>(dyn);
  if (a.state && a.state->done) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n = a.bl_n;
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
  for (int e = warp; e < n; e += W) sm[e][lane] = valid ? a.K[base + e * stride] : make_float2(0.f, 0.f);
  __syncthreads();
  bluestein_run<M, W, INV>(warp, lane, sm, a.tw, a.bl_chirp, a.bl_bhat, n);
  __syncthreads();
  if (valid)
    for (int e = warp; e < n; e += W) a.K[base + e * stride] = sm[e][lane];
}

// Axis-0 pass: forward transform, multiplier, inverse transform (MID_PROP,
// MID_LSYM), or one direction (MID_FWD, MID_INV with the 1/(n0 n1 n2) scale).
template <int M>
__global__ void __launch_bounds__(32 * warps_for(M), fft_min_blocks(M)) k_mid_bl(const __grid_constant__ PassArgs a) {
  constexpr int W = warps_for(M);
  extern __shared__ float2 dyn[];
  float2 (*sm)[kPad] = tile_of<M>(dyn);
  if (a.state && a.state->done) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n = a.bl_n;
  const MidPencil m = mid_pencil(a, blk_here());
  const int mode = a.mode;
  const float scl = mode == MID_INV ? m.sc : 1.f;
  for (int e = warp; e < n; e += W)
    sm[e][lane] = m.valid ? cscale(a.K[m.base + e * m.stride], scl) : make_float2(0.f, 0.f);
  __syncthreads();
  if (mode != MID_INV) {
    bluestein_run<M, W, false>(warp, lane, sm, a.tw, a.bl_chirp, a.bl_bhat, n);
    __syncthreads();
  }
  if (mode == MID_PROP || mode == MID_LSYM) {
    const float2 c = a.c, ck0 = a.ck0;
    // c is purely imaginary (Eq. c_scale2), so Re c(k0^2 - |p|^2) = Re(c k0^2) for every p
    const float dx = ck0.x, ex = dx + 1.f;
    for (int k = warp; k < n; k += W) {
      const float p2 = __ldg(m.p20 + k) + m.pl;
      const float dy = fmaf(-c.y, p2, ck0.y);  // Im c(k0^2 - |p|^2)
      float2 mul;
      if (mode == MID_PROP) {
        const float inv = m.sc * __frcp_rn(fmaf(ex, ex, dy * dy));
        mul = make_float2(ex * inv, -dy * inv);
      } else {
        mul = make_float2(dx * m.sc, dy * m.sc);
      }
      sm[k][lane] = cmul(sm[k][lane], mul);
    }
    __syncthreads();
  }
  if (mode != MID_FWD) {
    bluestein_run<M, W, true>(warp, lane, sm, a.tw, a.bl_chirp, a.bl_bhat, n);
    __syncthreads();
  }
  if (m.valid)
    for (int e = warp; e < n; e += W) a.K[m.base + e * m.stride] = sm[e][lane];
}

template <int M>
cudaError_t run_bluestein(int kind, int axis, bool inv, const PassArgs& a, int nrb, cudaStream_t st) {
  const size_t sm = tile_bytes(M);
  const dim3 blk(32 * warps_for(M));
  const unsigned gx = (unsigned)((a.g.N2 + 31) / 32);
  cudaError_t e = cudaSuccess;
  switch (kind) {
    case 0:
      e = set_smem(k_rows_first_bl<M>, sm);
      if (e) return e;
      k_rows_first_bl<M><<<dim3(nrb, a.nsub), blk, sm, st>>>(a);
      break;
    case 1:
      if (a.mode == LAST_RES) {
        e = set_smem(k_rows_last_bl<M, true>, sm);
        if (e) return e;
        k_rows_last_bl<M, true><<<dim3(nrb, a.nsub), blk, sm, st>>>(a);
      } else {
        e = set_smem(k_rows_last_bl<M, false>, sm);
        if (e) return e;
        k_rows_last_bl<M, false><<<dim3(nrb, a.nsub), blk, sm, st>>>(a);
      }
      break;
    case 2:
      if (axis == 1) {
        if (inv) {
          e = set_smem(k_strided_bl<M, 1, true>, sm);
          if (e) return e;
          k_strided_bl<M, 1, true><<<dim3(gx, (unsigned)a.g.N0, a.nsub), blk, sm, st>>>(a);
        } else {
          e = set_smem(k_strided_bl<M, 1, false>, sm);
          if (e) return e;
          k_strided_bl<M, 1, false><<<dim3(gx, (unsigned)a.g.N0, a.nsub), blk, sm, st>>>(a);
        }
      } else {
        if (inv) {
          e = set_smem(k_strided_bl<M, 0, true>, sm);
          if (e) return e;
          k_strided_bl<M, 0, true><<<dim3(gx, (unsigned)a.g.N1, a.nsub), blk, sm, st>>>(a);
        } else {
          e = set_smem(k_strided_bl<M, 0, false>, sm);
          if (e) return e;
          k_strided_bl<M, 0, false><<<dim3(gx, (unsigned)a.g.N1, a.nsub), blk, sm, st>>>(a);
        }
      }
      break;
    case 3:
      e = set_smem(k_mid_bl<M>, sm);
      if (e) return e;
      k_mid_bl<M><<<dim3(gx, (unsigned)a.g.N1, a.nsub), blk, sm, st>>>(a);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace mbs
