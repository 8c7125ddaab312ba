// Edge-correction, residual and set-up kernels of the MBS library.
#include <math.h>

#include "mbs_fft.cuh"
#include "mbs_internal.h"
#include "mbs_reduce.cuh"
#include "../../include/mbs.h"

namespace mbs {

// ---------------------------------------------------------------------------
// Edge corrections (Sec. 3, Figs. 4-5; Sec. 3.1 steps 1-5).
//
// For every pencil along a corrected axis d and every subdomain s on it, with
// f_s[b] the b-th voxel of s along the pencil (n = its size):
//   last t layers  (row a of W):   (E f)_s[n-t+a] = sum_b cW[a][b] (f_right[b]      - f_s[b])
//   first t layers (row a of W^T): (E f)_s[a]     = sum_b cW[b][a] (f_left[n_l-t+b] - f_s[n-t+b])
// A missing neighbour contributes nothing (wrap removal only, step 4); a present
// one adds its transfer (step 5). If n < 2t a voxel can be in both ranges and
// gets both terms. The terms of different axes add: axes run in order 0, 1, 2
// and a launch adds to the buffer where an earlier axis already wrote.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void put(float2* C, long long v, float2 val, bool add) {
  C[v] = add ? cadd(C[v], val) : val;
}

// W is Toeplitz, W[a][b] = D(t + b - a): 2t - 1 distinct entries, indexed here
// by m = b - a + t - 1 (row a = max(0, t - 1 - m), column b = a + m - (t - 1)).
// c is purely imaginary (Eq. c_scale2) and W real, so c W = i w with
// w = Im(c W) real and sum_b cW_b f_b = i v with v = sum_b w_b f_b (two FMAs per
// term); load_toeplitz_im returns the 2t - 1 values of w.
template <int T>
__device__ __forceinline__ void load_toeplitz_im(const float2* __restrict__ cW, float (&w)[2 * T - 1]) {
#pragma unroll
  for (int m = 0; m < 2 * T - 1; m++) {
    const int aa = m < T - 1 ? T - 1 - m : 0;
    const int bb = aa + m - (T - 1);
    w[m] = __ldg(&cW[aa * T + bb].y);
  }
}
__device__ __forceinline__ float2 times_i(float vx, float vy) { return make_float2(-vy, vx); }

// Axes 0 and 1: one thread per (pencil, subdomain); consecutive threads take
// consecutive axis-2 positions, so every load and store is coalesced.
template <int T>
__global__ void __launch_bounds__(128) k_corr_strided(const __grid_constant__ CorrArgs a) {
  if (a.state && a.state->done) return;
  const int d = a.axis;
  const AxisDesc& ax = a.g.ax[d];
  const long long N0 = a.g.N0, N1 = a.g.N1, N2 = a.g.N2;
  const long long npen = d == 0 ? N1 * N2 : N0 * N2;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= npen * ax.S) return;
  const int s = (int)(gid / npen);
  const long long p = gid - (long long)s * npen;
  long long base, stride;
  bool add = false;
  if (d == 0) {
    base = p;
    stride = N1 * N2;
  } else {
    const long long i0 = p / N2, i2 = p - i0 * N2;
    base = i0 * N1 * N2 + i2;
    stride = N2;
    add = a.tb.shell[0][i0];
  }
  const int off = ax.off[s], n = ax.n[s];
  const int L = ax.left[s], R = ax.right[s];
  // the pencil along the whole axis covers the own subdomain and both neighbours
  if (!grid_range_ok(a.g, base, base + (long long)(ax.N - 1) * stride, BC_CORR)) return;
  const float2* __restrict__ F = a.F;
  float2 D[T], E[T];
#pragma unroll
  for (int b = 0; b < T; b++) {
    const float2 A = F[base + (long long)(off + b) * stride];
    const float2 Z = F[base + (long long)(off + n - T + b) * stride];
    const float2 Rv = R >= 0 ? F[base + (long long)(ax.off[R] + b) * stride] : make_float2(0.f, 0.f);
    const float2 Lv = L >= 0 ? F[base + (long long)(ax.off[L] + ax.n[L] - T + b) * stride] : make_float2(0.f, 0.f);
    D[b] = csub(Rv, A);
    E[b] = csub(Lv, Z);
  }
  float w[2 * T - 1];
  load_toeplitz_im<T>(a.cW, w);
  float2* C = a.C;
  // first t layers: (W^T E)[q] = sum_b W[b][q] E[b] = sum_b w[q - b + T - 1] E[b]
  float2 outf[T];
#pragma unroll
  for (int q = 0; q < T; q++) {
    float vx = 0.f, vy = 0.f;
#pragma unroll
    for (int b = 0; b < T; b++) {
      vx = fmaf(w[q - b + T - 1], E[b].x, vx);
      vy = fmaf(w[q - b + T - 1], E[b].y, vy);
    }
    outf[q] = times_i(vx, vy);
  }
  // last t layers: (W D)[aa] = sum_b W[aa][b] D[b] = sum_b w[b - aa + T - 1] D[b]
#pragma unroll
  for (int aa = 0; aa < T; aa++) {
    float vx = 0.f, vy = 0.f;
#pragma unroll
    for (int b = 0; b < T; b++) {
      vx = fmaf(w[b - aa + T - 1], D[b].x, vx);
      vy = fmaf(w[b - aa + T - 1], D[b].y, vy);
    }
    const float2 v = times_i(vx, vy);
    const int q = n - T + aa;
    if (q < T) {
      outf[q] = cadd(outf[q], v);  // n < 2t: the voxel is in both ranges (q == n - T + aa)
    } else {
      put(C, base + (long long)(off + q) * stride, v, add);
    }
  }
#pragma unroll
  for (int q = 0; q < T; q++) put(C, base + (long long)(off + q) * stride, outf[q], add);
}

// Axes 0 and 1 when every subdomain on the axis has n >= 2t (the first and last
// layer ranges do not overlap): one thread per (pencil, subdomain, side), so
// each thread holds only t inputs (twice the threads, half the registers).
//   side 0 (first t):  out[q]        = sum_b w[q - b + t - 1] (f_left[n_l-t+b] - f_s[n-t+b])
//   side 1 (last t):   out[n-t+aa]   = sum_b w[b - aa + t - 1] (f_right[b]      - f_s[b])
template <int T>
__device__ __forceinline__ void corr_side_body(const CorrArgs& a, long long gid) {
  if (a.state && a.state->done) return;
  const int d = a.axis;
  const AxisDesc& ax = a.g.ax[d];
  const long long N0 = a.g.N0, N1 = a.g.N1, N2 = a.g.N2;
  const long long npen = d == 0 ? N1 * N2 : N0 * N2;
  if (gid >= 2 * npen * ax.S) return;
  const int ss = (int)(gid / npen);  // subdomain * 2 + side
  const int s = ss >> 1, side = ss & 1;
  const long long p = gid - (long long)ss * npen;
  long long base, stride;
  bool add = false;
  if (d == 0) {
    base = p;
    stride = N1 * N2;
  } else {
    const long long i0 = p / N2, i2 = p - i0 * N2;
    base = i0 * N1 * N2 + i2;
    stride = N2;
    add = a.tb.shell[0][i0];
  }
  const int off = ax.off[s], n = ax.n[s];
  const int nb = side ? ax.right[s] : ax.left[s];
  const long long own0 = base + (long long)(side ? off : off + n - T) * stride;
  const long long nb0 = nb >= 0 ? base + (long long)(side ? ax.off[nb] : ax.off[nb] + ax.n[nb] - T) * stride : 0;
  if (!grid_range_ok(a.g, base, base + (long long)(ax.N - 1) * stride, BC_CORR)) return;  // the whole pencil
  const float2* __restrict__ F = a.F;
  float2 G[T];
#pragma unroll
  for (int b = 0; b < T; b++) {
    const float2 o = F[own0 + (long long)b * stride];
    const float2 v = nb >= 0 ? F[nb0 + (long long)b * stride] : make_float2(0.f, 0.f);
    G[b] = csub(v, o);
  }
  float w[2 * T - 1];
  load_toeplitz_im<T>(a.cW, w);
  float2* C = a.C;
  const long long out0 = base + (long long)(side ? off + n - T : off) * stride;
#pragma unroll
  for (int q = 0; q < T; q++) {
    float vx = 0.f, vy = 0.f;
#pragma unroll
    for (int b = 0; b < T; b++) {
      const float wb = side ? w[b - q + T - 1] : w[q - b + T - 1];
      vx = fmaf(wb, G[b].x, vx);
      vy = fmaf(wb, G[b].y, vy);
    }
    put(C, out0 + (long long)q * stride, times_i(vx, vy), add);
  }
}

template <int T>
__global__ void __launch_bounds__(128) k_corr_side(const __grid_constant__ CorrArgs a) {
  corr_side_body<T>(a, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

// Batched form: plan blockIdx.y of d (threads past its pencils leave at once).
template <int T>
__global__ void __launch_bounds__(128) k_corr_side_batch(const CorrArgs* __restrict__ d) {
  __shared__ CorrArgs a;
  stage_args(&a, &d[blockIdx.y]);
  corr_side_body<T>(a, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

// Axis 2: one warp per grid row; the row's 2t layer values of every subdomain
// are staged in shared memory with coalesced loads, then each lane produces
// outputs from shared memory.
template <int T>
__global__ void __launch_bounds__(256) k_corr_rows(const __grid_constant__ CorrArgs a) {
  extern __shared__ float2 cs[];
  if (a.state && a.state->done) return;
  const AxisDesc& ax = a.g.ax[2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int S = ax.S, M = S * 2 * T;
  float2* sm = cs + warp * M;
  const long long N1 = a.g.N1, N2 = a.g.N2, rows = a.g.N0 * N1;
  const float2* __restrict__ F = a.F;
  __shared__ float w[2 * T - 1];  // lanes index it with their own (runtime) output position
  if (threadIdx.x == 0) {
    float wr[2 * T - 1];
    load_toeplitz_im<T>(a.cW, wr);
#pragma unroll
    for (int m = 0; m < 2 * T - 1; m++) w[m] = wr[m];
  }
  __syncthreads();
  float2* C = a.C;
  for (long long rho = (long long)blockIdx.x * 8 + warp; rho < rows; rho += (long long)gridDim.x * 8) {
    const long long i0 = rho / N1, i1 = rho - i0 * N1;
    const bool add = a.tb.shell[0][i0] || a.tb.shell[1][i1];
    const long long rb = rho * N2;
    if (!grid_range_ok(a.g, rb, rb + N2 - 1, BC_CORR)) continue;  // the warp's row
    for (int idx = lane; idx < M; idx += 32) {
      const int s = idx / (2 * T), k = idx - s * 2 * T;
      const int q = k < T ? k : ax.n[s] - T + (k - T);
      sm[idx] = F[rb + ax.off[s] + q];
    }
    __syncwarp();
    for (int idx = lane; idx < M; idx += 32) {
      const int s = idx / (2 * T), k = idx - s * 2 * T;
      const int n = ax.n[s];
      const float2* own = sm + s * 2 * T;  // own[0..t): first t layers, own[t..2t): last t layers
      const int lft = ax.left[s], rgt = ax.right[s];
      // local position q of this output; in the last range, voxels that are also
      // in the first range (n < 2t) are produced by the first-range lane
      const int q = k < T ? k : n - T + (k - T);
      if (k >= T && q < T) continue;
      float vx = 0.f, vy = 0.f;
      if (q < T) {  // first t layers: row q of W^T on (left's last t - own last t)
#pragma unroll
        for (int b = 0; b < T; b++) {
          float2 f = make_float2(-own[T + b].x, -own[T + b].y);
          if (lft >= 0) f = cadd(f, sm[lft * 2 * T + T + b]);
          vx = fmaf(w[q - b + T - 1], f.x, vx);
          vy = fmaf(w[q - b + T - 1], f.y, vy);
        }
      }
      if (q >= n - T) {  // last t layers: row q-(n-t) of W on (right's first t - own first t)
        const int aa = q - (n - T);
#pragma unroll
        for (int b = 0; b < T; b++) {
          float2 f = make_float2(-own[b].x, -own[b].y);
          if (rgt >= 0) f = cadd(f, sm[rgt * 2 * T + b]);
          vx = fmaf(w[b - aa + T - 1], f.x, vx);
          vy = fmaf(w[b - aa + T - 1], f.y, vy);
        }
      }
      put(C, rb + ax.off[s] + q, times_i(vx, vy), add);
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Tensor-core form of the edge corrections (3xTF32, FP32 accumulation).
// c is purely imaginary and W real, so E f = c (W g) with g the real and the
// imaginary parts of the gathered differences as separate columns. One warp
// handles 32 pencils of one (subdomain, side): A = [64 pencil-components][TP]
// (row 2p: real part, 2p+1: imaginary part; TP = t rounded up to 8, zero
// padded), B[k][n] = W^T or W, D = A B with mma.sync m16n8k8 TF32 in three
// products a_hi b_hi + a_hi b_lo + a_lo b_hi (Ootomo & Yokota's split, hi =
// round-to-nearest TF32, lo = TF32 of the remainder), then out = c D.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned tf32_hi(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// TC: the truncation width when known at compile time (t == TP == 8), 0 otherwise.
template <int TP, int TC>
__global__ void __launch_bounds__(128) k_corr_tc(const __grid_constant__ CorrArgs a) {
  // per warp, transposed: As[k][row] (row 2p: real part of pencil p, 2p + 1: imaginary part).
  // The pitch 72 (= 8 mod 32 banks) keeps the fragment reads (8 rows x 4 k per
  // instruction) conflict-free, and every lane's pencil is one float2 per k, so the
  // gather and the final reads move 256 contiguous bytes per warp.
  __shared__ __align__(16) float As[4][TP][72];
  __shared__ float Wr[TP][TP + 1];     // real W (not scaled by c), zero padded
  if (a.state && a.state->done) return;
  const int d = a.axis, t = TC > 0 ? TC : a.g.t;
  const AxisDesc& ax = a.g.ax[d];
  const long long N0 = a.g.N0, N1 = a.g.N1, N2 = a.g.N2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // W from c W: c = i c_im (c_re = 0), so W = Im(cW) / c_im
  const float cim = a.c.y;
  for (int i = threadIdx.x; i < TP * TP; i += blockDim.x) {
    const int r = i / TP, q = i - r * TP;
    Wr[r][q] = (r < t && q < t) ? a.cW[r * t + q].y / cim : 0.f;
  }
  __syncthreads();
  const long long npen = d == 0 ? N1 * N2 : (d == 1 ? N0 * N2 : N0 * N1);
  const long long ngroups = (npen + 31) / 32;
  const long long wid = (long long)blockIdx.x * 4 + warp;  // (group, subdomain, side)
  if (wid >= ngroups * ax.S * 2) return;
  const int ss = (int)(wid / ngroups);
  const int s = ss >> 1, side = ss & 1;
  const long long p = (wid - (long long)ss * ngroups) * 32 + lane;
  bool valid = p < npen;
  long long base = 0, stride;
  bool add = false;
  if (d == 0) {
    base = p;
    stride = N1 * N2;
  } else if (d == 1) {
    const long long i0 = p / N2, i2 = p - i0 * N2;
    base = i0 * N1 * N2 + i2;
    stride = N2;
    if (valid) add = a.tb.shell[0][i0];
  } else {
    const long long i0 = p / N1, i1 = p - i0 * N1;
    base = p * N2;
    stride = 1;
    if (valid) add = a.tb.shell[0][i0] || a.tb.shell[1][i1];
  }
  const int off = ax.off[s], n = ax.n[s];
  const int nb = side ? ax.right[s] : ax.left[s];
  const long long own0 = base + (long long)(side ? off : off + n - t) * stride;
  const long long nb0 = nb >= 0 ? base + (long long)(side ? ax.off[nb] : ax.off[nb] + ax.n[nb] - t) * stride : 0;
  if (valid) valid = grid_range_ok(a.g, base, base + (long long)(ax.N - 1) * stride, BC_CORR);  // the pencil
  // gather g = f_neighbour - f_own into the warp's A rows 2*lane, 2*lane+1
  for (int b = 0; b < TP; b++) {
    float2 g = make_float2(0.f, 0.f);
    if (valid && b < t) {
      const float2 o = a.F[own0 + (long long)b * stride];
      const float2 v = nb >= 0 ? a.F[nb0 + (long long)b * stride] : make_float2(0.f, 0.f);
      g = csub(v, o);
    }
    *reinterpret_cast<float2*>(&As[warp][b][2 * lane]) = g;
  }
  __syncwarp();
  const int gq = lane >> 2, tg = lane & 3;
  float D[4][TP / 8][4];  // [m-tile][n-tile][fragment]
#pragma unroll
  for (int mt = 0; mt < 4; mt++)
#pragma unroll
    for (int nt = 0; nt < TP / 8; nt++)
#pragma unroll
      for (int i = 0; i < 4; i++) D[mt][nt][i] = 0.f;
#pragma unroll
  for (int ks = 0; ks < TP / 8; ks++) {
    // B fragments: side 0 (first t): out[q] = sum_b W[b][q] g[b]  -> B[k=b][n=q] = W[b][q]
    //              side 1 (last t):  out[q] = sum_b W[q][b] g[b]  -> B[k=b][n=q] = W[q][b]
    unsigned bh[TP / 8][2], bl[TP / 8][2];
#pragma unroll
    for (int nt = 0; nt < TP / 8; nt++) {
#pragma unroll
      for (int j = 0; j < 2; j++) {
        const int k = ks * 8 + tg + 4 * j, q = nt * 8 + gq;
        const float w = side ? Wr[q][k] : Wr[k][q];
        bh[nt][j] = tf32_hi(w);
        bl[nt][j] = tf32_hi(w - __uint_as_float(bh[nt][j]));
      }
    }
#pragma unroll
    for (int mt = 0; mt < 4; mt++) {
      unsigned ah[4], al[4];
#pragma unroll
      for (int i = 0; i < 4; i++) {
        const int r = mt * 16 + gq + 8 * (i & 1), k = ks * 8 + tg + 4 * (i >> 1);
        const float v = As[warp][k][r];
        ah[i] = tf32_hi(v);
        al[i] = tf32_hi(v - __uint_as_float(ah[i]));
      }
#pragma unroll
      for (int nt = 0; nt < TP / 8; nt++) {
        mma_tf32(D[mt][nt], al, bh[nt]);
        mma_tf32(D[mt][nt], ah, bl[nt]);
        mma_tf32(D[mt][nt], ah, bh[nt]);
      }
    }
  }
  __syncwarp();
  // D fragments back to the warp's rows (A is no longer needed)
#pragma unroll
  for (int mt = 0; mt < 4; mt++)
#pragma unroll
    for (int nt = 0; nt < TP / 8; nt++)
#pragma unroll
      for (int i = 0; i < 4; i++) {
        const int r = mt * 16 + gq + 8 * (i >> 1), q = nt * 8 + 2 * tg + (i & 1);
        As[warp][q][r] = D[mt][nt][i];
      }
  __syncwarp();
  if (!valid) return;
  const float2 c = a.c;
  const long long out0 = base + (long long)(side ? off + n - t : off) * stride;
  if constexpr (TC > 0) {
    // every load of the outputs the earlier axes wrote is issued before any store
    float2 prev[TC];
#pragma unroll
    for (int q = 0; q < TC; q++) prev[q] = add ? a.C[out0 + (long long)q * stride] : make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < TC; q++) {
      const float2 v = cmul(c, *reinterpret_cast<const float2*>(&As[warp][q][2 * lane]));
      a.C[out0 + (long long)q * stride] = cadd(prev[q], v);
    }
  } else {
    for (int q = 0; q < t; q++) {
      const float2 v = cmul(c, *reinterpret_cast<const float2*>(&As[warp][q][2 * lane]));
      put(a.C, out0 + (long long)q * stride, v, add);
    }
  }
}

// Any t (1..kMaxT) on any axis, for the widths without a compiled kernel: one
// thread per (pencil, subdomain) does both sides, reading its inputs from
// global memory for every term (O(t^2) cached loads; widths above 32 are for
// the truncation sweep of Fig. 7 only). Both sides run in the same thread, so a
// voxel in both ranges (n < 2t) gets both terms without a race.
__global__ void __launch_bounds__(128) k_corr_generic(const __grid_constant__ CorrArgs a) {
  __shared__ float w[2 * kMaxT];
  if (a.state && a.state->done) return;
  const int t = a.g.t;
  if (threadIdx.x < 2 * t - 1) {
    const int m = threadIdx.x, aa = m < t - 1 ? t - 1 - m : 0, bb = aa + m - (t - 1);
    w[m] = a.cW[aa * t + bb].y;
  }
  __syncthreads();
  const int d = a.axis;
  const AxisDesc& ax = a.g.ax[d];
  const long long N0 = a.g.N0, N1 = a.g.N1, N2 = a.g.N2;
  const long long npen = d == 0 ? N1 * N2 : (d == 1 ? N0 * N2 : N0 * N1);
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= npen * ax.S) return;
  const int s = (int)(gid / npen);
  const long long p = gid - (long long)s * npen;
  long long base, stride;
  bool add = false;
  if (d == 0) {
    base = p;
    stride = N1 * N2;
  } else if (d == 1) {
    const long long i0 = p / N2, i2 = p - i0 * N2;
    base = i0 * N1 * N2 + i2;
    stride = N2;
    add = a.tb.shell[0][i0];
  } else {
    const long long i0 = p / N1, i1 = p - i0 * N1;
    base = p * N2;
    stride = 1;
    add = a.tb.shell[0][i0] || a.tb.shell[1][i1];
  }
  const int off = ax.off[s], n = ax.n[s];
  const int L = ax.left[s], R = ax.right[s];
  if (!grid_range_ok(a.g, base, base + (long long)(ax.N - 1) * stride, BC_CORR)) return;  // the whole pencil
  const float2* __restrict__ F = a.F;
  float2* C = a.C;
  auto at = [&](int pos) { return F[base + (long long)pos * stride]; };
  // first t layers: out[q] = sum_b w[q - b + t - 1] (f_left[n_l - t + b] - f_s[n - t + b])
  for (int q = 0; q < t; q++) {
    float vx = 0.f, vy = 0.f;
    for (int b = 0; b < t; b++) {
      float2 f = at(off + n - t + b);
      f = make_float2(-f.x, -f.y);
      if (L >= 0) f = cadd(f, at(ax.off[L] + ax.n[L] - t + b));
      vx = fmaf(w[q - b + t - 1], f.x, vx);
      vy = fmaf(w[q - b + t - 1], f.y, vy);
    }
    put(C, base + (long long)(off + q) * stride, times_i(vx, vy), add);
  }
  // last t layers: out[n - t + aa] = sum_b w[b - aa + t - 1] (f_right[b] - f_s[b])
  for (int aa = 0; aa < t; aa++) {
    float vx = 0.f, vy = 0.f;
    for (int b = 0; b < t; b++) {
      float2 f = at(off + b);
      f = make_float2(-f.x, -f.y);
      if (R >= 0) f = cadd(f, at(ax.off[R] + b));
      vx = fmaf(w[b - aa + t - 1], f.x, vx);
      vy = fmaf(w[b - aa + t - 1], f.y, vy);
    }
    const int q = n - t + aa;
    // a voxel also in the first range (n < 2t) was written just above by this thread
    put(C, base + (long long)(off + q) * stride, times_i(vx, vy), add || q < t);
  }
}

template <int T>
cudaError_t launch_corr_t(const CorrArgs& a, cudaStream_t st) {
  const AxisDesc& ax = a.g.ax[a.axis];
  if (a.axis == 2) {
    const size_t smem = (size_t)8 * ax.S * 2 * T * sizeof(float2);
    if (smem > 48 * 1024) {
      const cudaError_t e = cudaFuncSetAttribute(k_corr_rows<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e) return e;
    }
    const long long rows = a.g.N0 * a.g.N1;
    const long long blocks = (rows + 7) / 8 < 152 * 16 ? (rows + 7) / 8 : 152 * 16;
    k_corr_rows<T><<<(unsigned)blocks, 256, smem, st>>>(a);
    return cudaGetLastError();
  }
  const long long npen = a.axis == 0 ? a.g.N1 * a.g.N2 : a.g.N0 * a.g.N2;
  bool split = a.variant == 0;
  for (int s = 0; s < ax.S; s++) split = split && ax.n[s] >= 2 * T;
  const int bs = a.block == 64 ? 64 : 128;
  if (split) {
    const unsigned blocks = (unsigned)((2 * npen * ax.S + bs - 1) / bs);
    k_corr_side<T><<<blocks, bs, 0, st>>>(a);
  } else {
    const unsigned blocks = (unsigned)((npen * ax.S + bs - 1) / bs);
    k_corr_strided<T><<<blocks, bs, 0, st>>>(a);
  }
  return cudaGetLastError();
}

// Widths with specialised kernels: 1..16, 20, 24, 32; any other t up to kMaxT
// takes k_corr_generic (t = 0 has no corrections at all).
bool corr_t_supported(int t) { return t >= 0 && t <= kMaxT; }

cudaError_t launch_corr_tc(const CorrArgs& a, cudaStream_t st) {
  const AxisDesc& ax = a.g.ax[a.axis];
  const long long npen = a.axis == 0 ? a.g.N1 * a.g.N2 : (a.axis == 1 ? a.g.N0 * a.g.N2 : a.g.N0 * a.g.N1);
  const long long warps = (npen + 31) / 32 * ax.S * 2;
  const unsigned blocks = (unsigned)((warps + 3) / 4);
  const int t = a.g.t;
  if (t == 8)
    k_corr_tc<8, 8><<<blocks, 128, 0, st>>>(a);
  else if (t <= 8)
    k_corr_tc<8, 0><<<blocks, 128, 0, st>>>(a);
  else if (t <= 16)
    k_corr_tc<16, 0><<<blocks, 128, 0, st>>>(a);
  else if (t <= 24)
    k_corr_tc<24, 0><<<blocks, 128, 0, st>>>(a);
  else
    k_corr_tc<32, 0><<<blocks, 128, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_corr(const CorrArgs& a, cudaStream_t st) {
  if (a.tc) {
    // the two ranges must not overlap (every subdomain on the axis has n >= 2t)
    for (int s = 0; s < a.g.ax[a.axis].S; s++)
      if (a.g.ax[a.axis].n[s] < 2 * a.g.t) return cudaErrorInvalidValue;
    return launch_corr_tc(a, st);
  }
  switch (a.g.t) {
#define MBS_T(T) \
  case T:        \
    return launch_corr_t<T>(a, st);
    MBS_T(1) MBS_T(2) MBS_T(3) MBS_T(4) MBS_T(5) MBS_T(6) MBS_T(7) MBS_T(8)
    MBS_T(9) MBS_T(10) MBS_T(11) MBS_T(12) MBS_T(13) MBS_T(14) MBS_T(15) MBS_T(16)
    MBS_T(20) MBS_T(24) MBS_T(32)
#undef MBS_T
    default: {
      if (a.g.t < 1 || a.g.t > kMaxT) return cudaErrorInvalidValue;
      const AxisDesc& ax = a.g.ax[a.axis];
      const long long npen = a.axis == 0 ? a.g.N1 * a.g.N2 : (a.axis == 1 ? a.g.N0 * a.g.N2 : a.g.N0 * a.g.N1);
      k_corr_generic<<<(unsigned)((npen * ax.S + 127) / 128), 128, 0, st>>>(a);
      return cudaGetLastError();
    }
  }
}

// Boundary-layer voxels, with E = C[v] (the summed corrections of the voxel):
//   UPDATE_ITER:    r = B e - E, x <- x - alpha r, FP64 |r|^2   (e from the last pass)
//   UPDATE_PRECOND: out = -(B e - E)
//   ADD_E:          out += E          SET_E: out = E
// Two index spaces, both walked in batches of U voxels per thread with every
// load issued first: (1) whole grid rows inside an axis-0/1 layer (warp per
// row), (2) the axis-2 layer positions of all other rows, flattened.
template <int U, int MODE>
__device__ __forceinline__ float shell_batch(const ShellArgs& a, const long long (&v)[U]) {
  constexpr int mode = MODE;
  const bool upd = mode == SHELL_UPDATE_ITER || mode == SHELL_UPDATE_PRECOND || mode == SHELL_UPDATE_RES;
  float2 ev[U], cv[U], xv[U], bv[U];
#pragma unroll
  for (int u = 0; u < U; u++) {
    if (v[u] < 0) continue;
    cv[u] = a.C[v[u]];
    if (upd) {
      ev[u] = a.E[v[u]];
      bv[u] = a.B[v[u]];
      if (mode == SHELL_UPDATE_ITER || mode == SHELL_UPDATE_RES) xv[u] = a.X[v[u]];
    } else if (mode == SHELL_ADD_E) {
      xv[u] = a.out[v[u]];
    }
  }
  float racc = 0.f;
#pragma unroll
  for (int u = 0; u < U; u++) {
    if (v[u] < 0) continue;
    if (mode == SHELL_UPDATE_RES) {
      // residual form: r'_{n+1} = r'_n - alpha (B e - E e); its |r'_n|^2 was summed by the last pass
      const float2 r = csub(cmul(bv[u], ev[u]), cv[u]);
      a.X[v[u]] = make_float2(fmaf(-a.alpha, r.x, xv[u].x), fmaf(-a.alpha, r.y, xv[u].y));
    } else if (upd) {
      const float2 r = csub(cmul(bv[u], ev[u]), cv[u]);
      racc = fmaf(r.x, r.x, fmaf(r.y, r.y, racc));
      if (mode == SHELL_UPDATE_ITER)
        a.X[v[u]] = make_float2(fmaf(-a.alpha, r.x, xv[u].x), fmaf(-a.alpha, r.y, xv[u].y));
      else
        a.out[v[u]] = make_float2(-r.x, -r.y);
    } else if (mode == SHELL_ADD_E) {
      a.out[v[u]] = cadd(xv[u], cv[u]);
    } else {
      a.out[v[u]] = cv[u];
    }
  }
  return racc;
}

template <int MODE>
__global__ void __launch_bounds__(256, 4) k_shell(const __grid_constant__ ShellArgs a) {
  __shared__ double red[8];
  if (a.state && a.state->done) return;
  constexpr int U = 4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long N2 = a.g.N2;
  double acc = 0.0;  // FP64 across batches; each batch's (<= U voxels) partial is FP32
  // (1) rows inside an axis-0/1 layer: warp per row
  const long long nfull = (long long)a.tb.nl0 * a.g.N1 + (long long)(a.g.N0 - a.tb.nl0) * a.tb.nl1;
  for (long long fr = (long long)blockIdx.x * 8 + warp; fr < nfull; fr += (long long)gridDim.x * 8) {
    long long i0, i1;
    const long long f0 = (long long)a.tb.nl0 * a.g.N1;
    if (fr < f0) {  // i0 in an axis-0 layer, any i1
      i0 = a.tb.l0[fr / a.g.N1];
      i1 = fr - (fr / a.g.N1) * a.g.N1;
    } else {        // i0 outside, i1 in an axis-1 layer
      const long long q = fr - f0;
      i0 = a.tb.c0[q / a.tb.nl1];
      i1 = a.tb.l1[q - (q / a.tb.nl1) * a.tb.nl1];
    }
    const long long rb = (i0 * a.g.N1 + i1) * N2;
    if (!grid_range_ok(a.g, rb, rb + N2 - 1, BC_SHELL)) continue;  // the warp's row
    for (long long k0 = 0; k0 < N2; k0 += 32 * U) {
      long long v[U];
#pragma unroll
      for (int u = 0; u < U; u++) {
        const long long k = k0 + lane + 32 * u;
        v[u] = k < N2 ? rb + k : -1;
      }
      acc += (double)shell_batch<U, MODE>(a, v);
    }
  }
  // (2) axis-2 layer positions of rows outside the axis-0/1 layers, flattened
  // (32-bit index arithmetic while the flattened count fits: 64-bit division
  // per voxel would dominate this loop)
  const long long nc1 = a.g.N1 - a.tb.nl1;
  const long long npart = (a.g.N0 - a.tb.nl0) * nc1 * a.tb.nsh2;
  const long long nth = (long long)gridDim.x * blockDim.x;
  const bool narrow = npart < (1ll << 31);
  const unsigned nsh2 = (unsigned)a.tb.nsh2, nc1u = (unsigned)nc1;
  for (long long j0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; j0 < npart; j0 += nth * U) {
    long long v[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      const long long j = j0 + nth * u;
      v[u] = -1;
      if (j < npart) {
        long long i0, i1, k;
        if (narrow) {
          const unsigned ju = (unsigned)j, row = ju / nsh2, q = row / nc1u;
          k = ju - row * nsh2;
          i0 = a.tb.c0[q];
          i1 = a.tb.c1[row - q * nc1u];
        } else {
          const long long row = j / a.tb.nsh2;
          k = j - row * a.tb.nsh2;
          i0 = a.tb.c0[row / nc1];
          i1 = a.tb.c1[row - (row / nc1) * nc1];
        }
        v[u] = (i0 * a.g.N1 + i1) * N2 + a.tb.sh2list[k];
        if (!grid_range_ok(a.g, v[u], v[u], BC_SHELL)) v[u] = -1;
      }
    }
    acc += (double)shell_batch<U, MODE>(a, v);
  }
  if (a.partials) {
    const double s = block_sum(acc, red);
    finish_block(Finish{a.partials, a.slot0, a.n_total, a.fin, a.hist}, s, red);
  }
}

// Layer update with the axis-2 corrections fused in (SHELL_UPDATE_ITER or
// SHELL_UPDATE_RES), in two independent parts of one launch:
//   (a) rows inside an axis-0/1 layer, their voxels outside the axis-2 layers:
//       E e = C (the axis-0/1 terms), warp per row, U voxels per lane in flight;
//   (b) the axis-2 layer voxels of every row ("slots": per subdomain s its
//       first t, then its last t voxels; M = 2tS <= 32 J, J per lane), warp per
//       pair of rows: all loads of both rows are issued first (e, B, x and, on
//       rows inside an axis-0/1 layer, C), e is staged in shared memory, then
//       each slot's axis-2 correction (Sec. 3.1 steps 1-5, the formulas of
//       k_corr_rows) gives E e = C + E_2 e and the update.
// c is purely imaginary and W real: c W = i w with w = Im(c W), so
// sum_b cW_b f_b = i v with v = sum_b w_b f_b.
constexpr int kShellRowsMaxSlots = 64;

template <int TC>
__device__ __forceinline__ float2 axis2_corr_sum(const float* w, int t, int q, int n, const float2* own,
                                                 const float2* nbl, const float2* nbr) {
  float vx = 0.f, vy = 0.f;
  const int T = TC > 0 ? TC : t;
  if (q < T) {  // first t layers: row q of W^T on (left's last t - own last t)
#pragma unroll (TC > 0 ? TC : 1)
    for (int b = 0; b < T; b++) {
      float2 f = make_float2(-own[T + b].x, -own[T + b].y);
      if (nbl) f = cadd(f, nbl[b]);
      vx = fmaf(w[q - b + T - 1], f.x, vx);
      vy = fmaf(w[q - b + T - 1], f.y, vy);
    }
  }
  if (q >= n - T) {  // last t layers: row q-(n-t) of W on (right's first t - own first t)
    const int aa = q - (n - T);
#pragma unroll (TC > 0 ? TC : 1)
    for (int b = 0; b < T; b++) {
      float2 f = make_float2(-own[b].x, -own[b].y);
      if (nbr) f = cadd(f, nbr[b]);
      vx = fmaf(w[b - aa + T - 1], f.x, vx);
      vy = fmaf(w[b - aa + T - 1], f.y, vy);
    }
  }
  return make_float2(-vy, vx);  // i v
}

template <int MODE>
__device__ __forceinline__ float2 layer_step(float2 b, float2 e, float2 corr, float2 x, float alpha, float& racc) {
  const float2 r = csub(cmul(b, e), corr);
  if (MODE == SHELL_UPDATE_ITER) racc = fmaf(r.x, r.x, fmaf(r.y, r.y, racc));
  return make_float2(fmaf(-alpha, r.x, x.x), fmaf(-alpha, r.y, x.y));
}

// bx, nx: this block and the block count of the plan's launch (the loops stride by nx).
template <int MODE, int TC, int J>
__device__ __forceinline__ void shell_rows_body(const ShellArgs& a, unsigned bx, unsigned nx) {
  extern __shared__ float2 ws[];  // [8 warps][2 rows][M] staged e
  __shared__ double red[8];
  __shared__ float w[2 * kMaxT];  // w[m] = Im(c W) at column - row = m - (t - 1)
  if (a.state && a.state->done) return;
  constexpr int U = 4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int t = TC > 0 ? TC : a.g.t;
  const AxisDesc& ax = a.g.ax[2];
  const int M = (ax.a > 0 && t > 0) ? 2 * t * ax.S : 0;
  if (threadIdx.x < 2 * t - 1) {
    const int m = threadIdx.x, aa = m < t - 1 ? t - 1 - m : 0, bb = aa + m - (t - 1);
    w[m] = a.cW[aa * t + bb].y;
  }
  __syncthreads();
  const unsigned N1 = (unsigned)a.g.N1;
  const unsigned n2 = (unsigned)a.g.N2;
  const unsigned char* __restrict__ sh2 = a.tb.shell[2];
  double acc = 0.0;
  // (a) rows inside an axis-0/1 layer, voxels outside the axis-2 layers
  {
    const unsigned nl0 = (unsigned)a.tb.nl0, nl1 = (unsigned)a.tb.nl1;
    const unsigned f0 = nl0 * N1;
    const unsigned nfull = f0 + ((unsigned)a.g.N0 - nl0) * nl1;
    for (unsigned fr = bx * 8u + warp; fr < nfull; fr += nx * 8u) {
      unsigned i0, i1;
      if (fr < f0) {
        i0 = (unsigned)a.tb.l0[fr / N1];
        i1 = fr - (fr / N1) * N1;
      } else {
        const unsigned q = fr - f0;
        i0 = (unsigned)a.tb.c0[q / nl1];
        i1 = (unsigned)a.tb.l1[q - (q / nl1) * nl1];
      }
      const long long rb = ((long long)i0 * N1 + i1) * (long long)n2;
      if (!grid_range_ok(a.g, rb, rb + n2 - 1, BC_SHELL)) continue;  // the warp's row
      const float2* Cr = a.C + rb;
      const float2* Er = a.E + rb;
      const float2* __restrict__ Br = a.B + rb;
      float2* Xr = a.X + rb;
      const int j0 = a.active ? a.tb.sub[0][i0] : 0, j1 = a.active ? a.tb.sub[1][i1] : 0;
      for (unsigned k0 = lane; k0 < n2; k0 += 32 * U) {
        float2 e[U], c[U], b[U], x[U];
        bool ok[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
          const unsigned k = k0 + 32 * u;
          ok[u] = k < n2 && !sh2[k] && (!a.active || sub_active(a.active, a.g, j0, j1, a.tb.sub[2][k]));
          if (ok[u]) {
            c[u] = Cr[k];
            e[u] = Er[k];
            b[u] = __ldg(Br + k);
            x[u] = Xr[k];
          }
        }
        float r2 = 0.f;
#pragma unroll
        for (int u = 0; u < U; u++)
          if (ok[u]) Xr[k0 + 32 * u] = layer_step<MODE>(b[u], e[u], c[u], x[u], a.alpha, r2);
        acc += (double)r2;
      }
    }
  }
  // (b) the axis-2 layer voxels of every row, with their axis-2 corrections
  if (M > 0) {
    float2* evw = ws + warp * 2 * M;
    int sj[J], qj[J];
    bool use[J];
#pragma unroll
    for (int j = 0; j < J; j++) {
      const int idx = lane + 32 * j;
      use[j] = idx < M;
      sj[j] = use[j] ? idx / (2 * t) : 0;
      const int k = idx - sj[j] * 2 * t, n = ax.n[sj[j]];
      qj[j] = k < t ? k : n - t + (k - t);
      if (k >= t && qj[j] < t) use[j] = false;  // n < 2t: the voxel is the first-range slot q (still staged)
    }
    const unsigned rows = (unsigned)(a.g.N0 * a.g.N1);
    const unsigned step = nx * 8u;
    for (unsigned rho0 = bx * 8u + warp; rho0 < rows; rho0 += 2 * step) {
      const unsigned rho1 = rho0 + step;
      const bool live1 = rho1 < rows;
      const unsigned i00 = rho0 / N1, i10 = rho0 - i00 * N1;
      const unsigned i01 = live1 ? rho1 / N1 : 0, i11 = live1 ? rho1 - i01 * N1 : 0;
      const bool full0 = a.tb.shell[0][i00] | a.tb.shell[1][i10];
      const bool full1 = live1 && (a.tb.shell[0][i01] | a.tb.shell[1][i11]);
      // subdomains along axes 0, 1 of the two rows (activation: inactive slots keep x = 0; their
      // e, zero, still enters the neighbours' corrections)
      const int r00 = a.active ? a.tb.sub[0][i00] : 0, r10 = a.active ? a.tb.sub[1][i10] : 0;
      const int r01 = a.active && live1 ? a.tb.sub[0][i01] : 0, r11 = a.active && live1 ? a.tb.sub[1][i11] : 0;
      const long long rb0 = (long long)rho0 * n2, rb1 = (long long)rho1 * n2;
      if (!grid_range_ok(a.g, rb0, (live1 ? rb1 : rb0) + n2 - 1, BC_SHELL)) continue;  // the warp's two rows
      float2 e0[J], b0[J], x0[J], c0[J], e1[J], b1[J], x1[J], c1[J];
#pragma unroll
      for (int j = 0; j < J; j++) {
        if (lane + 32 * j < M) {
          const long long o = ax.off[sj[j]] + qj[j];
          e0[j] = a.E[rb0 + o];
          b0[j] = __ldg(a.B + rb0 + o);
          x0[j] = a.X[rb0 + o];
          c0[j] = full0 ? a.C[rb0 + o] : make_float2(0.f, 0.f);
          if (live1) {
            e1[j] = a.E[rb1 + o];
            b1[j] = __ldg(a.B + rb1 + o);
            x1[j] = a.X[rb1 + o];
            c1[j] = full1 ? a.C[rb1 + o] : make_float2(0.f, 0.f);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < J; j++) {
        if (lane + 32 * j < M) {
          evw[lane + 32 * j] = e0[j];
          if (live1) evw[M + lane + 32 * j] = e1[j];
        }
      }
      __syncwarp();
      float racc = 0.f;
#pragma unroll
      for (int j = 0; j < J; j++) {
        if (!use[j]) continue;
        const int s = sj[j], lft = ax.left[s], rgt = ax.right[s];
        const long long o = ax.off[s] + qj[j];
        if (sub_active(a.active, a.g, r00, r10, s)) {
          const float2* ev = evw;
          const float2 corr = axis2_corr_sum<TC>(w, t, qj[j], ax.n[s], ev + s * 2 * t,
                                                 lft >= 0 ? ev + lft * 2 * t + t : nullptr,
                                                 rgt >= 0 ? ev + rgt * 2 * t : nullptr);
          a.X[rb0 + o] = layer_step<MODE>(b0[j], e0[j], cadd(c0[j], corr), x0[j], a.alpha, racc);
        }
        if (live1 && sub_active(a.active, a.g, r01, r11, s)) {
          const float2* ev = evw + M;
          const float2 corr = axis2_corr_sum<TC>(w, t, qj[j], ax.n[s], ev + s * 2 * t,
                                                 lft >= 0 ? ev + lft * 2 * t + t : nullptr,
                                                 rgt >= 0 ? ev + rgt * 2 * t : nullptr);
          a.X[rb1 + o] = layer_step<MODE>(b1[j], e1[j], cadd(c1[j], corr), x1[j], a.alpha, racc);
        }
      }
      acc += (double)racc;
      __syncwarp();
    }
  }
  if (a.partials) {
    const double sum = block_sum(acc, red);
    finish_block_at(Finish{a.partials, a.slot0, a.n_total, a.fin, a.hist}, sum, red, bx, nx);
  }
}

template <int MODE, int TC, int J>
__global__ void __launch_bounds__(256, J == 1 ? 4 : 3) k_shell_rows(const __grid_constant__ ShellArgs a) {
  shell_rows_body<MODE, TC, J>(a, blockIdx.x, gridDim.x);
}

template <int MODE, int TC, int J>
__global__ void __launch_bounds__(256, J == 1 ? 4 : 3) k_shell_rows_batch(const ShellArgs* __restrict__ d) {
  __shared__ ShellArgs a;
  const unsigned nb = (unsigned)d[blockIdx.y].nblocks;
  if (blockIdx.x >= nb) return;
  stage_args(&a, &d[blockIdx.y]);
  shell_rows_body<MODE, TC, J>(a, blockIdx.x, nb);
}

bool shell_rows_supported(const GridDesc& g) {
  const int M = (g.ax[2].a > 0 && g.t > 0) ? 2 * g.t * g.ax[2].S : 0;
  return M <= kShellRowsMaxSlots && g.N0 * g.N1 < (1ll << 31);
}

cudaError_t launch_shell_rows(const ShellArgs& a, int blocks, cudaStream_t st) {
  if (!shell_rows_supported(a.g)) return cudaErrorInvalidValue;
  const int M = (a.g.ax[2].a > 0 && a.g.t > 0) ? 2 * a.g.t * a.g.ax[2].S : 0;
  const size_t smem = (size_t)8 * 2 * M * sizeof(float2);  // <= 8 KB
  const bool t8 = a.g.t == 8, one = M <= 32;
#define MBS_SHELL_ROWS(MODE)                                                                       \
  if (t8 && one) k_shell_rows<MODE, 8, 1><<<blocks, 256, smem, st>>>(a);                           \
  else if (t8) k_shell_rows<MODE, 8, 2><<<blocks, 256, smem, st>>>(a);                             \
  else if (one) k_shell_rows<MODE, 0, 1><<<blocks, 256, smem, st>>>(a);                            \
  else k_shell_rows<MODE, 0, 2><<<blocks, 256, smem, st>>>(a);
  if (a.mode == SHELL_UPDATE_ITER) {
    MBS_SHELL_ROWS(SHELL_UPDATE_ITER)
  } else if (a.mode == SHELL_UPDATE_RES) {
    MBS_SHELL_ROWS(SHELL_UPDATE_RES)
  } else {
    return cudaErrorInvalidValue;
  }
#undef MBS_SHELL_ROWS
  return cudaGetLastError();
}

// Batched layer update of the iteration (x form, SHELL_UPDATE_ITER) over the
// plans of d (grid blocks x m); every plan must fit the fused form, with t and
// the row-pair staging (M <= 32 or not) given for all of them.
cudaError_t launch_shell_rows_batch(const ShellArgs* d, int m, int t, int max_slots, int blocks, cudaStream_t st) {
  const size_t smem = (size_t)8 * 2 * max_slots * sizeof(float2);
  const dim3 grid((unsigned)blocks, (unsigned)m);
  const bool t8 = t == 8, one = max_slots <= 32;
  if (t8 && one) k_shell_rows_batch<SHELL_UPDATE_ITER, 8, 1><<<grid, 256, smem, st>>>(d);
  else if (t8) k_shell_rows_batch<SHELL_UPDATE_ITER, 8, 2><<<grid, 256, smem, st>>>(d);
  else if (one) k_shell_rows_batch<SHELL_UPDATE_ITER, 0, 1><<<grid, 256, smem, st>>>(d);
  else k_shell_rows_batch<SHELL_UPDATE_ITER, 0, 2><<<grid, 256, smem, st>>>(d);
  return cudaGetLastError();
}

// Batched FP32 edge corrections of one axis (0 or 1) with the side-split kernel
// (every subdomain edge on the axis >= 2t) over the plans of d; max_threads: the
// largest 2 * pencils * subdomains of the plans.
cudaError_t launch_corr_side_batch(const CorrArgs* d, int m, int t, long long max_threads, cudaStream_t st) {
  const dim3 grid((unsigned)((max_threads + 127) / 128), (unsigned)m);
  switch (t) {
#define MBS_TB(T)                                         \
  case T:                                                 \
    k_corr_side_batch<T><<<grid, 128, 0, st>>>(d);        \
    return cudaGetLastError();
    MBS_TB(1) MBS_TB(2) MBS_TB(3) MBS_TB(4) MBS_TB(5) MBS_TB(6) MBS_TB(7) MBS_TB(8)
    MBS_TB(9) MBS_TB(10) MBS_TB(11) MBS_TB(12) MBS_TB(13) MBS_TB(14) MBS_TB(15) MBS_TB(16)
    MBS_TB(20) MBS_TB(24) MBS_TB(32)
#undef MBS_TB
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_shell(const ShellArgs& a, int blocks, cudaStream_t st) {
  switch (a.mode) {
    case SHELL_UPDATE_ITER: k_shell<SHELL_UPDATE_ITER><<<blocks, 256, 0, st>>>(a); break;
    case SHELL_UPDATE_PRECOND: k_shell<SHELL_UPDATE_PRECOND><<<blocks, 256, 0, st>>>(a); break;
    case SHELL_UPDATE_RES: k_shell<SHELL_UPDATE_RES><<<blocks, 256, 0, st>>>(a); break;
    case SHELL_ADD_E: k_shell<SHELL_ADD_E><<<blocks, 256, 0, st>>>(a); break;
    default: k_shell<SHELL_SET_E><<<blocks, 256, 0, st>>>(a); break;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Activation check (Sec. 3.1, "Implementation"): squared norm of the field an
// active neighbour transfers into an inactive subdomain's boundary layers.
// Block row y handles face y; its threads walk the face's pencils along the
// face axis. The transfer from a left neighbour is c W^T on its last t layers,
// from a right neighbour c W on its first t layers; with c W = i w (w real) its
// squared modulus is |w v|^2.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_act_norms(const float2* __restrict__ X, const ActFace* faces, GridDesc g,
                                                   const float2* __restrict__ cW, double* norms) {
  __shared__ float w[2 * kMaxT];
  __shared__ double red[8];
  const int t = g.t;
  if (threadIdx.x < 2 * t - 1) {
    const int m = threadIdx.x, aa = m < t - 1 ? t - 1 - m : 0, bb = aa + m - (t - 1);
    w[m] = cW[aa * t + bb].y;
  }
  __syncthreads();
  const ActFace f = faces[blockIdx.y];
  const int d = f.axis;
  int jn[3];  // the neighbour's subdomain coordinates
  {
    const int S1 = g.ax[1].S, S2 = g.ax[2].S;
    jn[0] = f.nb / (S1 * S2);
    jn[1] = (f.nb / S2) % S1;
    jn[2] = f.nb % S2;
  }
  const int da = d == 0 ? 1 : 0, db = d == 2 ? 1 : 2;  // the two face axes
  const long long st[3] = {g.N1 * g.N2, g.N2, 1};
  const int na = g.ax[da].n[jn[da]], nb = g.ax[db].n[jn[db]];
  const long long org = (long long)g.ax[da].off[jn[da]] * st[da] + (long long)g.ax[db].off[jn[db]] * st[db];
  const int nd = g.ax[d].n[jn[d]];
  const long long l0 = (long long)(g.ax[d].off[jn[d]] + (f.left ? nd - t : 0)) * st[d];
  float acc = 0.f;
  double dacc = 0.0;
  for (long long pp = (long long)blockIdx.x * blockDim.x + threadIdx.x; pp < (long long)na * nb;
       pp += (long long)gridDim.x * blockDim.x) {
    const long long ia = pp / nb, ib = pp - ia * nb;
    const long long base = org + ia * st[da] + ib * st[db] + l0;
    if (!grid_range_ok(g, base, base + (long long)(t - 1) * st[d], BC_CORR)) continue;
    for (int q = 0; q < t; q++) {
      float vx = 0.f, vy = 0.f;
      for (int b = 0; b < t; b++) {
        const float2 xv = X[base + (long long)b * st[d]];
        // left neighbour: row q of W^T (W[b][q]); right neighbour: row q of W (W[q][b])
        const float wv = f.left ? w[q - b + t - 1] : w[b - q + t - 1];
        vx = fmaf(wv, xv.x, vx);
        vy = fmaf(wv, xv.y, vy);
      }
      acc = fmaf(vx, vx, fmaf(vy, vy, acc));
    }
    dacc += (double)acc;  // FP32 over one pencil's t outputs, then FP64
    acc = 0.f;
  }
  const double s = block_sum(dacc, red);
  if (threadIdx.x == 0 && s > 0.0) atomicAdd(norms + f.s, s);
}

cudaError_t launch_act_norms(const float2* X, const ActFace* faces, int nfaces, const GridDesc& g, const float2* cW,
                             double* norms, cudaStream_t st) {
  if (nfaces <= 0) return cudaSuccess;
  const dim3 grid(64, (unsigned)nfaces);
  k_act_norms<<<grid, 256, 0, st>>>(X, faces, g, cW, norms);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The plain form: one launch per step of Eq. wavesim_iter over the whole grid.
// A block walks grid rows (i0, i1); its threads take the row's axis-2 positions.
// Corrections (C) are valid on the boundary-layer voxels only.
// ---------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(256) k_plain_step(const __grid_constant__ PlainArgs a) {
  __shared__ double red[8];
  const long long N1 = a.g.N1, N2 = a.g.N2, rows = a.g.N0 * N1;
  double acc = 0.0;
  for (long long rho = blockIdx.x; rho < rows; rho += gridDim.x) {
    const long long i0 = rho / N1, i1 = rho - i0 * N1;
    const bool lay01 = a.tb.shell[0][i0] | a.tb.shell[1][i1];
    const bool srow = a.S && i0 >= a.sbox[0] && i0 < a.sbox[1] && i1 >= a.sbox[2] && i1 < a.sbox[3];
    const long long rb = rho * N2;
    if (!grid_range_ok(a.g, rb, rb + N2 - 1, BC_PLAIN)) continue;  // the block's row
    float racc = 0.f;
    for (long long i2 = threadIdx.x; i2 < N2; i2 += blockDim.x) {
      const long long v = rb + i2;
      const bool lay = lay01 || a.tb.shell[2][i2];
      if (MODE == PLAIN_U) {
        float2 u = cmul(a.B[v], a.X[v]);
        if (lay) u = csub(u, a.C[v]);
        if (srow && i2 >= a.sbox[4] && i2 < a.sbox[5]) u = cadd(u, cmul(a.mc, a.S[v]));
        a.K[v] = u;
      } else if (MODE == PLAIN_PROP) {
        const float p2 = a.tb.p2[0][i0] + a.tb.p2[1][i1] + a.tb.p2[2][i2];
        // c (k0^2 - |p|^2) + 1
        const float2 den = make_float2(fmaf(-a.c.x, p2, a.ck0.x) + 1.f, fmaf(-a.c.y, p2, a.ck0.y));
        const float inv = 1.f / (den.x * den.x + den.y * den.y);
        a.K[v] = cmul(a.K[v], make_float2(den.x * inv, -den.y * inv));
      } else if (MODE == PLAIN_D) {
        a.K[v] = csub(a.X[v], a.K[v]);
      } else if (MODE == PLAIN_R) {
        float2 r = cmul(a.B[v], a.K[v]);
        if (lay) r = csub(r, a.C[v]);
        a.K[v] = r;
      } else if (MODE == PLAIN_NORM) {
        const float2 r = a.K[v];
        racc = fmaf(r.x, r.x, fmaf(r.y, r.y, racc));
      } else {
        const float2 r = a.K[v], x = a.X[v];
        a.X[v] = make_float2(fmaf(-a.alpha, r.x, x.x), fmaf(-a.alpha, r.y, x.y));
      }
    }
    if (MODE == PLAIN_NORM) acc += (double)racc;  // FP32 over at most N2 / 256 voxels, then FP64
  }
  if (MODE == PLAIN_NORM) {
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) a.partials[blockIdx.x] = s;
  }
}

cudaError_t launch_plain_step(const PlainArgs& a, cudaStream_t st) {
  switch (a.mode) {
    case PLAIN_U: k_plain_step<PLAIN_U><<<kPlainBlocks, 256, 0, st>>>(a); break;
    case PLAIN_PROP: k_plain_step<PLAIN_PROP><<<kPlainBlocks, 256, 0, st>>>(a); break;
    case PLAIN_D: k_plain_step<PLAIN_D><<<kPlainBlocks, 256, 0, st>>>(a); break;
    case PLAIN_R: k_plain_step<PLAIN_R><<<kPlainBlocks, 256, 0, st>>>(a); break;
    case PLAIN_NORM: k_plain_step<PLAIN_NORM><<<kPlainBlocks, 256, 0, st>>>(a); break;
    case PLAIN_UPD: k_plain_step<PLAIN_UPD><<<kPlainBlocks, 256, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

__global__ void k_state_arm(DevState* st, int add_iter, double tol, int reset, int hist_cap) {
  if (reset) {
    st->iter = 0;
    st->R0 = 0.0;
    st->r0_fixed = 0;
    st->eps = 1.0;
    st->best = 1e300;
    st->rise = 0;
    st->status = 0;
    st->hist_cap = hist_cap;
    st->ticket = 0u;
  }
  st->max_iter = st->iter + add_iter;
  st->tol = tol;
  st->done = (add_iter > 0 && st->status == 0) ? 0 : 1;
}

cudaError_t launch_state_arm(DevState* state, int add_iter, double tol, int reset, int hist_cap, cudaStream_t st) {
  k_state_arm<<<1, 1, 0, st>>>(state, add_iter, tol, reset, hist_cap);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Plan set-up in FP64: absorbing ramp, k^2, bounds, contrast and B.
// ---------------------------------------------------------------------------
// Linear absorbing ramp of one axis: (w - i)/w at depth i from a face of width
// w, the larger of the two faces' values; the voxel's ramp is the largest over
// the three axes (faces meeting at edges and corners do not add).
struct Ramp {
  __device__ static double at(long long i, long long N, int lo, int hi) {
    double r = 0.0;
    if (lo > 0 && i < lo) r = fmax(r, (double)(lo - i) / lo);
    const long long j = N - 1 - i;
    if (hi > 0 && j < hi) r = fmax(r, (double)(hi - j) / hi);
    return r;
  }
};

__device__ __forceinline__ void k2_at(const float2* n, long long v, const GridDesc& g, const int* w, double kappa,
                                      double lambda, double& kr, double& ki) {
  const long long i0 = v / (g.N1 * g.N2), rem = v - i0 * g.N1 * g.N2, i1 = rem / g.N2, i2 = rem - i1 * g.N2;
  const double ramp = fmax(fmax(Ramp::at(i0, g.N0, w[0], w[1]), Ramp::at(i1, g.N1, w[2], w[3])),
                           Ramp::at(i2, g.N2, w[4], w[5]));
  const float2 nn = n[v];
  const double nr = nn.x, ni = (double)nn.y + kappa * ramp;
  const double s = 2.0 * 3.14159265358979323846 / lambda;
  const double kr0 = s * nr, ki0 = s * ni;
  kr = kr0 * kr0 - ki0 * ki0;
  ki = 2.0 * kr0 * ki0;
}

struct Widths {
  int w[6];
};

// Per-block bounds of k^2 over the grid: min/max of Re and Im, max |k^2| and a
// count of non-finite values (6 doubles per block).
__global__ void k_k2_bounds(const float2* __restrict__ n, GridDesc g, Widths w, double kappa, double lambda,
                            double* partials) {
  __shared__ double red[6][8];
  const long long total = g.N0 * g.N1 * g.N2;
  double v6[6] = {1e300, -1e300, 1e300, -1e300, 0.0, 0.0};
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < total; v += (long long)gridDim.x * blockDim.x) {
    double kr, ki;
    k2_at(n, v, g, w.w, kappa, lambda, kr, ki);
    if (!(isfinite(kr) && isfinite(ki))) {
      v6[5] += 1.0;
      continue;
    }
    v6[0] = fmin(v6[0], kr);
    v6[1] = fmax(v6[1], kr);
    v6[2] = fmin(v6[2], ki);
    v6[3] = fmax(v6[3], ki);
    v6[4] = fmax(v6[4], hypot(kr, ki));
  }
  for (int o = 16; o > 0; o >>= 1) {
    v6[0] = fmin(v6[0], __shfl_xor_sync(0xffffffffu, v6[0], o));
    v6[1] = fmax(v6[1], __shfl_xor_sync(0xffffffffu, v6[1], o));
    v6[2] = fmin(v6[2], __shfl_xor_sync(0xffffffffu, v6[2], o));
    v6[3] = fmax(v6[3], __shfl_xor_sync(0xffffffffu, v6[3], o));
    v6[4] = fmax(v6[4], __shfl_xor_sync(0xffffffffu, v6[4], o));
    v6[5] += __shfl_xor_sync(0xffffffffu, v6[5], o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0)
    for (int k = 0; k < 6; k++) red[k][warp] = v6[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); i++) {
      v6[0] = fmin(red[0][0], red[0][i]);
      red[0][0] = v6[0];
      red[1][0] = fmax(red[1][0], red[1][i]);
      red[2][0] = fmin(red[2][0], red[2][i]);
      red[3][0] = fmax(red[3][0], red[3][i]);
      red[4][0] = fmax(red[4][0], red[4][i]);
      red[5][0] += red[5][i];
    }
    for (int k = 0; k < 6; k++) partials[6 * blockIdx.x + k] = red[k][0];
  }
}

cudaError_t launch_k2_bounds(const float2* n, GridDesc g, const int* widths, double kappa, double lambda,
                             double* partials, int blocks, cudaStream_t st) {
  Widths w;
  for (int i = 0; i < 6; i++) w.w[i] = widths[i];
  k_k2_bounds<<<blocks, 256, 0, st>>>(n, g, w, kappa, lambda, partials);
  return cudaGetLastError();
}

__global__ void k_contrast(const float2* __restrict__ n, GridDesc g, Widths w, double kappa, double lambda,
                           double k0r, double k0i, double* partials) {
  __shared__ double red[8];
  const long long total = g.N0 * g.N1 * g.N2;
  double mx = 0.0;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < total; v += (long long)gridDim.x * blockDim.x) {
    double kr, ki;
    k2_at(n, v, g, w.w, kappa, lambda, kr, ki);
    mx = fmax(mx, hypot(kr - k0r, ki - k0i));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = red[0];
    for (int i = 1; i < (int)(blockDim.x >> 5); i++) m = fmax(m, red[i]);
    partials[blockIdx.x] = m;
  }
}

cudaError_t launch_contrast(const float2* n, GridDesc g, const int* widths, double kappa, double lambda,
                            double k0re, double k0im, double* partials, int blocks, cudaStream_t st) {
  Widths w;
  for (int i = 0; i < 6; i++) w.w[i] = widths[i];
  k_contrast<<<blocks, 256, 0, st>>>(n, g, w, kappa, lambda, k0re, k0im, partials);
  return cudaGetLastError();
}

// B = 1 - c (k^2 - k0^2) (Sec. 2: the medium factor I - V of Eq. wavesim_iter),
// evaluated in FP64 and rounded to complex64. May run in place (B == n).
__global__ void k_make_B(const float2* n, float2* B, GridDesc g, Widths w, double kappa, double lambda, double k0r,
                         double k0i, double cr, double ci) {
  const long long total = g.N0 * g.N1 * g.N2;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < total; v += (long long)gridDim.x * blockDim.x) {
    double kr, ki;
    k2_at(n, v, g, w.w, kappa, lambda, kr, ki);
    const double dr = kr - k0r, di = ki - k0i;
    B[v] = make_float2((float)(1.0 - (cr * dr - ci * di)), (float)(-(cr * di + ci * dr)));
  }
}

cudaError_t launch_make_B(const float2* n, float2* B, GridDesc g, const int* widths, double kappa, double lambda,
                          double k0re, double k0im, double cre, double cim, int blocks, cudaStream_t st) {
  Widths w;
  for (int i = 0; i < 6; i++) w.w[i] = widths[i];
  k_make_B<<<blocks, 256, 0, st>>>(n, B, g, w, kappa, lambda, k0re, k0im, cre, cim);
  return cudaGetLastError();
}

// Bounding box of the non-zero source voxels (atomic min/max of the indices).
__global__ void k_source_box(const float2* __restrict__ S, GridDesc g, int* box) {
  const long long total = g.N0 * g.N1 * g.N2;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < total; v += (long long)gridDim.x * blockDim.x) {
    const float2 s = S[v];
    if (s.x != 0.f || s.y != 0.f) {
      const long long i0 = v / (g.N1 * g.N2), rem = v - i0 * g.N1 * g.N2, i1 = rem / g.N2, i2 = rem - i1 * g.N2;
      atomicMin(box + 0, (int)i0);
      atomicMax(box + 1, (int)i0 + 1);
      atomicMin(box + 2, (int)i1);
      atomicMax(box + 3, (int)i1 + 1);
      atomicMin(box + 4, (int)i2);
      atomicMax(box + 5, (int)i2 + 1);
    }
  }
}

cudaError_t launch_source_box(const float2* S, GridDesc g, int* box, int blocks, cudaStream_t st) {
  k_source_box<<<blocks, 256, 0, st>>>(S, g, box);
  return cudaGetLastError();
}

__global__ void k_zero(float2* p, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = make_float2(0.f, 0.f);
}

cudaError_t launch_zero(float2* p, int64_t n, cudaStream_t st) {
  const long long blocks = n / 256 + 1 < 152 * 16 ? n / 256 + 1 : 152 * 16;
  k_zero<<<(unsigned)blocks, 256, 0, st>>>(p, n);
  return cudaGetLastError();
}

__global__ void k_negate_copy(const float2* __restrict__ in, float2* out, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float2 v = in[i];
    out[i] = make_float2(-v.x, -v.y);
  }
}

cudaError_t launch_negate_copy(const float2* in, float2* out, int64_t n, cudaStream_t st) {
  const long long blocks = n / 256 + 1 < 152 * 16 ? n / 256 + 1 : 152 * 16;
  k_negate_copy<<<(unsigned)blocks, 256, 0, st>>>(in, out, n);
  return cudaGetLastError();
}

// out = (1 - B) x = c (k^2 - k0^2) x, the potential part of V.
__global__ void k_pointwise_V(const float2* __restrict__ X, const float2* __restrict__ B, float2* out, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float2 b = B[i];
    out[i] = cmul(make_float2(1.f - b.x, -b.y), X[i]);
  }
}

cudaError_t launch_pointwise_V(const float2* X, const float2* B, float2* out, int64_t n, cudaStream_t st) {
  const long long blocks = n / 256 + 1 < 152 * 16 ? n / 256 + 1 : 152 * 16;
  k_pointwise_V<<<(unsigned)blocks, 256, 0, st>>>(X, B, out, n);
  return cudaGetLastError();
}

}  // namespace mbs
