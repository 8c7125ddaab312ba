// Shared-memory-staged mixed-radix FFT used for the per-subdomain transforms of
// the modified Born series (Sec. 2, Eq. L-convolution; Sec. 3.1: the fast
// convolution with (L_ss + I)^-1 is taken separately on every subdomain s).
//
// Organisation (GB300): one CTA transforms a tile of 32 pencils. Lane l of every
// warp owns pencil l; warp w owns butterflies j = w, w + W, ... of each radix
// stage. Stages follow the self-sorting (Stockham) decimation-in-time scheme
// with mixed radices, so the output is in natural order and no bit reversal
// pass is needed. Between stages the tile lives in shared memory laid out
// [element][33] (one pad column), which keeps both the per-lane element
// accesses and the coalesced row staging free of bank conflicts. The first
// and last stages may read/write global memory directly (strided axes), which
// removes two shared-memory round trips per pass.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mbs {

struct cf { float x, y; };

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <bool INV> __device__ __forceinline__ float2 mul_mi(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// ---------------------------------------------------------------------------
// Small DFT kernels X_k = sum_m a_m exp(-+ 2 pi i m k / R) (sign - forward).
// ---------------------------------------------------------------------------
template <int R, bool INV> struct Dft;

template <bool INV> struct Dft<1, INV> { __device__ __forceinline__ static void run(float2 (&)[1]) {} };

template <bool INV> struct Dft<2, INV> {
  __device__ __forceinline__ static void run(float2 (&v)[2]) {
    float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <bool INV> struct Dft<4, INV> {
  __device__ __forceinline__ static void run(float2 (&v)[4]) {
    float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    float2 t2 = cadd(v[1], v[3]), t3 = mul_mi<INV>(csub(v[1], v[3]));
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
  }
};

template <bool INV> struct Dft<8, INV> {
  __device__ __forceinline__ static void run(float2 (&v)[8]) {
    const float h = 0.70710678118654752f;
    float2 e[4] = {v[0], v[2], v[4], v[6]};
    float2 o[4] = {v[1], v[3], v[5], v[7]};
    Dft<4, INV>::run(e);
    Dft<4, INV>::run(o);
    // twiddles W8^k, k = 0..3
    float2 o1 = INV ? make_float2(h * (o[1].x - o[1].y), h * (o[1].x + o[1].y))
                    : make_float2(h * (o[1].x + o[1].y), h * (o[1].y - o[1].x));
    float2 o2 = mul_mi<INV>(o[2]);
    float2 o3 = INV ? make_float2(-h * (o[3].x + o[3].y), h * (o[3].x - o[3].y))
                    : make_float2(h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y));
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);
    v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);
    v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);
    v[7] = csub(e[3], o3);
  }
};

template <bool INV> struct Dft<16, INV> {
  __device__ __forceinline__ static void run(float2 (&v)[16]) {
    const float c1 = 0.92387953251128676f, s1 = 0.38268343236508977f, h = 0.70710678118654752f;
    float2 e[8], o[8];
#pragma unroll
    for (int i = 0; i < 8; i++) { e[i] = v[2 * i]; o[i] = v[2 * i + 1]; }
    Dft<8, INV>::run(e);
    Dft<8, INV>::run(o);
    const float sg = INV ? 1.f : -1.f;
    // W16^k = cos(pi k/8) + sg*i*sin(pi k/8)
    const float cw[8] = {1.f, c1, h, s1, 0.f, -s1, -h, -c1};
    const float sw[8] = {0.f, s1, h, c1, 1.f, c1, h, s1};
#pragma unroll
    for (int k = 0; k < 8; k++) {
      float2 w = make_float2(cw[k], sg * sw[k]);
      float2 t = (k == 0) ? o[0] : cmul(o[k], w);
      v[k] = cadd(e[k], t);
      v[k + 8] = csub(e[k], t);
    }
  }
};

// Odd primes 3, 5, 7: pairwise symmetric form.
template <int P> struct OddConst;
template <> struct OddConst<3> {
  __device__ __forceinline__ static float c(int k) { return -0.5f; }
  __device__ __forceinline__ static float s(int k) { return k == 1 ? 0.86602540378443865f : -0.86602540378443865f; }
};
template <> struct OddConst<5> {
  __device__ __forceinline__ static float c(int k) {
    return (k == 1 || k == 4) ? 0.30901699437494742f : -0.80901699437494742f;
  }
  __device__ __forceinline__ static float s(int k) {
    return k == 1 ? 0.95105651629515357f : k == 2 ? 0.58778525229247313f
         : k == 3 ? -0.58778525229247313f : -0.95105651629515357f;
  }
};
template <> struct OddConst<7> {
  __device__ __forceinline__ static float c(int k) {
    return (k == 1 || k == 6) ? 0.62348980185873353f : (k == 2 || k == 5) ? -0.22252093395631440f
         : -0.90096886790241913f;
  }
  __device__ __forceinline__ static float s(int k) {
    return k == 1 ? 0.78183148246802981f : k == 2 ? 0.97492791218182361f : k == 3 ? 0.43388373911755812f
         : k == 4 ? -0.43388373911755812f : k == 5 ? -0.97492791218182361f : -0.78183148246802981f;
  }
};

template <int P, bool INV> struct DftOdd {
  __device__ __forceinline__ static void run(float2 (&v)[P]) {
    constexpr int H = (P - 1) / 2;
    float2 s[H], d[H];
    float2 x0 = v[0];
    float2 sum = x0;
#pragma unroll
    for (int m = 1; m <= H; m++) {
      s[m - 1] = cadd(v[m], v[P - m]);
      d[m - 1] = csub(v[m], v[P - m]);
      sum = cadd(sum, s[m - 1]);
    }
    v[0] = sum;
#pragma unroll
    for (int k = 1; k <= H; k++) {
      float2 re = x0, im = make_float2(0.f, 0.f);
#pragma unroll
      for (int m = 1; m <= H; m++) {
        const int idx = (m * k) % P;
        const float cc = OddConst<P>::c(idx), ss = OddConst<P>::s(idx);
        re.x = fmaf(cc, s[m - 1].x, re.x);
        re.y = fmaf(cc, s[m - 1].y, re.y);
        im.x = fmaf(ss, d[m - 1].x, im.x);
        im.y = fmaf(ss, d[m - 1].y, im.y);
      }
      // forward: X_k = re - i*im, X_{P-k} = re + i*im
      float2 mi = make_float2(im.y, -im.x);  // -i*im
      if (!INV) {
        v[k] = cadd(re, mi);
        v[P - k] = csub(re, mi);
      } else {
        v[k] = csub(re, mi);
        v[P - k] = cadd(re, mi);
      }
    }
  }
};
template <bool INV> struct Dft<3, INV> { __device__ __forceinline__ static void run(float2 (&v)[3]) { DftOdd<3, INV>::run(v); } };
template <bool INV> struct Dft<5, INV> { __device__ __forceinline__ static void run(float2 (&v)[5]) { DftOdd<5, INV>::run(v); } };
template <bool INV> struct Dft<7, INV> { __device__ __forceinline__ static void run(float2 (&v)[7]) { DftOdd<7, INV>::run(v); } };

// ---------------------------------------------------------------------------
// Radix plans. Greedy choice of radix 16, 8, 4, 2, then 3, 5, 7; sizes with a
// prime factor above 7 are not supported by this engine.
// ---------------------------------------------------------------------------
struct RadixPlan {
  int nr;
  int r[12];
};

__host__ __device__ constexpr RadixPlan make_plan(int n) {
  RadixPlan p{0, {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0}};
  int m = n;
  while (m > 1 && p.nr < 12) {
    int r = 0;
    if (m % 16 == 0 && m != 32) r = 16;
    else if (m % 8 == 0) r = 8;
    else if (m % 4 == 0) r = 4;
    else if (m % 2 == 0) r = 2;
    else if (m % 3 == 0) r = 3;
    else if (m % 5 == 0) r = 5;
    else if (m % 7 == 0) r = 7;
    else return RadixPlan{-1, {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0}};
    p.r[p.nr++] = r;
    m /= r;
  }
  return p;
}

__host__ __device__ constexpr bool fft_size_supported(int n) { return n >= 1 && make_plan(n).nr >= 0; }

// Warps per CTA for a length-N tile: about 16 elements per thread, and four
// warps from N = 33 to 63, where two or three warps left the first pass
// limited to a third of the SM's warp slots by its shared memory (the tile and
// the staged neighbour layers of the fused corrections take about 20 KB).
__host__ __device__ constexpr int warps_for(int n) {
  return n <= 32 ? 2 : (n < 64 ? 4 : (n / 16 > 32 ? 32 : n / 16));
}

constexpr int kPad = 33;  // shared tile row pitch in float2

// ---------------------------------------------------------------------------
// One radix stage of a length-N transform over the 32 pencils of a tile.
// Ld(e) returns element e of this lane's pencil, St(e, v) stores it.
// SYNC_MID: reads and writes alias (in-place shared tile) -> barrier between.
// ---------------------------------------------------------------------------
template <int N, int R, int NS, int W, bool INV, bool SYNC_MID, class Ld, class St>
__device__ __forceinline__ void fft_stage(int warp, const float2* __restrict__ tw, Ld ld, St st) {
  constexpr int NB = N / R;
  constexpr int PER = (NB + W - 1) / W;
  float2 v[PER][R];
#pragma unroll
  for (int b = 0; b < PER; b++) {
    const int j = warp + b * W;
    if ((NB % W) == 0 || j < NB) {
#pragma unroll
      for (int r = 0; r < R; r++) v[b][r] = ld(j + r * NB);
      if (NS > 1) {
        const int k = j % NS;
#pragma unroll
        for (int r = 1; r < R; r++) {
          const float2 w = __ldg(tw + r * k * (N / (NS * R)));
          v[b][r] = INV ? cmulc(v[b][r], w) : cmul(v[b][r], w);
        }
      }
      Dft<R, INV>::run(v[b]);
    }
  }
  if (SYNC_MID) __syncthreads();
#pragma unroll
  for (int b = 0; b < PER; b++) {
    const int j = warp + b * W;
    if ((NB % W) == 0 || j < NB) {
      const int k = j % NS;
      const int d = (j / NS) * NS * R + k;
#pragma unroll
      for (int r = 0; r < R; r++) st(d + r * NS, v[b][r]);
    }
  }
}

template <int N, bool REV> struct PlanOf;
template <int N> struct PlanOf<N, false> { static constexpr RadixPlan value = make_plan(N); };
__host__ __device__ constexpr RadixPlan reversed(RadixPlan p) {
  RadixPlan q = p;
  for (int i = 0; i < p.nr; i++) q.r[i] = p.r[p.nr - 1 - i];
  return q;
}
template <int N> struct PlanOf<N, true> { static constexpr RadixPlan value = reversed(make_plan(N)); };

// Stage driver: stage S of the plan with NS = product of the previous radices.
// FIRST_SMEM / LAST_SMEM say whether the first stage's loader and the last
// stage's storer touch the shared tile (then the stage needs its mid barrier).
template <int N, int W, bool INV, bool REV, int S, int NS, bool FIRST_SMEM, bool LAST_SMEM, int PITCH, class Ld,
          class St>
__device__ __forceinline__ void fft_run(int warp, int lane, float2 (*sm)[PITCH], const float2* __restrict__ tw,
                                        Ld first_ld, St last_st) {
  constexpr RadixPlan P = PlanOf<N, REV>::value;
  constexpr int R = P.r[S];
  auto sld = [&](int e) { return sm[e][lane]; };
  auto sst = [&](int e, float2 v) { sm[e][lane] = v; };
  if constexpr (P.nr == 1) {
    fft_stage<N, R, NS, W, INV, FIRST_SMEM || LAST_SMEM>(warp, tw, first_ld, last_st);
  } else if constexpr (S == 0) {
    fft_stage<N, R, NS, W, INV, FIRST_SMEM>(warp, tw, first_ld, sst);
    __syncthreads();
    fft_run<N, W, INV, REV, S + 1, NS * R, FIRST_SMEM, LAST_SMEM>(warp, lane, sm, tw, first_ld, last_st);
  } else if constexpr (S == P.nr - 1) {
    fft_stage<N, R, NS, W, INV, LAST_SMEM>(warp, tw, sld, last_st);
  } else {
    fft_stage<N, R, NS, W, INV, true>(warp, tw, sld, sst);
    __syncthreads();
    fft_run<N, W, INV, REV, S + 1, NS * R, FIRST_SMEM, LAST_SMEM>(warp, lane, sm, tw, first_ld, last_st);
  }
}

// Forward stages S..nr-2 of plan(N) (all but the last), leaving the tile in
// shared memory. Used before the turn of fft_fwd_mul_inv.
template <int N, int W, int S, int NS, bool FIRST_SMEM, int PITCH, class Ld>
__device__ __forceinline__ void fft_run_partial(int warp, int lane, float2 (*sm)[PITCH], const float2* __restrict__ tw,
                                                Ld first_ld) {
  constexpr RadixPlan P = make_plan(N);
  constexpr int R = P.r[S];
  auto sld = [&](int e) { return sm[e][lane]; };
  auto sst = [&](int e, float2 v) { sm[e][lane] = v; };
  if constexpr (S == 0) {
    fft_stage<N, R, NS, W, false, FIRST_SMEM>(warp, tw, first_ld, sst);
  } else {
    fft_stage<N, R, NS, W, false, true>(warp, tw, sld, sst);
  }
  if constexpr (S + 1 < P.nr - 1) {
    __syncthreads();
    fft_run_partial<N, W, S + 1, NS * R, FIRST_SMEM>(warp, lane, sm, tw, first_ld);
  }
}

// The turn of a forward-multiply-inverse transform: the last forward stage
// (NS * R == N) leaves X[j + q*NS] in the registers of butterfly j, which are
// exactly the inputs of butterfly j of a first inverse stage of the same radix
// (NS = 1). So the k-space multiplier and that inverse stage run in registers.
template <int N, int R, int W, bool SYNC_MID, class Ld, class St, class Mul>
__device__ __forceinline__ void turn_stage(int warp, const float2* __restrict__ tw, Ld ld, St st, Mul mul) {
  constexpr int NB = N / R;  // == NS of the last forward stage
  constexpr int PER = (NB + W - 1) / W;
  float2 v[PER][R];
#pragma unroll
  for (int b = 0; b < PER; b++) {
    const int j = warp + b * W;
    if ((NB % W) == 0 || j < NB) {
#pragma unroll
      for (int r = 0; r < R; r++) v[b][r] = ld(j + r * NB);
      if (NB > 1) {
#pragma unroll
        for (int r = 1; r < R; r++) v[b][r] = cmul(v[b][r], __ldg(tw + r * j));
      }
      Dft<R, false>::run(v[b]);
#pragma unroll
      for (int r = 0; r < R; r++) v[b][r] = mul(j + r * NB, v[b][r]);
      Dft<R, true>::run(v[b]);
    }
  }
  if (SYNC_MID) __syncthreads();
#pragma unroll
  for (int b = 0; b < PER; b++) {
    const int j = warp + b * W;
    if ((NB % W) == 0 || j < NB) {
#pragma unroll
      for (int r = 0; r < R; r++) st(j * R + r, v[b][r]);
    }
  }
}

// Forward stages 0..nr-2 of plan(N), the turn, then inverse stages 1..nr-1 of
// the reversed plan. Loader/storer semantics as in fft_run.
template <int N, int W, bool FIRST_SMEM, bool LAST_SMEM, int PITCH, class Ld, class St, class Mul>
__device__ __forceinline__ void fft_fwd_mul_inv(int warp, int lane, float2 (*sm)[PITCH], const float2* __restrict__ tw,
                                                Ld first_ld, St last_st, Mul mul) {
  constexpr RadixPlan P = make_plan(N);
  constexpr int RL = P.r[P.nr - 1];
  auto sld = [&](int e) { return sm[e][lane]; };
  auto sst = [&](int e, float2 v) { sm[e][lane] = v; };
  if constexpr (P.nr == 1) {
    turn_stage<N, RL, W, FIRST_SMEM || LAST_SMEM>(warp, tw, first_ld, last_st, mul);
  } else {
    // forward stages except the last, ending in shared memory
    if constexpr (P.nr == 2) {
      fft_stage<N, P.r[0], 1, W, false, FIRST_SMEM>(warp, tw, first_ld, sst);
    } else {
      fft_run_partial<N, W, 0, 1, FIRST_SMEM>(warp, lane, sm, tw, first_ld);
    }
    __syncthreads();
    turn_stage<N, RL, W, true>(warp, tw, sld, sst, mul);
    __syncthreads();
    // inverse stages 1.. of the reversed plan, NS starts at RL
    fft_run<N, W, true, true, 1, RL, true, LAST_SMEM>(warp, lane, sm, tw, sld, last_st);
  }
}

}  // namespace mbs
