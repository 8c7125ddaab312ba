// FP64 residual reduction and the stop test of one iteration (Sec. 3.1: the
// relative residual eps = ||Gamma^-1 (y - A x_n)|| / ||Gamma^-1 y|| against a
// threshold; the global residual sums the squared norms of all subdomains).
//
// Every block of the iteration's last kernel writes its FP64 partial; the block
// that takes the last ticket sums all partials of the iteration in a fixed
// order (deterministic), updates the solver state and resets the ticket. This
// removes a separate single-block launch per iteration.
#pragma once
#include <math.h>

#include "mbs_internal.h"
#include "../../include/mbs.h"

namespace mbs {

// Sum over the block (valid in thread 0). Fixed order: warp shuffles, then warps.
__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < nw; i++) s += red[i];
  return s;
}

// Update of the solver state from the summed |r_n|^2 (thread 0 only).
__device__ __forceinline__ void state_update(DevState* st, double R, double* hist) {
  const int it = st->iter;
  if (it == 0 && !st->r0_fixed) st->R0 = R;
  const double eps = st->R0 > 0.0 ? sqrt(R / st->R0) : 0.0;
  if (hist && it < st->hist_cap) hist[it] = eps;
  st->eps = eps;
  st->iter = it + 1;
  if (!isfinite(eps) || !isfinite(R)) {
    st->status = MBS_ENAN;
    st->done = 1;
    return;
  }
  // the iteration is monotone in exact arithmetic (Sec. 2): a sustained rise
  // far above the best value so far means a breakdown
  if (eps < st->best) {
    st->best = eps;
    st->rise = 0;
  } else if (eps > 4.0 * st->best && eps > 1e-3) {
    st->rise += 1;
  } else {
    st->rise = 0;
  }
  if (st->rise >= 20) {
    st->status = MBS_EDIVERGE;
    st->done = 1;
  } else if (eps < st->tol || st->iter >= st->max_iter) {
    st->done = 1;
  }
}

struct Finish {
  double* partials;  // all partials of the iteration; this launch's block b writes partials[slot0 + b]
  int slot0;
  int n_total;
  DevState* state;   // non-null: this launch ends the iteration
  double* hist;
};

// Store this block's partial; the last block of the launch finishes the iteration.
// b: this block's index among the nb blocks of its plan's launch (a batched launch
// holds several plans' blocks; each plan counts its own).
__device__ __forceinline__ void finish_block_at(const Finish& f, double block_total, double* red, unsigned b,
                                                unsigned nb) {
  __shared__ unsigned int ticket;
  if (threadIdx.x == 0) {
    f.partials[f.slot0 + b] = block_total;
    if (f.state) {
      __threadfence();  // the partial is visible before the ticket is taken
      ticket = atomicAdd(&f.state->ticket, 1u);
    }
  }
  if (!f.state) return;
  __syncthreads();
  if (ticket != nb - 1) return;
  __threadfence();
  double s = 0.0;
  const volatile double* P = f.partials;
  for (int i = threadIdx.x; i < f.n_total; i += blockDim.x) s += P[i];
  const double R = block_sum(s, red);
  if (threadIdx.x == 0) {
    state_update(f.state, R, f.hist);
    f.state->ticket = 0u;
  }
}

__device__ __forceinline__ void finish_block(const Finish& f, double block_total, double* red) {
  finish_block_at(f, block_total, red, blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z),
                  gridDim.x * gridDim.y * gridDim.z);
}

}  // namespace mbs
