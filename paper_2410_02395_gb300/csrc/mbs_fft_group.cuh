// Body of one FFT size-group translation unit: the including file defines
// MBS_FFT_GROUP = k and gets
//   bool fft_group_<k>(n, kind, axis, inv, args, row blocks, stream, &err)
//     launches the pass kernel of that kind for edge n when n is in group k;
//   bool fft_group_<k>_batch(n, kind, inv, tc, descriptors, grid, smem, stream, &err)
//     the batched form of a pass for edge n (see run_size_batch);
//   bool fft_group_<k>_has(n)
//     whether n is in group k.
#pragma once
#include "mbs_fft_sizes.h"
#include "mbs_passes.cuh"

#ifndef MBS_FFT_GROUP
#error "define MBS_FFT_GROUP before including mbs_fft_group.cuh"
#endif

#define MBS_CAT_(a, b) a##b
#define MBS_CAT(a, b) MBS_CAT_(a, b)
#define MBS_HAS_CASE(n) case n:

namespace mbs {
bool MBS_CAT(fft_group_, MBS_FFT_GROUP)(int n, int kind, int axis, bool inv, const PassArgs& a, int nrb,
                                        cudaStream_t st, cudaError_t* err) {
  switch (n) {
    MBS_CAT(MBS_FFT_GROUP_, MBS_FFT_GROUP)(MBS_CASE)
    default:
      return false;
  }
}
bool MBS_CAT(MBS_CAT(fft_group_, MBS_FFT_GROUP), _batch)(int n, int kind, bool inv, int tc, const PassArgs* d, dim3 grid,
                                                          size_t smem, cudaStream_t st, cudaError_t* err) {
  switch (n) {
    MBS_CAT(MBS_FFT_GROUP_, MBS_FFT_GROUP)(MBS_CASE_BATCH)
    default:
      return false;
  }
}
bool MBS_CAT(MBS_CAT(fft_group_, MBS_FFT_GROUP), _has)(int n) {
  switch (n) {
    MBS_CAT(MBS_FFT_GROUP_, MBS_FFT_GROUP)(MBS_HAS_CASE) return true;
    default:
      return false;
  }
}
}  // namespace mbs
