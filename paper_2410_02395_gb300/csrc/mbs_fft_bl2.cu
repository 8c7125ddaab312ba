// Bluestein pass kernels on the M-point FFTs M = 256, 384 (mbs_bluestein.cuh).
#include "mbs_bluestein.cuh"

namespace mbs {
bool bluestein_group_2(int M, int kind, int axis, bool inv, const PassArgs& a, int nrb, cudaStream_t st,
                        cudaError_t* err) {
  switch (M) {
    case 256:
      *err = run_bluestein<256>(kind, axis, inv, a, nrb, st);
      return true;
    case 384:
      *err = run_bluestein<384>(kind, axis, inv, a, nrb, st);
      return true;
    default:
      return false;
  }
}
}  // namespace mbs
