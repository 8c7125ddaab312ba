// Bluestein pass kernels on the M-point FFTs M = 96, 128, 192 (mbs_bluestein.cuh).
#include "mbs_bluestein.cuh"

namespace mbs {
bool bluestein_group_1(int M, int kind, int axis, bool inv, const PassArgs& a, int nrb, cudaStream_t st,
                        cudaError_t* err) {
  switch (M) {
    case 96:
      *err = run_bluestein<96>(kind, axis, inv, a, nrb, st);
      return true;
    case 128:
      *err = run_bluestein<128>(kind, axis, inv, a, nrb, st);
      return true;
    case 192:
      *err = run_bluestein<192>(kind, axis, inv, a, nrb, st);
      return true;
    default:
      return false;
  }
}
}  // namespace mbs
