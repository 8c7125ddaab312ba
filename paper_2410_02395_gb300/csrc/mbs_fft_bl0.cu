// Bluestein pass kernels on the M-point FFTs M = 32, 48, 64, 512 (mbs_bluestein.cuh).
#include "mbs_bluestein.cuh"

namespace mbs {
bool bluestein_group_0(int M, int kind, int axis, bool inv, const PassArgs& a, int nrb, cudaStream_t st,
                        cudaError_t* err) {
  switch (M) {
    case 32:
      *err = run_bluestein<32>(kind, axis, inv, a, nrb, st);
      return true;
    case 48:
      *err = run_bluestein<48>(kind, axis, inv, a, nrb, st);
      return true;
    case 64:
      *err = run_bluestein<64>(kind, axis, inv, a, nrb, st);
      return true;
    case 512:
      *err = run_bluestein<512>(kind, axis, inv, a, nrb, st);
      return true;
    default:
      return false;
  }
}
}  // namespace mbs
