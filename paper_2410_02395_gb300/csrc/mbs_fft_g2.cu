// FFT pass kernels for subdomain edges 40, 42, 45, 48, 49, 50, 54, 56, 60, 63, 64.
#include "mbs_passes.cuh"

namespace mbs {
bool fft_group_2(int n, int kind, int axis, bool inv, const PassArgs& a, int nrb, cudaStream_t st,
                   cudaError_t* err) {
  switch (n) {
    MBS_CASE(40)
    MBS_CASE(42)
    MBS_CASE(45)
    MBS_CASE(48)
    MBS_CASE(49)
    MBS_CASE(50)
    MBS_CASE(54)
    MBS_CASE(56)
    MBS_CASE(60)
    MBS_CASE(63)
    MBS_CASE(64)
    default:
      return false;
  }
}
bool fft_group_2_has(int n) {
  switch (n) {
    case 40:
    case 42:
    case 45:
    case 48:
    case 49:
    case 50:
    case 54:
    case 56:
    case 60:
    case 63:
    case 64:
      return true;
    default:
      return false;
  }
}
}  // namespace mbs
