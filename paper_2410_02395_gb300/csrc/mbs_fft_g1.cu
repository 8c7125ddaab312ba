// FFT pass kernels for subdomain edges 18, 20, 21, 24, 25, 27, 28, 30, 32, 35, 36.
#include "mbs_passes.cuh"

namespace mbs {
bool fft_group_1(int n, int kind, int axis, bool inv, const PassArgs& a, int nrb, cudaStream_t st,
                   cudaError_t* err) {
  switch (n) {
    MBS_CASE(18)
    MBS_CASE(20)
    MBS_CASE(21)
    MBS_CASE(24)
    MBS_CASE(25)
    MBS_CASE(27)
    MBS_CASE(28)
    MBS_CASE(30)
    MBS_CASE(32)
    MBS_CASE(35)
    MBS_CASE(36)
    default:
      return false;
  }
}
bool fft_group_1_has(int n) {
  switch (n) {
    case 18:
    case 20:
    case 21:
    case 24:
    case 25:
    case 27:
    case 28:
    case 30:
    case 32:
    case 35:
    case 36:
      return true;
    default:
      return false;
  }
}
}  // namespace mbs
