// FFT pass kernels for subdomain edges 70, 72, 75, 80, 84, 90, 96, 100, 112, 120.
#include "mbs_passes.cuh"

namespace mbs {
bool fft_group_3(int n, int kind, int axis, bool inv, const PassArgs& a, int nrb, cudaStream_t st,
                   cudaError_t* err) {
  switch (n) {
    MBS_CASE(70)
    MBS_CASE(72)
    MBS_CASE(75)
    MBS_CASE(80)
    MBS_CASE(84)
    MBS_CASE(90)
    MBS_CASE(96)
    MBS_CASE(100)
    MBS_CASE(112)
    MBS_CASE(120)
    default:
      return false;
  }
}
bool fft_group_3_has(int n) {
  switch (n) {
    case 70:
    case 72:
    case 75:
    case 80:
    case 84:
    case 90:
    case 96:
    case 100:
    case 112:
    case 120:
      return true;
    default:
      return false;
  }
}
}  // namespace mbs
