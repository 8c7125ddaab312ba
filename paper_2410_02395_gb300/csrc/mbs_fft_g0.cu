// FFT pass kernels for subdomain edges 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 14, 15, 16.
#include "mbs_passes.cuh"

namespace mbs {
bool fft_group_0(int n, int kind, int axis, bool inv, const PassArgs& a, int nrb, cudaStream_t st,
                   cudaError_t* err) {
  switch (n) {
    MBS_CASE(1)
    MBS_CASE(2)
    MBS_CASE(3)
    MBS_CASE(4)
    MBS_CASE(5)
    MBS_CASE(6)
    MBS_CASE(7)
    MBS_CASE(8)
    MBS_CASE(9)
    MBS_CASE(10)
    MBS_CASE(12)
    MBS_CASE(14)
    MBS_CASE(15)
    MBS_CASE(16)
    default:
      return false;
  }
}
bool fft_group_0_has(int n) {
  switch (n) {
    case 1:
    case 2:
    case 3:
    case 4:
    case 5:
    case 6:
    case 7:
    case 8:
    case 9:
    case 10:
    case 12:
    case 14:
    case 15:
    case 16:
      return true;
    default:
      return false;
  }
}
}  // namespace mbs
