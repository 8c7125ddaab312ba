// FFT pass kernels for subdomain edges 320, 384, 448, 512.
#include "mbs_passes.cuh"

namespace mbs {
bool fft_group_5(int n, int kind, int axis, bool inv, const PassArgs& a, int nrb, cudaStream_t st,
                   cudaError_t* err) {
  switch (n) {
    MBS_CASE(320)
    MBS_CASE(384)
    MBS_CASE(448)
    MBS_CASE(512)
    default:
      return false;
  }
}
bool fft_group_5_has(int n) {
  switch (n) {
    case 320:
    case 384:
    case 448:
    case 512:
      return true;
    default:
      return false;
  }
}
}  // namespace mbs
