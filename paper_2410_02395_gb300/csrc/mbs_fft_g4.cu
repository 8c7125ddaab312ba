// FFT pass kernels for subdomain edges 128, 160, 192, 256.
#include "mbs_passes.cuh"

namespace mbs {
bool fft_group_4(int n, int kind, int axis, bool inv, const PassArgs& a, int nrb, cudaStream_t st,
                   cudaError_t* err) {
  switch (n) {
    MBS_CASE(128)
    MBS_CASE(160)
    MBS_CASE(192)
    MBS_CASE(256)
    default:
      return false;
  }
}
bool fft_group_4_has(int n) {
  switch (n) {
    case 128:
    case 160:
    case 192:
    case 256:
      return true;
    default:
      return false;
  }
}
}  // namespace mbs
