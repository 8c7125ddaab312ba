// Dispatch of the FFT pass kernels by subdomain edge length.
#include "mbs_fft_sizes.h"
#include "mbs_internal.h"

namespace mbs {
#define MBS_DECLARE_GROUP(k)                                                                           \
  bool fft_group_##k(int, int, int, bool, const PassArgs&, int, cudaStream_t, cudaError_t*);           \
  bool fft_group_##k##_has(int);
MBS_FFT_GROUP_IDS(MBS_DECLARE_GROUP)
#undef MBS_DECLARE_GROUP

static cudaError_t dispatch(int n, int kind, int axis, bool inv, const PassArgs& a, int nrb, cudaStream_t st) {
  cudaError_t err = cudaErrorInvalidValue;
#define MBS_TRY_GROUP(k) \
  if (fft_group_##k(n, kind, axis, inv, a, nrb, st, &err)) return err;
  MBS_FFT_GROUP_IDS(MBS_TRY_GROUP)
#undef MBS_TRY_GROUP
  return cudaErrorInvalidValue;
}

bool fft_size_compiled(int n) {
#define MBS_HAS_GROUP(k) \
  if (fft_group_##k##_has(n)) return true;
  MBS_FFT_GROUP_IDS(MBS_HAS_GROUP)
#undef MBS_HAS_GROUP
  return false;
}

cudaError_t launch_rows_first(int n, const PassArgs& a, int nrb, cudaStream_t st) { return dispatch(n, 0, 2, false, a, nrb, st); }
cudaError_t launch_rows_last(int n, const PassArgs& a, int nrb, cudaStream_t st) { return dispatch(n, 1, 2, true, a, nrb, st); }
cudaError_t launch_strided(int n, int axis, bool inv, const PassArgs& a, cudaStream_t st) {
  return dispatch(n, 2, axis, inv, a, 0, st);
}
cudaError_t launch_mid(int n, const PassArgs& a, cudaStream_t st) { return dispatch(n, 3, 0, false, a, 0, st); }
}  // namespace mbs
