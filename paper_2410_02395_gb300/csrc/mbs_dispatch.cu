// Dispatch of the FFT pass kernels by subdomain edge length.
#include "mbs_internal.h"

namespace mbs {
bool fft_group_0(int, int, int, bool, const PassArgs&, int, cudaStream_t, cudaError_t*);
bool fft_group_0_has(int);
bool fft_group_1(int, int, int, bool, const PassArgs&, int, cudaStream_t, cudaError_t*);
bool fft_group_1_has(int);
bool fft_group_2(int, int, int, bool, const PassArgs&, int, cudaStream_t, cudaError_t*);
bool fft_group_2_has(int);
bool fft_group_3(int, int, int, bool, const PassArgs&, int, cudaStream_t, cudaError_t*);
bool fft_group_3_has(int);
bool fft_group_4(int, int, int, bool, const PassArgs&, int, cudaStream_t, cudaError_t*);
bool fft_group_4_has(int);
bool fft_group_5(int, int, int, bool, const PassArgs&, int, cudaStream_t, cudaError_t*);
bool fft_group_5_has(int);

static cudaError_t dispatch(int n, int kind, int axis, bool inv, const PassArgs& a, int nrb, cudaStream_t st) {
  cudaError_t err = cudaErrorInvalidValue;
  if (fft_group_0(n, kind, axis, inv, a, nrb, st, &err)) return err;
  if (fft_group_1(n, kind, axis, inv, a, nrb, st, &err)) return err;
  if (fft_group_2(n, kind, axis, inv, a, nrb, st, &err)) return err;
  if (fft_group_3(n, kind, axis, inv, a, nrb, st, &err)) return err;
  if (fft_group_4(n, kind, axis, inv, a, nrb, st, &err)) return err;
  if (fft_group_5(n, kind, axis, inv, a, nrb, st, &err)) return err;
  return cudaErrorInvalidValue;
}

bool fft_size_compiled(int n) { return fft_group_0_has(n) || fft_group_1_has(n) || fft_group_2_has(n) || fft_group_3_has(n) || fft_group_4_has(n) || fft_group_5_has(n); }

cudaError_t launch_rows_first(int n, const PassArgs& a, int nrb, cudaStream_t st) { return dispatch(n, 0, 2, false, a, nrb, st); }
cudaError_t launch_rows_last(int n, const PassArgs& a, int nrb, cudaStream_t st) { return dispatch(n, 1, 2, true, a, nrb, st); }
cudaError_t launch_strided(int n, int axis, bool inv, const PassArgs& a, cudaStream_t st) {
  return dispatch(n, 2, axis, inv, a, 0, st);
}
cudaError_t launch_mid(int n, const PassArgs& a, cudaStream_t st) { return dispatch(n, 3, 0, false, a, 0, st); }
}  // namespace mbs
