// Dispatch of the FFT pass kernels by subdomain edge length.
#include "mbs_fft_sizes.h"
#include "mbs_internal.h"

namespace mbs {
#define MBS_DECLARE_GROUP(k)                                                                           \
  bool fft_group_##k(int, int, int, bool, const PassArgs&, int, cudaStream_t, cudaError_t*);           \
  bool fft_group_##k##_batch(int, int, bool, int, const PassArgs*, dim3, size_t, cudaStream_t, cudaError_t*); \
  bool fft_group_##k##_has(int);
MBS_FFT_GROUP_IDS(MBS_DECLARE_GROUP)
#undef MBS_DECLARE_GROUP

bool bluestein_group_0(int, int, int, bool, const PassArgs&, int, cudaStream_t, cudaError_t*);
bool bluestein_group_1(int, int, int, bool, const PassArgs&, int, cudaStream_t, cudaError_t*);
bool bluestein_group_2(int, int, int, bool, const PassArgs&, int, cudaStream_t, cudaError_t*);

static cudaError_t dispatch(int n, int kind, int axis, bool inv, const PassArgs& a, int nrb, cudaStream_t st) {
  cudaError_t err = cudaErrorInvalidValue;
#define MBS_TRY_GROUP(k) \
  if (fft_group_##k(n, kind, axis, inv, a, nrb, st, &err)) return err;
  MBS_FFT_GROUP_IDS(MBS_TRY_GROUP)
#undef MBS_TRY_GROUP
  if (bluestein_launch(n, kind, axis, inv, a, nrb, st, &err)) return err;
  return cudaErrorInvalidValue;
}

// Convolution lengths of the Bluestein kernels (compiled FFT lengths).
static const int kBluesteinM[] = {32, 48, 64, 96, 128, 192, 256, 384, 512};

int bluestein_len(int n) {
  if (n < 2 || n > 256) return 0;
  for (int m : kBluesteinM)
    if (m >= 2 * n - 1) return m;
  return 0;
}

bool bluestein_launch(int n, int kind, int axis, bool inv, const PassArgs& a, int nrb, cudaStream_t st,
                      cudaError_t* err) {
  const int M = bluestein_len(n);
  if (!M || !a.bl_chirp || !a.bl_bhat || a.bl_n != n) return false;
  return bluestein_group_0(M, kind, axis, inv, a, nrb, st, err) || bluestein_group_1(M, kind, axis, inv, a, nrb, st, err) ||
         bluestein_group_2(M, kind, axis, inv, a, nrb, st, err);
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

cudaError_t launch_pass_batch(int n, int kind, bool inv, int tc, const PassArgs* d, dim3 grid, size_t smem,
                              cudaStream_t st) {
  cudaError_t err = cudaErrorInvalidValue;
#define MBS_TRY_BATCH(k) \
  if (fft_group_##k##_batch(n, kind, inv, tc, d, grid, smem, st, &err)) return err;
  MBS_FFT_GROUP_IDS(MBS_TRY_BATCH)
#undef MBS_TRY_BATCH
  return cudaErrorInvalidValue;
}
}  // namespace mbs
