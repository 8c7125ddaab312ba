// FFT pass kernels for the subdomain edges of size group 0 (mbs_fft_sizes.h).
#define MBS_FFT_GROUP 0
#include "mbs_fft_group.cuh"
