// FFT pass kernels for the subdomain edges of size group 12 (mbs_fft_sizes.h).
#define MBS_FFT_GROUP 12
#include "mbs_fft_group.cuh"
