// Reading the edge-correction slabs (Sec. 3.1 steps 4-5: the corrections of the
// first and last t layers of every subdomain along every corrected axis, summed).
#pragma once
#include "mbs_fft.cuh"
#include "mbs_internal.h"

namespace mbs {

// Slab rows of a grid row (i0, i1) along axes 0 and 1.
struct RowSlab {
  int kf0, kl0, kf1, kl1;
};

__device__ __forceinline__ RowSlab row_slab(const AxisTables& tb, long long i0, long long i1) {
  RowSlab r;
  r.kf0 = tb.kf[0][i0];
  r.kl0 = tb.kl[0][i0];
  r.kf1 = tb.kf[1][i1];
  r.kl1 = tb.kl[1][i1];
  return r;
}

// Sum of the correction slabs at voxel (i0, i1, i2) (row index rho = i0*N1 + i1).
__device__ __forceinline__ float2 slab_sum(const AxisTables& tb, const GridDesc& g, const RowSlab& rs, long long i0,
                                           long long i1, long long rho, long long i2) {
  float2 E = make_float2(0.f, 0.f);
  const long long N1 = g.N1, N2 = g.N2;
  if (rs.kf0 >= 0) E = cadd(E, tb.C[0][((long long)rs.kf0 * N1 + i1) * N2 + i2]);
  if (rs.kl0 >= 0) E = cadd(E, tb.C[0][((long long)rs.kl0 * N1 + i1) * N2 + i2]);
  if (rs.kf1 >= 0) E = cadd(E, tb.C[1][(i0 * tb.Wd[1] + rs.kf1) * N2 + i2]);
  if (rs.kl1 >= 0) E = cadd(E, tb.C[1][(i0 * tb.Wd[1] + rs.kl1) * N2 + i2]);
  const int kf2 = tb.kf[2][i2], kl2 = tb.kl[2][i2];
  if (kf2 >= 0) E = cadd(E, tb.C[2][rho * tb.Wd[2] + kf2]);
  if (kl2 >= 0) E = cadd(E, tb.C[2][rho * tb.Wd[2] + kl2]);
  return E;
}

}  // namespace mbs
