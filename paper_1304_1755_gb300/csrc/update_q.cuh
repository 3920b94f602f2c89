// FP64 U += sum_l y_l z'_l over the N_x nodes of PC block b, z'_l the grid values of FP32 columns
// (shared by the solver's and the batch graph's solution updates).  kc[l] (shared memory): y_l as
// double-float and the block's grid scale and quantum; columns past nz carry zeros there and re-read
// column nz - 1.  The sum over l is accumulated in double-float from the exact grid values (FP32
// instructions; an FP64 multiply-add per term would make this pass FP64-bound on GB300) and added to
// U in FP64 once.  The block's elements [s0, s1) of the columns (each column starts on a 16-byte
// boundary) go four at a time by 16-byte loads over the aligned middle [a0, a1), so a warp reads 512
// contiguous bytes of a column per load; the up to three elements before a0 and after a1 go by plain
// loads in the first CTA of the block.
#pragma once
#include "df64.cuh"
#include "sg_internal.h"

__device__ __forceinline__ float qgrid_value(float z, float s, float q) {
  return __fmul_rn(__fsub_rn(__fmaf_rn(z, s, SG_QBIAS), SG_QBIAS), q);
}

template <int NV>
__device__ __forceinline__ void update_q_block(double* __restrict__ U, const float* __restrict__ Z, size_t ldz,
                                               const float4* kc, int nz, size_t Nx, int b) {
  const size_t s0 = (size_t)b * Nx, s1 = s0 + Nx;
  const size_t a0 = min((s0 + 3) & ~(size_t)3, s1), a1 = max(s1 & ~(size_t)3, a0);
  if (blockIdx.x == 0 && threadIdx.x < 8) {
    const size_t s = threadIdx.x < 4 ? s0 + threadIdx.x : a1 + (threadIdx.x - 4);
    if ((threadIdx.x < 4 && s < a0) || (threadIdx.x >= 4 && s < s1)) {
      dacc a = dacc_zero();
#pragma unroll
      for (int l = 0; l < NV; ++l) {
        const float4 k = kc[l];
        dacc_fma(a, df2{k.x, k.y}, qgrid_value(Z[(size_t)min(l, nz - 1) * ldz + s], k.z, k.w));
      }
      const df2 r = dacc_get(a);
      U[s] = (U[s] + (double)r.hi) + (double)r.lo;
    }
  }
  for (size_t q = a0 / 4 + blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < a1 / 4;
       q += (size_t)gridDim.x * blockDim.x) {
    dacc a[4] = {dacc_zero(), dacc_zero(), dacc_zero(), dacc_zero()};
#pragma unroll
    for (int l = 0; l < NV; ++l) {
      const float4 z = reinterpret_cast<const float4*>(Z + (size_t)min(l, nz - 1) * ldz)[q];
      const float4 k = kc[l];
      const df2 c{k.x, k.y};
      dacc_fma(a[0], c, qgrid_value(z.x, k.z, k.w));
      dacc_fma(a[1], c, qgrid_value(z.y, k.z, k.w));
      dacc_fma(a[2], c, qgrid_value(z.z, k.z, k.w));
      dacc_fma(a[3], c, qgrid_value(z.w, k.z, k.w));
    }
    double* u = U + 4 * q;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const df2 r = dacc_get(a[e]);
      u[e] = (u[e] + (double)r.hi) + (double)r.lo;
    }
  }
}
