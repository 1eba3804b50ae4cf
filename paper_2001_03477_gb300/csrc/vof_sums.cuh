// vof_sums.cuh -- block-wide sums in the library's one row layout (see
// SumOut in vof_launch.h).
#pragma once
#include "vof_launch.h"

namespace vofgb {

// Sums v[] over the block (up to 32 warps) in a fixed order and writes the
// row to out.partials, or adds the mapped nonzero values to out.diag with
// atomics.  Whole warps of zeros skip the FP64 shuffle tree (FP64 adds are
// the scarce operation on this part, and most warps of most kernels sum
// zeros).  Every thread of the block must call it.
__device__ __forceinline__ void block_sums(double (&v)[kNSums], const SumOut& out, unsigned block_lin) {
  __shared__ double red[kNSums][32];
  if (!out.partials && !out.diag) return;  // uniform over the block
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nw = (int)(blockDim.x * blockDim.y * blockDim.z) >> 5;
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int k = 0; k < kNSums; ++k) {
    double x = v[k];
    if (__any_sync(0xffffffffu, dnz(x))) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    } else {
      x = 0.0;
    }
    if (lane == 0) red[k][warp] = x;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < kNSums; ++k) {
      double x = lane < nw ? red[k][lane] : 0.0;
      if (__any_sync(0xffffffffu, dnz(x))) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      } else {
        x = 0.0;
      }
      if (lane == 0) {
        if (out.partials) out.partials[(size_t)block_lin * out.stride + k] = x;
        else if (out.map[k] >= 0 && dnz(x)) atomicAdd(out.diag + out.map[k], x);
      }
    }
  }
}

}  // namespace vofgb
