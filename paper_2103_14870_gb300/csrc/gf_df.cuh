// Double-float (float pair) arithmetic on the FP32 pipe: error-free
// transformations, warp and grid reductions, and the Dot2-style block product
// of the refinement residual.  Shared by the kernel-by-kernel refinement and
// the persistent solve.
#pragma once

#include "gf_device.h"

namespace gf {
namespace {

// error-free product and sum (Dekker / Knuth) for double-float accumulation
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = a * b;
  e = fmaf(a, b, -p);
}
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void df_add(float& hi, float& lo, float p, float pe) {
  float s, e;
  two_sum(hi, p, s, e);
  e += lo + pe;
  hi = s + e;
  lo = e - (hi - s);
}

// Double-float (float pair) warp and grid reductions: ~48-bit sums on the FP32
// pipe.  The FP64 pipe of GB300 costs a full 64-cycle slot per warp
// instruction even with one active lane, so the refinement keeps FP64-level
// accuracy with float pairs and converts to double only for the final scalars.
__device__ __forceinline__ void df_warp_sum(float& hi, float& lo) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_down_sync(0xffffffffu, hi, o);
    const float ol = __shfl_down_sync(0xffffffffu, lo, o);
    df_add(hi, lo, oh, ol);
  }
}

template <int NV>
__device__ __forceinline__ bool grid_reduce_df(float (&hi)[NV], float (&lo)[NV], double* partials, unsigned* ticket,
                                               double (&out)[NV], unsigned bid, unsigned nb) {
  __shared__ float sh[NV][2][32];
  __shared__ bool last;
  float2* part = reinterpret_cast<float2*>(partials);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    df_warp_sum(hi[i], lo[i]);
    if (lane == 0) {
      sh[i][0][wid] = hi[i];
      sh[i][1][wid] = lo[i];
    }
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      float h = lane < nw ? sh[i][0][lane] : 0.f, l = lane < nw ? sh[i][1][lane] : 0.f;
      df_warp_sum(h, l);
      if (lane == 0) part[bid * NV + i] = make_float2(h, l);
    }
  }
  if (threadIdx.x == 0) {
    __threadfence();
    last = (atomicAdd(ticket, 1u) == nb - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    float h = 0.f, l = 0.f;
    for (unsigned j = threadIdx.x; j < nb; j += blockDim.x) {
      const float2 v = __ldcg(&part[j * NV + i]);
      df_add(h, l, v.x, v.y);
    }
    df_warp_sum(h, l);
    __syncthreads();
    if (lane == 0) {
      sh[i][0][wid] = h;
      sh[i][1][wid] = l;
    }
    __syncthreads();
    if (wid == 0) {
      h = lane < nw ? sh[i][0][lane] : 0.f;
      l = lane < nw ? sh[i][1][lane] : 0.f;
      df_warp_sum(h, l);
      if (lane == 0) out[i] = double(h) + double(l);
    }
  }
  if (threadIdx.x == 0) *ticket = 0u;
  return true;
}

__device__ __forceinline__ void df_acc_prod(float& hi, float& lo, float a, float b) {
  float p, pe;
  two_prod(a, b, p, pe);
  df_add(hi, lo, p, pe);
}

// One 3x3 block times a double-float vector (xh + xl), accumulated in the
// manner of Dot2 (Ogita, Rump and Oishi, 2005): s the rounded sums, c the exact
// product and addition errors; s + c is as accurate as a doubled precision.
__device__ __forceinline__ void dot2_block(float (&s)[4], float (&c)[4], const float (&a)[9], const float (&xh)[3],
                                           const float (&xl)[3]) {
#pragma unroll
  for (int rr = 0; rr < 3; ++rr)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float av = a[3 * rr + k];
      const float p = av * xh[k];
      const float pe = fmaf(av, xl[k], fmaf(av, xh[k], -p));   // product error + the dv_lo term
      const float t = s[rr] + p;
      const float bp = t - s[rr];
      const float e = (s[rr] - (t - bp)) + (p - bp);              // TwoSum error
      s[rr] = t;
      c[rr] += e + pe;
    }
}

}  // namespace
}  // namespace gf
