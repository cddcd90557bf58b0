// Device helpers shared by the kernel translation units: warp sums, a
// deterministic grid reduction and warp-aggregated counters.
#pragma once

#include "gf_device.h"

namespace gf {

// Sum of src[stride r] over the rows r in [r0, r1), in ascending r.  The
// values are loaded B at a time before any add, so each thread keeps B
// independent loads in flight; the adds still run one by one in row order.
// `src` must not be written during the kernel.
template <int B, typename T>
__device__ __forceinline__ T row_sum(const T* __restrict__ src, int stride, int r0, int r1) {
  if (r0 >= r1) return T(0);
  // the sum starts from the first row (0 + x would cost an add on a pipe that
  // binds the FP64 gathers); later batches add in row order as before
  T acc;
  {
    T v[B];
#pragma unroll
    for (int k = 0; k < B; ++k) v[k] = r0 + k < r1 ? __ldg(src + int64_t(stride) * (r0 + k)) : T(0);
    acc = v[0];
#pragma unroll
    for (int k = 1; k < B; ++k) {
      if (r0 + k >= r1) break;
      acc += v[k];
    }
  }
  for (int r = r0 + B; r < r1; r += B) {
    T v[B];
#pragma unroll
    for (int k = 0; k < B; ++k) v[k] = r + k < r1 ? __ldg(src + int64_t(stride) * (r + k)) : T(0);
#pragma unroll
    for (int k = 0; k < B; ++k) {   // stop at the row count: no add issues once every lane is done
      if (r + k >= r1) break;
      acc += v[k];
    }
  }
  return acc;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic grid reduction of NV doubles: per-CTA partials, then the last
// CTA to arrive sums all partials in CTA order.  Every thread of every CTA must
// call it.  Returns true in the last CTA, with the totals in out[] (valid in
// thread 0).  Nothing waits on another CTA.
template <int NV>
__device__ __forceinline__ bool grid_reduce(double (&v)[NV], double* partials, unsigned* ticket, double (&out)[NV],
                                            unsigned bid, unsigned nb) {
  __shared__ double sh[NV][32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double t = warp_sum(v[i]);
    if (lane == 0) sh[i][wid] = t;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double t = warp_sum(lane < nw ? sh[i][lane] : 0.0);
      if (lane == 0) partials[bid * NV + i] = t;
    }
  }
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned k = atomicAdd(ticket, 1u);
    last = (k == nb - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double t = 0.0;
    for (unsigned j = threadIdx.x; j < nb; j += blockDim.x) t += __ldcg(&partials[j * NV + i]);
    t = warp_sum(t);
    __syncthreads();
    if (lane == 0) sh[i][wid] = t;
    __syncthreads();
    if (wid == 0) {
      t = warp_sum(lane < nw ? sh[i][lane] : 0.0);
      if (lane == 0) out[i] = t;
    }
  }
  if (threadIdx.x == 0) *ticket = 0u;
  return true;
}

__device__ __forceinline__ void warp_count(unsigned long long c, unsigned long long* dst) {
  unsigned v = __reduce_add_sync(0xffffffffu, unsigned(c));
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(dst, (unsigned long long)v);
}

}  // namespace gf
