// Persistent solve of the mixed-precision step (sm_103a).
//
// The kernel-by-kernel refinement launches five to six kernels per inner PCG
// iteration; on a stiff system (tens of iterations per step) those launches
// and their tails cost more than the arithmetic.  Here one cooperative launch
// runs the whole solver loop.  Its phases are the same as the kernels' (inner
// start, SpMV, update, apply, double-float residual), over the same row
// partition per mesh, and a grid barrier separates them.  Two changes:
//   * the direction update p = z + beta p is formed inside the next SpMV
//     (p of a neighbour row on the fly, own rows written to the other of two
//     p buffers), which saves a phase and a barrier per iteration;
//   * every phase serves all meshes of a batch at once and only those that
//     need it: the CTAs take the phase's blocks of the active meshes in
//     turn, so a converged mesh costs nothing while the others iterate.
// Vectors written by other CTAs are read only after the grid barrier that
// ends their phase, whose acquire fence (as in a cooperative grid sync) makes
// those writes visible; the solver scalars, which a phase's last block writes,
// are read and written through volatile accesses.  Reductions keep the
// kernels' per-block partials and fixed-order sums (the last block of a mesh
// sums them), so a mesh's scalars do not depend on how many meshes share the
// launch.  Measured on GB300 a barrier over 456 CTAs costs about 3.2 us, about
// a kernel boundary inside a CUDA graph, so the persistent form does not beat
// the graph of phase kernels on one mesh; its use is the batch, where phases
// skip the meshes that have converged.
#include <cmath>

#include "gf_device.h"
#include "gf_df.cuh"

namespace gf {
namespace {

constexpr int kPThreads = 256;
enum PersistPhase : int { kPhInit = 0, kPhSpmv, kPhUpdate, kPhApply, kPhResidual, kPhases };
__constant__ int kPhaseKind[kPhases] = {kB_ir_inner_init, kB_ir_spmv, kB_ir_update, kB_ir_apply, kB_ir_residual};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier over the launch's CTAs (all resident: cooperative launch).
// Arrivals count up across the launch; barrier g waits for g * gridDim.x.
// The wait is bounded: after kPersistWaitNs it sets ctl->error and the CTA
// gives up, and a CTA that sees the error gives up too.  Returns false then.
__device__ bool grid_barrier(PersistCtl* ctl, unsigned& gen) {
  __shared__ int ok_s;
  __syncthreads();
  gen += 1;   // every thread keeps the count: it selects the flag slot
  if (threadIdx.x == 0) {
    const unsigned target = gen * gridDim.x;
    __threadfence();
    const bool skip = ctl->test_skip && blockIdx.x == 0 && gen == 1;
    if (!skip) atomicAdd(&ctl->arrive, 1u);
    int ok = 1;
    const unsigned long long t0 = global_ns();
    while (ld_acquire_u32(&ctl->arrive) < target) {
      if (*reinterpret_cast<volatile int*>(&ctl->error)) {
        ok = 0;
        break;
      }
      if (global_ns() - t0 > kPersistWaitNs) {
        atomicExch(&ctl->error, 1);
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

__device__ __forceinline__ void ld3(const float* a, int64_t i, float (&o)[3]) {
  o[0] = a[3 * i];
  o[1] = a[3 * i + 1];
  o[2] = a[3 * i + 2];
}

// The solver scalars a phase's work reads, as the previous phase left them
// (its last block writes them before the barrier).
struct IrView {
  int in_iters;
  float alpha32, beta32;
};
__device__ __forceinline__ IrView ir_view(const IrState* S) {
  const volatile IrState* V = S;
  return {V->in_iters, V->alpha32, V->beta32};
}
// Which meshes take part in a phase, from a flag slot (done, in_done, applied).
__device__ __forceinline__ bool phase_needed(int ph, const volatile int* f) {
  const int done = f[0], in_done = f[1], applied = f[2];
  if (done) return false;
  switch (ph) {
    case kPhInit: return applied != 0;
    case kPhSpmv: case kPhUpdate: return in_done == 0;
    default: return in_done != 0 && applied == 0;   // apply, then the residual
  }
}
__device__ __forceinline__ void set_flags(int* f, const volatile IrState* S) {
  f[0] = S->done;
  f[1] = S->in_done;
  f[2] = S->applied;
}

// inner PCG start after a fresh residual: r32 = r, z = P r, d = 0; r . z.
// (p = z is formed by the first SpMV of the inner solve.)
__device__ void ph_init(const DevMesh& m, unsigned bid, unsigned nb, int* fnext) {
  const MixDev& x = m.mx;
  float h[1] = {0.f}, l[1] = {0.f};
  for (int64_t i = bid * int64_t(blockDim.x) + threadIdx.x; i < m.N; i += int64_t(nb) * blockDim.x) {
    float r[3] = {0, 0, 0}, z[3] = {0, 0, 0};
    if (!__ldg(m.pinned + i)) {
      ld3(x.rres, i, r);
      const float* pi = x.pinv32 + 9 * i;
#pragma unroll
      for (int c = 0; c < 3; ++c)
        z[c] = __ldg(pi + 3 * c) * r[0] + __ldg(pi + 3 * c + 1) * r[1] + __ldg(pi + 3 * c + 2) * r[2];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      x.r32[3 * i + c] = r[c];
      x.z32[3 * i + c] = z[c];
      x.d32[3 * i + c] = 0.f;
      df_acc_prod(h[0], l[0], r[c], z[c]);
    }
  }
  double out[1];
  if (grid_reduce_df<1>(h, l, m.partials, m.tickets + 5, out, bid, nb) && threadIdx.x == 0) {
    volatile IrState* S = x.ir;   // written by other SMs in this launch: no L1 copies
    S->rz = out[0];
    S->in_rr0 = S->rr;
    S->in_iters = 0;
    S->in_done = (out[0] == 0.0) ? 1 : 0;
    S->applied = 0;
    set_flags(fnext, S);
  }
}

// q = A32 p with p = z (first iteration) or z + beta p_prev formed on the fly
// for every column; half a warp per block row.  Own rows' p goes to the buffer
// of this iteration (p32 for even, p32b for odd iterations).  p . q.
__device__ void ph_spmv(const DevMesh& m, const IrView& v, unsigned bid, unsigned nb, int* fnext) {
  const MixDev& x = m.mx;
  const int k = v.in_iters;
  const float beta = v.beta32;
  const float* pprev = (k & 1) ? x.p32 : x.p32b;
  float* pnew = (k & 1) ? x.p32b : x.p32;
  const int j16 = threadIdx.x & 15;
  const unsigned hmask = (threadIdx.x & 16) ? 0xffff0000u : 0x0000ffffu;
  float h[1] = {0.f}, l[1] = {0.f};
  const int64_t nh = (int64_t(nb) * blockDim.x) >> 4;
  for (int64_t i = (bid * int64_t(blockDim.x) + threadIdx.x) >> 4; i < m.N; i += nh) {
    float y0 = 0.f, y1 = 0.f, y2 = 0.f;
    const int b1 = __ldg(m.row_ptr + i + 1);
    for (int b = __ldg(m.row_ptr + i) + j16; b < b1; b += 16) {
      const int64_t j = __ldg(m.col + b);
      const float* a = x.val32 + 9 * int64_t(b);
      float p[3];
      ld3(x.z32, j, p);
      if (k > 0) {
        float q[3];
        ld3(pprev, j, q);
#pragma unroll
        for (int c = 0; c < 3; ++c) p[c] = fmaf(beta, q[c], p[c]);
      }
      y0 += __ldg(a) * p[0] + __ldg(a + 1) * p[1] + __ldg(a + 2) * p[2];
      y1 += __ldg(a + 3) * p[0] + __ldg(a + 4) * p[1] + __ldg(a + 5) * p[2];
      y2 += __ldg(a + 6) * p[0] + __ldg(a + 7) * p[1] + __ldg(a + 8) * p[2];
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
      y0 += __shfl_xor_sync(hmask, y0, o);
      y1 += __shfl_xor_sync(hmask, y1, o);
      y2 += __shfl_xor_sync(hmask, y2, o);
    }
    if (j16 == 0) {
      float p[3];
      ld3(x.z32, i, p);
      if (k > 0) {
        float q[3];
        ld3(pprev, i, q);
#pragma unroll
        for (int c = 0; c < 3; ++c) p[c] = fmaf(beta, q[c], p[c]);
      }
      const float y[3] = {y0, y1, y2};
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        pnew[3 * i + c] = p[c];
        x.q32[3 * i + c] = y[c];
        df_acc_prod(h[0], l[0], p[c], y[c]);
      }
    }
  }
  double out[1];
  if (grid_reduce_df<1>(h, l, m.partials, m.tickets + 6, out, bid, nb) && threadIdx.x == 0) {
    volatile IrState* S = x.ir;   // written by other SMs in this launch: no L1 copies
    S->pq = out[0];
    if (!(out[0] > 0.0)) {
      if (!isfinite(out[0])) {
        S->status = GF_NAN;
        S->done = 1;
      } else if (S->in_iters == 0) {
        S->status = GF_CG_BREAKDOWN;
        S->done = 1;
      }
      S->in_done = 1;   // lost positive definiteness in FP32: hand back to the refinement
    } else {
      S->alpha = S->rz / out[0];
      S->alpha32 = float(S->alpha);
    }
    set_flags(fnext, S);
  }
}

// d += alpha p, r -= alpha q, z = P r on free rows (p of this iteration's
// buffer); r . z and r . r.
__device__ void ph_update(const DevMesh& m, const IrView& v, unsigned bid, unsigned nb, int* fnext) {
  const MixDev& x = m.mx;
  const float alpha = v.alpha32;
  const float* p = (v.in_iters & 1) ? x.p32b : x.p32;
  float h[2] = {0.f, 0.f}, l[2] = {0.f, 0.f};
  for (int64_t i = bid * int64_t(blockDim.x) + threadIdx.x; i < m.N; i += int64_t(nb) * blockDim.x) {
    if (__ldg(m.pinned + i)) continue;
    float r[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      x.d32[3 * i + c] = x.d32[3 * i + c] + alpha * p[3 * i + c];
      r[c] = x.r32[3 * i + c] - alpha * x.q32[3 * i + c];
      x.r32[3 * i + c] = r[c];
    }
    const float* pi = x.pinv32 + 9 * i;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float z = __ldg(pi + 3 * c) * r[0] + __ldg(pi + 3 * c + 1) * r[1] + __ldg(pi + 3 * c + 2) * r[2];
      x.z32[3 * i + c] = z;
      df_acc_prod(h[0], l[0], r[c], z);
      df_acc_prod(h[1], l[1], r[c], r[c]);
    }
  }
  double out[2];
  if (grid_reduce_df<2>(h, l, m.partials, m.tickets + 7, out, bid, nb) && threadIdx.x == 0) {
    volatile IrState* S = x.ir;   // written by other SMs in this launch: no L1 copies
    S->in_iters += 1;
    S->total_iters += 1;
    S->beta = out[0] / S->rz;
    S->beta32 = float(S->beta);
    S->rz = out[0];
    S->in_rr = out[1];
    if (!(out[1] > S->in_tol2 * S->in_rr0) || S->in_iters >= S->in_maxit || S->total_iters >= S->maxit)
      S->in_done = 1;
    set_flags(fnext, S);
  }
}

// dv += d on free rows, kept as a float pair (dv_hi + dv_lo).  No reduction.
__device__ void ph_apply(const DevMesh& m, unsigned bid, unsigned nb) {
  for (int64_t i = bid * int64_t(blockDim.x) + threadIdx.x; i < 3 * m.N; i += int64_t(nb) * blockDim.x) {
    if (__ldg(m.pinned + i / 3)) continue;
    float hi = m.mx.dv_hi[i], lo = m.mx.dv_lo[i];
    df_add(hi, lo, m.mx.d32[i], 0.f);
    m.mx.dv_hi[i] = hi;
    m.mx.dv_lo[i] = lo;
  }
}

// r = b - A32 dv on free rows in double-float, eight lanes per block row (the
// refinement residual of the kernel-by-kernel form, reading dv through L2);
// ||r||^2 decides convergence.
__device__ void ph_residual(const DevMesh& m, unsigned bid, unsigned nb, int* fnext) {
  const MixDev& x = m.mx;
  const int j8 = threadIdx.x & 7;
  const unsigned gmask = 0xffu << (threadIdx.x & 24);
  float nh_[1] = {0.f}, nl_[1] = {0.f};
  const int64_t ng = (int64_t(nb) * blockDim.x) >> 3;
  for (int64_t i = (bid * int64_t(blockDim.x) + threadIdx.x) >> 3; i < m.N; i += ng) {
    float hi[4] = {0, 0, 0, 0}, lo[4] = {0, 0, 0, 0};
    const bool fixed = __ldg(m.pinned + i);
    const int b1 = __ldg(m.row_ptr + i + 1);
    const int cw = j8 >> 1;
    const float bh = ((j8 & 1) == 0 && cw < 3) ? __ldg(x.rhs32 + 3 * i + cw) : 0.f;
    float sacc[4] = {0, 0, 0, 0}, cacc[4] = {0, 0, 0, 0};
    for (int b = __ldg(m.row_ptr + i) + j8; b < b1; b += 16) {
      const bool two = b + 8 < b1;
      const int64_t j0 = __ldg(m.col + b), j1 = two ? __ldg(m.col + b + 8) : j0;
      float a0[9], a1[9], xh0[3], xl0[3], xh1[3], xl1[3];
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        a0[q] = __ldg(x.val32 + 9 * int64_t(b) + q);
        a1[q] = two ? __ldg(x.val32 + 9 * int64_t(b + 8) + q) : 0.f;
      }
      ld3(x.dv_hi, j0, xh0);
      ld3(x.dv_lo, j0, xl0);
      ld3(x.dv_hi, j1, xh1);
      ld3(x.dv_lo, j1, xl1);
      dot2_block(sacc, cacc, a0, xh0, xl0);
      if (two) dot2_block(sacc, cacc, a1, xh1, xl1);
    }
#pragma unroll
    for (int rr = 0; rr < 3; ++rr) two_sum(sacc[rr], cacc[rr], hi[rr], lo[rr]);
    {
      const bool h2 = j8 & 4, h1 = j8 & 2;
      float uh[2], ul[2];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const float sh = h2 ? hi[k] : hi[2 + k], sl = h2 ? lo[k] : lo[2 + k];
        uh[k] = h2 ? hi[2 + k] : hi[k];
        ul[k] = h2 ? lo[2 + k] : lo[k];
        df_add(uh[k], ul[k], __shfl_xor_sync(gmask, sh, 4), __shfl_xor_sync(gmask, sl, 4));
      }
      float vh = h1 ? uh[1] : uh[0], vl = h1 ? ul[1] : ul[0];
      df_add(vh, vl, __shfl_xor_sync(gmask, h1 ? uh[0] : uh[1], 2), __shfl_xor_sync(gmask, h1 ? ul[0] : ul[1], 2));
      df_add(vh, vl, __shfl_xor_sync(gmask, vh, 1), __shfl_xor_sync(gmask, vl, 1));
      hi[0] = vh;
      lo[0] = vl;
    }
    if ((j8 & 1) == 0 && cw < 3) {
      float rh = 0.f, rl = 0.f;
      if (!fixed) {
        rh = bh;
        df_add(rh, rl, -hi[0], -lo[0]);
      }
      x.rres[3 * i + cw] = rh;
      df_acc_prod(nh_[0], nl_[0], rh, rh);
      df_add(nh_[0], nl_[0], 2.f * rh * rl, 0.f);
    }
  }
  double out[1];
  if (grid_reduce_df<1>(nh_, nl_, m.partials, m.tickets + 4, out, bid, nb) && threadIdx.x == 0) {
    volatile IrState* S = x.ir;   // written by other SMs in this launch: no L1 copies
    S->sweeps += 1;
    S->applied = 1;
    S->rr = out[0];
    S->done = (out[0] == 0.0 || out[0] <= S->tol2 * S->bb) ? 1 : 0;
    if (!isfinite(out[0])) {
      S->status = GF_NAN;
      S->done = 1;
    } else if (!S->done && S->total_iters >= S->maxit) {
      S->status = GF_CG_MAXITER;
      S->done = 1;
    }
    set_flags(fnext, S);
  }
}

// Exclusive prefix sum of one int per thread over the block (blockDim.x =
// kPThreads); s_off[t] receives thread t's offset, s_off[blockDim.x] the total.
__device__ int block_offsets(int v, int* s_off, int* s_warp) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) s_warp[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int w = lane < kPThreads / 32 ? s_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += u;
    }
    if (lane < kPThreads / 32) s_warp[lane] = w;   // inclusive warp totals
  }
  __syncthreads();
  const int base = wid ? s_warp[wid - 1] : 0;
  s_off[threadIdx.x] = base + incl - v;
  if (threadIdx.x == blockDim.x - 1) s_off[blockDim.x] = base + incl;
  __syncthreads();
  return s_off[blockDim.x];
}

// The whole solver loop of every mesh of `tab`.  A round runs the phases
// inner start, SpMV, update, apply, residual; a phase runs only if some mesh
// needs it, over the blocks of those meshes (the same per-mesh block counts as
// the kernel-by-kernel launches), and ends at a grid barrier.
__global__ void __launch_bounds__(kPThreads, 3) k_ir_persist(const BatchTab* __restrict__ tab, PersistCtl* ctl,
                                                             int cap) {
  __shared__ int s_off[kPThreads + 1];
  __shared__ int s_warp[kPThreads / 32];
  const int n = tab->n;
  unsigned gen = 0;
  int round = 0;
  for (; round < cap; ++round) {
    for (int ph = 0; ph < kPhases; ++ph) {
      const int* fcur = &ctl->flags[gen & 1][0][0];
      int* fnext = &ctl->flags[(gen + 1) & 1][0][0];
      const int k = threadIdx.x;
      int cnt = 0;
      if (k < n && phase_needed(ph, fcur + 3 * k)) {
        const int kind = kPhaseKind[ph];
        cnt = tab->off[kind][k + 1] - tab->off[kind][k];
      }
      const int total = block_offsets(cnt, s_off, s_warp);
      if (total == 0) continue;   // the same on every CTA: no barrier
      // block 0 carries the flags of the meshes this phase leaves unchanged
      if (blockIdx.x == 0 && k < n && (cnt == 0 || ph == kPhApply)) {
        const volatile int* f = fcur + 3 * k;
        fnext[3 * k] = f[0];
        fnext[3 * k + 1] = f[1];
        fnext[3 * k + 2] = f[2];
      }
      for (int w = blockIdx.x; w < total; w += gridDim.x) {
        int lo = 0, hi = n;   // the mesh of item w: the last lo with s_off[lo] <= w
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (s_off[mid] <= w) lo = mid;
          else hi = mid;
        }
        const unsigned bid = unsigned(w - s_off[lo]), nb = unsigned(s_off[lo + 1] - s_off[lo]);
        const DevMesh& m = tab->mesh[lo];
        int* fn = fnext + 3 * lo;
        switch (ph) {
          case kPhInit: ph_init(m, bid, nb, fn); break;
          case kPhSpmv: ph_spmv(m, ir_view(m.mx.ir), bid, nb, fn); break;
          case kPhUpdate: ph_update(m, ir_view(m.mx.ir), bid, nb, fn); break;
          case kPhApply: ph_apply(m, bid, nb); break;
          default: ph_residual(m, bid, nb, fn); break;
        }
        __syncthreads();   // the reductions' shared memory serves the next item
      }
      if (!grid_barrier(ctl, gen)) return;
    }
    // stop once every mesh is done (the same decision on every CTA)
    const int* fcur = &ctl->flags[gen & 1][0][0];
    const int active = threadIdx.x < n && !reinterpret_cast<const volatile int*>(fcur)[3 * threadIdx.x];
    if (!__syncthreads_or(active)) break;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) ctl->rounds = round;
}

// Reset the control block and take every mesh's flags after the first residual.
__global__ void k_persist_begin(const BatchTab* __restrict__ tab, PersistCtl* ctl, int test_skip) {
  const int k = threadIdx.x;
  if (k == 0) {
    ctl->arrive = 0u;
    ctl->error = 0;
    ctl->rounds = 0;
    ctl->test_skip = test_skip;
  }
  if (k < tab->n) {
    const IrState* S = tab->mesh[k].mx.ir;
    ctl->flags[0][k][0] = S->done;
    ctl->flags[0][k][1] = S->in_done;
    ctl->flags[0][k][2] = S->applied;
  }
}

}  // namespace

unsigned persist_grid() {
  static unsigned grid[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  if (!grid[dev]) {
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ir_persist, kPThreads, 0) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || per_sm < 1)
      return 0;
    grid[dev] = unsigned(per_sm) * unsigned(sms);
  }
  return grid[dev];
}

int launch_ir_persist(const BatchTab* tab, int n, PersistCtl* ctl, int cap, int test_skip, cudaStream_t s) {
  const unsigned grid = persist_grid();
  if (grid == 0 || n < 1 || n > kPThreads) return -1;
  k_persist_begin<<<1, kPThreads, 0, s>>>(tab, ctl, test_skip);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kPThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, k_ir_persist, tab, ctl, cap) != cudaSuccess) return -1;
  return 2;
}

}  // namespace gf
