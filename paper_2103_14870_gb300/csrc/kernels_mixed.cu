// Mixed-precision kernels of one graph-FEM fracture step (sm_103a).
//
// Element tangents, stresses, the non-local average and the inner PCG run in
// FP32 (the FP32 pipe is ~61x the FP64 pipe on GB300); the state (x, v, dv),
// the residual of the iterative refinement, the dot-product accumulation and
// the damage threshold test stay FP64.  Small strains keep full FP32 relative
// accuracy because squared-length changes are formed from displacements:
// ds = De . (2 E0 + De), De = u_b - u_a (never |e|^2 - |E0|^2).
#include <cfloat>
#include <cmath>

#include "gf_device.h"
#include "gf_df.cuh"
#include "gf_reduce.cuh"

namespace gf {
namespace {

constexpr int kThreads = 256;

// one 32-byte row in a single 256-bit load (sm_100+; the row must be 32-byte aligned)
__device__ __forceinline__ void ld8f(const float* p, float o[8]) {
  asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=f"(o[0]), "=f"(o[1]), "=f"(o[2]), "=f"(o[3]), "=f"(o[4]), "=f"(o[5]), "=f"(o[6]), "=f"(o[7])
      : "l"(p));
}

__device__ __forceinline__ void ld3f(const float* __restrict__ a, int64_t i, float o[3]) {
  const float* p = a + 3 * i;
  o[0] = p[0];
  o[1] = p[1];
  o[2] = p[2];
}

// one tet's 128-byte rest row: 8 x 16-byte loads
__device__ __forceinline__ void load_restA(const float* __restrict__ rA, int64_t t, float A[32]) {
  const float4* p = reinterpret_cast<const float4*>(rA + kRAStride * t);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const float4 v = __ldg(p + q);
    A[4 * q] = v.x;
    A[4 * q + 1] = v.y;
    A[4 * q + 2] = v.z;
    A[4 * q + 3] = v.w;
  }
}

// rest edge vectors of the 6 local edges from the three stored (X1-X0, X2-X0, X3-X0)
__device__ __forceinline__ void rest_edges(const float A[32], float E0[6][3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) E0[k][c] = A[kRAE0 + 3 * k + c];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    E0[3][c] = E0[1][c] - E0[0][c];
    E0[4][c] = E0[2][c] - E0[0][c];
    E0[5][c] = E0[2][c] - E0[1][c];
  }
}

// current edge vectors e and squared-length changes ds from nodal displacements
__device__ __forceinline__ void edge_state(const float E0[6][3], const float du[4][3], float e[6][3], float ds[6]) {
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    float De[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      De[c] = du[edge_b(k)][c] - du[edge_a(k)][c];
      e[k][c] = E0[k][c] + De[c];
    }
    ds[k] = De[0] * (E0[k][0] + e[k][0]) + De[1] * (E0[k][1] + e[k][1]) + De[2] * (E0[k][2] + e[k][2]);
  }
}

__device__ __forceinline__ float normal_stress32(const float e[3], float s, const float S[6], float kappa) {
  float q = e[0] * e[0] * S[0] + e[1] * e[1] * S[1] + e[2] * e[2] * S[2] +
            kappa * (e[0] * e[1] * S[3] + e[0] * e[2] * S[4] + e[1] * e[2] * S[5]);
  return q / s;
}

// ---------------------------------------------------------------------------
// damage (Eq. 14-25) in FP32, threshold test in FP64
// ---------------------------------------------------------------------------

// The tet's current edge vectors e_k (from displacements) and its second
// Piola-Kirchhoff stress S (Voigt xx yy zz xy xz yz), in FP32.
__device__ __forceinline__ void tet_current_stress32(const DevMesh& m, const Material& mt, int64_t t, float (&e)[6][3],
                                                     float (&S)[6]) {
  const float lam = mt.lam32, mu = mt.mu32;
  const MixDev& x = m.mx;
  const int4 n = m.tets[t];
  const int nid[4] = {n.x, n.y, n.z, n.w};
  float du[4][3];
#pragma unroll
  for (int a = 0; a < 4; ++a) ld3f(x.u32, nid[a], du[a]);
  float A[32];
  load_restA(x.restA, t, A);
  float E0[6][3], ds[6];
  rest_edges(A, E0);
  edge_state(E0, du, e, ds);
  float B[9];
  {
    const float4* pb = reinterpret_cast<const float4*>(x.restB + kRBStride * t);
    const float4 b0 = __ldg(pb), b1 = __ldg(pb + 1), b2 = __ldg(pb + 2);
    B[0] = b0.x; B[1] = b0.y; B[2] = b0.z; B[3] = b0.w;
    B[4] = b1.x; B[5] = b1.y; B[6] = b1.z; B[7] = b1.w;
    B[8] = b2.x;
  }
  // C - I = B^T G(ds) B  (G linear in s, G(s0) = Dm^T Dm)
  float G[3][3];
  G[0][0] = ds[0];
  G[1][1] = ds[1];
  G[2][2] = ds[2];
  G[0][1] = G[1][0] = 0.5f * (ds[0] + ds[1] - ds[3]);
  G[0][2] = G[2][0] = 0.5f * (ds[0] + ds[2] - ds[4]);
  G[1][2] = G[2][1] = 0.5f * (ds[1] + ds[2] - ds[5]);
  float Y[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) Y[r][c] = G[r][0] * B[c] + G[r][1] * B[3 + c] + G[r][2] * B[6 + c];
  const int I[6] = {0, 1, 2, 0, 0, 1}, J[6] = {0, 1, 2, 1, 2, 2};
  float Eg[6];   // Green strain (C - I)/2
#pragma unroll
  for (int v = 0; v < 6; ++v)
    Eg[v] = 0.5f * (B[I[v]] * Y[0][J[v]] + B[3 + I[v]] * Y[1][J[v]] + B[6 + I[v]] * Y[2][J[v]]);
  const float tr = lam * (Eg[0] + Eg[1] + Eg[2]);
  S[0] = tr + 2.f * mu * Eg[0];
  S[1] = tr + 2.f * mu * Eg[1];
  S[2] = tr + 2.f * mu * Eg[2];
  S[3] = 2.f * mu * Eg[3];
  S[4] = 2.f * mu * Eg[4];
  S[5] = 2.f * mu * Eg[5];
}

// Eq. 14 per tet: the stress fed to the Eq. 20 average (chi S, or S); the
// edge-normal stresses of Eq. 22-25 are formed in k_tet_chi32, only for the
// tets that have a broken edge.
__device__ __forceinline__ void tet_stress32_body(const DevMesh& m, const Material& mt, const StepScalars& sp, unsigned bid, unsigned nb) {
  const int64_t t = bid * int64_t(blockDim.x) + threadIdx.x;
  if (t >= m.T) return;
  const MixDev& x = m.mx;
  float e[6][3], S[6];
  tet_current_stress32(m, mt, t, e, S);
  const float w = mt.average_degraded ? x.chi32[t] : 1.f;
  float4* si = reinterpret_cast<float4*>(x.sig_in32 + 8 * t);
  si[0] = make_float4(w * S[0], w * S[1], w * S[2], w * S[3]);
  si[1] = make_float4(w * S[4], w * S[5], 0.f, 0.f);
}
__global__ void __launch_bounds__(kThreads) k_tet_stress32(DevMesh m, Material mt, StepScalars sp) {
  tet_stress32_body(m, mt, sp, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kThreads) kb_tet_stress32(const BatchTab* __restrict__ tab) {
  unsigned bid, nb;
  const int k = batch_locate(tab, kB_tet_stress32, blockIdx.x, bid, nb);
  tet_stress32_body(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb);
}

// Eq. 20 sum in FP32, tiled.  A CTA takes a tile of consecutive tets (128, or
// 64 where the radius makes the unions wide: the mesh's nl_tile) and first
// stages the union of their neighbour sets (ascending tet ids, six floats a
// row) in shared memory; a tile whose union exceeds the staged capacity reads
// the rows from global memory instead.  A single-mesh launch stages as many
// rows as the mesh's largest union (at most kNlCapMax), so its occupancy
// follows the radius; a batched launch stages kNlCap rows for every mesh.  Each pair of tets (2q, 2q+1) has a joint list:
// the union of the two neighbour lists, per entry a 16-bit union position and
// the two FP32 weights (zero where a tet lacks that neighbour), so one staged
// row read serves both tets (0.61 row reads per (tet, neighbour) pair on the
// loaf instead of 1).  Each list is padded to a multiple of four entries (pads
// repeat a position of the list with zero weights) and read in groups of four
// consecutive entries.  A warp works on four pairs at once, eight lanes per
// pair: lane s of a pair takes the groups s, s + 8, s + 16, ..., each with one
// 8-byte load of its four positions and two 16-byte loads of their weights
// (a block of 32 entries keeps the weights of the lanes' first two entries,
// then of their last two, so each load of a pair's eight lanes is one
// contiguous 128-byte line), kNlGroups groups loaded while the previous ones
// are summed.  The twelve sums
// of a pair are then reduced over its eight lanes by a transposing butterfly
// (three steps, each lane keeping half of its values), which leaves two output
// columns in each lane: one 8-byte store per lane writes the two 32-byte
// output rows.  The host orders each list so that the eight entries a pair
// sums at once fall on distinct shared-memory bank pairs, and the two pairs of
// a half-warp on opposite halves of the banks.
constexpr int kNlThreads = 256;
constexpr unsigned kNlSmem = kNlCap * 24;           // batched launches
constexpr unsigned kNlSmemMax = kNlCapMax * 24;     // single-mesh launches at most
constexpr int kNlGroups = 1;  // groups of four entries of a lane in flight per load batch

struct NlBatch {
  uint2 loc[kNlGroups];       // four 16-bit positions per group
  float4 wt[kNlGroups][2];    // (w_2q, w_2q+1) of entries 0, 1 and of entries 2, 3
  bool ok[kNlGroups];
};
// groups G, G + 8, ..., G + 8 (kNlGroups - 1) of a list of n entries at beg
__device__ __forceinline__ void nl_load(const MixDev& x, int64_t beg, int64_t n, int64_t G, NlBatch& q) {
#pragma unroll
  for (int c = 0; c < kNlGroups; ++c) {
    const int64_t e = 4 * (G + 8 * c);
    q.ok[c] = e < n;
    if (q.ok[c]) {
      const int64_t blk = e & ~int64_t(31), sl = (e & 31) >> 2;
      const int64_t m = n - blk < 32 ? (n - blk) >> 2 : 8;   // lanes with a group in this block
      q.loc[c] = __ldg(reinterpret_cast<const uint2*>(x.nb_loc + beg + e));
      q.wt[c][0] = __ldg(reinterpret_cast<const float4*>(x.nb_w2 + beg + blk + 2 * sl));
      q.wt[c][1] = __ldg(reinterpret_cast<const float4*>(x.nb_w2 + beg + blk + 2 * m + 2 * sl));
    }
  }
}
__device__ __forceinline__ void nl_row(const MixDev& x, const float2* su, bool staged, int64_t u0, int loc, float2& r0,
                                       float2& r1, float2& r2) {
  if (staged) {
    r0 = su[3 * loc];
    r1 = su[3 * loc + 1];
    r2 = su[3 * loc + 2];
  } else {
    float sj[8];
    ld8f(x.sig_in32 + 8 * int64_t(__ldg(x.nl_uidx + u0 + loc)), sj);
    r0 = make_float2(sj[0], sj[1]);
    r1 = make_float2(sj[2], sj[3]);
    r2 = make_float2(sj[4], sj[5]);
  }
}
// Packed FP32 FMA (two lanes of fma.rn.f32x2, sm_100 and later): c.x += a.x b.x,
// c.y += a.y b.y, each rounded once like a scalar FMA.
__device__ __forceinline__ void fma2(float2& c, float2 a, float2 b) {
  asm("{\n\t.reg .b64 ra, rb, rc;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%0, %1};\n\t"
      "fma.rn.f32x2 rc, ra, rb, rc;\n\tmov.b64 {%0, %1}, rc;\n\t}"
      : "+f"(c.x), "+f"(c.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
}
// acc[0..2]: the first tet of the pair (columns 0-5 as pairs), acc[3..5]: the second
__device__ __forceinline__ void nl_accumulate(const MixDev& x, const float2* su, bool staged, int64_t u0, const NlBatch& q,
                                              float2 (&acc)[6]) {
#pragma unroll
  for (int c = 0; c < kNlGroups; ++c) {
    if (!q.ok[c]) continue;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const unsigned word = k < 2 ? q.loc[c].x : q.loc[c].y;
      const int loc = int((word >> (16 * (k & 1))) & 0xffffu);
      const float4 w = q.wt[c][k >> 1];
      const float w0 = (k & 1) ? w.z : w.x, w1 = (k & 1) ? w.w : w.y;
      float2 r0, r1, r2;
      nl_row(x, su, staged, u0, loc, r0, r1, r2);
      const float2 wa = make_float2(w0, w0), wb = make_float2(w1, w1);
      fma2(acc[0], wa, r0);
      fma2(acc[1], wa, r1);
      fma2(acc[2], wa, r2);
      fma2(acc[3], wb, r0);
      fma2(acc[4], wb, r1);
      fma2(acc[5], wb, r2);
    }
  }
}
// Reduce v[0..15] (columns 0-7 of the first tet, then of the second) over the
// eight lanes of a group: afterwards lane s holds columns 2 (s & 3) and
// 2 (s & 3) + 1 of tet s >> 2 (each step keeps the half named by a bit of s).
__device__ __forceinline__ float2 group_transpose_sum(const float (&v)[16], int s, unsigned gmask) {
  const bool b2 = s & 4, b1 = s & 2, b0 = s & 1;
  float u[8], w[4];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float snd = b2 ? v[k] : v[8 + k];
    u[k] = (b2 ? v[8 + k] : v[k]) + __shfl_xor_sync(gmask, snd, 4);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float snd = b1 ? u[k] : u[4 + k];
    w[k] = (b1 ? u[4 + k] : u[k]) + __shfl_xor_sync(gmask, snd, 2);
  }
  const float s0 = b0 ? w[0] : w[2], s1 = b0 ? w[1] : w[3];
  const float k0 = (b0 ? w[2] : w[0]) + __shfl_xor_sync(gmask, s0, 1);
  const float k1 = (b0 ? w[3] : w[1]) + __shfl_xor_sync(gmask, s1, 1);
  return make_float2(k0, k1);
}

// cap: rows this launch stages (its dynamic shared memory / 24 B)
__device__ __forceinline__ void nonlocal32_body(const DevMesh& m, const Material& mt, const StepScalars& sp, unsigned bid, unsigned nb,
                                                int cap) {
  extern __shared__ float2 su[];   // [cap][3]: stress rows of the tile's union
  constexpr int kStage = 8;        // union rows of a thread in flight together
  const MixDev& x = m.mx;
  const int64_t t0 = int64_t(bid) * x.nl_tile;
  const int warp_pairs = x.nl_tile / 2 / (kNlThreads / 32);   // tet pairs of a warp: 8 (128-tet tiles) or 4
  const int64_t u0 = x.nl_uptr[bid], un = x.nl_uptr[bid + 1] - u0;
  const bool staged = un <= cap;
  if (staged) {   // a thread's union ids, then their rows, kStage at a time in flight together
    for (int64_t r0 = 0; r0 < un; r0 += int64_t(kStage) * kNlThreads) {
      int64_t j[kStage];
#pragma unroll
      for (int c = 0; c < kStage; ++c) {
        const int64_t r = r0 + threadIdx.x + int64_t(c) * kNlThreads;
        j[c] = r < un ? __ldg(x.nl_uidx + u0 + r) : -1;
      }
#pragma unroll
      for (int c = 0; c < kStage; ++c) {
        if (j[c] < 0) continue;
        const int64_t r = r0 + threadIdx.x + int64_t(c) * kNlThreads;
        float sj[8];
        ld8f(x.sig_in32 + 8 * j[c], sj);
        su[3 * r] = make_float2(sj[0], sj[1]);
        su[3 * r + 1] = make_float2(sj[2], sj[3]);
        su[3 * r + 2] = make_float2(sj[4], sj[5]);
      }
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, g = lane >> 3, sl = lane & 7;
  const unsigned gmask = 0xffu << (lane & 24);
  // this warp's pairs: q in [qw, qw + np) (pair q = tets 2q, 2q+1), four at a time
  const int64_t NQ = (m.T + 1) / 2;
  const int64_t qw = t0 / 2 + int64_t(warp_pairs) * (threadIdx.x >> 5);
  if (qw >= NQ) return;
  const int np = int(NQ - qw < warp_pairs ? NQ - qw : warp_pairs);
  for (int r0 = 0; r0 < np; r0 += 4) {
    const int64_t q = qw + r0 + g;
    const bool live = r0 + g < np;
    const int64_t beg = live ? x.nb_ptr[q] : 0, n = live ? x.nb_ptr[q + 1] - beg : 0;
    // batches of this lane's groups; every lane of the warp runs the longest lane's count
    const int64_t groups = n / 4;
    const int mine = groups > sl ? int((groups - sl + 7) / 8) : 0;
    const int rounds = __reduce_max_sync(0xffffffffu, (mine + kNlGroups - 1) / kNlGroups);
    float2 acc2[6];
#pragma unroll
    for (int v = 0; v < 6; ++v) acc2[v] = make_float2(0.f, 0.f);
    NlBatch cur, nxt;
    nl_load(x, beg, n, sl, cur);
    for (int b = 0; b < rounds; ++b) {
      if (b + 1 < rounds) nl_load(x, beg, n, sl + 8 * kNlGroups * (b + 1), nxt);
      nl_accumulate(x, su, staged, u0, cur, acc2);
      cur = nxt;
    }
    float acc[16];
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      acc[2 * v] = acc2[v].x;
      acc[2 * v + 1] = acc2[v].y;
      acc[8 + 2 * v] = acc2[3 + v].x;
      acc[8 + 2 * v + 1] = acc2[3 + v].y;
    }
    acc[6] = acc[7] = acc[14] = acc[15] = 0.f;
    const float2 tot = group_transpose_sum(acc, sl, gmask);
    const int64_t t = 2 * q + (sl >> 2);
    if (live && t < m.T) reinterpret_cast<float2*>(x.sig_bar32 + 8 * t)[sl & 3] = tot;
  }
}
__global__ void __launch_bounds__(kNlThreads, 4) k_nonlocal32(DevMesh m, Material mt, StepScalars sp) {
  nonlocal32_body(m, mt, sp, blockIdx.x, gridDim.x, m.mx.nl_cap);
}
__global__ void __launch_bounds__(kNlThreads, 3) kb_nonlocal32(const BatchTab* __restrict__ tab) {
  unsigned bid, nb;
  const int k = batch_locate(tab, kB_nonlocal32, blockIdx.x, bid, nb);
  nonlocal32_body(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb, kNlCap);
}

__device__ __forceinline__ void edge_driver32_body(const DevMesh& m, const Material& mt, const StepScalars& sp, unsigned bid, unsigned nb) {
  const float kappa = mt.kappa32, inv_young = mt.inv_young32;
  const int stress_mode = mt.driver_stress;
  const double threshold = mt.threshold;

  const int64_t i = bid * int64_t(blockDim.x) + threadIdx.x;
  unsigned long long n_brk = 0, n_new = 0;
  if (i < m.NE) {
    const int2 ab = m.edges[i];
    float ua[3], ub[3], e0[3];
    ld3f(m.mx.u32, ab.x, ua);
    ld3f(m.mx.u32, ab.y, ub);
    ld3f(m.mx.edge_e0, i, e0);
    const float e[3] = {e0[0] + (ub[0] - ua[0]), e0[1] + (ub[1] - ua[1]), e0[2] + (ub[2] - ua[2])};
    const float s = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
    // max of (e.S.e) / s over the incident tets: one division of the largest numerator
    float mq = -INFINITY;
    for (int p = m.et_ptr[i]; p < m.et_ptr[i + 1]; ++p) {
      float S[8];
      ld8f(m.mx.sig_bar32 + 8 * int64_t(m.et_tet[p]), S);
      mq = fmaxf(mq, normal_stress32(e, 1.f, S, kappa));
    }
    const float mx = mq / s;
    const double d = double(stress_mode ? mx : mx * inv_young);
    m.driver[i] = d;
    const uint8_t old = m.labels[i];
    const uint8_t now = (old || d >= threshold) ? 1 : 0;   // threshold test in FP64
    if (now != old) m.labels[i] = now;
    n_brk = now;
    n_new = now && !old;
  }
  warp_count(n_brk, m.counters + kCntBroken);
  warp_count(n_new, m.counters + kCntNewBroken);
}
__global__ void __launch_bounds__(kThreads) k_edge_driver32(DevMesh m, Material mt, StepScalars sp) {
  edge_driver32_body(m, mt, sp, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kThreads) kb_edge_driver32(const BatchTab* __restrict__ tab) {
  unsigned bid, nb;
  const int k = batch_locate(tab, kB_edge_driver32, blockIdx.x, bid, nb);
  edge_driver32_body(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb);
}

__device__ __forceinline__ void tet_chi32_body(const DevMesh& m, const Material& mt, const StepScalars& sp, unsigned bid, unsigned nb) {
  const float young = mt.young32;
  const uint64_t lut = mt.lut;

  const int64_t t = bid * int64_t(blockDim.x) + threadIdx.x;
  unsigned long long zero = 0;
  if (t < m.T) {
    int mask = 0;
#pragma unroll
    for (int k = 0; k < 6; ++k) mask |= int(m.labels[m.tet_edges[6 * t + k]] != 0) << k;
    float c = 1.f;
    if (mask) {
      if ((lut >> mask) & 1ull) {
        c = 0.f;
      } else {
        float e[6][3], S[6];
        tet_current_stress32(m, mt, t, e, S);
        float num = 0.f, den = 0.f;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          const float a =
              fabsf(normal_stress32(e[k], e[k][0] * e[k][0] + e[k][1] * e[k][1] + e[k][2] * e[k][2], S, mt.kappa32));
          den += a;
          if (!((mask >> k) & 1)) num += a;
        }
        c = (den <= 1e-12f * young) ? float(6 - __popc(mask)) / 6.f : num / den;
      }
    }
    m.mx.chi32[t] = c;
    m.chi[t] = double(c);
    zero = (c == 0.f);
  }
  warp_count(zero, m.counters + kCntChiZero);
}
__global__ void __launch_bounds__(kThreads) k_tet_chi32(DevMesh m, Material mt, StepScalars sp) {
  tet_chi32_body(m, mt, sp, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kThreads) kb_tet_chi32(const BatchTab* __restrict__ tab) {
  unsigned bid, nb;
  const int k = batch_locate(tab, kB_tet_chi32, blockIdx.x, bid, nb);
  tet_chi32_body(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb);
}

// ---------------------------------------------------------------------------
// Two-phase assembly, no colours and no atomics.
// Phase 1 (k_elem32, one thread per tet): the tet's six off-diagonal 3x3
// blocks (a < b) of (dt beta + dt^2) chi k_e and its four nodal rhs shares
// dt chi (f_a - (beta + dt) (k_e v)_a), built in a shared-memory row of
// kElemW floats, then written by the CTA into the assembly rows they belong
// to: local node a's rhs share to node row nrow[4t+a] (3 floats and a pad),
// local edge k's block to edge row erow[6t+k] (9 floats, oriented for the
// global edge (i, j), i < j).
// Phase 2 (k_gather32): a thread per off-diagonal matrix entry or rhs
// component streams through the contiguous rows of its edge or node in
// ascending tet order and adds the external and damping terms.
// Phase 3 (k_diag32): the diagonal blocks as minus the sum of their row's
// off-diagonal blocks (every block row of the stiffness sums to zero) plus
// the mass, and their inverses (block Jacobi).
// ---------------------------------------------------------------------------

constexpr int kElemW = 68;   // 54 block floats + 12 rhs floats + 2 pad
constexpr int kNodeRow = 4, kEdgeRow = 9;
// Each thread's row is built in shared memory (stride 69 floats: conflict-free
// for 32 consecutive threads), each block already oriented for its global edge
// (transposed where the tet's local order of the edge's nodes is the reverse
// of the global one); each warp then writes its 32 rows out, the node rows as
// one 16-byte store each and the edge rows as runs of 9 consecutive floats,
// with the destination rows passed between lanes by shuffles.
constexpr int kElemThreads = 128, kElemSS = kElemW + 1;
constexpr unsigned kElemSmem = kElemThreads * kElemSS * 4;

// one tet's row: the six off-diagonal 3x3 blocks (scaled; local edge k's block
// at 9 k), four rhs shares, two zeros
__device__ __forceinline__ void elem32_row(const DevMesh& m, const StepScalars& sp, int64_t t, float* o) {
  const float sKv = sp.sKv, cv = sp.cv, dtf = sp.dtf;
  const MixDev& x = m.mx;
  const float chi = x.chi32[t];
  if (chi == 0.f) {
    for (int q = 0; q < kElemW; ++q) o[q] = 0.f;
    return;
  }
  const int4 n = m.tets[t];
  const int nid[4] = {n.x, n.y, n.z, n.w};
  float du[4][3], vv[4][3];
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    ld3f(x.u32, nid[b], du[b]);
    ld3f(x.v32, nid[b], vv[b]);
  }
  float A[32];
  load_restA(x.restA, t, A);
  float E0[6][3], e[6][3], ds[6];
  rest_edges(A, E0);
  edge_state(E0, du, e, ds);
  const float* H = A + kRAH;
  auto h = [&](int k, int l) { return k <= l ? H[tri6(k, l)] : H[tri6(l, k)]; };
  float g[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    float s = 0.f;
#pragma unroll
    for (int l = 0; l < 6; ++l) s += h(k, l) * ds[l];
    g[k] = s;
  }
  unsigned flip = 0u;   // bit q: local edge q runs against the global (i < j) order
  {
    const int4 n2 = m.tets[t];
    const int nid2[4] = {n2.x, n2.y, n2.z, n2.w};
#pragma unroll
    for (int k = 0; k < 6; ++k) flip |= nid2[edge_a(k)] > nid2[edge_b(k)] ? (1u << k) : 0u;
  }
  // Y_b[k][c] = sum_{l in b} H_kl sgn_lb e_l[c]  (sgn = -1 if b is the first node of l)
  // only the off-diagonal blocks (a < b): the block rows sum to zero, and
  // k_diag32 forms the assembled diagonal blocks
  float Kv[4][3] = {};
#pragma unroll
  for (int b = 1; b < 4; ++b) {
    float Y[6][3];
#pragma unroll
    for (int k = 0; k < 6; ++k)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float y = 0.f;
#pragma unroll
        for (int l = 0; l < 6; ++l) {
          if (edge_a(l) != b && edge_b(l) != b) continue;
          y += (edge_a(l) == b ? -h(k, l) : h(k, l)) * e[l][c];
        }
        Y[k][c] = y;
      }
#pragma unroll
    for (int a = 0; a < b; ++a) {
      float blk[3][3];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          float v = 0.f;
#pragma unroll
          for (int k = 0; k < 6; ++k) {
            if (edge_a(k) != a && edge_b(k) != a) continue;
            v += (edge_a(k) == a ? -e[k][r] : e[k][r]) * Y[k][c];
          }
          blk[r][c] = 4.f * v;
        }
      float geo = 0.f;
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        const bool ina = edge_a(k) == a || edge_b(k) == a, inb = edge_a(k) == b || edge_b(k) == b;
        if (a == b && ina) geo += 2.f * g[k];
        if (a != b && ina && inb) geo -= 2.f * g[k];
      }
      blk[0][0] += geo;
      blk[1][1] += geo;
      blk[2][2] += geo;
      // K v with relative velocities (rigid translations are in the null space)
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        Kv[a][r] += blk[r][0] * (vv[b][0] - vv[a][0]) + blk[r][1] * (vv[b][1] - vv[a][1]) +
                    blk[r][2] * (vv[b][2] - vv[a][2]);
        if (a != b)
          Kv[b][r] += blk[0][r] * (vv[a][0] - vv[b][0]) + blk[1][r] * (vv[a][1] - vv[b][1]) +
                      blk[2][r] * (vv[a][2] - vv[b][2]);
      }
      const int q = a == 0 ? b - 1 : a + b;   // local edge of (a, b)
      const float sk = sKv * chi;
      const bool tr = (flip >> q) & 1u;
      float* ob = o + 9 * q;
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) ob[tr ? 3 * c + r : 3 * r + c] = sk * blk[r][c];
    }
  }
  // rhs shares: dt chi (f_a - cv (K v)_a), f_a = -2 sum_{k in a} sgn_ka g_k e_k
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      float f = 0.f;
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        if (edge_a(k) == a) f += 2.f * g[k] * e[k][r];
        if (edge_b(k) == a) f -= 2.f * g[k] * e[k][r];
      }
      o[54 + 3 * a + r] = dtf * chi * (f - cv * Kv[a][r]);
    }
  o[66] = 0.f;
  o[67] = 0.f;
}
__device__ __forceinline__ void elem32_body(const DevMesh& m, const Material& mt, const StepScalars& sp, unsigned bid, unsigned nb) {
  extern __shared__ float sh_rows[];
  const int64_t t0 = bid * int64_t(blockDim.x), t = t0 + threadIdx.x;
  const int lane = threadIdx.x & 31, wbase = threadIdx.x & ~31;
  const MixDev& x = m.mx;
  int32_t nr[4] = {0, 0, 0, 0}, er[6] = {0, 0, 0, 0, 0, 0};
  if (t < m.T) {
    elem32_row(m, sp, t, sh_rows + threadIdx.x * kElemSS);
#pragma unroll
    for (int k = 0; k < 6; ++k) er[k] = m.erow[6 * t + k];
#pragma unroll
    for (int a = 0; a < 4; ++a) nr[a] = m.nrow[4 * t + a];
  }
  __syncwarp();
  // each warp writes out its own 32 rows; the row indices come from the owning lane
  const int64_t rem = m.T - (t0 + wbase);
  const int nw = rem < 32 ? int(rem) : 32;   // live rows of this warp (the whole warp agrees)
  if (nw <= 0) return;
  const float* wrows = sh_rows + wbase * kElemSS;
  // node rows: one float4 each (the rhs share of node a and a pad); lane r
  // writes its own row's four node rows
  float4* nbuf = reinterpret_cast<float4*>(x.ebuf);
  if (lane < nw) {
    const float* src = wrows + lane * kElemSS;
#pragma unroll
    for (int a = 0; a < 4; ++a)
      nbuf[nr[a]] = make_float4(src[54 + 3 * a], src[54 + 3 * a + 1], src[54 + 3 * a + 2], 0.f);
  }
  // edge rows: 9 consecutive floats each (float q of row r is j = 9 r + q)
  float* ebuf = x.ebuf + int64_t(kNodeRow) * 4 * m.T;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
#pragma unroll
    for (int j = lane; j < 288; j += 32) {
      const int r = j / 9, q = j - 9 * r;
      const int32_t row = __shfl_sync(0xffffffffu, er[k], r);
      if (r < nw) ebuf[int64_t(kEdgeRow) * row + q] = wrows[r * kElemSS + 9 * k + q];
    }
  }
}

__global__ void __launch_bounds__(128, 6) k_elem32(DevMesh m, Material mt, StepScalars sp) {
  elem32_body(m, mt, sp, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(128, 6) kb_elem32(const BatchTab* __restrict__ tab) {
  unsigned bid, nb;
  const int k = batch_locate(tab, kB_elem32, blockIdx.x, bid, nb);
  elem32_body(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb);
}

// Phase 2 in the layout of the FP64 gather: threads [0, 9 NE) take one entry
// of an edge's block (the 4-6 tets around the edge, rows contiguous) and write
// it to (i, j) and, transposed, (j, i); threads [9 NE, 9 NE + 3 N) take a
// node's rhs components (the ~24 tets around the node).  Sums run in
// ascending tet order (deterministic).
__device__ __forceinline__ void gather32_body(const DevMesh& m, const Material& mt, const StepScalars& sp, unsigned bid, unsigned nb) {
  const float dtf = sp.dtf, alphaf = sp.alphaf;
  const MixDev& x = m.mx;
  const int64_t t = bid * int64_t(blockDim.x) + threadIdx.x;
  const int64_t n_edge = 9 * m.NE;
  if (t < n_edge) {
    const int64_t e = t / 9;
    const int q = int(t - 9 * e);
    const float acc = row_sum<8>(x.ebuf + int64_t(kNodeRow) * 4 * m.T + q, kEdgeRow, m.et_ptr[e], m.et_ptr[e + 1]);
    const int2 sl = m.edge_slot[e];
    x.val32[9 * int64_t(sl.x) + q] = acc;
    x.val32[9 * int64_t(sl.y) + 3 * (q % 3) + q / 3] = acc;
    return;
  }
  const int64_t u = t - n_edge;
  if (u >= 3 * m.N) return;
  const int64_t i = u / 3;
  const int c3 = int(u - 3 * i);
  const float acc = row_sum<8>(x.ebuf + c3, kNodeRow, m.np_ptr[i], m.np_ptr[i + 1]);
  const float fe = sp.has_fext ? float(m.f_ext[3 * i + c3]) : 0.f;   // f_ext in FP32
  float mv = x.mass32[i] * x.v32[3 * i + c3];
  if (x.mass_blk32) {
    mv = 0.f;
    for (int b = m.row_ptr[i]; b < m.row_ptr[i + 1]; ++b) mv += x.mass_blk32[b] * x.v32[3 * int64_t(m.col[b]) + c3];
  }
  x.rhs32[3 * i + c3] = acc + dtf * (fe - alphaf * mv);
}

// Phase 3: A_ii = -sum_{j != i} A_ij (zero block-row sums of the stiffness)
// plus the mass (lumped on the diagonal, or the consistent m_ij of Eq. 5 on
// every block of the row, added after the sum), then the block-Jacobi inverse
// of A_ii in FP32.  Nine threads per node (entry q), 32 nodes per CTA of
// kDiagThreads: the node's nine entries meet in shared memory and thread q
// writes entry q of the inverse (cofactor q over the determinant).
constexpr int kDiagThreads = 288;
__device__ __forceinline__ void diag32_body(const DevMesh& m, const Material& mt, const StepScalars& sp, unsigned bid, unsigned nb) {
  __shared__ float dsh[kDiagThreads];
  const MixDev& x = m.mx;
  const int64_t t = bid * int64_t(kDiagThreads) + threadIdx.x;
  const bool live = t < 9 * m.N;
  const int64_t i = t / 9;
  const int q = int(t - 9 * i);
  float diag = 0.f;
  if (live) {
    const int d = m.diag_blk[i], b0 = m.row_ptr[i], b1 = m.row_ptr[i + 1];
    float acc = 0.f;
    for (int b = b0; b < b1; ++b)
      if (b != d) acc += x.val32[9 * int64_t(b) + q];
    diag = -acc;
    if (q == 0 || q == 4 || q == 8) {
      const float cmf = sp.cmf;
      diag += cmf * (x.mass_blk32 ? x.mass_blk32[d] : x.mass32[i]);
      if (x.mass_blk32)
        for (int b = b0; b < b1; ++b)
          if (b != d) x.val32[9 * int64_t(b) + q] += cmf * x.mass_blk32[b];   // Eq. 5
    }
    x.val32[9 * int64_t(d) + q] = diag;
  }
  dsh[threadIdx.x] = diag;
  __syncthreads();
  if (!live) return;
  const float* d = dsh + (threadIdx.x - q);
  const float c00 = d[4] * d[8] - d[5] * d[7], c01 = d[2] * d[7] - d[1] * d[8], c02 = d[1] * d[5] - d[2] * d[4];
  const float c10 = d[5] * d[6] - d[3] * d[8], c11 = d[0] * d[8] - d[2] * d[6], c12 = d[2] * d[3] - d[0] * d[5];
  const float c20 = d[3] * d[7] - d[4] * d[6], c21 = d[1] * d[6] - d[0] * d[7], c22 = d[0] * d[4] - d[1] * d[3];
  const float id = 1.f / (d[0] * c00 + d[1] * c10 + d[2] * c20);
  const float cq = q == 0 ? c00 : q == 1 ? c01 : q == 2 ? c02 : q == 3 ? c10 : q == 4 ? c11 : q == 5 ? c12
                 : q == 6 ? c20 : q == 7 ? c21 : c22;
  x.pinv32[9 * i + q] = cq * id;
}
__global__ void __launch_bounds__(kDiagThreads) k_diag32(DevMesh m, Material mt, StepScalars sp) {
  diag32_body(m, mt, sp, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kDiagThreads) kb_diag32(const BatchTab* __restrict__ tab) {
  unsigned bid, nb;
  const int k = batch_locate(tab, kB_diag32, blockIdx.x, bid, nb);
  diag32_body(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb);
}
__global__ void __launch_bounds__(256) k_gather32(DevMesh m, Material mt, StepScalars sp) {
  gather32_body(m, mt, sp, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(256) kb_gather32(const BatchTab* __restrict__ tab) {
  unsigned bid, nb;
  const int k = batch_locate(tab, kB_gather32, blockIdx.x, bid, nb);
  gather32_body(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb);
}

// ---------------------------------------------------------------------------
// FP64 iterative refinement around an FP32 PCG
// ---------------------------------------------------------------------------

// r = b - A32 dv on free rows, with A32 dv formed to double-float accuracy
// (dv = dv_hi + dv_lo) and b - A dv in double-float; eight lanes per block row
// (lane j takes blocks j, j+8, ..., two at a time so that both blocks' loads
// are in flight before the arithmetic).  Each lane accumulates in the manner of
// Dot2 (Ogita, Rump and Oishi, "Accurate sum and dot product", 2005): s collects
// the rounded products, c the exact error of each product (an FMA) and of each
// addition (TwoSum), and s + c is as accurate as a sum in twice the precision;
// the pair is renormalised once per lane.  A transposing double-float butterfly
// then leaves component c of row i in lanes 2c and 2c + 1, and lane 2c forms
// r_c.  The inner solve's right-hand side is the leading float of r; ||r||^2
// accumulates in double-float.
__device__ __forceinline__ void ir_residual_body(const DevMesh& m, const Material& mt, const StepScalars& sp, unsigned bid, unsigned nb, int first) {

  IrState* S = m.mx.ir;
  // after the first call: only right after a correction was applied (inner solve
  // finished, residual not yet formed); flags are written by the last CTA only
  if (!first && (S->done || !S->in_done || S->applied)) return;
  const MixDev& x = m.mx;
  const int j8 = threadIdx.x & 7;
  const unsigned gmask = 0xffu << (threadIdx.x & 24);
  float nh_[1] = {0.f}, nl_[1] = {0.f};
  const int64_t ng = (int64_t(nb) * blockDim.x) >> 3;
  for (int64_t i = (bid * int64_t(blockDim.x) + threadIdx.x) >> 3; i < m.N; i += ng) {
    float hi[4] = {0, 0, 0, 0}, lo[4] = {0, 0, 0, 0};
    // independent loads first; pinned rows run the loop too and are zeroed at the end
    const bool fixed = m.pinned[i];
    const int b1 = m.row_ptr[i + 1];
    const int cw = j8 >> 1;   // the component this lane ends with (3: none)
    const float bh = ((j8 & 1) == 0 && cw < 3) ? x.rhs32[3 * i + cw] : 0.f;
    // the first residual of a step without pinned nodes has dv = 0 exactly:
    // A dv = 0 and b - 0 = b, so the product is skipped (same bits)
    if (!(first && sp.n_pinned == 0)) {
      float sacc[4] = {0, 0, 0, 0}, cacc[4] = {0, 0, 0, 0};
      for (int b = m.row_ptr[i] + j8; b < b1; b += 16) {
        const bool two = b + 8 < b1;
        const int64_t j0 = m.col[b], j1 = two ? m.col[b + 8] : j0;
        float a0[9], a1[9], xh0[3], xl0[3], xh1[3], xl1[3];
#pragma unroll
        for (int q = 0; q < 9; ++q) {
          a0[q] = x.val32[9 * int64_t(b) + q];
          a1[q] = two ? x.val32[9 * int64_t(b + 8) + q] : 0.f;
        }
        ld3f(x.dv_hi, j0, xh0);
        ld3f(x.dv_lo, j0, xl0);
        ld3f(x.dv_hi, j1, xh1);
        ld3f(x.dv_lo, j1, xl1);
        dot2_block(sacc, cacc, a0, xh0, xl0);
        if (two) dot2_block(sacc, cacc, a1, xh1, xl1);
      }
#pragma unroll
      for (int rr = 0; rr < 3; ++rr) two_sum(sacc[rr], cacc[rr], hi[rr], lo[rr]);
    }
    // transposing butterfly over the 8 lanes: keep 2 of 4 values, then 1 of 2, then pair up
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
    if (first) {
      S->bb = out[0];
      S->sweeps = 0;
      S->total_iters = 0;
      S->status = GF_OK;
    } else {
      S->sweeps += 1;
    }
    S->applied = 1;   // a fresh residual is ready for the next inner solve
    S->rr = out[0];
    S->done = (out[0] == 0.0 || out[0] <= S->tol2 * S->bb) ? 1 : 0;
    if (!isfinite(out[0])) {
      S->status = GF_NAN;
      S->done = 1;
    } else if (!S->done && S->total_iters >= S->maxit) {
      S->status = GF_CG_MAXITER;
      S->done = 1;
    }
  }
}
__global__ void __launch_bounds__(kThreads, 5) k_ir_residual(DevMesh m, Material mt, StepScalars sp, int first) {
  ir_residual_body(m, mt, sp, blockIdx.x, gridDim.x, first);
}
__global__ void __launch_bounds__(kThreads, 5) kb_ir_residual(const BatchTab* __restrict__ tab, int first) {
  unsigned bid, nb;
  const int k = batch_locate(tab, kB_ir_residual, blockIdx.x, bid, nb);
  ir_residual_body(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb, first);
}

// inner PCG start (only after a fresh residual; otherwise the current inner
// solve continues): r32 = r, z = P r (z32 and z4), p = z, d = 0
__device__ __forceinline__ void ir_inner_init_body(const DevMesh& m, const Material& mt, const StepScalars& sp, unsigned bid, unsigned nb) {

  IrState* S = m.mx.ir;
  if (S->done || !S->applied) return;
  const MixDev& x = m.mx;
  float h[1] = {0.f}, l[1] = {0.f};
  for (int64_t i = bid * int64_t(blockDim.x) + threadIdx.x; i < m.N; i += int64_t(nb) * blockDim.x) {
    float r[3] = {0, 0, 0}, z[3] = {0, 0, 0};
    if (!m.pinned[i]) {
#pragma unroll
      for (int c = 0; c < 3; ++c) r[c] = x.rres[3 * i + c];
      const float* pi = x.pinv32 + 9 * i;
#pragma unroll
      for (int c = 0; c < 3; ++c) z[c] = pi[3 * c] * r[0] + pi[3 * c + 1] * r[1] + pi[3 * c + 2] * r[2];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      x.r32[3 * i + c] = r[c];
      x.z32[3 * i + c] = z[c];
      x.p32[3 * i + c] = z[c];
      x.d32[3 * i + c] = 0.f;
      df_acc_prod(h[0], l[0], r[c], z[c]);
    }
    x.z4[i] = make_float4(z[0], z[1], z[2], 0.f);   // z of the two-kernel form
  }
  double out[1];
  if (grid_reduce_df<1>(h, l, m.partials, m.tickets + 5, out, bid, nb) && threadIdx.x == 0) {
    S->rz = out[0];
    S->in_rr0 = S->rr;
    S->in_iters = 0;
    S->in_done = (out[0] == 0.0) ? 1 : 0;
    S->applied = 0;
  }
}
__global__ void __launch_bounds__(kThreads) k_ir_inner_init(DevMesh m, Material mt, StepScalars sp) {
  ir_inner_init_body(m, mt, sp, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kThreads) kb_ir_inner_init(const BatchTab* __restrict__ tab) {
  unsigned bid, nb;
  const int k = batch_locate(tab, kB_ir_inner_init, blockIdx.x, bid, nb);
  ir_inner_init_body(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb);
}

// y = A32 v over all rows with half a warp per block row (coalesced block
// loads) and two rows (i0, i0 + nh) in flight per half-warp; lane c < 3 ends
// with component c of both rows, stores it to y and adds v_i . y_i to (h, l)
// in double-float (own v loaded up front).  The same bits for y as one row at a
// time: every lane sums its blocks in the same order.
// A node's three components of a vector stored as [N][3] floats or as one
// 16-byte row per node (float4, w unused: a single load per gather)
__device__ __forceinline__ void vrow(const float* __restrict__ v, int64_t j, float& a, float& b, float& c) {
  a = v[3 * j];
  b = v[3 * j + 1];
  c = v[3 * j + 2];
}
__device__ __forceinline__ void vrow(const float4* __restrict__ v, int64_t j, float& a, float& b, float& c) {
  const float4 t = v[j];
  a = t.x;
  b = t.y;
  c = t.z;
}
__device__ __forceinline__ float vcomp(const float* __restrict__ v, int64_t i, int c) { return v[3 * i + c]; }
__device__ __forceinline__ float vcomp(const float4* __restrict__ v, int64_t i, int c) {
  return reinterpret_cast<const float*>(v)[4 * i + c];
}

template <typename V>
__device__ __forceinline__ void spmv32_rows(const DevMesh& m, const V* __restrict__ v, float* __restrict__ y,
                                            unsigned bid, unsigned nb, float& h, float& l) {
  const float* __restrict__ val = m.mx.val32;
  const int j16 = threadIdx.x & 15;
  const unsigned hmask = (threadIdx.x & 16) ? 0xffff0000u : 0x0000ffffu;
  const int64_t nh = (int64_t(nb) * blockDim.x) >> 4;
  for (int64_t i0 = (bid * int64_t(blockDim.x) + threadIdx.x) >> 4; i0 < m.N; i0 += 2 * nh) {
    const int64_t i1 = i0 + nh;
    const bool two = i1 < m.N;
    const int s0 = m.row_ptr[i0], e0 = m.row_ptr[i0 + 1];
    const int s1 = two ? m.row_ptr[i1] : 0, e1 = two ? m.row_ptr[i1 + 1] : 0;
    const float vi0 = j16 < 3 ? vcomp(v, i0, j16) : 0.f;
    const float vi1 = (two && j16 < 3) ? vcomp(v, i1, j16) : 0.f;
    float y0 = 0.f, y1 = 0.f, y2 = 0.f, u0 = 0.f, u1 = 0.f, u2 = 0.f;
    const int len = max(e0 - s0, e1 - s1);
    for (int k = j16; k < len; k += 16) {
      if (s0 + k < e0) {
        const int b = s0 + k;
        const int64_t j = m.col[b];
        const float* a = val + 9 * int64_t(b);
        float x0, x1, x2;
        vrow(v, j, x0, x1, x2);
        y0 += a[0] * x0 + a[1] * x1 + a[2] * x2;
        y1 += a[3] * x0 + a[4] * x1 + a[5] * x2;
        y2 += a[6] * x0 + a[7] * x1 + a[8] * x2;
      }
      if (s1 + k < e1) {
        const int b = s1 + k;
        const int64_t j = m.col[b];
        const float* a = val + 9 * int64_t(b);
        float x0, x1, x2;
        vrow(v, j, x0, x1, x2);
        u0 += a[0] * x0 + a[1] * x1 + a[2] * x2;
        u1 += a[3] * x0 + a[4] * x1 + a[5] * x2;
        u2 += a[6] * x0 + a[7] * x1 + a[8] * x2;
      }
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
      y0 += __shfl_xor_sync(hmask, y0, o);
      y1 += __shfl_xor_sync(hmask, y1, o);
      y2 += __shfl_xor_sync(hmask, y2, o);
      u0 += __shfl_xor_sync(hmask, u0, o);
      u1 += __shfl_xor_sync(hmask, u1, o);
      u2 += __shfl_xor_sync(hmask, u2, o);
    }
    if (j16 < 3) {
      const float yc = j16 == 0 ? y0 : (j16 == 1 ? y1 : y2);
      y[3 * i0 + j16] = yc;
      df_acc_prod(h, l, vi0, yc);
      if (two) {
        const float uc = j16 == 0 ? u0 : (j16 == 1 ? u1 : u2);
        y[3 * i1 + j16] = uc;
        df_acc_prod(h, l, vi1, uc);
      }
    }
  }
}

// q = A32 p, p . q in double-float
__device__ __forceinline__ void ir_spmv_body(const DevMesh& m, const Material& mt, const StepScalars& sp, unsigned bid, unsigned nb) {

  IrState* S = m.mx.ir;
  if (S->done || S->in_done) return;
  const MixDev& x = m.mx;
  float h[1] = {0.f}, l[1] = {0.f};
  spmv32_rows(m, x.p32, x.q32, bid, nb, h[0], l[0]);
  double out[1];
  if (grid_reduce_df<1>(h, l, m.partials, m.tickets + 6, out, bid, nb) && threadIdx.x == 0) {
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
  }
}
__global__ void __launch_bounds__(kThreads) k_ir_spmv(DevMesh m, Material mt, StepScalars sp) {
  ir_spmv_body(m, mt, sp, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kThreads) kb_ir_spmv(const BatchTab* __restrict__ tab) {
  unsigned bid, nb;
  const int k = batch_locate(tab, kB_ir_spmv, blockIdx.x, bid, nb);
  ir_spmv_body(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb);
}

__device__ __forceinline__ void ir_update_body(const DevMesh& m, const Material& mt, const StepScalars& sp, unsigned bid, unsigned nb) {

  IrState* S = m.mx.ir;
  if (S->done || S->in_done) return;
  const MixDev& x = m.mx;
  const float alpha = S->alpha32;
  float h[2] = {0.f, 0.f}, l[2] = {0.f, 0.f};
  for (int64_t i = bid * int64_t(blockDim.x) + threadIdx.x; i < m.N; i += int64_t(nb) * blockDim.x) {
    if (m.pinned[i]) continue;
    // every load before the first store (the vectors may alias as far as the
    // compiler knows)
    float d[3], p[3], r[3], q[3], pi[9];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      d[c] = x.d32[3 * i + c];
      p[c] = x.p32[3 * i + c];
      r[c] = x.r32[3 * i + c];
      q[c] = x.q32[3 * i + c];
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) pi[k] = x.pinv32[9 * i + k];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      x.d32[3 * i + c] = d[c] + alpha * p[c];
      r[c] = r[c] - alpha * q[c];
      x.r32[3 * i + c] = r[c];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float z = pi[3 * c] * r[0] + pi[3 * c + 1] * r[1] + pi[3 * c + 2] * r[2];
      x.z32[3 * i + c] = z;
      df_acc_prod(h[0], l[0], r[c], z);
      df_acc_prod(h[1], l[1], r[c], r[c]);
    }
  }
  double out[2];
  if (grid_reduce_df<2>(h, l, m.partials, m.tickets + 7, out, bid, nb) && threadIdx.x == 0) {
    S->in_iters += 1;
    S->total_iters += 1;
    S->beta = out[0] / S->rz;
    S->beta32 = float(S->beta);
    S->rz = out[0];
    S->in_rr = out[1];
    if (!(out[1] > S->in_tol2 * S->in_rr0) || S->in_iters >= S->in_maxit || S->total_iters >= S->maxit)
      S->in_done = 1;
  }
}
__global__ void __launch_bounds__(kThreads) k_ir_update(DevMesh m, Material mt, StepScalars sp) {
  ir_update_body(m, mt, sp, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kThreads) kb_ir_update(const BatchTab* __restrict__ tab) {
  unsigned bid, nb;
  const int k = batch_locate(tab, kB_ir_update, blockIdx.x, bid, nb);
  ir_update_body(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb);
}

__device__ __forceinline__ void ir_p_body(const DevMesh& m, const Material& mt, const StepScalars& sp, unsigned bid, unsigned nb) {

  IrState* S = m.mx.ir;
  if (S->done || S->in_done) return;
  const float beta = S->beta32;
  for (int64_t i = bid * int64_t(blockDim.x) + threadIdx.x; i < 3 * m.N; i += int64_t(nb) * blockDim.x)
    m.mx.p32[i] = m.mx.z32[i] + beta * m.mx.p32[i];
}
__global__ void __launch_bounds__(kThreads) k_ir_p(DevMesh m, Material mt, StepScalars sp) {
  ir_p_body(m, mt, sp, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kThreads) kb_ir_p(const BatchTab* __restrict__ tab) {
  unsigned bid, nb;
  const int k = batch_locate(tab, kB_ir_p, blockIdx.x, bid, nb);
  ir_p_body(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb);
}

// Inner PCG in two kernels per iteration (GF_SOLVE_CG), the iterates of the
// three-kernel form in exact arithmetic.  The search direction's image
// q = A p follows the recurrence q = w + beta q with w = A z, and p.A.p =
// z.A.z - beta gamma / alpha_old (the identity of Chronopoulos and Gear, J.
// Comput. Appl. Math. 25, 1989; gamma = r.z), so the direction update joins the
// vector update.  k_ir_cg_spmv forms w = A32 z and z.w in double-float; its
// last CTA takes alpha = gamma / p.A.p.  k_ir_cg_update applies p = z + beta p,
// q = w + beta q, d += alpha p, r -= alpha q, z = P r and reduces r.z and r.r
// in double-float; its last CTA counts the iteration, stops the inner solve at
// in_rtol (or the iteration limits) and takes beta = gamma_new / gamma.  Each
// kernel keeps the three-kernel form's single dot product per row in its tail.
__device__ __forceinline__ void ir_cg_spmv_body(const DevMesh& m, const Material& mt, const StepScalars& sp, unsigned bid,
                                                unsigned nb) {
  IrState* S = m.mx.ir;
  if (S->done || S->in_done) return;
  const MixDev& x = m.mx;
  float h[1] = {0.f}, l[1] = {0.f};
  spmv32_rows(m, x.z4, x.w32, bid, nb, h[0], l[0]);   // w = A32 z, z . w (z is zero on pinned rows)
  double out[1];
  if (grid_reduce_df<1>(h, l, m.partials, m.tickets + 11, out, bid, nb) && threadIdx.x == 0) {
    const double den = S->in_iters > 0 ? out[0] - S->beta * S->rz / S->alpha : out[0];   // p.A.p
    S->pq = den;
    if (!(den > 0.0)) {
      if (!isfinite(den)) {
        S->status = GF_NAN;
        S->done = 1;
      } else if (S->in_iters == 0) {
        S->status = GF_CG_BREAKDOWN;
        S->done = 1;
      }
      S->in_done = 1;   // lost positive definiteness in FP32: hand back to the refinement
    } else {
      S->alpha = S->rz / den;
      S->alpha32 = float(S->alpha);
    }
  }
}
__global__ void __launch_bounds__(kThreads) k_ir_cg_spmv(DevMesh m, Material mt, StepScalars sp) {
  ir_cg_spmv_body(m, mt, sp, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kThreads) kb_ir_cg_spmv(const BatchTab* __restrict__ tab) {
  unsigned bid, nb;
  const int k = batch_locate(tab, kB_ir_cg_spmv, blockIdx.x, bid, nb);
  ir_cg_spmv_body(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb);
}

__device__ __forceinline__ void ir_cg_update_body(const DevMesh& m, const Material& mt, const StepScalars& sp,
                                                  unsigned bid, unsigned nb) {
  IrState* S = m.mx.ir;
  if (S->done || S->in_done) return;
  const MixDev& x = m.mx;
  const float alpha = S->alpha32, beta = S->beta32;
  const bool first = S->in_iters == 0;   // p = z, q = w
  float h[2] = {0.f, 0.f}, l[2] = {0.f, 0.f};
  for (int64_t i = bid * int64_t(blockDim.x) + threadIdx.x; i < m.N; i += int64_t(nb) * blockDim.x) {
    // every load first (the vectors may alias as far as the compiler knows, so
    // loads after a store would wait for it); p' and q' are not used on the
    // first iteration, and d, r and the inverse not on pinned rows
    const bool fixed = m.pinned[i];
    float zo[3], w[3], pq[3], qo[3], d[3], r[3], pi[9];
    {
      const float4 t = x.z4[i];
      zo[0] = t.x;
      zo[1] = t.y;
      zo[2] = t.z;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      w[c] = x.w32[3 * i + c];
      pq[c] = x.p32[3 * i + c];
      qo[c] = x.q32[3 * i + c];
      d[c] = x.d32[3 * i + c];
      r[c] = x.r32[3 * i + c];
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) pi[k] = x.pinv32[9 * i + k];
    float p[3], q[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      p[c] = first ? zo[c] : zo[c] + beta * pq[c];
      q[c] = first ? w[c] : w[c] + beta * qo[c];
      x.p32[3 * i + c] = p[c];
      x.q32[3 * i + c] = q[c];
    }
    if (fixed) continue;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      x.d32[3 * i + c] = d[c] + alpha * p[c];
      r[c] = r[c] - alpha * q[c];
      x.r32[3 * i + c] = r[c];
    }
    float zn[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      zn[c] = pi[3 * c] * r[0] + pi[3 * c + 1] * r[1] + pi[3 * c + 2] * r[2];
      df_acc_prod(h[0], l[0], r[c], zn[c]);
      df_acc_prod(h[1], l[1], r[c], r[c]);
    }
    x.z4[i] = make_float4(zn[0], zn[1], zn[2], 0.f);
  }
  double out[2];
  if (grid_reduce_df<2>(h, l, m.partials, m.tickets + 12, out, bid, nb) && threadIdx.x == 0) {
    S->in_iters += 1;
    S->total_iters += 1;
    S->beta = out[0] / S->rz;
    S->beta32 = float(S->beta);
    S->rz = out[0];
    S->in_rr = out[1];
    if (!isfinite(out[0]) || !isfinite(out[1])) {
      S->status = GF_NAN;
      S->done = 1;
      S->in_done = 1;
    } else if (!(out[1] > S->in_tol2 * S->in_rr0) || S->in_iters >= S->in_maxit || S->total_iters >= S->maxit) {
      S->in_done = 1;
    }
  }
}
__global__ void __launch_bounds__(kThreads) k_ir_cg_update(DevMesh m, Material mt, StepScalars sp) {
  ir_cg_update_body(m, mt, sp, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kThreads) kb_ir_cg_update(const BatchTab* __restrict__ tab) {
  unsigned bid, nb;
  const int k = batch_locate(tab, kB_ir_cg_update, blockIdx.x, bid, nb);
  ir_cg_update_body(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb);
}

// dv += d on free rows once the inner solve has finished, kept as a float pair
// (dv_hi + dv_lo) on the FP32 pipe.  Writes no flag: every CTA decides from the
// same state (the residual that follows marks the correction as applied).
__device__ __forceinline__ void ir_apply_body(const DevMesh& m, const Material& mt, const StepScalars& sp, unsigned bid, unsigned nb) {

  IrState* S = m.mx.ir;
  if (S->done || !S->in_done || S->applied) return;
  for (int64_t i = bid * int64_t(blockDim.x) + threadIdx.x; i < 3 * m.N; i += int64_t(nb) * blockDim.x) {
    if (m.pinned[i / 3]) continue;
    float hi = m.mx.dv_hi[i], lo = m.mx.dv_lo[i];
    df_add(hi, lo, m.mx.d32[i], 0.f);
    m.mx.dv_hi[i] = hi;
    m.mx.dv_lo[i] = lo;
  }
}
__global__ void __launch_bounds__(kThreads) k_ir_apply(DevMesh m, Material mt, StepScalars sp) {
  ir_apply_body(m, mt, sp, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kThreads) kb_ir_apply(const BatchTab* __restrict__ tab) {
  unsigned bid, nb;
  const int k = batch_locate(tab, kB_ir_apply, blockIdx.x, bid, nb);
  ir_apply_body(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb);
}

// v += dv (dv = dv_hi + dv_lo), x += dt v; refresh the FP32 copies of u = x - X and v
__device__ __forceinline__ void integrate32_body(const DevMesh& m, const Material& mt, const StepScalars& sp, unsigned bid, unsigned nb) {
  const double dt = sp.dt;

  const int64_t i = bid * int64_t(blockDim.x) + threadIdx.x;
  if (i >= 3 * m.N) return;
  const double dv = double(m.mx.dv_hi[i]) + double(m.mx.dv_lo[i]);
  m.dv[i] = dv;
  const double v = m.v[i] + dv;
  m.v[i] = v;
  const double xn = m.x[i] + dt * v;
  m.x[i] = xn;
  m.mx.u32[i] = float(xn - m.mx.X[i]);
  m.mx.v32[i] = float(v);
}
__global__ void __launch_bounds__(kThreads) k_integrate32(DevMesh m, Material mt, StepScalars sp) {
  integrate32_body(m, mt, sp, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kThreads) kb_integrate32(const BatchTab* __restrict__ tab) {
  unsigned bid, nb;
  const int k = batch_locate(tab, kB_integrate32, blockIdx.x, bid, nb);
  integrate32_body(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb);
}

// FP32 copies after a state change; also the float-pair split of dv
__device__ __forceinline__ void refresh32_body(const DevMesh& m, const Material& mt, const StepScalars& sp, unsigned bid, unsigned nb) {

  const int64_t i = bid * int64_t(blockDim.x) + threadIdx.x;
  if (i >= 3 * m.N) return;
  m.mx.u32[i] = float(m.x[i] - m.mx.X[i]);
  m.mx.v32[i] = float(m.v[i]);
  const double d = m.dv[i];
  const float hi = float(d);
  m.mx.dv_hi[i] = hi;
  m.mx.dv_lo[i] = float(d - double(hi));
}
__global__ void __launch_bounds__(kThreads) k_refresh32(DevMesh m, Material mt, StepScalars sp) {
  refresh32_body(m, mt, sp, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kThreads) kb_refresh32(const BatchTab* __restrict__ tab) {
  unsigned bid, nb;
  const int k = batch_locate(tab, kB_refresh32, blockIdx.x, bid, nb);
  refresh32_body(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb);
}

__device__ __forceinline__ void chi_to32_body(const DevMesh& m, const Material& mt, const StepScalars& sp, unsigned bid, unsigned nb) {

  const int64_t t = bid * int64_t(blockDim.x) + threadIdx.x;
  if (t < m.T) m.mx.chi32[t] = float(m.chi[t]);
}
__global__ void k_chi_to32(DevMesh m, Material mt, StepScalars sp) {
  chi_to32_body(m, mt, sp, blockIdx.x, gridDim.x);
}
__global__ void kb_chi_to32(const BatchTab* __restrict__ tab) {
  unsigned bid, nb;
  const int k = batch_locate(tab, kB_chi_to32, blockIdx.x, bid, nb);
  chi_to32_body(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb);
}

// Distributed solver-loop kernels of a batch: a fixed grid whose CTAs take the
// blocks listed in the work table in turn (the same bodies, the same per-mesh
// block index and count as the per-kind launches).
#define GF_DIST_KERNEL(name, bounds, kind, body)                                                       \
  __global__ void __launch_bounds__ bounds name(const BatchTab* __restrict__ tab, const BatchAct* __restrict__ act) { \
    const int total = act->off[kind][act->n];                                                          \
    for (int w = blockIdx.x; w < total; w += gridDim.x) {                                              \
      unsigned bid, nb;                                                                                \
      const int k = act_locate(act, kind, unsigned(w), bid, nb);                                       \
      body;                                                                                            \
      __syncthreads();                                                                                 \
    }                                                                                                  \
  }
GF_DIST_KERNEL(kd_ir_residual, (kThreads, 5), kB_ir_residual,
               ir_residual_body(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb, 0))
GF_DIST_KERNEL(kd_ir_inner_init, (kThreads), kB_ir_inner_init,
               ir_inner_init_body(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb))
GF_DIST_KERNEL(kd_ir_spmv, (kThreads), kB_ir_spmv, ir_spmv_body(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb))
GF_DIST_KERNEL(kd_ir_update, (kThreads), kB_ir_update, ir_update_body(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb))
GF_DIST_KERNEL(kd_ir_p, (kThreads), kB_ir_p, ir_p_body(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb))
GF_DIST_KERNEL(kd_ir_apply, (kThreads), kB_ir_apply, ir_apply_body(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb))
#undef GF_DIST_KERNEL

}  // namespace

int launch_dist_mixed(int kind, const BatchTab* tab, const BatchAct* act, unsigned grid, cudaStream_t s) {
  switch (kind) {
    case kB_ir_residual: kd_ir_residual<<<grid, kThreads, 0, s>>>(tab, act); break;
    case kB_ir_inner_init: kd_ir_inner_init<<<grid, kThreads, 0, s>>>(tab, act); break;
    case kB_ir_spmv: kd_ir_spmv<<<grid, kThreads, 0, s>>>(tab, act); break;
    case kB_ir_update: kd_ir_update<<<grid, kThreads, 0, s>>>(tab, act); break;
    case kB_ir_p: kd_ir_p<<<grid, kThreads, 0, s>>>(tab, act); break;
    case kB_ir_apply: kd_ir_apply<<<grid, kThreads, 0, s>>>(tab, act); break;
    default: return 0;
  }
  return 1;
}

// the element kernels stage 53.8 KB of rows in shared memory, a single-mesh
// Eq. 20 launch up to 216 KB of union rows: raise the limits once per device
void elem32_smem_attr() {
  static bool done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64 || done[dev]) return;
  cudaFuncSetAttribute(k_elem32, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kElemSmem));
  cudaFuncSetAttribute(kb_elem32, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kElemSmem));
  cudaFuncSetAttribute(k_nonlocal32, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kNlSmemMax));
  done[dev] = true;
}

int launch_kind_mixed(int kind, const DevMesh& m, const Material& mt, const StepScalars& sp, cudaStream_t s, int first) {
  const LaunchDims d = launch_dims(kind, m, mt, sp);
  if (d.blocks == 0) return 0;
  switch (kind) {
    case kB_tet_stress32: k_tet_stress32<<<d.blocks, d.threads, 0, s>>>(m, mt, sp); break;
    case kB_nonlocal32:   // stages nl_cap rows of 24 B
      elem32_smem_attr();
      k_nonlocal32<<<d.blocks, d.threads, unsigned(m.mx.nl_cap) * 24u, s>>>(m, mt, sp);
      break;
    case kB_edge_driver32: k_edge_driver32<<<d.blocks, d.threads, 0, s>>>(m, mt, sp); break;
    case kB_tet_chi32: k_tet_chi32<<<d.blocks, d.threads, 0, s>>>(m, mt, sp); break;
    case kB_elem32:
      elem32_smem_attr();
      k_elem32<<<d.blocks, d.threads, kElemSmem, s>>>(m, mt, sp);
      break;
    case kB_gather32: k_gather32<<<d.blocks, d.threads, 0, s>>>(m, mt, sp); break;
    case kB_diag32: k_diag32<<<d.blocks, d.threads, 0, s>>>(m, mt, sp); break;
    case kB_ir_residual: k_ir_residual<<<d.blocks, d.threads, 0, s>>>(m, mt, sp, first); break;
    case kB_ir_inner_init: k_ir_inner_init<<<d.blocks, d.threads, 0, s>>>(m, mt, sp); break;
    case kB_ir_spmv: k_ir_spmv<<<d.blocks, d.threads, 0, s>>>(m, mt, sp); break;
    case kB_ir_update: k_ir_update<<<d.blocks, d.threads, 0, s>>>(m, mt, sp); break;
    case kB_ir_p: k_ir_p<<<d.blocks, d.threads, 0, s>>>(m, mt, sp); break;
    case kB_ir_apply: k_ir_apply<<<d.blocks, d.threads, 0, s>>>(m, mt, sp); break;
    case kB_ir_cg_spmv: k_ir_cg_spmv<<<d.blocks, d.threads, 0, s>>>(m, mt, sp); break;
    case kB_ir_cg_update: k_ir_cg_update<<<d.blocks, d.threads, 0, s>>>(m, mt, sp); break;
    case kB_integrate32: k_integrate32<<<d.blocks, d.threads, 0, s>>>(m, mt, sp); break;
    case kB_refresh32: k_refresh32<<<d.blocks, d.threads, 0, s>>>(m, mt, sp); break;
    case kB_chi_to32: k_chi_to32<<<d.blocks, d.threads, 0, s>>>(m, mt, sp); break;
    default: return -1;
  }
  return 1;
}

int launch_batch_mixed(int kind, const BatchTab* tab, unsigned blocks, unsigned threads, cudaStream_t s, int first) {
  if (blocks == 0) return 0;
  switch (kind) {
    case kB_tet_stress32: kb_tet_stress32<<<blocks, threads, 0, s>>>(tab); break;
    case kB_nonlocal32: kb_nonlocal32<<<blocks, threads, kNlSmem, s>>>(tab); break;
    case kB_edge_driver32: kb_edge_driver32<<<blocks, threads, 0, s>>>(tab); break;
    case kB_tet_chi32: kb_tet_chi32<<<blocks, threads, 0, s>>>(tab); break;
    case kB_elem32:
      elem32_smem_attr();
      kb_elem32<<<blocks, threads, kElemSmem, s>>>(tab);
      break;
    case kB_gather32: kb_gather32<<<blocks, threads, 0, s>>>(tab); break;
    case kB_diag32: kb_diag32<<<blocks, threads, 0, s>>>(tab); break;
    case kB_ir_residual: kb_ir_residual<<<blocks, threads, 0, s>>>(tab, first); break;
    case kB_ir_inner_init: kb_ir_inner_init<<<blocks, threads, 0, s>>>(tab); break;
    case kB_ir_spmv: kb_ir_spmv<<<blocks, threads, 0, s>>>(tab); break;
    case kB_ir_update: kb_ir_update<<<blocks, threads, 0, s>>>(tab); break;
    case kB_ir_p: kb_ir_p<<<blocks, threads, 0, s>>>(tab); break;
    case kB_ir_apply: kb_ir_apply<<<blocks, threads, 0, s>>>(tab); break;
    case kB_ir_cg_spmv: kb_ir_cg_spmv<<<blocks, threads, 0, s>>>(tab); break;
    case kB_ir_cg_update: kb_ir_cg_update<<<blocks, threads, 0, s>>>(tab); break;
    case kB_integrate32: kb_integrate32<<<blocks, threads, 0, s>>>(tab); break;
    case kB_refresh32: kb_refresh32<<<blocks, threads, 0, s>>>(tab); break;
    case kB_chi_to32: kb_chi_to32<<<blocks, threads, 0, s>>>(tab); break;
    default: return -1;
  }
  return 1;
}

}  // namespace gf
