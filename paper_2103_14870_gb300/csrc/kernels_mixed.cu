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

__global__ void __launch_bounds__(kThreads) k_tet_stress32(DevMesh m, float lam, float mu, float kappa, int avg) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= m.T) return;
  const MixDev& x = m.mx;
  const int4 n = m.tets[t];
  const int nid[4] = {n.x, n.y, n.z, n.w};
  float du[4][3];
#pragma unroll
  for (int a = 0; a < 4; ++a) ld3f(x.u32, nid[a], du[a]);
  float A[32];
  load_restA(x.restA, t, A);
  float E0[6][3], e[6][3], ds[6];
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
  const float S[6] = {tr + 2.f * mu * Eg[0], tr + 2.f * mu * Eg[1], tr + 2.f * mu * Eg[2],
                      2.f * mu * Eg[3], 2.f * mu * Eg[4], 2.f * mu * Eg[5]};
  const float w = avg ? x.chi32[t] : 1.f;
  float4* si = reinterpret_cast<float4*>(x.sig_in32 + 8 * t);
  si[0] = make_float4(w * S[0], w * S[1], w * S[2], w * S[3]);
  si[1] = make_float4(w * S[4], w * S[5], 0.f, 0.f);
  float* sf = x.sigf32 + 6 * t;
#pragma unroll
  for (int k = 0; k < 6; ++k)
    sf[k] = normal_stress32(e[k], e[k][0] * e[k][0] + e[k][1] * e[k][1] + e[k][2] * e[k][2], S, kappa);
}

// Eq. 20 sum in FP32: one warp per tet over its CSR neighbour list (coalesced
// index and weight loads; the gathered 32-byte stress rows of a tet's
// neighbours come from short runs of consecutive tets), then a fixed-order
// warp reduction (deterministic).
__global__ void __launch_bounds__(kThreads) k_nonlocal32(DevMesh m) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t t = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; t < m.T; t += nw) {
    const int64_t beg = m.mx.nb_ptr[t], end = m.mx.nb_ptr[t + 1];
    float acc[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t p = beg + lane; p < end; p += 32) {
      const int j = __ldg(m.mx.nb_csr + p);
      const float w = __ldg(m.mx.nb_wc + p);
      float sj[8];
      ld8f(m.mx.sig_in32 + 8 * int64_t(j), sj);
#pragma unroll
      for (int q = 0; q < 6; ++q) acc[q] += w * sj[q];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int q = 0; q < 6; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
    if (lane == 0) {
      float4* o = reinterpret_cast<float4*>(m.mx.sig_bar32 + 8 * t);
      o[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
      o[1] = make_float4(acc[4], acc[5], 0.f, 0.f);
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_edge_driver32(DevMesh m, float kappa, float inv_young, int stress_mode,
                                                            double threshold) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  unsigned long long nb = 0, nn = 0;
  if (i < m.NE) {
    const int2 ab = m.edges[i];
    float ua[3], ub[3], e0[3];
    ld3f(m.mx.u32, ab.x, ua);
    ld3f(m.mx.u32, ab.y, ub);
    ld3f(m.mx.edge_e0, i, e0);
    const float e[3] = {e0[0] + (ub[0] - ua[0]), e0[1] + (ub[1] - ua[1]), e0[2] + (ub[2] - ua[2])};
    const float s = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
    float mx = -INFINITY;
    for (int p = m.et_ptr[i]; p < m.et_ptr[i + 1]; ++p) {
      float S[8];
      ld8f(m.mx.sig_bar32 + 8 * int64_t(m.et_tet[p]), S);
      mx = fmaxf(mx, normal_stress32(e, s, S, kappa));
    }
    const double d = double(stress_mode ? mx : mx * inv_young);
    m.driver[i] = d;
    const uint8_t old = m.labels[i];
    const uint8_t now = (old || d >= threshold) ? 1 : 0;   // threshold test in FP64
    if (now != old) m.labels[i] = now;
    nb = now;
    nn = now && !old;
  }
  warp_count(nb, m.counters + kCntBroken);
  warp_count(nn, m.counters + kCntNewBroken);
}

__global__ void __launch_bounds__(kThreads) k_tet_chi32(DevMesh m, float young, uint64_t lut) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
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
        float num = 0.f, den = 0.f;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          const float a = fabsf(m.mx.sigf32[6 * t + k]);
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

// ---------------------------------------------------------------------------
// Two-phase assembly, no colours and no atomics.
// Phase 1 (k_elem32, one thread per tet): the tet's ten upper-triangle 3x3
// blocks (a <= b) of (dt beta + dt^2) chi k_e and its four nodal rhs shares
// dt chi (f_a - (beta + dt) (k_e v)_a), written to a per-tet row of kElemW floats.
// Phase 2 (k_gather32, one warp per node row): lane p sums the contributions of
// block slot p in a fixed, precomputed order (transposing lower blocks), adds
// the lumped mass, and lane 0 inverts the diagonal block (block Jacobi); lanes
// 0..2 sum the node's rhs shares and add the external and damping terms.
// ---------------------------------------------------------------------------

constexpr int kElemW = 104;   // 90 block floats + 12 rhs floats + 2 pad (16-byte rows)

__global__ void __launch_bounds__(128) k_elem32(DevMesh m, float sKv, float cv, float dtf) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= m.T) return;
  const MixDev& x = m.mx;
  float4* out = reinterpret_cast<float4*>(x.ebuf + kElemW * t);
  const float chi = x.chi32[t];
  if (chi == 0.f) {
#pragma unroll
    for (int q = 0; q < kElemW / 4; ++q) out[q] = make_float4(0.f, 0.f, 0.f, 0.f);
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
  // Y_b[k][c] = sum_{l in b} H_kl sgn_lb e_l[c]  (sgn = -1 if b is the first node of l)
  float o[kElemW];
  float Kv[4][3] = {};
#pragma unroll
  for (int b = 0; b < 4; ++b) {
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
    for (int a = 0; a <= b; ++a) {
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
      const int q = blk_q(a, b);
      const float sk = sKv * chi;
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) o[9 * q + 3 * r + c] = sk * blk[r][c];
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
      o[90 + 3 * a + r] = dtf * chi * (f - cv * Kv[a][r]);
    }
  o[102] = 0.f;
  o[103] = 0.f;
#pragma unroll
  for (int q = 0; q < kElemW / 4; ++q) out[q] = make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
}

__global__ void __launch_bounds__(256) k_gather32(DevMesh m, float dtf, float alphaf, float cmf) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  if (i >= m.N) return;                               // whole warp leaves together
  __shared__ float dg[8][9];
  const int wib = threadIdx.x >> 5;
  const MixDev& x = m.mx;
  const int rb = m.row_ptr[i], rl = m.row_ptr[i + 1] - rb;
  const int dslot = m.diag_blk[i];
  const float mi = x.mass32[i];
  // lane o takes entry (r, c) = o % 9 of block slot rb + o / 9: the lanes of one
  // pass read 3-4 whole element blocks per request
  for (int o = lane; o < 9 * rl; o += 32) {
    const int p = o / 9, e = o - 9 * p;
    const int slot = rb + p;
    const int et = 3 * (e % 3) + e / 3;          // entry of the transposed block
    float acc = 0.f;
    for (int c = m.sc_ptr[slot]; c < m.sc_ptr[slot + 1]; ++c) {
      const int ent = m.sc_ent[c];
      acc += x.ebuf[kElemW * int64_t(ent >> 5) + 9 * (ent & 15) + ((ent & 16) ? et : e)];
    }
    if (slot == dslot) {
      if (e == 0 || e == 4 || e == 8) acc += cmf * mi;
      dg[wib][e] = acc;
    }
    x.val32[9 * int64_t(slot) + e] = acc;
  }
  if (lane < 3) {
    float acc = 0.f;
    for (int k = m.np_ptr[i]; k < m.np_ptr[i + 1]; ++k) {
      const int pr = m.np_pair[k];
      acc += x.ebuf[kElemW * int64_t(pr >> 2) + 90 + 3 * (pr & 3) + lane];
    }
    const float fe = x.fext32 ? x.fext32[3 * i + lane] : 0.f;
    x.rhs32[3 * i + lane] = acc + dtf * (fe - alphaf * mi * x.v32[3 * i + lane]);
  }
  __syncwarp();
  if (lane == 0) {
    const float* d = dg[wib];
    const float c00 = d[4] * d[8] - d[5] * d[7], c01 = d[2] * d[7] - d[1] * d[8], c02 = d[1] * d[5] - d[2] * d[4];
    const float c10 = d[5] * d[6] - d[3] * d[8], c11 = d[0] * d[8] - d[2] * d[6], c12 = d[2] * d[3] - d[0] * d[5];
    const float c20 = d[3] * d[7] - d[4] * d[6], c21 = d[1] * d[6] - d[0] * d[7], c22 = d[0] * d[4] - d[1] * d[3];
    const float id = 1.f / (d[0] * c00 + d[1] * c10 + d[2] * c20);
    float* pi = x.pinv32 + 9 * i;
    pi[0] = c00 * id; pi[1] = c01 * id; pi[2] = c02 * id;
    pi[3] = c10 * id; pi[4] = c11 * id; pi[5] = c12 * id;
    pi[6] = c20 * id; pi[7] = c21 * id; pi[8] = c22 * id;
  }
}

// f_ext in FP32 for the gather (one conversion per entry)
__global__ void __launch_bounds__(kThreads) k_fext32(DevMesh m, const double* f) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i < 3 * m.N) m.mx.fext32[i] = float(f[i]);
}

// ---------------------------------------------------------------------------
// FP64 iterative refinement around an FP32 PCG
// ---------------------------------------------------------------------------

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
                                               double (&out)[NV]) {
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
      if (lane == 0) part[blockIdx.x * NV + i] = make_float2(h, l);
    }
  }
  if (threadIdx.x == 0) {
    __threadfence();
    last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    float h = 0.f, l = 0.f;
    for (unsigned j = threadIdx.x; j < gridDim.x; j += blockDim.x) {
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

// r = b - A32 dv on free rows, with A32 dv formed in double-float (dv = dv_hi +
// dv_lo) and b - A dv in double-float; half a warp per block row (lane j takes
// blocks j, j+16, ...), then a 16-lane double-float reduction.  The inner
// solve's right-hand side is the leading float of r; ||r||^2 accumulates in
// double-float.
__global__ void __launch_bounds__(kThreads) k_ir_residual(DevMesh m, int first) {
  IrState* S = m.mx.ir;
  if (!first && (S->done || !S->applied)) return;   // no new correction yet: nothing to check
  const MixDev& x = m.mx;
  const int j16 = threadIdx.x & 15;
  const unsigned hmask = (threadIdx.x & 16) ? 0xffff0000u : 0x0000ffffu;
  float nh_[1] = {0.f}, nl_[1] = {0.f};
  const int64_t nh = (int64_t(gridDim.x) * blockDim.x) >> 4;
  for (int64_t i = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 4; i < m.N; i += nh) {
    float hi[3] = {0, 0, 0}, lo[3] = {0, 0, 0};
    const bool fixed = m.pinned[i];
    if (!fixed) {
      for (int b = m.row_ptr[i] + j16; b < m.row_ptr[i + 1]; b += 16) {
        const int64_t j = m.col[b];
        const float* a = x.val32 + 9 * int64_t(b);
        float xh[3], xl[3];
        ld3f(x.dv_hi, j, xh);
        ld3f(x.dv_lo, j, xl);
#pragma unroll
        for (int rr = 0; rr < 3; ++rr)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            float p, pe;
            two_prod(a[3 * rr + c], xh[c], p, pe);
            pe = fmaf(a[3 * rr + c], xl[c], pe);
            df_add(hi[rr], lo[rr], p, pe);
          }
      }
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1)
#pragma unroll
      for (int rr = 0; rr < 3; ++rr) {
        const float oh = __shfl_xor_sync(hmask, hi[rr], o);
        const float ol = __shfl_xor_sync(hmask, lo[rr], o);
        df_add(hi[rr], lo[rr], oh, ol);
      }
    if (j16 == 0) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float rh = 0.f, rl = 0.f;
        if (!fixed) {
          rh = x.rhs32[3 * i + c];
          df_add(rh, rl, -hi[c], -lo[c]);
        }
        x.rres[3 * i + c] = rh;
        df_acc_prod(nh_[0], nl_[0], rh, rh);
        df_add(nh_[0], nl_[0], 2.f * rh * rl, 0.f);
      }
    }
  }
  double out[1];
  if (grid_reduce_df<1>(nh_, nl_, m.partials, m.tickets + 4, out) && threadIdx.x == 0) {
    if (first) {
      S->bb = out[0];
      S->sweeps = 0;
      S->total_iters = 0;
      S->status = GF_OK;
    } else {
      S->sweeps += 1;
    }
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

// inner PCG start (only after a fresh residual; otherwise the current inner
// solve continues): r32 = r, z = P r, p = z, d = 0
__global__ void __launch_bounds__(kThreads) k_ir_inner_init(DevMesh m) {
  IrState* S = m.mx.ir;
  if (S->done || !S->applied) return;
  const MixDev& x = m.mx;
  float h[1] = {0.f}, l[1] = {0.f};
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < m.N; i += int64_t(gridDim.x) * blockDim.x) {
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
  }
  double out[1];
  if (grid_reduce_df<1>(h, l, m.partials, m.tickets + 5, out) && threadIdx.x == 0) {
    S->rz = out[0];
    S->in_rr0 = S->rr;
    S->in_iters = 0;
    S->in_done = (out[0] == 0.0) ? 1 : 0;
    S->applied = 0;
  }
}

// q = A32 p with half a warp per block row (coalesced block loads), p . q in double-float
__global__ void __launch_bounds__(kThreads) k_ir_spmv(DevMesh m) {
  IrState* S = m.mx.ir;
  if (S->done || S->in_done) return;
  const MixDev& x = m.mx;
  const int j16 = threadIdx.x & 15;
  const unsigned hmask = (threadIdx.x & 16) ? 0xffff0000u : 0x0000ffffu;
  float h[1] = {0.f}, l[1] = {0.f};
  const int64_t nh = (int64_t(gridDim.x) * blockDim.x) >> 4;
  for (int64_t i = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 4; i < m.N; i += nh) {
    float y0 = 0.f, y1 = 0.f, y2 = 0.f;
    for (int b = m.row_ptr[i] + j16; b < m.row_ptr[i + 1]; b += 16) {
      const int64_t j = m.col[b];
      const float* a = x.val32 + 9 * int64_t(b);
      const float p0 = x.p32[3 * j], p1 = x.p32[3 * j + 1], p2 = x.p32[3 * j + 2];
      y0 += a[0] * p0 + a[1] * p1 + a[2] * p2;
      y1 += a[3] * p0 + a[4] * p1 + a[5] * p2;
      y2 += a[6] * p0 + a[7] * p1 + a[8] * p2;
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
      y0 += __shfl_xor_sync(hmask, y0, o);
      y1 += __shfl_xor_sync(hmask, y1, o);
      y2 += __shfl_xor_sync(hmask, y2, o);
    }
    if (j16 == 0) {
      const float y[3] = {y0, y1, y2};
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        x.q32[3 * i + c] = y[c];
        df_acc_prod(h[0], l[0], x.p32[3 * i + c], y[c]);
      }
    }
  }
  double out[1];
  if (grid_reduce_df<1>(h, l, m.partials, m.tickets + 6, out) && threadIdx.x == 0) {
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

__global__ void __launch_bounds__(kThreads) k_ir_update(DevMesh m) {
  IrState* S = m.mx.ir;
  if (S->done || S->in_done) return;
  const MixDev& x = m.mx;
  const float alpha = S->alpha32;
  float h[2] = {0.f, 0.f}, l[2] = {0.f, 0.f};
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < m.N; i += int64_t(gridDim.x) * blockDim.x) {
    if (m.pinned[i]) continue;
    float r[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      x.d32[3 * i + c] += alpha * x.p32[3 * i + c];
      r[c] = x.r32[3 * i + c] - alpha * x.q32[3 * i + c];
      x.r32[3 * i + c] = r[c];
    }
    const float* pi = x.pinv32 + 9 * i;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float z = pi[3 * c] * r[0] + pi[3 * c + 1] * r[1] + pi[3 * c + 2] * r[2];
      x.z32[3 * i + c] = z;
      df_acc_prod(h[0], l[0], r[c], z);
      df_acc_prod(h[1], l[1], r[c], r[c]);
    }
  }
  double out[2];
  if (grid_reduce_df<2>(h, l, m.partials, m.tickets + 7, out) && threadIdx.x == 0) {
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

__global__ void __launch_bounds__(kThreads) k_ir_p(DevMesh m) {
  IrState* S = m.mx.ir;
  if (S->done || S->in_done) return;
  const float beta = S->beta32;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < 3 * m.N; i += int64_t(gridDim.x) * blockDim.x)
    m.mx.p32[i] = m.mx.z32[i] + beta * m.mx.p32[i];
}

// dv += d on free rows, kept as a float pair (dv_hi + dv_lo) on the FP32 pipe
__global__ void __launch_bounds__(kThreads) k_ir_apply(DevMesh m) {
  IrState* S = m.mx.ir;
  if (S->done || !S->in_done || S->applied) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) S->applied = 1;   // read by the next kernels only
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < 3 * m.N; i += int64_t(gridDim.x) * blockDim.x) {
    if (m.pinned[i / 3]) continue;
    float hi = m.mx.dv_hi[i], lo = m.mx.dv_lo[i];
    df_add(hi, lo, m.mx.d32[i], 0.f);
    m.mx.dv_hi[i] = hi;
    m.mx.dv_lo[i] = lo;
  }
}

// v += dv (dv = dv_hi + dv_lo), x += dt v; refresh the FP32 copies of u = x - X and v
__global__ void __launch_bounds__(kThreads) k_integrate32(DevMesh m, double dt) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
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

// FP32 copies after a state change; also the float-pair split of dv
__global__ void __launch_bounds__(kThreads) k_refresh32(DevMesh m) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= 3 * m.N) return;
  m.mx.u32[i] = float(m.x[i] - m.mx.X[i]);
  m.mx.v32[i] = float(m.v[i]);
  const double d = m.dv[i];
  const float hi = float(d);
  m.mx.dv_hi[i] = hi;
  m.mx.dv_lo[i] = float(d - double(hi));
}

__global__ void k_chi_to32(DevMesh m) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t < m.T) m.mx.chi32[t] = float(m.chi[t]);
}

inline unsigned blocks_for(int64_t n, int threads) { return unsigned((n + threads - 1) / threads); }
// reducing kernels of the refinement: at most 4 CTAs per SM (grid-stride loops),
// so the final double-float pass over the partials stays short
inline unsigned ir_grid(int64_t n) {
  int64_t b = (n + kThreads - 1) / kThreads;
  return unsigned(b < 1 ? 1 : (b > 4 * 152 ? 4 * 152 : b));
}
inline unsigned reduce_grid(int64_t n) {
  int64_t b = (n + kThreads - 1) / kThreads;
  return unsigned(b < 1 ? 1 : (b > kMaxPartials ? kMaxPartials : b));
}

}  // namespace

int launch_tet_stress32(const DevMesh& m, const Material& mt, cudaStream_t s) {
  k_tet_stress32<<<blocks_for(m.T, kThreads), kThreads, 0, s>>>(m, float(mt.lam), float(mt.mu), float(mt.kappa),
                                                               mt.average_degraded);
  return 1;
}
int launch_nonlocal32(const DevMesh& m, cudaStream_t s) {
  k_nonlocal32<<<blocks_for(32 * m.T, kThreads), kThreads, 0, s>>>(m);
  return 1;
}
int launch_edge_driver32(const DevMesh& m, const Material& mt, cudaStream_t s) {
  k_edge_driver32<<<blocks_for(m.NE, kThreads), kThreads, 0, s>>>(m, float(mt.kappa), float(1.0 / mt.young),
                                                                 mt.driver_stress, mt.threshold);
  return 1;
}
int launch_tet_chi32(const DevMesh& m, const Material& mt, uint64_t lut, cudaStream_t s) {
  k_tet_chi32<<<blocks_for(m.T, kThreads), kThreads, 0, s>>>(m, float(mt.young), lut);
  return 1;
}
int launch_assemble32(const DevMesh& m, const Material& mt, double dt, const double* f_ext, cudaStream_t s) {
  int n = 0;
  k_elem32<<<blocks_for(m.T, 128), 128, 0, s>>>(m, float(dt * mt.beta + dt * dt), float(mt.beta + dt), float(dt));
  ++n;
  DevMesh v = m;
  if (f_ext) {
    k_fext32<<<blocks_for(3 * m.N, kThreads), kThreads, 0, s>>>(m, f_ext);
    ++n;
  } else {
    v.mx.fext32 = nullptr;
  }
  k_gather32<<<blocks_for(32 * m.N, 256), 256, 0, s>>>(v, float(dt), float(mt.alpha), float(1.0 + dt * mt.alpha));
  return n + 1;
}
int launch_ir_residual(const DevMesh& m, int first, cudaStream_t s) {
  k_ir_residual<<<ir_grid(16 * m.N), kThreads, 0, s>>>(m, first);
  return 1;
}
int launch_ir_inner_init(const DevMesh& m, cudaStream_t s) {
  k_ir_inner_init<<<ir_grid(m.N), kThreads, 0, s>>>(m);
  return 1;
}
int launch_ir_inner_iter(const DevMesh& m, cudaStream_t s, int which) {
  if (which == 0) k_ir_spmv<<<ir_grid(16 * m.N), kThreads, 0, s>>>(m);
  else if (which == 1) k_ir_update<<<ir_grid(m.N), kThreads, 0, s>>>(m);
  else k_ir_p<<<ir_grid(3 * m.N), kThreads, 0, s>>>(m);
  return 1;
}
int launch_ir_apply(const DevMesh& m, cudaStream_t s) {
  k_ir_apply<<<ir_grid(3 * m.N), kThreads, 0, s>>>(m);
  return 1;
}
int launch_integrate32(const DevMesh& m, double dt, cudaStream_t s) {
  k_integrate32<<<blocks_for(3 * m.N, kThreads), kThreads, 0, s>>>(m, dt);
  return 1;
}
int launch_chi_to32(const DevMesh& m, cudaStream_t s) {
  k_chi_to32<<<blocks_for(m.T, kThreads), kThreads, 0, s>>>(m);
  return 1;
}
int launch_refresh32(const DevMesh& m, cudaStream_t s) {
  k_refresh32<<<blocks_for(3 * m.N, kThreads), kThreads, 0, s>>>(m);
  return 1;
}

}  // namespace gf
