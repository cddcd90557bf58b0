// Learned warm start and block preconditioner: a 3-layer message-passing
// network over the mesh graph (hidden width 64), bfloat16 weights, FP32
// activations and accumulation.  Feature construction, forward, backward and
// Adam; every sum is taken in a fixed order, so results are deterministic.
//
//   node inputs f_i: log(t_i / mean t), A_ii / t_i - I (xx yy zz xy xz yz),
//                    log(m_i / mean m), pinned, degree / 16, y_i / s, 0 0 0
//   edge inputs e_ij (message j -> i): (X_j - X_i) / mean edge length,
//                    A_ij / sqrt(t_i t_j) (row-major), 0 0 0 0
//   h = relu(W0 f + b0);  per layer: a = Wa h,  M_i = mean_j relu(a_j + We e_ij + bm),
//   h += relu(Wu [h; M] + bu);  out = Wd h + bd = (delta (3), ell (6))
//   P_i = C_i (L_i L_i^T + eps I) C_i^T with C_i C_i^T = A_ii^-1,  x0_i = P_i b_i + s delta_i
// where t_i = trace(A_ii) / 3, y_i = A_ii^-1 b_i (0 on pinned nodes), s = rms |y_i|.
#include <cuda_bf16.h>

#include <cmath>

#include "gf_gnn.h"
#include "gf_reduce.cuh"

namespace gf {
namespace {

constexpr int kT = 256;
constexpr int kMaxParts = 1216;   // 8 CTAs per SM
__device__ __forceinline__ float bf(const __nv_bfloat16 v) { return __bfloat162float(v); }

__device__ __forceinline__ void load_diag(const DevMesh& m, int64_t i, float (&d)[9]) {
  const double* a = m.val + 9 * int64_t(m.diag_blk[i]);
#pragma unroll
  for (int k = 0; k < 9; ++k) d[k] = float(a[k]);
}

// D^-1 (symmetrised), its lower Cholesky factor and t = trace(D) / 3
__device__ __forceinline__ void diag_factors(const float (&d)[9], float (&inv)[6], float (&C)[6]) {
  const float c00 = d[4] * d[8] - d[5] * d[7], c01 = d[2] * d[7] - d[1] * d[8], c02 = d[1] * d[5] - d[2] * d[4];
  const float c10 = d[5] * d[6] - d[3] * d[8], c11 = d[0] * d[8] - d[2] * d[6], c12 = d[2] * d[3] - d[0] * d[5];
  const float c20 = d[3] * d[7] - d[4] * d[6], c21 = d[1] * d[6] - d[0] * d[7], c22 = d[0] * d[4] - d[1] * d[3];
  const float id = 1.f / (d[0] * c00 + d[1] * c10 + d[2] * c20);
  inv[0] = c00 * id;                      // xx
  inv[1] = c11 * id;                      // yy
  inv[2] = c22 * id;                      // zz
  inv[3] = 0.5f * (c01 + c10) * id;       // xy
  inv[4] = 0.5f * (c02 + c20) * id;       // xz
  inv[5] = 0.5f * (c12 + c21) * id;       // yz
  const float l00 = sqrtf(inv[0]);
  const float l10 = inv[3] / l00, l20 = inv[4] / l00;
  const float l11 = sqrtf(fmaxf(inv[1] - l10 * l10, 1e-30f));
  const float l21 = (inv[5] - l20 * l10) / l11;
  const float l22 = sqrtf(fmaxf(inv[2] - l20 * l20 - l21 * l21, 1e-30f));
  C[0] = l00; C[1] = l10; C[2] = l11; C[3] = l20; C[4] = l21; C[5] = l22;
}

// per node: t, C, y, b; totals sum t, sum |y|^2 and the free count -> s, mean t
__global__ void __launch_bounds__(kT) k_gnn_prep(GnnDev g, DevMesh m, const double* b) {
  double acc[3] = {0.0, 0.0, 0.0};
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < g.N; i += int64_t(gridDim.x) * blockDim.x) {
    float d[9], inv[6], C[6];
    load_diag(m, i, d);
    diag_factors(d, inv, C);
    const float t = (d[0] + d[4] + d[8]) * (1.f / 3.f);
    g.T[i] = t;
#pragma unroll
    for (int k = 0; k < 6; ++k) g.C[6 * i + k] = C[k];
    const bool fr = !m.pinned[i];
    g.freem[i] = fr ? 1 : 0;
    float bb[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) bb[c] = float(b[3 * i + c]);
    float y[3] = {0.f, 0.f, 0.f};
    if (fr) {
      y[0] = inv[0] * bb[0] + inv[3] * bb[1] + inv[4] * bb[2];
      y[1] = inv[3] * bb[0] + inv[1] * bb[1] + inv[5] * bb[2];
      y[2] = inv[4] * bb[0] + inv[5] * bb[1] + inv[2] * bb[2];
      acc[1] += double(y[0]) * y[0] + double(y[1]) * y[1] + double(y[2]) * y[2];
      acc[2] += 1.0;
    }
    acc[0] += double(t);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      g.Y[3 * i + c] = y[c];
      g.B[3 * i + c] = bb[c];
    }
  }
  double out[3];
  if (grid_reduce<3>(acc, g.red, g.ticket + 0, out, blockIdx.x, gridDim.x) && threadIdx.x == 0) {
    double s = out[2] > 0 ? sqrt(out[1] / out[2]) : 1.0;
    if (!(s > 0) || !isfinite(s)) s = 1.0;
    g.scal[0] = float(s);
    g.scal[2] = float(out[0] / double(g.N));
  }
}

__global__ void __launch_bounds__(kT) k_gnn_nodefeat(GnnDev g, DevMesh m) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= g.N) return;
  const float inv_s = 1.f / g.scal[0];
  float d[9];
  load_diag(m, i, d);
  const float t = g.T[i], it = 1.f / t;
  float x[kNin];
  x[0] = logf(t / g.scal[2]);
  x[1] = d[0] * it - 1.f;
  x[2] = d[4] * it - 1.f;
  x[3] = d[8] * it - 1.f;
  x[4] = d[1] * it;
  x[5] = d[2] * it;
  x[6] = d[5] * it;
  x[7] = g.nstat[2 * i];
  x[8] = g.freem[i] ? 0.f : 1.f;
  x[9] = g.nstat[2 * i + 1];
#pragma unroll
  for (int c = 0; c < 3; ++c) x[10 + c] = g.Y[3 * i + c] * inv_s;
  x[13] = x[14] = x[15] = 0.f;
  float4* dst = reinterpret_cast<float4*>(g.X0 + kNin * i);
#pragma unroll
  for (int q = 0; q < kNin / 4; ++q) dst[q] = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
}

__global__ void __launch_bounds__(kT) k_gnn_edgefeat(GnnDev g, DevMesh m) {
  const int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (p >= g.E) return;
  const int64_t i = g.dst[p], j = g.col[p];
  const float sc = rsqrtf(g.T[i] * g.T[j]);
  const double* a = m.val + 9 * int64_t(g.amap[p]);
  float e[kEin];
#pragma unroll
  for (int c = 0; c < 3; ++c) e[c] = g.relpos[3 * p + c];
#pragma unroll
  for (int k = 0; k < 9; ++k) e[3 + k] = float(a[k]) * sc;
  e[12] = e[13] = e[14] = e[15] = 0.f;
  float4* dst = reinterpret_cast<float4*>(g.efeat + kEin * p);
#pragma unroll
  for (int q = 0; q < kEin / 4; ++q) dst[q] = make_float4(e[4 * q], e[4 * q + 1], e[4 * q + 2], e[4 * q + 3]);
}

// Z = [X1 | X2] W' (+ bias) over 64-node x 64-output tiles, 256 threads, 4 x 4
// (X1, X2 row strides ld1, ld2)
// outputs per thread, K staged in chunks of 32 through shared memory.
// X rows are read as float4: ld1, ld2 multiples of 4 and K1 a multiple of 4
// (entries past K inside a row are read and dropped).
// W' (k, o) = W[k * ldw + o], or W[(k0 + o) * ldw + k] when trans (the
// backward pass dX = dZ W[k0 : k0 + 64, :]^T).  K1 is a multiple of 32 when
// K2 > 0.  Epilogue: mode 0 Z = acc (+ Z when accumulate), 1 also
// Hout = relu(Z), 2 also Hout = Hres + relu(Z).
constexpr int kDT = 64, kDK = 32;
__global__ void __launch_bounds__(256, 3) k_dense(int64_t N, const float* X1, int K1, int ld1, const float* X2, int K2,
                                               int ld2, const __nv_bfloat16* W, int ldw, int k0, int trans,
                                               const __nv_bfloat16* bias, int NO, float* Z, int ldz,
                                               const float* Hres, float* Hout, int mode, int accumulate) {
  __shared__ float xs[kDT][kDK + 1];
  __shared__ __align__(16) float ws[kDK][kDT];
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int64_t r0 = int64_t(blockIdx.x) * kDT;
  const int K = K1 + K2;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int kc = 0; kc < K; kc += kDK) {
    __syncthreads();
#pragma unroll
    for (int q0 = 0; q0 < kDT * kDK / 4; q0 += 256) {   // float4 per thread: rows are 16-byte aligned
      const int q = q0 + tid, r = q / (kDK / 4), kk = 4 * (q % (kDK / 4)), k = kc + kk;
      const int64_t row = r0 + r;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (row < N && k < K)
        v = k < K1 ? *reinterpret_cast<const float4*>(X1 + int64_t(ld1) * row + k)
                   : *reinterpret_cast<const float4*>(X2 + int64_t(ld2) * row + (k - K1));
      xs[r][kk] = k < K ? v.x : 0.f;
      xs[r][kk + 1] = k + 1 < K ? v.y : 0.f;
      xs[r][kk + 2] = k + 2 < K ? v.z : 0.f;
      xs[r][kk + 3] = k + 3 < K ? v.w : 0.f;
    }
#pragma unroll
    for (int q0 = 0; q0 < kDK * kDT; q0 += 256) {
      const int q = q0 + tid, kk = q / kDT, o = q % kDT, k = kc + kk;
      float v = 0.f;
      if (o < NO && k < K) v = __bfloat162float(trans ? W[int64_t(k0 + o) * ldw + k] : W[int64_t(k) * ldw + o]);
      ws[kk][o] = v;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < kDK; ++kk) {
      const float4 b = *reinterpret_cast<const float4*>(&ws[kk][4 * tx]);
      float a[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = xs[4 * ty + i][kk];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        acc[i][0] += a[i] * b.x;
        acc[i][1] += a[i] * b.y;
        acc[i][2] += a[i] * b.z;
        acc[i][3] += a[i] * b.w;
      }
    }
  }
  float bs[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int o = 4 * tx + j;
    bs[j] = (bias && o < NO) ? __bfloat162float(bias[o]) : 0.f;
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t row = r0 + 4 * ty + i;
    if (row >= N) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int o = 4 * tx + j;
      if (o >= NO) continue;
      float z = acc[i][j] + bs[j];
      float* zp = Z + int64_t(ldz) * row + o;
      if (accumulate) z += *zp;
      *zp = z;
      if (mode == 1) Hout[64 * row + o] = fmaxf(z, 0.f);
      else if (mode == 2) Hout[64 * row + o] = Hres[64 * row + o] + fmaxf(z, 0.f);
    }
  }
}

__device__ __forceinline__ void load_efeat(const float* ef, int64_t p, float (&e)[kEin]) {
  const float4* ev = reinterpret_cast<const float4*>(ef + int64_t(kEin) * p);
#pragma unroll
  for (int q = 0; q < kEin / 4; ++q) {
    const float4 v = ev[q];
    e[4 * q] = v.x; e[4 * q + 1] = v.y; e[4 * q + 2] = v.z; e[4 * q + 3] = v.w;
  }
}

// M_i = (1 / deg_i) sum_j relu(a_j + We e_ij + bm): one warp per node, lane o owns outputs 2o, 2o+1
__global__ void __launch_bounds__(kT) k_gnn_edge_fwd(GnnDev g, const float* a, const __nv_bfloat16* We,
                                                     const __nv_bfloat16* bm, float* M) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  if (i >= g.N) return;
  float we0[kEin], we1[kEin];
#pragma unroll
  for (int k = 0; k < kEin; ++k) {
    we0[k] = bf(We[64 * k + 2 * lane]);
    we1[k] = bf(We[64 * k + 2 * lane + 1]);
  }
  const float b0 = bf(bm[2 * lane]), b1 = bf(bm[2 * lane + 1]);
  float s0 = 0.f, s1 = 0.f;
  const int p0 = g.row_ptr[i], p1 = g.row_ptr[i + 1];
  int p = p0;
  for (; p + 1 < p1; p += 2) {   // two messages per pass: their loads overlap
    const int64_t ja = g.col[p], jb = g.col[p + 1];
    float ea[kEin], eb[kEin];
    load_efeat(g.efeat, p, ea);
    load_efeat(g.efeat, p + 1, eb);
    const float2 aa = reinterpret_cast<const float2*>(a + 64 * ja)[lane];
    const float2 ab = reinterpret_cast<const float2*>(a + 64 * jb)[lane];
    float za0 = aa.x + b0, za1 = aa.y + b1, zb0 = ab.x + b0, zb1 = ab.y + b1;
#pragma unroll
    for (int k = 0; k < kEin; ++k) {
      za0 += ea[k] * we0[k];
      za1 += ea[k] * we1[k];
      zb0 += eb[k] * we0[k];
      zb1 += eb[k] * we1[k];
    }
    s0 += fmaxf(za0, 0.f);
    s1 += fmaxf(za1, 0.f);
    s0 += fmaxf(zb0, 0.f);
    s1 += fmaxf(zb1, 0.f);
  }
  if (p < p1) {
    const int64_t j = g.col[p];
    float e[kEin];
    load_efeat(g.efeat, p, e);
    const float2 aj = reinterpret_cast<const float2*>(a + 64 * j)[lane];
    float z0 = aj.x + b0, z1 = aj.y + b1;
#pragma unroll
    for (int k = 0; k < kEin; ++k) {
      z0 += e[k] * we0[k];
      z1 += e[k] * we1[k];
    }
    s0 += fmaxf(z0, 0.f);
    s1 += fmaxf(z1, 0.f);
  }
  const float inv = 1.f / float(max(p1 - p0, 1));
  reinterpret_cast<float2*>(M + 64 * i)[lane] = make_float2(s0 * inv, s1 * inv);
}

// Per-node network outputs: C (lower), L (lower), P = C (L L^T + eps I) C^T, x0 = P b + s delta
struct NodeOut {
  float C[3][3], L[3][3], P[3][3], x0[3];
};
__device__ __forceinline__ void node_outputs(const GnnDev& g, int64_t i, float s, NodeOut& o) {
  const float* d = g.OUT + 16 * i;
  const float* c = g.C + 6 * i;
  const float C[3][3] = {{c[0], 0.f, 0.f}, {c[1], c[2], 0.f}, {c[3], c[4], c[5]}};
  const float L[3][3] = {{expf(d[3]), 0.f, 0.f}, {d[6], expf(d[4]), 0.f}, {d[7], d[8], expf(d[5])}};
  float G[3][3], CG[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      o.C[r][q] = C[r][q];
      o.L[r][q] = L[r][q];
      G[r][q] = L[r][0] * L[q][0] + L[r][1] * L[q][1] + L[r][2] * L[q][2] + (r == q ? kEps : 0.f);
    }
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int q = 0; q < 3; ++q) CG[r][q] = C[r][0] * G[0][q] + C[r][1] * G[1][q] + C[r][2] * G[2][q];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int q = 0; q < 3; ++q) o.P[r][q] = CG[r][0] * C[q][0] + CG[r][1] * C[q][1] + CG[r][2] * C[q][2];
  const float* b = g.B + 3 * i;
#pragma unroll
  for (int r = 0; r < 3; ++r) o.x0[r] = o.P[r][0] * b[0] + o.P[r][1] * b[1] + o.P[r][2] * b[2] + s * d[r];
}

// Inference: start dv = x_prev + x0 on free nodes (flag bit 0) and the learned
// blocks P into m.pinv (flag bit 1).  A node with non-finite outputs keeps block
// Jacobi and the start x_prev.  A system the plain initialisation already
// solved (b_free = 0) is left alone.
__global__ void __launch_bounds__(kT) k_gnn_apply(GnnDev g, DevMesh m, int flags) {
  if (m.pcg->done) return;
  const float s = g.scal[0];
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < g.N; i += int64_t(gridDim.x) * blockDim.x) {
    NodeOut o;
    node_outputs(g, i, s, o);
    bool ok = isfinite(o.x0[0]) && isfinite(o.x0[1]) && isfinite(o.x0[2]);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int q = 0; q < 3; ++q) ok = ok && isfinite(o.P[r][q]);
    if (!ok) {
#pragma unroll
      for (int r = 0; r < 3; ++r) {
#pragma unroll
        for (int q = 0; q < 3; ++q)
          o.P[r][q] = o.C[r][0] * o.C[q][0] + o.C[r][1] * o.C[q][1] + o.C[r][2] * o.C[q][2];
        o.x0[r] = 0.f;
      }
    }
    if (flags & 2) {
      double* pi = m.pinv + 9 * i;
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int q = 0; q < 3; ++q) pi[3 * r + q] = double(0.5f * (o.P[r][q] + o.P[q][r]));
    }
    if ((flags & 1) && g.freem[i])
#pragma unroll
      for (int r = 0; r < 3; ++r) m.dv[3 * i + r] = g.xprev[3 * i + r] + double(o.x0[r]);
  }
}

// P and x0 into g.Po, g.xo (nothing of the mesh changes)
__global__ void __launch_bounds__(kT) k_gnn_export(GnnDev g) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= g.N) return;
  NodeOut o;
  node_outputs(g, i, g.scal[0], o);
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    g.xo[3 * i + r] = o.x0[r];
#pragma unroll
    for (int q = 0; q < 3; ++q) g.Po[9 * i + 3 * r + q] = o.P[r][q];
  }
}

// training, 1: e = x0 - target on free nodes (0 on pinned)
__global__ void __launch_bounds__(kT) k_gnn_err(GnnDev g, const double* target) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= g.N) return;
  NodeOut o;
  node_outputs(g, i, g.scal[0], o);
  const bool fr = g.freem[i];
#pragma unroll
  for (int r = 0; r < 3; ++r) g.ebuf[3 * i + r] = fr ? double(o.x0[r]) - target[3 * i + r] : 0.0;
}

// training, 2: q = A_ff e, e^T A_ff e and target^T A_ff target; loss += the ratio
__global__ void __launch_bounds__(kT) k_gnn_aerr(GnnDev g, DevMesh m, const double* target) {
  double acc[2] = {0.0, 0.0};
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < g.N; i += int64_t(gridDim.x) * blockDim.x) {
    double q[3] = {0.0, 0.0, 0.0};
    if (g.freem[i]) {
      double u[3] = {0.0, 0.0, 0.0};
      for (int p = m.row_ptr[i]; p < m.row_ptr[i + 1]; ++p) {
        const int64_t j = m.col[p];
        if (!g.freem[j]) continue;
        const double* a = m.val + 9 * int64_t(p);
        const double* e = g.ebuf + 3 * j;
        const double* t = target + 3 * j;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          q[r] += a[3 * r] * e[0] + a[3 * r + 1] * e[1] + a[3 * r + 2] * e[2];
          u[r] += a[3 * r] * t[0] + a[3 * r + 1] * t[1] + a[3 * r + 2] * t[2];
        }
      }
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        acc[0] += g.ebuf[3 * i + r] * q[r];
        acc[1] += target[3 * i + r] * u[r];
      }
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) g.qbuf[3 * i + r] = q[r];
  }
  double out[2];
  if (grid_reduce<2>(acc, g.red, g.ticket + 1, out, blockIdx.x, gridDim.x) && threadIdx.x == 0) {
    const double den = out[1] > 0 ? out[1] : 1.0;
    g.scal[1] = float(den);
    g.dscal[0] = den;
    g.loss[0] += out[0] / den;
  }
}

// training, 3: d loss / d out from d loss / d x0 = 2 A_ff e / den
__global__ void __launch_bounds__(kT) k_gnn_train_bwd(GnnDev g) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= g.N) return;
  const float s = g.scal[0];
  const double den = g.dscal[0];
  NodeOut o;
  node_outputs(g, i, s, o);
  float dx[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) dx[r] = g.freem[i] ? float(2.0 * g.qbuf[3 * i + r] / den) : 0.f;
  const float* b = g.B + 3 * i;
  float* dout = g.dOUT + 16 * i;
#pragma unroll
  for (int r = 0; r < 3; ++r) dout[r] = s * dx[r];
  // d/dP of P b is dx b^T; P = C G C^T gives dG = C^T dP C; G = L L^T + eps I
  // gives dL = (dG + dG^T) L; ell_0..2 are the logs of diag(L)
  float T1[3][3], dG[3][3], dL[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int q = 0; q < 3; ++q) T1[r][q] = (o.C[0][r] * dx[0] + o.C[1][r] * dx[1] + o.C[2][r] * dx[2]) * b[q];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int q = 0; q < 3; ++q) dG[r][q] = T1[r][0] * o.C[0][q] + T1[r][1] * o.C[1][q] + T1[r][2] * o.C[2][q];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      float v = 0.f;
#pragma unroll
      for (int k = 0; k < 3; ++k) v += (dG[r][k] + dG[k][r]) * o.L[k][q];
      dL[r][q] = v;
    }
  dout[3] = dL[0][0] * o.L[0][0];
  dout[4] = dL[1][1] * o.L[1][1];
  dout[5] = dL[2][2] * o.L[2][2];
  dout[6] = dL[1][0];
  dout[7] = dL[2][0];
  dout[8] = dL[2][1];
}

// dZ = dY (.) [Z > 0], rows of 64
__global__ void __launch_bounds__(kT) k_relu_mask(int64_t n, const float* Z, const float* dY, float* dZ) {
  const int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (q < n) dZ[q] = Z[q] > 0.f ? dY[q] : 0.f;
}

// Per-CTA partial weight gradients over a grid-stride set of 32-node tiles:
// entry k * NO + o = sum_i X[i][k] dZ[i][o] (k < K), entry K * NO + o = sum_i dZ[i][o].
constexpr int kWgRows = 32;
constexpr int kWgPer = (129 * 64 + kT - 1) / kT;
__global__ void __launch_bounds__(kT) k_dense_wgrad(int64_t N, const float* X1, int K1, const float* X2, int K2,
                                                    const float* dZ, int ldz, int NO, float* gpart, int64_t stride) {
  __shared__ float xs[kWgRows][129];
  __shared__ float zs[kWgRows][65];
  const int K = K1 + K2;
  const int nout = (K + 1) * NO;
  float acc[kWgPer];
#pragma unroll
  for (int r = 0; r < kWgPer; ++r) acc[r] = 0.f;
  for (int64_t i0 = int64_t(blockIdx.x) * kWgRows; i0 < N; i0 += int64_t(gridDim.x) * kWgRows) {
    __syncthreads();
    for (int q = threadIdx.x; q < kWgRows * K; q += blockDim.x) {
      const int r = q / K, k = q - r * K;
      const int64_t i = i0 + r;
      float v = 0.f;
      if (i < N) v = k < K1 ? X1[int64_t(K1) * i + k] : X2[int64_t(K2) * i + (k - K1)];
      xs[r][k] = v;
    }
    for (int q = threadIdx.x; q < kWgRows * NO; q += blockDim.x) {
      const int r = q / NO, o = q - r * NO;
      const int64_t i = i0 + r;
      zs[r][o] = i < N ? dZ[int64_t(ldz) * i + o] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kWgPer; ++r) {
      const int q = threadIdx.x + r * kT;
      if (q < nout) {
        const int k = q / NO, o = q - k * NO;
        float a = 0.f;
        if (k < K) {
#pragma unroll 8
          for (int rr = 0; rr < kWgRows; ++rr) a += xs[rr][k] * zs[rr][o];
        } else {
#pragma unroll 8
          for (int rr = 0; rr < kWgRows; ++rr) a += zs[rr][o];
        }
        acc[r] += a;
      }
    }
  }
  float* out = gpart + int64_t(blockIdx.x) * stride;
#pragma unroll
  for (int r = 0; r < kWgPer; ++r) {
    const int q = threadIdx.x + r * kT;
    if (q < nout) out[q] = acc[r];
  }
}

// Backward of one message aggregation: one warp per source node j over its
// outgoing messages (j -> i, stored in row i at tpos): da_j, and per-CTA
// partials of dWe (16 x 64) followed by dbm (64).
__global__ void __launch_bounds__(kT) k_gnn_edge_bwd(GnnDev g, const float* a, const __nv_bfloat16* We,
                                                     const __nv_bfloat16* bm, const float* dM, float* da, float* gpart,
                                                     int64_t stride) {
  __shared__ float red[kT / 32][(kEin + 1) * 64];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  float we0[kEin], we1[kEin], gw0[kEin], gw1[kEin];
#pragma unroll
  for (int k = 0; k < kEin; ++k) {
    we0[k] = bf(We[64 * k + 2 * lane]);
    we1[k] = bf(We[64 * k + 2 * lane + 1]);
    gw0[k] = gw1[k] = 0.f;
  }
  const float b0 = bf(bm[2 * lane]), b1 = bf(bm[2 * lane + 1]);
  float gb0 = 0.f, gb1 = 0.f;
  const int64_t nwarps = int64_t(gridDim.x) * (blockDim.x >> 5);
  for (int64_t j = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; j < g.N; j += nwarps) {
    const float2 aj = reinterpret_cast<const float2*>(a + 64 * j)[lane];
    float d0 = 0.f, d1 = 0.f;
    for (int p = g.row_ptr[j]; p < g.row_ptr[j + 1]; ++p) {
      const int64_t i = g.col[p];
      float e[kEin];
      load_efeat(g.efeat, g.tpos[p], e);
      float z0 = aj.x + b0, z1 = aj.y + b1;
#pragma unroll
      for (int k = 0; k < kEin; ++k) {
        z0 += e[k] * we0[k];
        z1 += e[k] * we1[k];
      }
      const float inv = 1.f / float(max(g.row_ptr[i + 1] - g.row_ptr[i], 1));
      const float2 dm = reinterpret_cast<const float2*>(dM + 64 * i)[lane];
      const float g0 = z0 > 0.f ? dm.x * inv : 0.f, g1 = z1 > 0.f ? dm.y * inv : 0.f;
      d0 += g0;
      d1 += g1;
#pragma unroll
      for (int k = 0; k < kEin; ++k) {
        gw0[k] += e[k] * g0;
        gw1[k] += e[k] * g1;
      }
      gb0 += g0;
      gb1 += g1;
    }
    reinterpret_cast<float2*>(da + 64 * j)[lane] = make_float2(d0, d1);
  }
#pragma unroll
  for (int k = 0; k < kEin; ++k) {
    red[wib][64 * k + 2 * lane] = gw0[k];
    red[wib][64 * k + 2 * lane + 1] = gw1[k];
  }
  red[wib][64 * kEin + 2 * lane] = gb0;
  red[wib][64 * kEin + 2 * lane + 1] = gb1;
  __syncthreads();
  float* out = gpart + int64_t(blockIdx.x) * stride;
  for (int q = threadIdx.x; q < (kEin + 1) * 64; q += blockDim.x) {
    float acc = 0.f;
#pragma unroll
    for (int w = 0; w < kT / 32; ++w) acc += red[w][q];
    out[q] = acc;
  }
}

// grad[q] += sum_c gpart[c * stride + q], CTAs in order
__global__ void __launch_bounds__(kT) k_reduce_parts(const float* gpart, int64_t stride, int nparts, int len,
                                                     float* grad) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= len) return;
  float acc = 0.f;
  for (int c = 0; c < nparts; ++c) acc += gpart[int64_t(c) * stride + q];
  grad[q] += acc;
}

__global__ void __launch_bounds__(kT) k_adam(int64_t P, float* w, __nv_bfloat16* w16, float* m1, float* m2,
                                             const float* grad, float scale, float lr, float b1, float b2, float c1,
                                             float c2, float eps) {
  const int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (q >= P) return;
  const float gq = grad[q] * scale;
  const float a = b1 * m1[q] + (1.f - b1) * gq;
  const float v = b2 * m2[q] + (1.f - b2) * gq * gq;
  m1[q] = a;
  m2[q] = v;
  const float wn = w[q] - lr * (a / c1) / (sqrtf(v / c2) + eps);
  w[q] = wn;
  w16[q] = __float2bfloat16_rn(wn);
}

__global__ void __launch_bounds__(kT) k_to_bf16(int64_t P, const float* w, __nv_bfloat16* w16) {
  const int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (q < P) w16[q] = __float2bfloat16_rn(w[q]);
}

// Pair of a step: with w = dv on pinned nodes and x_prev on free ones,
// b_net = b - A w on free rows (0 on pinned rows); target = dv - x_prev on free
// nodes, 0 on pinned (target may be NULL)
__global__ void __launch_bounds__(kT) k_gnn_pair(DevMesh m, const double* xprev, double* bout, double* tout) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= m.N) return;
  double r[3] = {0.0, 0.0, 0.0}, t[3] = {0.0, 0.0, 0.0};
  if (!m.pinned[i]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      r[c] = m.rhs[3 * i + c];
      t[c] = m.dv[3 * i + c] - xprev[3 * i + c];
    }
    for (int p = m.row_ptr[i]; p < m.row_ptr[i + 1]; ++p) {
      const int64_t j = m.col[p];
      const double* w = m.pinned[j] ? m.dv + 3 * j : xprev + 3 * j;
      const double* a = m.val + 9 * int64_t(p);
#pragma unroll
      for (int c = 0; c < 3; ++c) r[c] -= a[3 * c] * w[0] + a[3 * c + 1] * w[1] + a[3 * c + 2] * w[2];
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    bout[3 * i + c] = r[c];
    if (tout) tout[3 * i + c] = t[c];
  }
}

inline unsigned cdiv(int64_t n, int d) { return unsigned((n + d - 1) / d); }
inline unsigned rgrid(int64_t n) {
  const int64_t b = (n + kT - 1) / kT;
  return unsigned(b < 1 ? 1 : (b > 4 * 152 ? 4 * 152 : b));
}
inline unsigned pgrid(int64_t units) { return unsigned(units < 1 ? 1 : (units > kMaxParts ? kMaxParts : units)); }

// Dense layer: the tcgen05 kernel when the network uses tensor cores and the
// shape has a tensor-core form, else the FP32 FMA kernel (same arguments).
int dense(const GnnDev& g, int64_t N, const float* X1, int K1, int ld1, const float* X2, int K2, int ld2,
          const __nv_bfloat16* W, int ldw, int k0, int trans, const __nv_bfloat16* bias, int NO, float* Z, int ldz,
          const float* Hres, float* Hout, int mode, int accumulate, cudaStream_t s) {
  if (g.use_tc) {
    const int L = dense_tc(N, X1, K1, ld1, X2, K2, ld2, W, ldw, k0, trans, bias, NO, Z, ldz, Hres, Hout, mode,
                           accumulate, g.err, s);
    if (L >= 0) return L;
  }
  if (N <= 0) return 0;
  k_dense<<<cdiv(N, kDT), 256, 0, s>>>(N, X1, K1, ld1, X2, K2, ld2, W, ldw, k0, trans, bias, NO, Z, ldz, Hres, Hout,
                                      mode, accumulate);
  return 1;
}

int edge_fwd(const GnnDev& g, const float* a, const __nv_bfloat16* We, const __nv_bfloat16* bm, float* M,
             cudaStream_t s) {
  if (g.use_tc) {
    const int L = gnn_edge_fwd_tc(g, a, We, bm, M, s);
    if (L >= 0) return L;
  }
  k_gnn_edge_fwd<<<cdiv(32 * g.N, kT), kT, 0, s>>>(g, a, We, bm, M);
  return 1;
}

}  // namespace

int gnn_max_parts() { return kMaxParts; }
int gnn_reduce_slots() { return 4 * 152; }

int gnn_forward(const GnnDev& g, const DevMesh& m, const double* b, cudaStream_t s) {
  const __nv_bfloat16* W = g.w16;
  const int64_t N = g.N;
  k_gnn_prep<<<rgrid(N), kT, 0, s>>>(g, m, b);
  k_gnn_nodefeat<<<cdiv(N, kT), kT, 0, s>>>(g, m);
  int L = 2;
  if (g.E > 0) {
    k_gnn_edgefeat<<<cdiv(g.E, kT), kT, 0, s>>>(g, m);
    ++L;
  }
  L += dense(g, N, g.X0, kNin, kNin, nullptr, 0, 0, W + g.off[kPW0], 64, 0, 0, W + g.off[kPb0], 64, g.Z0, 64, nullptr,
             g.H, 1, 0, s);
  for (int l = 0; l < 3; ++l) {
    const float* h = g.H + int64_t(l) * N * 64;
    float* a = g.Aa + int64_t(l) * N * 64;
    float* M = g.M + int64_t(l) * N * 64;
    L += dense(g, N, h, 64, 64, nullptr, 0, 0, W + g.off[kPWa + 5 * l], 64, 0, 0, nullptr, 64, a, 64, nullptr, nullptr,
               0, 0, s);
    L += edge_fwd(g, a, W + g.off[kPWe + 5 * l], W + g.off[kPbm + 5 * l], M, s);
    L += dense(g, N, h, 64, 64, M, 64, 64, W + g.off[kPWu + 5 * l], 64, 0, 0, W + g.off[kPbu + 5 * l], 64,
               g.ZU + int64_t(l) * N * 64, 64, h, g.H + int64_t(l + 1) * N * 64, 2, 0, s);
  }
  L += dense(g, N, g.H + 3 * N * 64, 64, 64, nullptr, 0, 0, W + g.off[kPWd], kNout, 0, 0, W + g.off[kPbd], kNout,
             g.OUT, 16, nullptr, nullptr, 0, 0, s);
  return L;
}

int gnn_apply_inference(const GnnDev& g, const DevMesh& m, int flags, cudaStream_t s) {
  k_gnn_apply<<<rgrid(g.N), kT, 0, s>>>(g, m, flags);
  return 1;
}

int gnn_apply_export(const GnnDev& g, cudaStream_t s) {
  k_gnn_export<<<cdiv(g.N, kT), kT, 0, s>>>(g);
  return 1;
}

int gnn_backward_pair(const GnnDev& g, const DevMesh& m, const double* target, cudaStream_t s) {
  const __nv_bfloat16* W = g.w16;
  const int64_t N = g.N;
  const int64_t st = g.part_stride;
  const unsigned wg = pgrid(cdiv(N, kWgRows)), eg = pgrid(cdiv(32 * N, kT));
  int L = 0;
  k_gnn_err<<<cdiv(N, kT), kT, 0, s>>>(g, target);
  k_gnn_aerr<<<rgrid(N), kT, 0, s>>>(g, m, target);
  k_gnn_train_bwd<<<cdiv(N, kT), kT, 0, s>>>(g);
  ++L;
  // decoder
  k_dense_wgrad<<<wg, kT, 0, s>>>(N, g.H + 3 * N * 64, 64, nullptr, 0, g.dOUT, 16, kNout, g.gpart, st);
  k_reduce_parts<<<cdiv(65 * kNout, kT), kT, 0, s>>>(g.gpart, st, int(wg), 65 * kNout, g.grad + g.off[kPWd]);
  L += 4 + dense(g, N, g.dOUT, kNout, 16, nullptr, 0, 0, W + g.off[kPWd], kNout, 0, 1, nullptr, 64, g.dH, 64, nullptr,
                 nullptr, 0, 0, s);
  for (int l = 2; l >= 0; --l) {
    const float* h = g.H + int64_t(l) * N * 64;
    const float* a = g.Aa + int64_t(l) * N * 64;
    const float* M = g.M + int64_t(l) * N * 64;
    k_relu_mask<<<cdiv(N * 64, kT), kT, 0, s>>>(N * 64, g.ZU + int64_t(l) * N * 64, g.dH, g.dZ);
    k_dense_wgrad<<<wg, kT, 0, s>>>(N, h, 64, M, 64, g.dZ, 64, 64, g.gpart, st);
    k_reduce_parts<<<cdiv(129 * 64, kT), kT, 0, s>>>(g.gpart, st, int(wg), 129 * 64, g.grad + g.off[kPWu + 5 * l]);
    // dM = dZU Wu[64:128]^T (the 1/deg factor is applied per edge); the residual keeps dH
    L += dense(g, N, g.dZ, 64, 64, nullptr, 0, 0, W + g.off[kPWu + 5 * l], 64, 64, 1, nullptr, 64, g.dM, 64, nullptr,
               nullptr, 0, 0, s);
    L += dense(g, N, g.dZ, 64, 64, nullptr, 0, 0, W + g.off[kPWu + 5 * l], 64, 0, 1, nullptr, 64, g.dH, 64, nullptr,
               nullptr, 0, 1, s);
    k_gnn_edge_bwd<<<eg, kT, 0, s>>>(g, a, W + g.off[kPWe + 5 * l], W + g.off[kPbm + 5 * l], g.dM, g.dA, g.gpart, st);
    k_reduce_parts<<<cdiv((kEin + 1) * 64, kT), kT, 0, s>>>(g.gpart, st, int(eg), (kEin + 1) * 64, g.grad + g.off[kPWe + 5 * l]);
    k_dense_wgrad<<<wg, kT, 0, s>>>(N, h, 64, nullptr, 0, g.dA, 64, 64, g.gpart, st);
    k_reduce_parts<<<cdiv(64 * 64, kT), kT, 0, s>>>(g.gpart, st, int(wg), 64 * 64, g.grad + g.off[kPWa + 5 * l]);
    L += dense(g, N, g.dA, 64, 64, nullptr, 0, 0, W + g.off[kPWa + 5 * l], 64, 0, 1, nullptr, 64, g.dH, 64, nullptr,
               nullptr, 0, 1, s);
    L += 7;
  }
  k_relu_mask<<<cdiv(N * 64, kT), kT, 0, s>>>(N * 64, g.Z0, g.dH, g.dZ);
  k_dense_wgrad<<<wg, kT, 0, s>>>(N, g.X0, kNin, nullptr, 0, g.dZ, 64, 64, g.gpart, st);
  k_reduce_parts<<<cdiv(17 * 64, kT), kT, 0, s>>>(g.gpart, st, int(wg), 17 * 64, g.grad + g.off[kPW0]);
  return L + 3;
}

int gnn_adam(const GnnDev& g, float scale, float lr, int t, cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, float(t)), c2 = 1.f - powf(b2, float(t));
  k_adam<<<cdiv(g.P, kT), kT, 0, s>>>(g.P, g.w32, g.w16, g.m1, g.m2, g.grad, scale, lr, b1, b2, c1, c2, 1e-8f);
  return 1;
}

int gnn_refresh_bf16(const GnnDev& g, cudaStream_t s) {
  k_to_bf16<<<cdiv(g.P, kT), kT, 0, s>>>(g.P, g.w32, g.w16);
  return 1;
}

int gnn_pair(const DevMesh& m, const double* xprev, double* b, double* target, cudaStream_t s) {
  k_gnn_pair<<<cdiv(m.N, kT), kT, 0, s>>>(m, xprev, b, target);
  return 1;
}

}  // namespace gf
