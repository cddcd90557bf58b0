// FP64 kernels of one graph-FEM fracture step (sm_103a).
//
// Order inside a step (Algorithm 1, Sec. 4.3):
//   k_tet_stress -> k_nonlocal -> k_edge_driver -> k_tet_chi     (Eq. 14-25)
//   memset(A) -> k_node_init -> k_assemble per colour            (Eq. 2, 12, 32-34)
//   k_set_pinned -> k_pcg_init -> {k_pcg_spmv, k_pcg_update, k_pcg_p}* -> k_true_residual -> k_integrate
//
// FP64 on GB300 runs at ~1/61 of the FP32 rate (measured 1.19 TFLOP/s), so
// these kernels are FP64-pipe bound rather than HBM bound; they are written to
// minimise FP64 operations: StVK in edge lengths is an exact quadratic form
// V Psi = 1/2 (s - s0)^T Hs (s - s0) with a per-tet constant Hs (precomputed),
// so forces and tangents need no C or F at all.
#include <cfloat>
#include <cmath>

#include "gf_device.h"
#include "gf_reduce.cuh"

#include <algorithm>

namespace gf {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ void ld3(const double* __restrict__ a, int64_t i, double o[3]) {
  const double* p = a + 3 * i;
  o[0] = p[0];
  o[1] = p[1];
  o[2] = p[2];
}

// C = B^T G B, G_ij = (s_0i + s_0j - s_ij)/2 (Thm 3.1 in closed form); Voigt out.
__device__ __forceinline__ void cauchy_green(const double s[6], const double B[9], double C[6]) {
  double G[3][3];
  G[0][0] = s[0];
  G[1][1] = s[1];
  G[2][2] = s[2];
  G[0][1] = G[1][0] = 0.5 * (s[0] + s[1] - s[3]);
  G[0][2] = G[2][0] = 0.5 * (s[0] + s[2] - s[4]);
  G[1][2] = G[2][1] = 0.5 * (s[1] + s[2] - s[5]);
  double Y[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) Y[r][c] = G[r][0] * B[c] + G[r][1] * B[3 + c] + G[r][2] * B[6 + c];
  const int I[6] = {0, 1, 2, 0, 0, 1}, J[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
  for (int v = 0; v < 6; ++v) C[v] = B[I[v]] * Y[0][J[v]] + B[3 + I[v]] * Y[1][J[v]] + B[6 + I[v]] * Y[2][J[v]];
}

// Normal stress along e (Eq. 16 with the current direction, Eq. 17): (e.S.e)/|e|^2,
// shear terms weighted by kappa.  edge_traction is the numerator e.S.e; callers
// divide by |e|^2 (an FP64 division is a multi-instruction sequence, so they
// share divisions where they can).
__device__ __forceinline__ double edge_traction(const double e[3], const double S[6], double kappa) {
  return e[0] * e[0] * S[0] + e[1] * e[1] * S[1] + e[2] * e[2] * S[2] +
         kappa * (e[0] * e[1] * S[3] + e[0] * e[2] * S[4] + e[1] * e[2] * S[5]);
}

// ---------------------------------------------------------------------------
// Damage: stress, non-local average, edge driver + relabel, chi
// ---------------------------------------------------------------------------

// The tet's current edge vectors e_k, squared lengths s_k and second
// Piola-Kirchhoff stress S (Voigt xx yy zz xy xz yz) from the positions x.
template <bool kSNH>
__device__ __forceinline__ void tet_current_stress(const DevMesh& m, const Material& mt, int64_t t, double (&e)[6][3],
                                                   double (&s)[6], double (&S)[6]) {
  const int4 n = m.tets[t];
  const int nid[4] = {n.x, n.y, n.z, n.w};
  double P[4][3];
#pragma unroll
  for (int a = 0; a < 4; ++a) ld3(m.x, nid[a], P[a]);
#pragma unroll
  for (int k = 0; k < 6; ++k) {
#pragma unroll
    for (int c = 0; c < 3; ++c) e[k][c] = P[edge_b(k)][c] - P[edge_a(k)][c];
    s[k] = e[k][0] * e[k][0] + e[k][1] * e[k][1] + e[k][2] * e[k][2];
  }
  double B[9];
#pragma unroll
  for (int f = 0; f < 9; ++f) B[f] = m.rest[(kRestB + f) * m.T + t];
  double C[6];
  cauchy_green(s, B, C);
  if constexpr (kSNH) {
    // Eq. 35: S = mu (1 - 1/(I_C + 1)) I + lam (J - a) J C^-1 = ... + lam (J - a) / J adj(C),
    // J = det F = det(Ds) det(B) (signed)
    const double ds = e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) -
                      e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
                      e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
    const double db = B[0] * (B[4] * B[8] - B[5] * B[7]) - B[1] * (B[3] * B[8] - B[5] * B[6]) +
                      B[2] * (B[3] * B[7] - B[4] * B[6]);
    const double J = ds * db, IC = C[0] + C[1] + C[2];
    const double d0 = mt.mu * (1.0 - 1.0 / (IC + 1.0)), d1 = mt.lam * (J - mt.snh_a) / J;
    // adjugate of the symmetric C (Voigt xx yy zz xy xz yz)
    S[0] = d0 + d1 * (C[1] * C[2] - C[5] * C[5]);
    S[1] = d0 + d1 * (C[0] * C[2] - C[4] * C[4]);
    S[2] = d0 + d1 * (C[0] * C[1] - C[3] * C[3]);
    S[3] = d1 * (C[4] * C[5] - C[3] * C[2]);
    S[4] = d1 * (C[3] * C[5] - C[4] * C[1]);
    S[5] = d1 * (C[3] * C[4] - C[0] * C[5]);
  } else {
    // second Piola-Kirchhoff stress of Eq. 37: lam/2 (tr C - 3) I + mu (C - I)
    const double h = 0.5 * mt.lam * (C[0] + C[1] + C[2] - 3.0);
    S[0] = h + mt.mu * (C[0] - 1.0);
    S[1] = h + mt.mu * (C[1] - 1.0);
    S[2] = h + mt.mu * (C[2] - 1.0);
    S[3] = mt.mu * C[3];
    S[4] = mt.mu * C[4];
    S[5] = mt.mu * C[5];
  }
}

// Eq. 14 per tet: the stress fed to the Eq. 20 average (chi S, or S).  The
// tet's own edge-normal stresses of Eq. 22-25 are formed in k_tet_chi, only for
// the tets that have a broken edge (chi = 1 needs none of them).
template <bool kSNH>
__device__ __forceinline__ void tet_stress_body(const DevMesh& m, const Material& mt, const StepScalars& sp, unsigned bid, unsigned nb) {

  const int64_t t = bid * int64_t(blockDim.x) + threadIdx.x;
  if (t >= m.T) return;
  double e[6][3], s[6], S[6];
  tet_current_stress<kSNH>(m, mt, t, e, s, S);
  const double w = mt.average_degraded ? m.chi[t] : 1.0;
  double2* si = reinterpret_cast<double2*>(m.sig_in + 6 * t);
  si[0] = make_double2(w * S[0], w * S[1]);
  si[1] = make_double2(w * S[2], w * S[3]);
  si[2] = make_double2(w * S[4], w * S[5]);
}
__global__ void __launch_bounds__(kThreads) k_tet_stress(DevMesh m, Material mt, StepScalars sp) {
  tet_stress_body<false>(m, mt, sp, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kThreads) k_tet_stress_snh(DevMesh m, Material mt, StepScalars sp) {
  tet_stress_body<true>(m, mt, sp, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kThreads) kb_tet_stress(const BatchTab* __restrict__ tab) {
  unsigned bid, nb;
  const int k = batch_locate(tab, kB_tet_stress, blockIdx.x, bid, nb);
  tet_stress_body<false>(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb);   // batches run the StVK energy
}

// Eq. 20 sum: thread per SELL-32 lane slot (coalesced index/weight loads; the
// neighbour stresses are gathered from L2).  Slot q holds tet nb_perm[q]: the
// tets of a window are ordered by list length, so a group pads little.
__device__ __forceinline__ void nonlocal_body(const DevMesh& m, const Material& mt, const StepScalars& sp, unsigned bid, unsigned nb) {

  const int64_t q = bid * int64_t(blockDim.x) + threadIdx.x;
  if (q >= m.T) return;
  const int64_t g = q >> 5;
  const int lane = int(q & 31);
  const int64_t t = m.nb_perm[q];
  const int64_t off = m.nb_off[g] + lane;
  const int len = m.nb_len[g];
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int k = 0; k < len; ++k) {
    const int j = __ldg(m.nb_idx + off + 32 * int64_t(k));
    const double w = __ldg(m.nb_w + off + 32 * int64_t(k));
    const double2* sj = reinterpret_cast<const double2*>(m.sig_in + 6 * int64_t(j));
    const double2 a = sj[0], b = sj[1], c = sj[2];
    acc[0] += w * a.x;
    acc[1] += w * a.y;
    acc[2] += w * b.x;
    acc[3] += w * b.y;
    acc[4] += w * c.x;
    acc[5] += w * c.y;
  }
  double2* o = reinterpret_cast<double2*>(m.sig_bar + 6 * t);
  o[0] = make_double2(acc[0], acc[1]);
  o[1] = make_double2(acc[2], acc[3]);
  o[2] = make_double2(acc[4], acc[5]);
}
__global__ void __launch_bounds__(kThreads) k_nonlocal(DevMesh m, Material mt, StepScalars sp) {
  nonlocal_body(m, mt, sp, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kThreads) kb_nonlocal(const BatchTab* __restrict__ tab) {
  unsigned bid, nb;
  const int k = batch_locate(tab, kB_nonlocal, blockIdx.x, bid, nb);
  nonlocal_body(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb);
}

// Per edge: sigma* = max over incident tets of the projected average (Eq. 20),
// driver = sigma*/E (or sigma*), then zeta |= (driver >= threshold) (Eq. 21).
__device__ __forceinline__ void edge_driver_body(const DevMesh& m, const Material& mt, const StepScalars& sp, unsigned bid, unsigned nb) {

  const int64_t g = bid * int64_t(blockDim.x) + threadIdx.x;
  unsigned long long n_brk = 0, n_new = 0;
  if (g < m.NE) {
    const int64_t i = m.edge_order[g];   // edges of equal incident-tet count side by side
    const int2 ab = m.edges[i];
    double pa[3], pb[3];
    ld3(m.x, ab.x, pa);
    ld3(m.x, ab.y, pb);
    const double e[3] = {pb[0] - pa[0], pb[1] - pa[1], pb[2] - pa[2]};
    const double s = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
    // e.S.e = sum_v w_v S_v with the edge's weights w (the shear ones carry
    // kappa), formed once per edge: one DMUL and five DFMA per incident tet
    const double w[6] = {e[0] * e[0], e[1] * e[1], e[2] * e[2], mt.kappa * (e[0] * e[1]), mt.kappa * (e[0] * e[2]),
                         mt.kappa * (e[1] * e[2])};
    // max over the incident tets of (e.S.e) / s: s > 0 and rounded division is
    // monotone, so dividing the largest numerator once gives the same value
    double mq = -INFINITY;
    for (int p = m.et_ptr[i]; p < m.et_ptr[i + 1]; ++p) {
      const double2* sb = reinterpret_cast<const double2*>(m.sig_bar + 6 * int64_t(m.et_tet[p]));
      const double2 a = sb[0], b = sb[1], c = sb[2];
      const double q = fma(w[5], c.y, fma(w[4], c.x, fma(w[3], b.y, fma(w[2], b.x, fma(w[1], a.y, w[0] * a.x)))));
      mq = fmax(mq, q);
    }
    // one FP64 division per edge (a multi-instruction sequence on the FP64
    // pipe): the strain driver divides by s E at once
    const double d = mq / (mt.driver_stress ? s : s * mt.young);
    m.driver[i] = d;
    const uint8_t old = m.labels[i];
    const uint8_t now = (old || d >= mt.threshold) ? 1 : 0;
    if (now != old) m.labels[i] = now;
    n_brk = now;
    n_new = now && !old;
  }
  warp_count(n_brk, m.counters + kCntBroken);
  warp_count(n_new, m.counters + kCntNewBroken);
}
__global__ void __launch_bounds__(kThreads) k_edge_driver(DevMesh m, Material mt, StepScalars sp) {
  edge_driver_body(m, mt, sp, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kThreads) kb_edge_driver(const BatchTab* __restrict__ tab) {
  unsigned bid, nb;
  const int k = batch_locate(tab, kB_edge_driver, blockIdx.x, bid, nb);
  edge_driver_body(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb);
}

// Eq. 22-25: chi from the tet's broken-edge mask and its local edge-normal
// stresses sigma_f = (e.S.e)/|e|^2 of its own (un-averaged) stress, formed
// here for the tets that have a broken edge and are not split apart.
template <bool kSNH>
__device__ __forceinline__ void tet_chi_body(const DevMesh& m, const Material& mt, const StepScalars& sp, unsigned bid, unsigned nb) {
  const uint64_t lut = mt.lut;

  const int64_t t = bid * int64_t(blockDim.x) + threadIdx.x;
  unsigned long long zero = 0;
  if (t < m.T) {
    int mask = 0;
#pragma unroll
    for (int k = 0; k < 6; ++k) mask |= int(m.labels[m.tet_edges[6 * t + k]] != 0) << k;
    double c = 1.0;
    if (mask) {
      if ((lut >> mask) & 1ull) {
        c = 0.0;
      } else {
        double e[6][3], s[6], S[6];
        tet_current_stress<kSNH>(m, mt, t, e, s, S);
        double num = 0.0, den = 0.0;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          const double a = fabs(edge_traction(e[k], S, mt.kappa) / s[k]);
          den += a;
          if (!((mask >> k) & 1)) num += a;
        }
        c = (den <= 1e-12 * mt.young) ? double(6 - __popc(mask)) / 6.0 : num / den;
      }
    }
    m.chi[t] = c;
    zero = (c == 0.0);
  }
  warp_count(zero, m.counters + kCntChiZero);
}
__global__ void __launch_bounds__(kThreads) k_tet_chi(DevMesh m, Material mt, StepScalars sp) {
  tet_chi_body<false>(m, mt, sp, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kThreads) k_tet_chi_snh(DevMesh m, Material mt, StepScalars sp) {
  tet_chi_body<true>(m, mt, sp, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kThreads) kb_tet_chi(const BatchTab* __restrict__ tab) {
  unsigned bid, nb;
  const int k = batch_locate(tab, kB_tet_chi, blockIdx.x, bid, nb);
  tet_chi_body<false>(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb);   // batches run the StVK energy
}

// ---------------------------------------------------------------------------
// Assembly of A = (1 + dt alpha) M + (dt beta + dt^2) K*, b = dt (f_ext + f* - alpha M v - (beta + dt) K* v)
// ---------------------------------------------------------------------------

__device__ __forceinline__ void node_init_body(const DevMesh& m, const Material& mt, const StepScalars& sp, unsigned bid, unsigned nb) {
  const double dt = sp.dt, alpha = mt.alpha;
  const double* f_ext = sp.has_fext ? m.f_ext : nullptr;

  const int64_t i = bid * int64_t(blockDim.x) + threadIdx.x;
  if (i >= m.N) return;
  if (m.mass_blk) {   // consistent mass: every block of the row, and M v over the row
    double mv[3] = {0.0, 0.0, 0.0};
    for (int b = m.row_ptr[i]; b < m.row_ptr[i + 1]; ++b) {
      const double mb = m.mass_blk[b];
      const int64_t j = m.col[b];
#pragma unroll
      for (int c = 0; c < 3; ++c) mv[c] += mb * m.v[3 * j + c];
      double* d = m.val + 9 * int64_t(b);
      const double cm = (1.0 + dt * alpha) * mb;
      d[0] += cm;
      d[4] += cm;
      d[8] += cm;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) m.rhs[3 * i + c] = dt * ((f_ext ? f_ext[3 * i + c] : 0.0) - alpha * mv[c]);
    return;
  }
  const double mi = m.mass[i];
#pragma unroll
  for (int c = 0; c < 3; ++c)
    m.rhs[3 * i + c] = dt * ((f_ext ? f_ext[3 * i + c] : 0.0) - alpha * mi * m.v[3 * i + c]);
  double* d = m.val + 9 * int64_t(m.diag_blk[i]);
  const double cm = (1.0 + dt * alpha) * mi;
  d[0] += cm;
  d[4] += cm;
  d[8] += cm;
}
__global__ void __launch_bounds__(kThreads) k_node_init(DevMesh m, Material mt, StepScalars sp) {
  node_init_body(m, mt, sp, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kThreads) kb_node_init(const BatchTab* __restrict__ tab) {
  unsigned bid, nb;
  const int k = batch_locate(tab, kB_node_init, blockIdx.x, bid, nb);
  node_init_body(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb);
}

// One colour: no two tets share a node, so the read-modify-write scatter into
// the block-CSR slots and into b is conflict-free without atomics.
__global__ void __launch_bounds__(128) k_assemble(DevMesh m, double dt, double beta, int t0, int t1) {
  const int64_t ct = t0 + blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (ct >= t1) return;
  const int64_t t = m.colour_tets[ct];
  const double chi = m.chi[t];
  if (chi == 0.0) return;   // chi = 0: the element carries no energy (Eq. 25)
  const int4 n = m.tets[t];
  const int nid[4] = {n.x, n.y, n.z, n.w};
  // incident local edges of each node and the sign of ds_k/dx_a = 2 sgn e_k
  const int inc[4][3] = {{0, 1, 2}, {0, 3, 4}, {1, 3, 5}, {2, 4, 5}};
  const double sgn[4][3] = {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {1, 1, 1}};
  const int kab[4][4] = {{-1, 0, 1, 2}, {0, -1, 3, 4}, {1, 3, -1, 5}, {2, 4, 5, -1}};

  double P[4][3], U[4][3];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    ld3(m.x, nid[a], P[a]);
    ld3(m.v, nid[a], U[a]);
  }
  double e[6][3], ds[6], Dv[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    double du[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      e[k][c] = P[edge_b(k)][c] - P[edge_a(k)][c];
      du[c] = U[edge_b(k)][c] - U[edge_a(k)][c];
    }
    ds[k] = e[k][0] * e[k][0] + e[k][1] * e[k][1] + e[k][2] * e[k][2] - m.rest[(kRestS0 + k) * m.T + t];
    Dv[k] = e[k][0] * du[0] + e[k][1] * du[1] + e[k][2] * du[2];   // half ds/dt (the 2 is taken with cv below)
  }
  double H[21];
#pragma unroll
  for (int f = 0; f < 21; ++f) H[f] = m.rest[(kRestH + f) * m.T + t];
  auto h = [&](int k, int l) { return k <= l ? H[tri6(k, l)] : H[tri6(l, k)]; };
  // g = dV Psi/ds = Hs (s - s0);  w = Hs (ds/dx . v) / 2
  double g[6], w[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    double gk = 0.0, wk = 0.0;
#pragma unroll
    for (int l = 0; l < 6; ++l) {
      gk += h(k, l) * ds[l];
      wk += h(k, l) * Dv[l];
    }
    g[k] = gk;
    w[k] = wk;
  }
  // right-hand side: per edge k (a->b), t_k = 2 dt chi [e_k (g_k + 2 c w_k) + c g_k (v_b - v_a)], c = beta + dt
  {
    const double cv = beta + dt, cv2 = 2.0 * cv, sc = 2.0 * dt * chi;
    double f[4][3] = {};
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const double a1 = sc * (g[k] + cv2 * w[k]), a2 = sc * cv * g[k];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double tk = a1 * e[k][c] + a2 * (U[edge_b(k)][c] - U[edge_a(k)][c]);
        f[edge_a(k)][c] += tk;
        f[edge_b(k)][c] -= tk;
      }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) m.rhs[3 * int64_t(nid[a]) + c] += f[a][c];
  }
  // tangent blocks: (a,b) = 4 sK sum_{k in a, l in b} sgn sgn H_kl e_k e_l^T + geometric part
  const double sK = (dt * beta + dt * dt) * chi;
  const int* sl = m.slot + 16 * t;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    double Y[6][3];   // Y[k][c] = 4 sK sum_j H(k, l_j) sgn_bj e_{l_j}[c]
#pragma unroll
    for (int k = 0; k < 6; ++k)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        double y = 0.0;
#pragma unroll
        for (int j = 0; j < 3; ++j) y += sgn[b][j] * h(k, inc[b][j]) * e[inc[b][j]][c];
        Y[k][c] = 4.0 * sK * y;
      }
#pragma unroll
    for (int a = 0; a <= b; ++a) {
      double blk[3][3];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          double v = 0.0;
#pragma unroll
          for (int i = 0; i < 3; ++i) v += sgn[a][i] * e[inc[a][i]][r] * Y[inc[a][i]][c];
          blk[r][c] = v;
        }
      double geo;
      if (a == b) {
        geo = 2.0 * sK * (g[inc[a][0]] + g[inc[a][1]] + g[inc[a][2]]);
      } else {
        geo = -2.0 * sK * g[kab[a][b]];
      }
      blk[0][0] += geo;
      blk[1][1] += geo;
      blk[2][2] += geo;
      double* dst = m.val + 9 * int64_t(sl[4 * a + b]);
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) dst[3 * r + c] += blk[r][c];
      if (a != b) {
        double* dt2 = m.val + 9 * int64_t(sl[4 * b + a]);
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int c = 0; c < 3; ++c) dt2[3 * r + c] += blk[c][r];
      }
    }
  }
}

// Two-phase FP64 assembly (no colours, no atomics).
// k_elem64 (thread per tet) computes the six off-diagonal blocks of
// (dt beta + dt^2) chi k_e and the four rhs shares dt chi (f_a - (beta+dt)(k_e v)_a)
// and writes each straight into the assembly row it belongs to: local edge
// k's block to edge row erow[6t+k] (9 values, oriented for the global edge
// (i, j), i < j), local node a's rhs share to node row nrow[4t+a] (3 values
// and a pad).  A node's or an edge's rows are contiguous, so k_gather64
// (thread per matrix entry or rhs component) streams through them in a fixed
// order.  The element energy depends on node differences only, so every
// block row of k_e sums to zero, and so does every block row of the assembled
// stiffness: k_diag64 forms the diagonal blocks as minus the sum of their
// row's off-diagonal blocks and adds the mass terms.
constexpr int kNodeRow = 4, kEdgeRow = 9;
constexpr int kElemThreads64 = 128;   // threads per CTA of the element kernels

// where a tet's contributions go (the writes scatter; the gather reads stream)
struct ElemRows64 {
  double* nb;        // node rows [4T][4]: rhs share, pad
  double* eb;        // edge rows [6T][9]
  const int32_t* nr; // nrow + 4t
  const int32_t* er; // erow + 6t
  unsigned flip;     // bit k: the tet lists local edge k against the global (i < j) order
  __device__ __forceinline__ ElemRows64(const DevMesh& m, int64_t t, const int (&nid)[4])
      : nb(m.ebuf), eb(m.ebuf + int64_t(kNodeRow) * 4 * m.T), nr(m.nrow + 4 * t), er(m.erow + 6 * t), flip(0u) {
#pragma unroll
    for (int k = 0; k < 6; ++k) flip |= nid[edge_a(k)] > nid[edge_b(k)] ? (1u << k) : 0u;
  }
  // off-diagonal block (a, b), a < b, of the tet's matrix
  __device__ __forceinline__ void block(int a, int b, const double (&blk)[3][3]) const {
    const int k = a == 0 ? b - 1 : a + b;   // local edge of (a, b)
    double* d = eb + int64_t(kEdgeRow) * __ldg(er + k);
    const bool tr = (flip >> k) & 1u;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) d[tr ? 3 * c + r : 3 * r + c] = blk[r][c];
  }
  __device__ __forceinline__ void rhs(int a, const double (&f)[3]) const {
    double2* d = reinterpret_cast<double2*>(nb + int64_t(kNodeRow) * __ldg(nr + a));
    d[0] = make_double2(f[0], f[1]);
    d[1] = make_double2(f[2], 0.0);
  }
  __device__ __forceinline__ void zero() const {
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      double2* d = reinterpret_cast<double2*>(nb + int64_t(kNodeRow) * __ldg(nr + a));
      d[0] = make_double2(0.0, 0.0);
      d[1] = make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      double* d = eb + int64_t(kEdgeRow) * __ldg(er + k);
#pragma unroll
      for (int q = 0; q < kEdgeRow; ++q) d[q] = 0.0;
    }
  }
};

// Stable Neo-Hookean element (Eq. 35, squared reading) from the deformation
// gradient F = Ds B (B = Dm^-1), with the gradient operator G_0 = -(B_0 + B_1 +
// B_2), G_{m+1} = B_m (rows of B), dF_ij / dx_{a,c} = delta_ic G_aj:
//   P = c1 F + c2 cof F,  c1 = mu (1 - w), c2 = lam (J - a), w = 1 / (I_C + 1);
//   f_a = -V P G_a = -V (c1 u_a + c2 z_a),  u_a = F G_a, z_a = cof(F) G_a;
//   K_ab = V [c1 (G_a . G_b) I + 2 mu w^2 u_a u_b^T + lam z_a z_b^T + c2 [t]_x],
//   t_m = det[G_a; G_b; F_m] (F_m row m of F), [t]_x (c, d) = eps_cdm t_m:
// the contraction of d2Psi/dF2 with G_a, G_b in closed form.  Output as the
// StVK body: the six off-diagonal blocks (a < b) of (dt beta + dt^2) chi K and
// the rhs shares dt chi (f_a - (beta + dt) (K v)_a).
__device__ __forceinline__ void elem_snh64(const DevMesh& m, const Material& mt, const StepScalars& sp, int64_t t,
                                           const int (&nid)[4], double chi) {
  const double dt = sp.dt, beta = mt.beta, mu = mt.mu, lam = mt.lam;
  const ElemRows64 out(m, t, nid);
  double Px[4][3], U[4][3];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    ld3(m.x, nid[a], Px[a]);
    ld3(m.v, nid[a], U[a]);
  }
  double B[9];
#pragma unroll
  for (int f = 0; f < 9; ++f) B[f] = m.rest[(kRestB + f) * m.T + t];
  const double V = m.rest[size_t(kRestV) * m.T + t];
  double G[4][3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    G[1][j] = B[j];
    G[2][j] = B[3 + j];
    G[3][j] = B[6 + j];
    G[0][j] = -(B[j] + B[3 + j] + B[6 + j]);
  }
  double F[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      F[i][j] = (Px[1][i] - Px[0][i]) * B[j] + (Px[2][i] - Px[0][i]) * B[3 + j] + (Px[3][i] - Px[0][i]) * B[6 + j];
  double cof[3][3];
  cof[0][0] = F[1][1] * F[2][2] - F[1][2] * F[2][1];
  cof[0][1] = F[1][2] * F[2][0] - F[1][0] * F[2][2];
  cof[0][2] = F[1][0] * F[2][1] - F[1][1] * F[2][0];
  cof[1][0] = F[0][2] * F[2][1] - F[0][1] * F[2][2];
  cof[1][1] = F[0][0] * F[2][2] - F[0][2] * F[2][0];
  cof[1][2] = F[0][1] * F[2][0] - F[0][0] * F[2][1];
  cof[2][0] = F[0][1] * F[1][2] - F[0][2] * F[1][1];
  cof[2][1] = F[0][2] * F[1][0] - F[0][0] * F[1][2];
  cof[2][2] = F[0][0] * F[1][1] - F[0][1] * F[1][0];
  const double J = F[0][0] * cof[0][0] + F[0][1] * cof[0][1] + F[0][2] * cof[0][2];
  double IC = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) IC += F[i][j] * F[i][j];
  const double w = 1.0 / (IC + 1.0);
  const double c1 = mu * (1.0 - w), c2 = lam * (J - mt.snh_a), c3 = 2.0 * mu * w * w;
  // the block scale (dt beta + dt^2) chi V is folded into the factors: blocks come out scaled
  const double sK = (dt * beta + dt * dt) * chi, sV = sK * V;
  const double k1 = sV * c1, k2 = sV * c2, k3 = sV * c3, k4 = sV * lam;
  double u[4][3], z[4][3], us[4][3], zs[4][3];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      u[a][c] = F[c][0] * G[a][0] + F[c][1] * G[a][1] + F[c][2] * G[a][2];
      z[a][c] = cof[c][0] * G[a][0] + cof[c][1] * G[a][1] + cof[c][2] * G[a][2];
      us[a][c] = k3 * u[a][c];
      zs[a][c] = k4 * z[a][c];
    }
  // Zero block-row sums (the energy depends on node differences only):
  // (K v)_a = sum_{b != a} K_ab (v_b - v_a); only the six off-diagonal blocks
  // are formed (k_diag64 forms the assembled diagonal blocks).
  double Kv[4][3] = {};
#pragma unroll
  for (int b = 1; b < 4; ++b)
#pragma unroll
    for (int a = 0; a < b; ++a) {
      const double gg = G[a][0] * G[b][0] + G[a][1] * G[b][1] + G[a][2] * G[b][2];
      double tm[3];
      {
        const double x0 = G[a][1] * G[b][2] - G[a][2] * G[b][1];
        const double x1 = G[a][2] * G[b][0] - G[a][0] * G[b][2];
        const double x2 = G[a][0] * G[b][1] - G[a][1] * G[b][0];
#pragma unroll
        for (int mm = 0; mm < 3; ++mm) tm[mm] = k2 * (x0 * F[mm][0] + x1 * F[mm][1] + x2 * F[mm][2]);
      }
      double blk[3][3];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) blk[r][c] = us[a][r] * u[b][c] + zs[a][r] * z[b][c];
      const double dg = k1 * gg;
      blk[0][0] += dg;
      blk[1][1] += dg;
      blk[2][2] += dg;
      blk[0][1] += tm[2];
      blk[1][0] -= tm[2];
      blk[0][2] -= tm[1];
      blk[2][0] += tm[1];
      blk[1][2] += tm[0];
      blk[2][1] -= tm[0];
      const double du[3] = {U[b][0] - U[a][0], U[b][1] - U[a][1], U[b][2] - U[a][2]};
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        Kv[a][r] += blk[r][0] * du[0] + blk[r][1] * du[1] + blk[r][2] * du[2];
        Kv[b][r] -= blk[0][r] * du[0] + blk[1][r] * du[1] + blk[2][r] * du[2];
      }
      out.block(a, b, blk);
    }
  // rhs shares dt chi (f_a - (beta + dt) (K v)_a): the blocks carry (dt beta + dt^2) chi = dt chi (beta + dt),
  // so the damping/velocity term is the scaled blocks' K v itself
  const double sf = dt * chi * V;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    double f[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) f[c] = -sf * (c1 * u[a][c] + c2 * z[a][c]) - Kv[a][c];
    out.rhs(a, f);
  }
}

__device__ __forceinline__ void elem64_body(const DevMesh& m, const Material& mt, const StepScalars& sp, unsigned bid, unsigned nb) {
  const double dt = sp.dt, beta = mt.beta;

  const int64_t t = bid * int64_t(blockDim.x) + threadIdx.x;
  if (t >= m.T) return;
  const int4 n = m.tets[t];
  const int nid[4] = {n.x, n.y, n.z, n.w};
  const ElemRows64 out(m, t, nid);
  const double chi = m.chi[t];
  if (chi == 0.0) {
    out.zero();
    return;
  }
  // The energy depends on node differences only, so every block row of the
  // tet's tangent sums to zero: only the six off-diagonal blocks are formed
  // (Y for b = 1..3), and k_diag64 forms the assembled diagonal blocks.
  const int inc[4][3] = {{0, 1, 2}, {0, 3, 4}, {1, 3, 5}, {2, 4, 5}};
  const double sgn[4][3] = {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {1, 1, 1}};
  const int kab[4][4] = {{-1, 0, 1, 2}, {0, -1, 3, 4}, {1, 3, -1, 5}, {2, 4, 5, -1}};
  double P[4][3], U[4][3];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    ld3(m.x, nid[a], P[a]);
    ld3(m.v, nid[a], U[a]);
  }
  double e[6][3], du[6][3], ds[6], Dv[6];   // edge vectors and edge velocity differences
#pragma unroll
  for (int k = 0; k < 6; ++k) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      e[k][c] = P[edge_b(k)][c] - P[edge_a(k)][c];
      du[k][c] = U[edge_b(k)][c] - U[edge_a(k)][c];
    }
    // summed in the order of the rest lengths' sums, so a tet at rest gives exactly 0
    ds[k] = e[k][0] * e[k][0] + e[k][1] * e[k][1] + e[k][2] * e[k][2] - m.rest[(kRestS0 + k) * m.T + t];
    // half the rate of change of the squared length (the factor 2 is taken with cv below)
    Dv[k] = e[k][0] * du[k][0] + e[k][1] * du[k][1] + e[k][2] * du[k][2];
  }
  double H[21];
#pragma unroll
  for (int f = 0; f < 21; ++f) H[f] = m.rest[(kRestH + f) * m.T + t];
  auto h = [&](int k, int l) { return k <= l ? H[tri6(k, l)] : H[tri6(l, k)]; };
  double g[6], w[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    double gk = 0.0, wk = 0.0;
#pragma unroll
    for (int l = 0; l < 6; ++l) {
      gk += h(k, l) * ds[l];
      wk += h(k, l) * Dv[l];
    }
    g[k] = gk;
    w[k] = wk;
  }
  {
    const double cv = beta + dt, cv2 = 2.0 * cv, sc = 2.0 * dt * chi;
    double f[4][3] = {};
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const double a1 = sc * (g[k] + cv2 * w[k]), a2 = sc * cv * g[k];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double tk = a1 * e[k][c] + a2 * du[k][c];
        f[edge_a(k)][c] += tk;
        f[edge_b(k)][c] -= tk;
      }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) out.rhs(a, f[a]);
  }
  const double sK = (dt * beta + dt * dt) * chi;
  double es[6][3];   // 4 sK e_l: the block scale taken once per edge, not once per Y entry
#pragma unroll
  for (int k = 0; k < 6; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) es[k][c] = 4.0 * sK * e[k][c];
#pragma unroll
  for (int b = 1; b < 4; ++b) {
    double Y[6][3];   // Y[k][c] = 4 sK sum_j H(k, l_j) sgn_bj e_{l_j}[c]
#pragma unroll
    for (int k = 0; k < 6; ++k)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        double y = 0.0;
#pragma unroll
        for (int j = 0; j < 3; ++j) y += sgn[b][j] * h(k, inc[b][j]) * es[inc[b][j]][c];
        Y[k][c] = y;
      }
#pragma unroll
    for (int a = 0; a < b; ++a) {
      // the geometric term -2 sK g_ab I starts the diagonal entries' sums
      const double geo = -2.0 * sK * g[kab[a][b]];
      double blk[3][3];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          double v = r == c ? geo : 0.0;
#pragma unroll
          for (int i = 0; i < 3; ++i) v += sgn[a][i] * e[inc[a][i]][r] * Y[inc[a][i]][c];
          blk[r][c] = v;
        }
      out.block(a, b, blk);
    }
  }
}
__device__ __forceinline__ void elem_snh64_body(const DevMesh& m, const Material& mt, const StepScalars& sp, unsigned bid,
                                                unsigned nb) {
  const int64_t t = bid * int64_t(blockDim.x) + threadIdx.x;
  if (t >= m.T) return;
  const int4 n = m.tets[t];
  const int nid[4] = {n.x, n.y, n.z, n.w};
  const double chi = m.chi[t];
  if (chi == 0.0) {
    ElemRows64(m, t, nid).zero();
    return;
  }
  elem_snh64(m, mt, sp, t, nid, chi);
}
__global__ void __launch_bounds__(kElemThreads64) k_elem64(DevMesh m, Material mt, StepScalars sp) {
  elem64_body(m, mt, sp, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(128) k_elem_snh64(DevMesh m, Material mt, StepScalars sp) {
  elem_snh64_body(m, mt, sp, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kElemThreads64) kb_elem64(const BatchTab* __restrict__ tab) {
  unsigned bid, nb;
  const int k = batch_locate(tab, kB_elem64, blockIdx.x, bid, nb);
  elem64_body(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb);   // batches run the StVK energy
}

// Phase 2 of the assembly: each off-diagonal matrix entry and rhs component is
// the sum, in ascending tet order, of its element contributions.  Threads
// [0, 9 NE) take one entry of an edge's block (the 4-6 tets around the edge,
// rows contiguous) and write it to both (i, j) and, transposed, (j, i);
// threads [9 NE, 9 NE + 3 N) take a node's rhs components (the ~24 tets around
// the node) and add the external force and mass damping of Eq. 2.
// Neighbouring threads read neighbouring values and sum lists of similar length.
__device__ __forceinline__ void gather64_body(const DevMesh& m, const Material& mt, const StepScalars& sp, unsigned bid, unsigned nb) {
  const double dt = sp.dt, alpha = mt.alpha;
  const int64_t t = bid * int64_t(blockDim.x) + threadIdx.x;
  const int64_t n_edge = 9 * m.NE;
  if (t < n_edge) {
    const int64_t g = t / 9;
    const int q = int(t - 9 * g);
    const int64_t e = m.edge_order[g];   // edges of equal row count side by side
    const double acc = row_sum<8>(m.ebuf + int64_t(kNodeRow) * 4 * m.T + q, kEdgeRow, m.et_ptr[e], m.et_ptr[e + 1]);
    const int2 sl = m.edge_slot[e];
    m.val[9 * int64_t(sl.x) + q] = acc;
    m.val[9 * int64_t(sl.y) + 3 * (q % 3) + q / 3] = acc;
    return;
  }
  const int64_t u = t - n_edge;
  if (u >= 3 * m.N) return;
  const int64_t g = u / 3;
  const int c3 = int(u - 3 * g);
  const int64_t i = m.node_order[g];
  const double acc = row_sum<8>(m.ebuf + c3, kNodeRow, m.np_ptr[i], m.np_ptr[i + 1]);
  const double* f_ext = sp.has_fext ? m.f_ext : nullptr;
  double mv = m.mass[i] * m.v[3 * i + c3];
  if (m.mass_blk) {   // consistent mass: (M v)_i over the row
    mv = 0.0;
    for (int b = m.row_ptr[i]; b < m.row_ptr[i + 1]; ++b) mv += m.mass_blk[b] * m.v[3 * int64_t(m.col[b]) + c3];
  }
  m.rhs[3 * i + c3] = acc + dt * ((f_ext ? f_ext[3 * i + c3] : 0.0) - alpha * mv);
}

// Phase 3: the diagonal blocks.  Every block row of the assembled stiffness
// sums to zero (each element's does: its energy depends on node differences
// only), so A_ii = -sum_{j != i} A_ij + the mass terms of Eq. 2 (lumped on the
// diagonal, or the consistent m_ij of Eq. 5 on every block of the row, added
// here after the sum).  Thread per (node, entry); a row's blocks are read in
// order (deterministic) and only its own thread writes them.
__device__ __forceinline__ void diag64_body(const DevMesh& m, const Material& mt, const StepScalars& sp, unsigned bid, unsigned nb) {
  const int64_t t = bid * int64_t(blockDim.x) + threadIdx.x;
  if (t >= 9 * m.N) return;
  const int64_t g = t / 9;
  const int q = int(t - 9 * g);
  const int64_t i = m.node_order[g];   // nodes of similar degree side by side
  const int d = m.diag_blk[i], b0 = m.row_ptr[i], b1 = m.row_ptr[i + 1];
  // the sum starts from the row's first off-diagonal block (none for a node
  // outside every tet)
  const int bf = b0 == d ? b0 + 1 : b0;
  double acc = bf < b1 ? m.val[9 * int64_t(bf) + q] : 0.0;
  for (int b = bf + 1; b < b1; ++b)
    if (b != d) acc += m.val[9 * int64_t(b) + q];
  double diag = -acc;
  const bool dg = q == 0 || q == 4 || q == 8;
  if (dg) {
    const double cm = (1.0 + sp.dt * mt.alpha) * sp.mscale;
    diag += cm * (m.mass_blk ? m.mass_blk[d] : m.mass[i]);
    if (m.mass_blk)
      for (int b = b0; b < b1; ++b)
        if (b != d) m.val[9 * int64_t(b) + q] += cm * m.mass_blk[b];
  }
  m.val[9 * int64_t(d) + q] = diag;
}
__global__ void __launch_bounds__(256) k_diag64(DevMesh m, Material mt, StepScalars sp) {
  diag64_body(m, mt, sp, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(256) kb_diag64(const BatchTab* __restrict__ tab) {
  unsigned bid, nb;
  const int k = batch_locate(tab, kB_diag64, blockIdx.x, bid, nb);
  diag64_body(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb);
}
__global__ void __launch_bounds__(256) k_gather64(DevMesh m, Material mt, StepScalars sp) {
  gather64_body(m, mt, sp, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(256) kb_gather64(const BatchTab* __restrict__ tab) {
  unsigned bid, nb;
  const int k = batch_locate(tab, kB_gather64, blockIdx.x, bid, nb);
  gather64_body(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb);
}

// Newton iterate k >= 1 (v^k = v + dv, the previous solve's total velocity
// change dv): positions xk = x + dt v^k for the element kernel, and the
// velocity w = v - dt v^k / (beta + dt) of its K v term, so that the assembled
// right-hand side is b(x^k, v) + dt^2 K(x^k) v^k and the unknown stays
// dv = v^{k+1} - v.
__global__ void __launch_bounds__(kThreads) k_newton_prep(int64_t n, const double* __restrict__ x,
                                                         const double* __restrict__ v, const double* __restrict__ dv,
                                                         double dt, double cw, double* xk, double* w) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  const double vk = v[i] + dv[i];
  xk[i] = x[i] + dt * vk;
  w[i] = v[i] - cw * vk;
}

// ---------------------------------------------------------------------------
// Quasi-static load step (Eq. 36; Newton with a line search, Sec. 4.3)
// ---------------------------------------------------------------------------

// E(x) = sum_e chi_e V_e Psi_e(x) - f_ext . x and sum |chi V Psi| + sum |f_i x_i|
// (the magnitude that sets E's rounding).  StVK: V Psi = 1/2 (s - s0)^T Hs (s - s0)
// exactly (Eq. 37 is quadratic in s, Hs includes V); SNH: V Psi(F) of Eq. 35.
__global__ void __launch_bounds__(kThreads) k_qs_energy(DevMesh m, Material mt, const double* __restrict__ x,
                                                       const double* __restrict__ f_ext, double* out) {
  double v[2] = {0.0, 0.0};
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < m.T; t += stride) {
    const double chi = m.chi[t];
    if (chi == 0.0) continue;
    const int4 n = m.tets[t];
    const int nid[4] = {n.x, n.y, n.z, n.w};
    double P[4][3];
#pragma unroll
    for (int a = 0; a < 4; ++a) ld3(x, nid[a], P[a]);
    double psi;
    if (mt.energy == GF_ENERGY_SNH) {
      double B[9];
#pragma unroll
      for (int f = 0; f < 9; ++f) B[f] = m.rest[(kRestB + f) * m.T + t];
      double F[3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
          F[i][j] = (P[1][i] - P[0][i]) * B[j] + (P[2][i] - P[0][i]) * B[3 + j] + (P[3][i] - P[0][i]) * B[6 + j];
      const double J = F[0][0] * (F[1][1] * F[2][2] - F[1][2] * F[2][1]) -
                       F[0][1] * (F[1][0] * F[2][2] - F[1][2] * F[2][0]) +
                       F[0][2] * (F[1][0] * F[2][1] - F[1][1] * F[2][0]);
      double IC = 0.0;
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) IC += F[i][j] * F[i][j];
      const double V = m.rest[size_t(kRestV) * m.T + t];
      psi = V * (0.5 * mt.mu * (IC - 3.0) + 0.5 * mt.lam * (J - mt.snh_a) * (J - mt.snh_a) -
                 0.5 * mt.mu * log(IC + 1.0));
    } else {
      double ds[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        double e2 = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const double e = P[edge_b(k)][c] - P[edge_a(k)][c];
          e2 += e * e;
        }
        ds[k] = e2 - m.rest[(kRestS0 + k) * m.T + t];
      }
      psi = 0.0;
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        double hk = 0.0;
#pragma unroll
        for (int l = 0; l < 6; ++l)
          hk += m.rest[(kRestH + (k <= l ? tri6(k, l) : tri6(l, k))) * m.T + t] * ds[l];
        psi += 0.5 * ds[k] * hk;
      }
    }
    v[0] += chi * psi;
    v[1] += fabs(chi * psi);
  }
  if (f_ext)
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < 3 * m.N; i += stride) {
      const double fx = f_ext[i] * x[i];
      v[0] -= fx;
      v[1] += fabs(fx);
    }
  double o[2];
  if (grid_reduce<2>(v, m.partials, m.tickets + 8, o, blockIdx.x, gridDim.x) && threadIdx.x == 0) {
    out[0] = o[0];
    out[1] = o[1];
  }
}

// r . d on free DOFs (the slope of E along the Newton direction d, r = -grad E)
__global__ void __launch_bounds__(kThreads) k_qs_slope(DevMesh m, double* out) {
  double v[1] = {0.0};
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < m.N; i += int64_t(gridDim.x) * blockDim.x)
    if (!m.pinned[i])
#pragma unroll
      for (int c = 0; c < 3; ++c) v[0] += m.rhs[3 * i + c] * m.dv[3 * i + c];
  double o[1];
  if (grid_reduce<1>(v, m.partials, m.tickets + 9, o, blockIdx.x, gridDim.x) && threadIdx.x == 0) out[2] = o[0];
}

__global__ void __launch_bounds__(kThreads) k_qs_trial(int64_t n, const double* __restrict__ x,
                                                      const double* __restrict__ d, double a, double* xt) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i < n) xt[i] = x[i] + a * d[i];
}

__global__ void __launch_bounds__(kThreads) k_qs_set_pins(DevMesh m, const int32_t* __restrict__ ids,
                                                         const double* __restrict__ pos, int64_t n_pinned) {
  const int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (p >= n_pinned) return;
  const int64_t id = ids[p];
  if (id < 0 || id >= m.N) return;   // reported by k_set_pinned
#pragma unroll
  for (int c = 0; c < 3; ++c) m.x[3 * id + c] = pos[3 * p + c];
}

// ---------------------------------------------------------------------------
// Projected block-Jacobi PCG (Sec. 4.3), all scalars on the device
// ---------------------------------------------------------------------------

__device__ __forceinline__ void spmv_row(const DevMesh& m, int64_t i, const double* __restrict__ x, double y[3]) {
  double y0 = 0.0, y1 = 0.0, y2 = 0.0;
  const int b1 = m.row_ptr[i + 1];
  for (int b = m.row_ptr[i]; b < b1; ++b) {
    const int64_t j = m.col[b];
    const double* a = m.val + 9 * int64_t(b);
    const double x0 = x[3 * j], x1 = x[3 * j + 1], x2 = x[3 * j + 2];
    // one FMA chain per output component: 9 FP64 instructions per block
    // (the grouped form y += (a0 x0 + a1 x1 + a2 x2) takes 12)
    y0 = fma(a[2], x2, fma(a[1], x1, fma(a[0], x0, y0)));
    y1 = fma(a[5], x2, fma(a[4], x1, fma(a[3], x0, y1)));
    y2 = fma(a[8], x2, fma(a[7], x1, fma(a[6], x0, y2)));
  }
  y[0] = y0;
  y[1] = y1;
  y[2] = y2;
}

__device__ __forceinline__ void set_pinned_body(const DevMesh& m, const Material& mt, const StepScalars& sp, unsigned bid, unsigned nb) {
  const int64_t n_pinned = sp.n_pinned;
  const double* pin_vel = sp.has_pvel ? m.pin_vel : nullptr;

  const int64_t p = bid * int64_t(blockDim.x) + threadIdx.x;
  if (p >= n_pinned) return;
  const int64_t id = m.pin_ids[p];
  if (id < 0 || id >= m.N) {
    atomicAdd(m.counters + 3, 1ull);   // reported as GF_BAD_ARG after the step
    return;
  }
  m.pinned[id] = 1;
#pragma unroll
  for (int c = 0; c < 3; ++c) m.dv[3 * id + c] = (pin_vel ? pin_vel[3 * p + c] : 0.0) - m.v[3 * id + c];
}
__global__ void __launch_bounds__(kThreads) k_set_pinned(DevMesh m, Material mt, StepScalars sp) {
  set_pinned_body(m, mt, sp, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kThreads) kb_set_pinned(const BatchTab* __restrict__ tab) {
  unsigned bid, nb;
  const int k = batch_locate(tab, kB_set_pinned, blockIdx.x, bid, nb);
  set_pinned_body(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb);
}

// r = b - A dv on free nodes, block-Jacobi inverse, z = P r, p = z; rz, rr.
// With sp.learned the preconditioner blocks and the start dv are the learned
// ones already in place, and the reference norm |b_free|^2 is kept from the
// plain initialisation that ran before them.
__device__ __forceinline__ void pcg_init_body(const DevMesh& m, const Material& mt, const StepScalars& sp, unsigned bid, unsigned nb) {

  double v[3] = {0.0, 0.0, 0.0};
  for (int64_t i = bid * int64_t(blockDim.x) + threadIdx.x; i < m.N; i += int64_t(nb) * blockDim.x) {
    double r[3] = {0, 0, 0}, z[3] = {0, 0, 0};
    if (!m.pinned[i] && sp.warm) {   // |b - A_fp dv_p|^2: the reference of a warm-started solve
      double bf[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) bf[c] = m.rhs[3 * i + c];
      for (int b = m.row_ptr[i]; b < m.row_ptr[i + 1]; ++b) {
        const int64_t j = m.col[b];
        if (!m.pinned[j]) continue;
        const double* a = m.val + 9 * int64_t(b);
#pragma unroll
        for (int c = 0; c < 3; ++c)
          bf[c] -= a[3 * c] * m.dv[3 * j] + a[3 * c + 1] * m.dv[3 * j + 1] + a[3 * c + 2] * m.dv[3 * j + 2];
      }
      v[2] += bf[0] * bf[0] + bf[1] * bf[1] + bf[2] * bf[2];
    }
    if (!m.pinned[i] && sp.learned) {
      double ad[3];
      spmv_row(m, i, m.dv, ad);
#pragma unroll
      for (int c = 0; c < 3; ++c) r[c] = m.rhs[3 * i + c] - ad[c];
      const double* pi = m.pinv + 9 * i;
#pragma unroll
      for (int c = 0; c < 3; ++c) z[c] = pi[3 * c] * r[0] + pi[3 * c + 1] * r[1] + pi[3 * c + 2] * r[2];
    } else if (!m.pinned[i]) {
      // every caller zeroes dv before k_set_pinned, so without pinned nodes and
      // without a warm start dv is exactly zero: A dv = 0 and b - 0 = b, and the
      // product is skipped (same bits)
      double ad[3] = {0.0, 0.0, 0.0};
      if (sp.n_pinned > 0 || sp.warm) spmv_row(m, i, m.dv, ad);
#pragma unroll
      for (int c = 0; c < 3; ++c) r[c] = m.rhs[3 * i + c] - ad[c];
      const double* a = m.val + 9 * int64_t(m.diag_blk[i]);
      const double c00 = a[4] * a[8] - a[5] * a[7], c01 = a[2] * a[7] - a[1] * a[8], c02 = a[1] * a[5] - a[2] * a[4];
      const double c10 = a[5] * a[6] - a[3] * a[8], c11 = a[0] * a[8] - a[2] * a[6], c12 = a[2] * a[3] - a[0] * a[5];
      const double c20 = a[3] * a[7] - a[4] * a[6], c21 = a[1] * a[6] - a[0] * a[7], c22 = a[0] * a[4] - a[1] * a[3];
      // a node with no stiffness and no mass (every tet around it at chi = 0 in a
      // quasi-static solve) has a zero block: a zero inverse keeps it in place
      const double det = a[0] * c00 + a[1] * c10 + a[2] * c20;
      const double id = det != 0.0 ? 1.0 / det : 0.0;
      double* pi = m.pinv + 9 * i;
      const double inv[9] = {c00 * id, c01 * id, c02 * id, c10 * id, c11 * id, c12 * id, c20 * id, c21 * id, c22 * id};
#pragma unroll
      for (int k = 0; k < 9; ++k) pi[k] = inv[k];
#pragma unroll
      for (int c = 0; c < 3; ++c) z[c] = inv[3 * c] * r[0] + inv[3 * c + 1] * r[1] + inv[3 * c + 2] * r[2];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      m.r[3 * i + c] = r[c];
      m.z[3 * i + c] = z[c];
      m.p[3 * i + c] = z[c];
      v[0] += r[c] * z[c];
      v[1] += r[c] * r[c];
    }
  }
  double out[3];
  if (grid_reduce<3>(v, m.partials, m.tickets + 0, out, bid, nb) && threadIdx.x == 0) {
    PcgState* s = m.pcg;
    s->rz = out[0];
    s->rr = out[1];
    s->rr0 = out[1];
    if (sp.warm) s->bb = out[2];
    else if (!sp.learned) s->bb = out[1];
    s->iters = 0;
    s->status = GF_OK;
    s->done = (out[1] == 0.0 || out[1] <= s->tol2 * s->bb) ? 1 : 0;
    if (!isfinite(out[1])) {
      s->status = GF_NAN;
      s->done = 1;
    }
  }
}
__global__ void __launch_bounds__(kThreads) k_pcg_init(DevMesh m, Material mt, StepScalars sp) {
  pcg_init_body(m, mt, sp, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kThreads) kb_pcg_init(const BatchTab* __restrict__ tab) {
  unsigned bid, nb;
  const int k = batch_locate(tab, kB_pcg_init, blockIdx.x, bid, nb);
  pcg_init_body(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb);
}

// q = A p; pq = p . q; alpha = rz / pq (breakdown when pq <= 0)
__device__ __forceinline__ void pcg_spmv_body(const DevMesh& m, const Material& mt, const StepScalars& sp, unsigned bid, unsigned nb) {

  if (m.pcg->done) return;
  double v[1] = {0.0};
  for (int64_t i = bid * int64_t(blockDim.x) + threadIdx.x; i < m.N; i += int64_t(nb) * blockDim.x) {
    double y[3];
    spmv_row(m, i, m.p, y);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      m.q[3 * i + c] = y[c];
      v[0] += m.p[3 * i + c] * y[c];
    }
  }
  double out[1];
  if (grid_reduce<1>(v, m.partials, m.tickets + 1, out, bid, nb) && threadIdx.x == 0) {
    PcgState* s = m.pcg;
    s->pq = out[0];
    if (!(out[0] > 0.0)) {
      s->status = isfinite(out[0]) ? GF_CG_BREAKDOWN : GF_NAN;
      s->done = 1;
    } else {
      s->alpha = s->rz / out[0];
    }
  }
}
__global__ void __launch_bounds__(kThreads) k_pcg_spmv(DevMesh m, Material mt, StepScalars sp) {
  pcg_spmv_body(m, mt, sp, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kThreads) kb_pcg_spmv(const BatchTab* __restrict__ tab) {
  unsigned bid, nb;
  const int k = batch_locate(tab, kB_pcg_spmv, blockIdx.x, bid, nb);
  pcg_spmv_body(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb);
}

// dv += alpha p; r -= alpha q; z = P r; rz_new, rr; convergence test
__device__ __forceinline__ void pcg_update_body(const DevMesh& m, const Material& mt, const StepScalars& sp, unsigned bid, unsigned nb) {

  if (m.pcg->done) return;
  const double alpha = m.pcg->alpha;
  double v[2] = {0.0, 0.0};
  for (int64_t i = bid * int64_t(blockDim.x) + threadIdx.x; i < m.N; i += int64_t(nb) * blockDim.x) {
    if (m.pinned[i]) continue;
    // every load before the first store (the vectors may alias as far as the
    // compiler knows)
    double dv[3], p[3], r[3], q[3], pi[9];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      dv[c] = m.dv[3 * i + c];
      p[c] = m.p[3 * i + c];
      r[c] = m.r[3 * i + c];
      q[c] = m.q[3 * i + c];
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) pi[k] = m.pinv[9 * i + k];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      m.dv[3 * i + c] = dv[c] + alpha * p[c];
      r[c] = r[c] - alpha * q[c];
      m.r[3 * i + c] = r[c];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double z = pi[3 * c] * r[0] + pi[3 * c + 1] * r[1] + pi[3 * c + 2] * r[2];
      m.z[3 * i + c] = z;
      v[0] += r[c] * z;
      v[1] += r[c] * r[c];
    }
  }
  double out[2];
  if (grid_reduce<2>(v, m.partials, m.tickets + 2, out, bid, nb) && threadIdx.x == 0) {
    PcgState* s = m.pcg;
    s->iters += 1;
    s->beta = out[0] / s->rz;
    s->rz = out[0];
    s->rr = out[1];
    if (!isfinite(out[1])) {
      s->status = GF_NAN;
      s->done = 1;
    } else if (out[1] <= s->tol2 * s->bb) {
      s->done = 1;
    } else if (s->iters >= s->maxit) {
      s->status = GF_CG_MAXITER;
      s->done = 1;
    }
  }
}
__global__ void __launch_bounds__(kThreads) k_pcg_update(DevMesh m, Material mt, StepScalars sp) {
  pcg_update_body(m, mt, sp, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kThreads) kb_pcg_update(const BatchTab* __restrict__ tab) {
  unsigned bid, nb;
  const int k = batch_locate(tab, kB_pcg_update, blockIdx.x, bid, nb);
  pcg_update_body(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb);
}

__device__ __forceinline__ void pcg_p_body(const DevMesh& m, const Material& mt, const StepScalars& sp, unsigned bid, unsigned nb) {

  if (m.pcg->done) return;
  const double beta = m.pcg->beta;
  for (int64_t i = bid * int64_t(blockDim.x) + threadIdx.x; i < 3 * m.N; i += int64_t(nb) * blockDim.x)
    m.p[i] = m.z[i] + beta * m.p[i];
}
__global__ void __launch_bounds__(kThreads) k_pcg_p(DevMesh m, Material mt, StepScalars sp) {
  pcg_p_body(m, mt, sp, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kThreads) kb_pcg_p(const BatchTab* __restrict__ tab) {
  unsigned bid, nb;
  const int k = batch_locate(tab, kB_pcg_p, blockIdx.x, bid, nb);
  pcg_p_body(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb);
}

// Quasi-static inner solve: the same projected block-Jacobi PCG in the
// Chronopoulos-Gear form (Chronopoulos & Gear, J. Comput. Appl. Math. 25, 1989),
// whose Krylov iterates equal the three-kernel form's in exact arithmetic but
// which needs one grid reduction per iteration instead of two.  With w = A z,
// gamma = r.z and delta = z.w: beta = gamma / gamma_old, p.A.p = delta -
// beta gamma / alpha_old, alpha = gamma / p.A.p, and q = A p follows the
// recurrence q = w + beta q.  k_qs_cg_spmv forms w and the three dots and sets
// the coefficients in its last CTA; k_qs_cg_update streams the vector updates
// with no reduction.  The mass-free quasi-static system takes hundreds of
// iterations per Newton iteration, so a reduction and a launch saved per
// iteration add up.
__global__ void __launch_bounds__(kThreads) k_qs_cg_spmv(DevMesh m) {
  PcgState* S = m.pcg;
  if (S->done) return;   // set only by a last CTA, after every CTA has passed here
  double v[3] = {0.0, 0.0, 0.0};
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < m.N; i += int64_t(gridDim.x) * blockDim.x) {
    double y[3];
    spmv_row(m, i, m.z, y);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double z = m.z[3 * i + c], r = m.r[3 * i + c];
      m.w[3 * i + c] = y[c];
      v[0] += r * z;      // z and r are zero on pinned rows
      v[1] += z * y[c];
      v[2] += r * r;
    }
  }
  double out[3];
  if (grid_reduce<3>(v, m.partials, m.tickets + 10, out, blockIdx.x, gridDim.x) && threadIdx.x == 0) {
    const int k = S->cg_k;   // updates applied so far
    S->cg_k = k + 1;
    S->iters = k;
    S->rr = out[2];
    const double gamma = out[0], delta = out[1];
    const double beta = k > 0 ? gamma / S->rz : 0.0;
    const double den = k > 0 ? delta - beta * gamma / S->alpha : delta;   // p.A.p
    if (!isfinite(out[2]) || !isfinite(delta)) {
      S->status = GF_NAN;
      S->done = 1;
    } else if (out[2] <= S->tol2 * S->bb) {
      S->done = 1;
    } else if (k >= S->maxit) {
      S->status = GF_CG_MAXITER;
      S->done = 1;
    } else if (!(den > 0.0)) {
      S->status = GF_CG_BREAKDOWN;
      S->done = 1;
    } else {
      S->beta = beta;
      S->alpha = gamma / den;
      S->rz = gamma;
      S->pq = den;
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_qs_cg_update(DevMesh m) {
  const PcgState* S = m.pcg;
  if (S->done) return;
  const double alpha = S->alpha, beta = S->beta;
  const bool first = S->cg_k == 1;   // p = z, q = w
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < m.N; i += int64_t(gridDim.x) * blockDim.x) {
    // every load first (the vectors may alias as far as the compiler knows);
    // p' and q' are not used on the first iteration, dv, r and the inverse not
    // on pinned rows
    const bool fixed = m.pinned[i];
    double zo[3], w[3], po[3], qo[3], dv[3], r[3], pi[9];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      zo[c] = m.z[3 * i + c];
      w[c] = m.w[3 * i + c];
      po[c] = m.p[3 * i + c];
      qo[c] = m.q[3 * i + c];
      dv[c] = m.dv[3 * i + c];
      r[c] = m.r[3 * i + c];
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) pi[k] = m.pinv[9 * i + k];
    double p[3], q[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      p[c] = first ? zo[c] : zo[c] + beta * po[c];
      q[c] = first ? w[c] : w[c] + beta * qo[c];
      m.p[3 * i + c] = p[c];
      m.q[3 * i + c] = q[c];
    }
    if (fixed) continue;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      m.dv[3 * i + c] = dv[c] + alpha * p[c];
      r[c] = r[c] - alpha * q[c];
      m.r[3 * i + c] = r[c];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) m.z[3 * i + c] = pi[3 * c] * r[0] + pi[3 * c + 1] * r[1] + pi[3 * c + 2] * r[2];
  }
}

// Quasi-static solve with an FP32 inner solve (GF_QS_SOLVE_NESTED; FP64
// meshes): flexible PCG in FP64 (Notay, SIAM J. Sci. Comput. 22, 2000; one
// previous direction kept) whose preconditioner is an inner PCG in FP32 on the
// matrix and block-Jacobi inverses rounded to FP32 (the mixed step's two-kernel
// inner iterations, on m.mx), run until its residual falls by the inner
// tolerance.  With z the inner solution for the outer residual r, w = A z and
// the previous direction p' (q' = A p'):
//   beta = z.q' / p'.q',  p = z - beta p',  q = w - beta q' (= A p),
//   p.q = z.w - 2 beta z.q' + beta^2 p'.q' (A symmetric),  alpha = p.r / p.q,
//   dv += alpha p,  r -= alpha q.
// The outer residual, iterate and coefficients are FP64, and the iteration
// stops at |r| <= cg_rtol |b| like the FP64 PCG.  Outer scalars live in m.pcg,
// the inner ones in m.mx.ir; ir->done ends both.

// val32 = fl(val), pinv32 = fl(pinv): once per Newton iteration, after the FP64
// assembly and block-Jacobi inverses
__global__ void __launch_bounds__(kThreads) k_qsr_to32(DevMesh m) {
  const int64_t nv = 9 * m.NB, stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < nv; k += stride) m.mx.val32[k] = float(m.val[k]);
  for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < 9 * m.N; k += stride)
    m.mx.pinv32[k] = float(m.pinv[k]);
}

// Inner start on row i from the outer residual r (zero on pinned rows), scaled
// by sc = 1 / |r_prev| so that the FP32 solve and its double-float sums work on
// values near 1 whatever the outer residual has fallen to (the flexible PCG is
// invariant to a scaling of the preconditioner's output): r32 = fl(sc r),
// z = P32 r32 (into z4, the two-kernel inner form's z), d32 = 0; adds
// r32 . z and r32 . r32 to g and n (exact products of floats, summed in FP64)
__device__ __forceinline__ void inner_start_row(const DevMesh& m, int64_t i, const double r[3], double sc, double& g,
                                                double& n) {
  const MixDev& x = m.mx;
  float r32[3], z32[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) r32[c] = float(sc * r[c]);
  const float* pi = x.pinv32 + 9 * i;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    z32[c] = pi[3 * c] * r32[0] + pi[3 * c + 1] * r32[1] + pi[3 * c + 2] * r32[2];
    g += double(r32[c]) * double(z32[c]);
    n += double(r32[c]) * double(r32[c]);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    x.r32[3 * i + c] = r32[c];
    x.d32[3 * i + c] = 0.f;
  }
  x.z4[i] = make_float4(z32[0], z32[1], z32[2], 0.f);
}

// the last CTA's bookkeeping after a new outer residual: the outer test, then
// the inner solve's start (reference |r32|^2, gamma, no iterations yet)
__device__ __forceinline__ void outer_residual_done(IrState* S, double rr, double gamma, double rr32, bool first) {
  if (first) {
    S->sweeps = 0;
    S->total_iters = 0;
    S->status = GF_OK;
  } else {
    S->sweeps += 1;
  }
  S->rr = rr;
  S->done = (rr == 0.0 || rr <= S->tol2 * S->bb) ? 1 : 0;
  if (!isfinite(rr) || !isfinite(gamma)) {
    S->status = GF_NAN;
    S->done = 1;
  } else if (!S->done && S->total_iters >= S->maxit) {
    S->status = GF_CG_MAXITER;
    S->done = 1;
  }
  S->in_rr0 = rr32;
  S->in_iters = 0;
  S->rz = gamma;
  S->in_done = (S->done || gamma == 0.0) ? 1 : 0;
}

// first inner start, from the residual r = b - A dv that k_pcg_init left in m.r
// (dv = 0, or a warm start), with the reference |b|^2 it left in m.pcg
__global__ void __launch_bounds__(kThreads) k_qsr_start(DevMesh m) {
  const double bb = m.pcg->bb, rr0 = m.pcg->rr;
  const double sc = rr0 > 0.0 ? 1.0 / sqrt(rr0) : 1.0;
  double v[3] = {0.0, 0.0, 0.0};
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < m.N; i += int64_t(gridDim.x) * blockDim.x) {
    double r[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      r[c] = m.r[3 * i + c];
      v[0] += r[c] * r[c];
    }
    inner_start_row(m, i, r, sc, v[1], v[2]);
  }
  double out[3];
  if (grid_reduce<3>(v, m.partials, m.tickets + 13, out, blockIdx.x, gridDim.x) && threadIdx.x == 0) {
    m.mx.ir->bb = bb;
    outer_residual_done(m.mx.ir, out[0], out[1], out[2], true);
  }
}

// the nested solve's outcome in the PCG state the step reads: iterations (inner),
// status, done
__global__ void k_nested_finish(DevMesh m) {
  if (threadIdx.x != 0) return;
  const IrState* S = m.mx.ir;
  m.pcg->iters = S->total_iters;
  m.pcg->status = S->done ? S->status : GF_CG_MAXITER;
  m.pcg->rr = S->rr;
  m.pcg->done = 1;
}

// z = fl64(d32) (the inner solution; zero on pinned rows), w = A z, and z.q',
// z.w, z.r, p'.r; the last CTA forms beta, p.q and alpha.  Runs only once the
// inner solve has finished (a graph body launches it after every group of
// inner iterations); the first outer iteration is the one with no sweep yet.
__global__ void __launch_bounds__(kThreads) k_fcg_spmv(DevMesh m) {
  const IrState* S = m.mx.ir;
  if (S->done || !S->in_done) return;
  const bool first = S->sweeps == 0;
  const float* __restrict__ d32 = m.mx.d32;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < m.N; i += int64_t(gridDim.x) * blockDim.x) {
    double y0 = 0.0, y1 = 0.0, y2 = 0.0;
    const int b1 = m.row_ptr[i + 1];
    for (int b = m.row_ptr[i]; b < b1; ++b) {
      const int64_t j = m.col[b];
      const double* a = m.val + 9 * int64_t(b);
      const double x0 = d32[3 * j], x1 = d32[3 * j + 1], x2 = d32[3 * j + 2];
      y0 = fma(a[2], x2, fma(a[1], x1, fma(a[0], x0, y0)));
      y1 = fma(a[5], x2, fma(a[4], x1, fma(a[3], x0, y1)));
      y2 = fma(a[8], x2, fma(a[7], x1, fma(a[6], x0, y2)));
    }
    const double y[3] = {y0, y1, y2};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double z = d32[3 * i + c], r = m.r[3 * i + c];
      m.z[3 * i + c] = z;
      m.w[3 * i + c] = y[c];
      v[1] += z * y[c];
      v[2] += z * r;
      if (!first) {
        v[0] += z * m.q[3 * i + c];
        v[3] += m.p[3 * i + c] * r;
      }
    }
  }
  double out[4];
  if (grid_reduce<4>(v, m.partials, m.tickets + 14, out, blockIdx.x, gridDim.x) && threadIdx.x == 0) {
    IrState* I = m.mx.ir;
    PcgState* P = m.pcg;
    const double beta = first ? 0.0 : out[0] / P->pq;
    const double pq = first ? out[1] : out[1] - 2.0 * beta * out[0] + beta * beta * P->pq;
    const double pr = first ? out[2] : out[2] - beta * out[3];
    if (!isfinite(pq) || !isfinite(pr)) {
      I->status = GF_NAN;
      I->done = 1;
    } else if (!(pq > 0.0)) {
      I->status = GF_CG_BREAKDOWN;
      I->done = 1;
    } else {
      P->beta = beta;
      P->pq = pq;
      P->alpha = pr / pq;
    }
  }
}

// p = z - beta p', q = w - beta q', dv += alpha p, r -= alpha q on free rows,
// then the next inner start from the new r, |r|^2 and the outer test (which
// counts the sweep and clears in_done: the flags are read by every CTA first)
__global__ void __launch_bounds__(kThreads) k_fcg_update(DevMesh m) {
  if (m.mx.ir->done || !m.mx.ir->in_done) return;
  const bool first = m.mx.ir->sweeps == 0;
  const double alpha = m.pcg->alpha, beta = m.pcg->beta;
  const double rr_prev = m.mx.ir->rr;   // written again only by this launch's last CTA
  const double sc = rr_prev > 0.0 ? 1.0 / sqrt(rr_prev) : 1.0;
  double v[3] = {0.0, 0.0, 0.0};
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < m.N; i += int64_t(gridDim.x) * blockDim.x) {
    double r[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double p = first ? m.z[3 * i + c] : m.z[3 * i + c] - beta * m.p[3 * i + c];
      const double q = first ? m.w[3 * i + c] : m.w[3 * i + c] - beta * m.q[3 * i + c];
      m.p[3 * i + c] = p;
      m.q[3 * i + c] = q;
      r[c] = 0.0;
      if (!m.pinned[i]) {
        m.dv[3 * i + c] += alpha * p;
        r[c] = m.r[3 * i + c] - alpha * q;
      }
      m.r[3 * i + c] = r[c];
      v[0] += r[c] * r[c];
    }
    inner_start_row(m, i, r, sc, v[1], v[2]);
  }
  double out[3];
  if (grid_reduce<3>(v, m.partials, m.tickets + 15, out, blockIdx.x, gridDim.x) && threadIdx.x == 0)
    outer_residual_done(m.mx.ir, out[0], out[1], out[2], false);
}

// ||b - A dv||^2 over free nodes, recomputed from scratch after the solve.
__device__ __forceinline__ void true_residual_body(const DevMesh& m, const Material& mt, const StepScalars& sp, unsigned bid, unsigned nb) {

  double v[1] = {0.0};
  for (int64_t i = bid * int64_t(blockDim.x) + threadIdx.x; i < m.N; i += int64_t(nb) * blockDim.x) {
    if (m.pinned[i]) continue;
    double y[3];
    spmv_row(m, i, m.dv, y);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double r = m.rhs[3 * i + c] - y[c];
      v[0] += r * r;
    }
  }
  double out[1];
  if (grid_reduce<1>(v, m.partials, m.tickets + 3, out, bid, nb) && threadIdx.x == 0) m.pcg->true_rr = out[0];
}
__global__ void __launch_bounds__(kThreads) k_true_residual(DevMesh m, Material mt, StepScalars sp) {
  true_residual_body(m, mt, sp, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kThreads) kb_true_residual(const BatchTab* __restrict__ tab) {
  unsigned bid, nb;
  const int k = batch_locate(tab, kB_true_residual, blockIdx.x, bid, nb);
  true_residual_body(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb);
}

__device__ __forceinline__ void integrate_body(const DevMesh& m, const Material& mt, const StepScalars& sp, unsigned bid, unsigned nb) {
  const double dt = sp.dt;

  const int64_t i = bid * int64_t(blockDim.x) + threadIdx.x;
  if (i >= 3 * m.N) return;
  const double v = m.v[i] + m.dv[i];
  m.v[i] = v;
  m.x[i] += dt * v;
}
__global__ void __launch_bounds__(kThreads) k_integrate(DevMesh m, Material mt, StepScalars sp) {
  integrate_body(m, mt, sp, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kThreads) kb_integrate(const BatchTab* __restrict__ tab) {
  unsigned bid, nb;
  const int k = batch_locate(tab, kB_integrate, blockIdx.x, bid, nb);
  integrate_body(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb);
}

// Distributed solver-loop kernels of a batch (see the mixed ones).
#define GF_DIST_KERNEL(name, kind, body)                                                               \
  __global__ void __launch_bounds__(kThreads) name(const BatchTab* __restrict__ tab, const BatchAct* __restrict__ act) { \
    const int total = act->off[kind][act->n];                                                          \
    for (int w = blockIdx.x; w < total; w += gridDim.x) {                                              \
      unsigned bid, nb;                                                                                \
      const int k = act_locate(act, kind, unsigned(w), bid, nb);                                       \
      body;                                                                                            \
      __syncthreads();                                                                                 \
    }                                                                                                  \
  }
GF_DIST_KERNEL(kd_pcg_spmv, kB_pcg_spmv, pcg_spmv_body(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb))
GF_DIST_KERNEL(kd_pcg_update, kB_pcg_update, pcg_update_body(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb))
GF_DIST_KERNEL(kd_pcg_p, kB_pcg_p, pcg_p_body(tab->mesh[k], tab->mt[k], tab->sp[k], bid, nb))
#undef GF_DIST_KERNEL

}  // namespace

// Quasi-static kernels: grid-stride over at most four CTAs per SM of the
// current device (and never more CTAs than the reduction partials hold).
inline unsigned qs_grid(int64_t n) {
  static int sm_count[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  int& sms = sm_count[dev & 63];
  if (sms == 0 && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sms = 152;
  const int64_t cap = std::min<int64_t>(4 * int64_t(sms), kMaxPartials);
  const int64_t b = (n + kThreads - 1) / kThreads;
  return unsigned(b < 1 ? 1 : (b > cap ? cap : b));
}
int launch_qs_energy(const DevMesh& m, const Material& mt, const double* x, const double* f_ext, double* out,
                     cudaStream_t s) {
  k_qs_energy<<<qs_grid(std::max(m.T, 3 * m.N)), kThreads, 0, s>>>(m, mt, x, f_ext, out);
  return 1;
}
int launch_qs_slope(const DevMesh& m, double* out, cudaStream_t s) {
  k_qs_slope<<<qs_grid(m.N), kThreads, 0, s>>>(m, out);
  return 1;
}
int launch_qs_cg_spmv(const DevMesh& m, cudaStream_t s) {
  k_qs_cg_spmv<<<qs_grid(m.N), kThreads, 0, s>>>(m);
  return 1;
}
int launch_qs_cg_update(const DevMesh& m, cudaStream_t s) {
  k_qs_cg_update<<<qs_grid(m.N), kThreads, 0, s>>>(m);
  return 1;
}
int launch_qsr_to32(const DevMesh& m, cudaStream_t s) {
  k_qsr_to32<<<qs_grid(9 * m.NB), kThreads, 0, s>>>(m);
  return 1;
}
int launch_qsr_start(const DevMesh& m, cudaStream_t s) {
  k_qsr_start<<<qs_grid(m.N), kThreads, 0, s>>>(m);
  return 1;
}
int launch_nested_finish(const DevMesh& m, cudaStream_t s) {
  k_nested_finish<<<1, 32, 0, s>>>(m);
  return 1;
}
int launch_fcg_spmv(const DevMesh& m, cudaStream_t s) {
  k_fcg_spmv<<<qs_grid(m.N), kThreads, 0, s>>>(m);
  return 1;
}
int launch_fcg_update(const DevMesh& m, cudaStream_t s) {
  k_fcg_update<<<qs_grid(m.N), kThreads, 0, s>>>(m);
  return 1;
}
int launch_qs_trial(int64_t n, const double* x, const double* d, double a, double* xt, cudaStream_t s) {
  k_qs_trial<<<unsigned((n + kThreads - 1) / kThreads), kThreads, 0, s>>>(n, x, d, a, xt);
  return 1;
}
int launch_qs_set_pins(const DevMesh& m, const int32_t* ids, const double* pos, int64_t n_pinned, cudaStream_t s) {
  if (n_pinned <= 0) return 0;
  k_qs_set_pins<<<unsigned((n_pinned + kThreads - 1) / kThreads), kThreads, 0, s>>>(m, ids, pos, n_pinned);
  return 1;
}

int launch_newton_prep(const DevMesh& m, const Material& mt, double dt, double* xk, double* w, cudaStream_t s) {
  const int64_t n = 3 * m.N;
  const double cw = dt / (mt.beta + dt);
  k_newton_prep<<<unsigned((n + kThreads - 1) / kThreads), kThreads, 0, s>>>(n, m.x, m.v, m.dv, dt, cw, xk, w);
  return 1;
}

int launch_assemble_colour(const DevMesh& m, const Material& mt, double dt, int t0, int t1, cudaStream_t s) {
  if (t1 <= t0) return 0;
  k_assemble<<<unsigned((t1 - t0 + 127) / 128), 128, 0, s>>>(m, dt, mt.beta, t0, t1);
  return 1;
}

// launches of the kinds implemented in this file
int launch_kind_fp64(int kind, const DevMesh& m, const Material& mt, const StepScalars& sp, cudaStream_t s) {
  const LaunchDims d = launch_dims(kind, m, mt, sp);
  if (d.blocks == 0) return 0;
  switch (kind) {
    case kB_tet_stress:
      if (mt.energy == GF_ENERGY_SNH) k_tet_stress_snh<<<d.blocks, d.threads, 0, s>>>(m, mt, sp);
      else k_tet_stress<<<d.blocks, d.threads, 0, s>>>(m, mt, sp);
      break;
    case kB_nonlocal: k_nonlocal<<<d.blocks, d.threads, 0, s>>>(m, mt, sp); break;
    case kB_edge_driver: k_edge_driver<<<d.blocks, d.threads, 0, s>>>(m, mt, sp); break;
    case kB_tet_chi:
      if (mt.energy == GF_ENERGY_SNH) k_tet_chi_snh<<<d.blocks, d.threads, 0, s>>>(m, mt, sp);
      else k_tet_chi<<<d.blocks, d.threads, 0, s>>>(m, mt, sp);
      break;
    case kB_node_init: k_node_init<<<d.blocks, d.threads, 0, s>>>(m, mt, sp); break;
    case kB_elem64:
      if (mt.energy == GF_ENERGY_SNH) k_elem_snh64<<<d.blocks, d.threads, 0, s>>>(m, mt, sp);
      else k_elem64<<<d.blocks, d.threads, 0, s>>>(m, mt, sp);
      break;
    case kB_gather64: k_gather64<<<d.blocks, d.threads, 0, s>>>(m, mt, sp); break;
    case kB_diag64: k_diag64<<<d.blocks, d.threads, 0, s>>>(m, mt, sp); break;
    case kB_set_pinned: k_set_pinned<<<d.blocks, d.threads, 0, s>>>(m, mt, sp); break;
    case kB_pcg_init: k_pcg_init<<<d.blocks, d.threads, 0, s>>>(m, mt, sp); break;
    case kB_pcg_spmv: k_pcg_spmv<<<d.blocks, d.threads, 0, s>>>(m, mt, sp); break;
    case kB_pcg_update: k_pcg_update<<<d.blocks, d.threads, 0, s>>>(m, mt, sp); break;
    case kB_pcg_p: k_pcg_p<<<d.blocks, d.threads, 0, s>>>(m, mt, sp); break;
    case kB_true_residual: k_true_residual<<<d.blocks, d.threads, 0, s>>>(m, mt, sp); break;
    case kB_integrate: k_integrate<<<d.blocks, d.threads, 0, s>>>(m, mt, sp); break;
    default: return -1;
  }
  return 1;
}

int launch_dist_fp64(int kind, const BatchTab* tab, const BatchAct* act, unsigned grid, cudaStream_t s) {
  switch (kind) {
    case kB_pcg_spmv: kd_pcg_spmv<<<grid, kThreads, 0, s>>>(tab, act); break;
    case kB_pcg_update: kd_pcg_update<<<grid, kThreads, 0, s>>>(tab, act); break;
    case kB_pcg_p: kd_pcg_p<<<grid, kThreads, 0, s>>>(tab, act); break;
    default: return 0;
  }
  return 1;
}

int launch_batch_fp64(int kind, const BatchTab* tab, unsigned blocks, unsigned threads, cudaStream_t s) {
  if (blocks == 0) return 0;
  switch (kind) {
    case kB_tet_stress: kb_tet_stress<<<blocks, threads, 0, s>>>(tab); break;
    case kB_nonlocal: kb_nonlocal<<<blocks, threads, 0, s>>>(tab); break;
    case kB_edge_driver: kb_edge_driver<<<blocks, threads, 0, s>>>(tab); break;
    case kB_tet_chi: kb_tet_chi<<<blocks, threads, 0, s>>>(tab); break;
    case kB_node_init: kb_node_init<<<blocks, threads, 0, s>>>(tab); break;
    case kB_elem64: kb_elem64<<<blocks, threads, 0, s>>>(tab); break;
    case kB_gather64: kb_gather64<<<blocks, threads, 0, s>>>(tab); break;
    case kB_diag64: kb_diag64<<<blocks, threads, 0, s>>>(tab); break;
    case kB_set_pinned: kb_set_pinned<<<blocks, threads, 0, s>>>(tab); break;
    case kB_pcg_init: kb_pcg_init<<<blocks, threads, 0, s>>>(tab); break;
    case kB_pcg_spmv: kb_pcg_spmv<<<blocks, threads, 0, s>>>(tab); break;
    case kB_pcg_update: kb_pcg_update<<<blocks, threads, 0, s>>>(tab); break;
    case kB_pcg_p: kb_pcg_p<<<blocks, threads, 0, s>>>(tab); break;
    case kB_true_residual: kb_true_residual<<<blocks, threads, 0, s>>>(tab); break;
    case kB_integrate: kb_integrate<<<blocks, threads, 0, s>>>(tab); break;
    default: return -1;
  }
  return 1;
}

}  // namespace gf
