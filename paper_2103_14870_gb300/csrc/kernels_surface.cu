// Split visualisation mesh for output (Sec. 4.1, Fig. 6): child nodes of
// edges, faces and tets, and the crack quads between the node-associated
// pieces of every tet.  Output only: nothing here feeds the dynamics.
//
// A broken edge splits into two child nodes at its midpoint, a face into
// three at its centroid, a tet into four at its centroid.  A child follows
// the parents it is still joined to through unbroken edges of its entity: it
// sits at the entity's rest centroid plus the mean displacement x - X of those
// parents (with no broken edge, all children are at the current centroid).
//
// Vertex numbering: [0, N) nodes (x); N + 2 e + s edge children;
// N + 2 NE + 3 f + c face children (faces sorted); N + 2 NE + 3 NF + 4 t + a
// tet children.  Quads: for tet t and broken local edge k = (a, b), c < d the
// other local nodes, [E(a), F(abc, a), T(a), F(abd, a)] and
// [E(b), F(abd, b), T(b), F(abc, b)], by tet, local edge, a-side first.
#include "gf_surface.h"

namespace gf {
namespace {

constexpr int kST = 256;

// components of n <= 4 nodes joined by unbroken pairs: root = smallest member
template <int n>
__device__ __forceinline__ void components(const bool (&brk)[n][n], int (&comp)[n]) {
#pragma unroll
  for (int i = 0; i < n; ++i) comp[i] = i;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      if (brk[i][j]) continue;
      int ri = i, rj = j;
      while (comp[ri] != ri) ri = comp[ri];
      while (comp[rj] != rj) rj = comp[rj];
      if (ri != rj) comp[ri > rj ? ri : rj] = ri < rj ? ri : rj;
    }
#pragma unroll
  for (int i = 0; i < n; ++i) {
    int r = i;
    while (comp[r] != r) r = comp[r];
    comp[i] = r;
  }
}

// 1 / k for the member counts of an entity (multiplications instead of FP64 divides; within an ulp)
__device__ __forceinline__ double inv_count(int k) { return k == 1 ? 1.0 : (k == 2 ? 0.5 : (k == 3 ? 1.0 / 3.0 : 0.25)); }

// children of one entity with nodes nid[0..n): rest centroid + mean displacement of each component
template <int n>
__device__ __forceinline__ void follow(const double* __restrict__ X, const double* __restrict__ x, const int (&nid)[n],
                                       const bool (&brk)[n][n], double* out) {
  int comp[n];
  components<n>(brk, comp);
  double Xc[3] = {0.0, 0.0, 0.0}, d[n][3];
#pragma unroll
  for (int i = 0; i < n; ++i)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double Xi = X[3 * int64_t(nid[i]) + c];
      Xc[c] += Xi;
      d[i][c] = x[3 * int64_t(nid[i]) + c] - Xi;
    }
#pragma unroll
  for (int c = 0; c < 3; ++c) Xc[c] *= inv_count(n);
#pragma unroll
  for (int i = 0; i < n; ++i) {
    double s[3] = {0.0, 0.0, 0.0};
    int cnt = 0;
#pragma unroll
    for (int j = 0; j < n; ++j)
      if (comp[j] == comp[i]) {
        ++cnt;
#pragma unroll
        for (int c = 0; c < 3; ++c) s[c] += d[j][c];
      }
    const double ic = inv_count(cnt);
#pragma unroll
    for (int c = 0; c < 3; ++c) out[3 * i + c] = Xc[c] + s[c] * ic;
  }
}

__global__ void __launch_bounds__(kST) k_surf_nodes_edges(DevMesh m, SurfDev sd, double* V) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i < 3 * m.N) V[i] = m.x[i];
  if (i >= m.NE) return;
  const int2 ab = m.edges[i];
  const int nid[2] = {ab.x, ab.y};
  const bool b = m.labels[i] != 0;
  const bool brk[2][2] = {{false, b}, {b, false}};
  follow<2>(sd.X, m.x, nid, brk, V + 3 * (m.N + 2 * i));
}

__global__ void __launch_bounds__(kST) k_surf_faces(DevMesh m, SurfDev sd, double* V) {
  const int64_t f = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (f >= sd.NF) return;
  const int3 t = sd.faces[f];
  const int3 e = sd.face_edges[f];
  const int nid[3] = {t.x, t.y, t.z};
  const bool b01 = m.labels[e.x] != 0, b02 = m.labels[e.y] != 0, b12 = m.labels[e.z] != 0;
  const bool brk[3][3] = {{false, b01, b02}, {b01, false, b12}, {b02, b12, false}};
  follow<3>(sd.X, m.x, nid, brk, V + 3 * (m.N + 2 * m.NE + 3 * f));
}

__global__ void __launch_bounds__(kST) k_surf_tets(DevMesh m, SurfDev sd, double* V) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= m.T) return;
  const int4 n = m.tets[t];
  const int nid[4] = {n.x, n.y, n.z, n.w};
  bool brk[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i) brk[i][i] = false;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const bool b = m.labels[m.tet_edges[6 * t + k]] != 0;
    brk[edge_a(k)][edge_b(k)] = brk[edge_b(k)][edge_a(k)] = b;
  }
  follow<4>(sd.X, m.x, nid, brk, V + 3 * (m.N + 2 * m.NE + 3 * sd.NF + 4 * t));
}

__device__ __forceinline__ unsigned tet_quads(const DevMesh& m, int64_t t) {
  unsigned c = 0;
#pragma unroll
  for (int k = 0; k < 6; ++k) c += m.labels[m.tet_edges[6 * t + k]] != 0 ? 2u : 0u;
  return c;
}

// inclusive block scan of one value per thread (kST threads); returns the block total in *total
__device__ __forceinline__ unsigned block_scan(unsigned v, unsigned* total) {
  __shared__ unsigned ws[kST / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  if (lane == 31) ws[w] = v;
  __syncthreads();
  if (w == 0) {
    unsigned s = lane < kST / 32 ? ws[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < kST / 32) ws[lane] = s;
  }
  __syncthreads();
  if (w > 0) v += ws[w - 1];
  *total = ws[kST / 32 - 1];
  return v;
}

// pass 1: quads per block of tets
__global__ void __launch_bounds__(kST) k_surf_count(DevMesh m, SurfDev sd) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  unsigned total;
  block_scan(t < m.T ? tet_quads(m, t) : 0u, &total);
  if (threadIdx.x == 0) sd.bsum[blockIdx.x] = total;
}

// pass 2 (one CTA): exclusive prefix of the block sums, total in bsum[nb]
__global__ void __launch_bounds__(kST) k_surf_scan_blocks(SurfDev sd, int64_t nb) {
  unsigned carry = 0;
  for (int64_t base = 0; base < nb; base += kST) {
    const int64_t i = base + threadIdx.x;
    const unsigned v = i < nb ? sd.bsum[i] : 0u;
    unsigned total;
    const unsigned inc = block_scan(v, &total);
    __syncthreads();
    if (i < nb) sd.bsum[i] = carry + inc - v;
    carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) sd.bsum[nb] = carry;
}

// pass 3: write every tet's quads at its offset
__global__ void __launch_bounds__(kST) k_surf_quads(DevMesh m, SurfDev sd, int32_t* Q, int64_t max_quads) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const unsigned c = t < m.T ? tet_quads(m, t) : 0u;
  unsigned total;
  const unsigned inc = block_scan(c, &total);
  if (t >= m.T || c == 0) return;
  int64_t q = int64_t(sd.bsum[blockIdx.x]) + inc - c;
  const int64_t oF = m.N + 2 * m.NE, oT = oF + 3 * sd.NF + 4 * t;
  const int4 n = m.tets[t];
  const int nid[4] = {n.x, n.y, n.z, n.w};
  const int4 tf = sd.tet_faces[t];
  const int fo[4] = {tf.x, tf.y, tf.z, tf.w};   // face opposite each local node
  auto E = [&](int64_t e, int node) { return int32_t(m.N + 2 * e + (m.edges[e].x == node ? 0 : 1)); };
  auto F = [&](int f, int node) {
    const int3 tri = sd.faces[f];
    return int32_t(oF + 3 * int64_t(f) + (tri.x == node ? 0 : (tri.y == node ? 1 : 2)));
  };
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const int64_t e = m.tet_edges[6 * t + k];
    if (m.labels[e] == 0) continue;
    const int a = edge_a(k), b = edge_b(k);
    int c0 = -1, d0 = -1;
#pragma unroll
    for (int v = 0; v < 4; ++v)
      if (v != a && v != b) {
        if (c0 < 0) c0 = v;
        else d0 = v;
      }
    const int f_abc = fo[d0], f_abd = fo[c0];
    if (q + 2 <= max_quads) {
      int32_t* qa = Q + 4 * q;
      qa[0] = E(e, nid[a]);
      qa[1] = F(f_abc, nid[a]);
      qa[2] = int32_t(oT + a);
      qa[3] = F(f_abd, nid[a]);
      int32_t* qb = Q + 4 * (q + 1);
      qb[0] = E(e, nid[b]);
      qb[1] = F(f_abd, nid[b]);
      qb[2] = int32_t(oT + b);
      qb[3] = F(f_abc, nid[b]);
    }
    q += 2;
  }
}

inline unsigned grid(int64_t n) { return unsigned((n + kST - 1) / kST); }

}  // namespace

int64_t surf_blocks(const DevMesh& m) { return (m.T + kST - 1) / kST; }

int launch_surface_count(const DevMesh& m, const SurfDev& sd, cudaStream_t s) {
  const int64_t nb = surf_blocks(m);
  if (nb > 0) k_surf_count<<<unsigned(nb), kST, 0, s>>>(m, sd);
  k_surf_scan_blocks<<<1, kST, 0, s>>>(sd, nb);
  return nb > 0 ? 2 : 1;
}

int launch_surface_vertices(const DevMesh& m, const SurfDev& sd, double* V, cudaStream_t s) {
  const int64_t n = std::max<int64_t>(3 * m.N, m.NE);
  int L = 0;
  if (n > 0) {
    k_surf_nodes_edges<<<grid(n), kST, 0, s>>>(m, sd, V);
    ++L;
  }
  if (sd.NF > 0) {
    k_surf_faces<<<grid(sd.NF), kST, 0, s>>>(m, sd, V);
    ++L;
  }
  if (m.T > 0) {
    k_surf_tets<<<grid(m.T), kST, 0, s>>>(m, sd, V);
    ++L;
  }
  return L;
}

int launch_surface_quads(const DevMesh& m, const SurfDev& sd, int32_t* Q, int64_t max_quads, cudaStream_t s) {
  if (m.T <= 0) return 0;
  k_surf_quads<<<unsigned(surf_blocks(m)), kST, 0, s>>>(m, sd, Q, max_quads);
  return 1;
}

}  // namespace gf
