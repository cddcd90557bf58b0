// Host precompute of the fixed mesh graph (run once per mesh in gf_mesh_create).
//
// The computational mesh is never remeshed (Sec. 1), so everything derived from
// the rest configuration is built here once: the edge list (graph of Sec. 3.2),
// rest data of every tet, the lumped mass (Eq. 5, row-sum lumped), the
// block-CSR pattern of the system matrix (its size never changes, Sec. 5.4),
// a tet colouring for a conflict-free scatter, and the neighbour lists and
// weights of the non-local average (Eq. 20).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <numeric>
#include <thread>

#include "gf_internal.h"

namespace gf {

namespace {

inline uint64_t key(int32_t a, int32_t b) { return (uint64_t(uint32_t(a)) << 32) | uint32_t(b); }

int hw_threads() {
  unsigned n = std::thread::hardware_concurrency();
  return n == 0 ? 1 : int(std::min(n, 64u));
}

template <class F>
void parallel_for(int64_t n, F f) {
  int nt = hw_threads();
  if (n < 4096 || nt == 1) {
    f(int64_t(0), n);
    return;
  }
  std::vector<std::thread> th;
  int64_t chunk = (n + nt - 1) / nt;
  for (int i = 0; i < nt; ++i) {
    int64_t b = i * chunk, e = std::min(n, b + chunk);
    if (b >= e) break;
    th.emplace_back([=] { f(b, e); });
  }
  for (auto& t : th) t.join();
}

// E_k = dG/ds_k for G_ij = (x_i - x_0).(x_j - x_0) written by polarisation:
// G_ii = s_0i, G_ij = (s_0i + s_0j - s_ij)/2.
void edge_basis(double E[6][3][3]) {
  std::memset(E, 0, sizeof(double) * 54);
  for (int i = 0; i < 3; ++i) {      // edges (0, i+1) are k = i
    E[i][i][i] = 1.0;
    for (int j = 0; j < 3; ++j)
      if (j != i) E[i][i][j] = E[i][j][i] = 0.5;
  }
  const int pk[3][2] = {{0, 1}, {0, 2}, {1, 2}};  // edges (1,2) (1,3) (2,3) are k = 3, 4, 5
  for (int m = 0; m < 3; ++m) {
    E[3 + m][pk[m][0]][pk[m][1]] = -0.5;
    E[3 + m][pk[m][1]][pk[m][0]] = -0.5;
  }
}

}  // namespace

uint64_t disconnect_table() {
  uint64_t t = 0;
  for (int m = 0; m < 64; ++m) {
    int parent[4] = {0, 1, 2, 3};
    auto find = [&](int v) {
      while (parent[v] != v) v = parent[v];
      return v;
    };
    for (int k = 0; k < 6; ++k)
      if (!((m >> k) & 1)) {
        int a = find(edge_a(k)), b = find(edge_b(k));
        if (a != b) parent[a] = b;
      }
    int roots = 0;
    for (int v = 0; v < 4; ++v) roots += (find(v) == v);
    if (roots > 1) t |= (uint64_t(1) << m);
  }
  return t;
}

gf_status build_host_mesh(const double* X, int64_t N, const int32_t* tets_in, int64_t T, const gf_material& mat,
                          HostMesh& hm, std::string& err) {
  if (N <= 0 || T <= 0 || N > (int64_t(1) << 30) || T > (int64_t(1) << 30)) {
    err = "n_nodes and n_tets must be in [1, 2^30]";
    return GF_BAD_ARG;
  }
  for (int64_t i = 0; i < 4 * T; ++i)
    if (tets_in[i] < 0 || tets_in[i] >= N) {
      err = "tet node id out of range at tets[" + std::to_string(i) + "]";
      return GF_BAD_ARG;
    }
  for (int64_t i = 0; i < 3 * N; ++i)
    if (!std::isfinite(X[i])) {
      err = "non-finite node coordinate";
      return GF_BAD_ARG;
    }
  hm.n_nodes = N;
  hm.n_tets = T;

  // ---- edges (sorted unique (min, max) pairs) and caller-order tet->edge ----
  std::vector<uint64_t> keys(6 * T);
  for (int64_t t = 0; t < T; ++t)
    for (int k = 0; k < 6; ++k) {
      int32_t a = tets_in[4 * t + edge_a(k)], b = tets_in[4 * t + edge_b(k)];
      if (a == b) {
        err = "tet " + std::to_string(t) + " repeats a node";
        return GF_BAD_ARG;
      }
      keys[6 * t + k] = key(std::min(a, b), std::max(a, b));
    }
  std::vector<uint64_t> ukeys(keys);
  std::sort(ukeys.begin(), ukeys.end());
  ukeys.erase(std::unique(ukeys.begin(), ukeys.end()), ukeys.end());
  hm.n_edges = int64_t(ukeys.size());
  hm.edges.resize(2 * hm.n_edges);
  for (int64_t e = 0; e < hm.n_edges; ++e) {
    hm.edges[2 * e] = int32_t(ukeys[e] >> 32);
    hm.edges[2 * e + 1] = int32_t(ukeys[e] & 0xffffffffu);
  }
  std::vector<int32_t> te_caller(6 * T);
  parallel_for(6 * T, [&](int64_t b, int64_t e) {
    for (int64_t i = b; i < e; ++i)
      te_caller[i] = int32_t(std::lower_bound(ukeys.begin(), ukeys.end(), keys[i]) - ukeys.begin());
  });
  keys.clear();
  keys.shrink_to_fit();

  // ---- block-CSR pattern: row i = {i} U graph neighbours of i, sorted ----
  std::vector<int32_t> deg(N, 1);
  for (int64_t e = 0; e < hm.n_edges; ++e) {
    deg[hm.edges[2 * e]]++;
    deg[hm.edges[2 * e + 1]]++;
  }
  hm.row_ptr.assign(N + 1, 0);
  for (int64_t i = 0; i < N; ++i) hm.row_ptr[i + 1] = hm.row_ptr[i] + deg[i];
  hm.n_blocks = hm.row_ptr[N];
  hm.col.assign(hm.n_blocks, 0);
  std::vector<int32_t> fill(hm.row_ptr.begin(), hm.row_ptr.end() - 1);
  for (int64_t i = 0; i < N; ++i) hm.col[fill[i]++] = int32_t(i);
  for (int64_t e = 0; e < hm.n_edges; ++e) {
    int32_t a = hm.edges[2 * e], b = hm.edges[2 * e + 1];
    hm.col[fill[a]++] = b;
    hm.col[fill[b]++] = a;
  }
  hm.diag_blk.resize(N);
  for (int64_t i = 0; i < N; ++i) {
    std::sort(hm.col.begin() + hm.row_ptr[i], hm.col.begin() + hm.row_ptr[i + 1]);
    hm.diag_blk[i] = int32_t(std::lower_bound(hm.col.begin() + hm.row_ptr[i], hm.col.begin() + hm.row_ptr[i + 1],
                                              int32_t(i)) - hm.col.begin());
  }

  // ---- greedy colouring: no two tets of one colour share a node ----
  std::vector<int32_t> colour(T);
  {
    std::vector<std::vector<uint64_t>> used(1, std::vector<uint64_t>(N, 0));  // 64 colours per word
    for (int64_t t = 0; t < T; ++t) {
      int c = -1;
      for (size_t w = 0; c < 0; ++w) {
        if (w == used.size()) used.emplace_back(N, 0);
        uint64_t m = 0;
        for (int v = 0; v < 4; ++v) m |= used[w][tets_in[4 * t + v]];
        if (~m) {
          int bit = __builtin_ctzll(~m);
          c = int(w) * 64 + bit;
          for (int v = 0; v < 4; ++v) used[w][tets_in[4 * t + v]] |= (uint64_t(1) << bit);
        }
      }
      colour[t] = c;
    }
  }
  int32_t n_col = *std::max_element(colour.begin(), colour.end()) + 1;
  hm.colour_ptr.assign(n_col + 1, 0);
  for (int64_t t = 0; t < T; ++t) hm.colour_ptr[colour[t] + 1]++;
  for (int c = 0; c < n_col; ++c) hm.colour_ptr[c + 1] += hm.colour_ptr[c];
  hm.colour_tets.resize(T);
  {
    std::vector<int32_t> pos(hm.colour_ptr.begin(), hm.colour_ptr.end() - 1);
    for (int64_t t = 0; t < T; ++t) hm.colour_tets[pos[colour[t]]++] = int32_t(t);   // ascending within a colour
  }
  // tets keep the caller's order (spatially coherent for the gathers)
  hm.perm.resize(T);
  for (int64_t t = 0; t < T; ++t) hm.perm[t] = int32_t(t);

  // ---- internal-order tets, tet->edge, block slots ----
  hm.tets.resize(4 * T);
  hm.tet_edges.resize(6 * T);
  hm.slot.resize(16 * T);
  parallel_for(T, [&](int64_t b, int64_t e) {
    for (int64_t i = b; i < e; ++i) {
      int64_t t = hm.perm[i];
      for (int v = 0; v < 4; ++v) hm.tets[4 * i + v] = tets_in[4 * t + v];
      for (int k = 0; k < 6; ++k) hm.tet_edges[6 * i + k] = te_caller[6 * t + k];
      for (int a = 0; a < 4; ++a)
        for (int c = 0; c < 4; ++c) {
          int32_t r = tets_in[4 * t + a], cc = tets_in[4 * t + c];
          hm.slot[16 * i + 4 * a + c] = int32_t(
              std::lower_bound(hm.col.begin() + hm.row_ptr[r], hm.col.begin() + hm.row_ptr[r + 1], cc) - hm.col.begin());
        }
    }
  });

  // ---- two-phase assembly rows ----
  // Node rows: node i owns rows [np_ptr[i], np_ptr[i+1]), one per incident tet
  // in ascending tet order; nrow[4t+a] is the row of (tet t, local node a).
  hm.np_ptr.assign(N + 1, 0);
  for (int64_t i = 0; i < 4 * T; ++i) hm.np_ptr[hm.tets[i] + 1]++;
  for (int64_t i = 0; i < N; ++i) hm.np_ptr[i + 1] += hm.np_ptr[i];
  hm.nrow.resize(4 * T);
  {
    std::vector<int32_t> pos(hm.np_ptr.begin(), hm.np_ptr.end() - 1);
    for (int64_t t = 0; t < T; ++t)
      for (int a = 0; a < 4; ++a) hm.nrow[4 * t + a] = pos[hm.tets[4 * t + a]]++;
  }
  // block slots of (i, j) and (j, i) for every edge i < j
  hm.edge_slot.resize(2 * hm.n_edges);
  for (int64_t e = 0; e < hm.n_edges; ++e) {
    const int32_t i = hm.edges[2 * e], j = hm.edges[2 * e + 1];
    hm.edge_slot[2 * e] =
        int32_t(std::lower_bound(hm.col.begin() + hm.row_ptr[i], hm.col.begin() + hm.row_ptr[i + 1], j) - hm.col.begin());
    hm.edge_slot[2 * e + 1] =
        int32_t(std::lower_bound(hm.col.begin() + hm.row_ptr[j], hm.col.begin() + hm.row_ptr[j + 1], i) - hm.col.begin());
  }
  if (T >= (int64_t(1) << 26)) {
    err = "at most 2^26 tets per mesh";
    return GF_BAD_ARG;
  }

  // ---- rest data per tet (internal order) ----
  const double lam = mat.young * mat.poisson / ((1.0 + mat.poisson) * (1.0 - 2.0 * mat.poisson));
  const double mu = mat.young / (2.0 * (1.0 + mat.poisson));
  double Eb[6][3][3];
  edge_basis(Eb);
  hm.rest.assign(size_t(kRestFields) * T, 0.0);
  hm.mass.assign(N, 0.0);
  std::vector<double> vol(T);
  std::atomic<bool> degenerate{false};
  std::atomic<int64_t> bad_tet{-1};
  parallel_for(T, [&](int64_t b, int64_t e) {
    for (int64_t i = b; i < e; ++i) {
      const int32_t* n = &hm.tets[4 * i];
      double Dm[3][3];
      for (int c = 0; c < 3; ++c)
        for (int r = 0; r < 3; ++r) Dm[r][c] = X[3 * n[c + 1] + r] - X[3 * n[0] + r];
      double det = Dm[0][0] * (Dm[1][1] * Dm[2][2] - Dm[1][2] * Dm[2][1]) -
                   Dm[0][1] * (Dm[1][0] * Dm[2][2] - Dm[1][2] * Dm[2][0]) +
                   Dm[0][2] * (Dm[1][0] * Dm[2][1] - Dm[1][1] * Dm[2][0]);
      double scale = 0;
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) scale = std::max(scale, std::fabs(Dm[r][c]));
      if (!(std::fabs(det) > 1e-12 * scale * scale * scale)) {
        degenerate.store(true);
        bad_tet.store(hm.perm[i]);
        continue;
      }
      double B[3][3];   // inverse by cofactors
      B[0][0] = (Dm[1][1] * Dm[2][2] - Dm[1][2] * Dm[2][1]) / det;
      B[0][1] = (Dm[0][2] * Dm[2][1] - Dm[0][1] * Dm[2][2]) / det;
      B[0][2] = (Dm[0][1] * Dm[1][2] - Dm[0][2] * Dm[1][1]) / det;
      B[1][0] = (Dm[1][2] * Dm[2][0] - Dm[1][0] * Dm[2][2]) / det;
      B[1][1] = (Dm[0][0] * Dm[2][2] - Dm[0][2] * Dm[2][0]) / det;
      B[1][2] = (Dm[0][2] * Dm[1][0] - Dm[0][0] * Dm[1][2]) / det;
      B[2][0] = (Dm[1][0] * Dm[2][1] - Dm[1][1] * Dm[2][0]) / det;
      B[2][1] = (Dm[0][1] * Dm[2][0] - Dm[0][0] * Dm[2][1]) / det;
      B[2][2] = (Dm[0][0] * Dm[1][1] - Dm[0][1] * Dm[1][0]) / det;
      double V = std::fabs(det) / 6.0;
      vol[i] = V;
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) hm.rest[size_t(kRestB + 3 * r + c) * T + i] = B[r][c];
      for (int k = 0; k < 6; ++k) {
        double s = 0;
        for (int c = 0; c < 3; ++c) {
          double d = X[3 * n[edge_b(k)] + c] - X[3 * n[edge_a(k)] + c];
          s += d * d;
        }
        hm.rest[size_t(kRestS0 + k) * T + i] = s;
      }
      // StVK (Eq. 37) is quadratic in C and C = B^T G(s) B is linear in s, so
      // V*Psi = 1/2 (s - s0)^T Hs (s - s0) with the constant
      // Hs_kl = V [lam/4 tr(M_k) tr(M_l) + mu/2 M_k : M_l],  M_k = B^T E_k B.
      // With P = B B^T: tr(M_k) = E_k : P and M_k : M_l = tr(E_k P E_l P).
      double P[3][3];
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) P[r][c] = B[r][0] * B[c][0] + B[r][1] * B[c][1] + B[r][2] * B[c][2];
      double a[6], EP[6][3][3];
      for (int k = 0; k < 6; ++k) {
        a[k] = 0;
        for (int r = 0; r < 3; ++r)
          for (int c = 0; c < 3; ++c) {
            a[k] += Eb[k][r][c] * P[r][c];
            EP[k][r][c] = Eb[k][r][0] * P[0][c] + Eb[k][r][1] * P[1][c] + Eb[k][r][2] * P[2][c];
          }
      }
      for (int k = 0; k < 6; ++k)
        for (int l = k; l < 6; ++l) {
          double tr = 0;   // tr(EP_k EP_l)
          for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) tr += EP[k][r][c] * EP[l][c][r];
          hm.rest[size_t(kRestH + tri6(k, l)) * T + i] = V * (lam / 4.0 * a[k] * a[l] + mu / 2.0 * tr);
        }
      hm.rest[size_t(kRestV) * T + i] = V;
    }
  });
  if (degenerate) {
    err = "degenerate (zero-volume) tet " + std::to_string(bad_tet.load());
    return GF_BAD_ARG;
  }
  for (int64_t i = 0; i < T; ++i)
    for (int v = 0; v < 4; ++v) hm.mass[hm.tets[4 * i + v]] += mat.density * vol[i] / 4.0;

  // ---- edge -> incident tets (internal tet ids, ascending) ----
  hm.et_ptr.assign(hm.n_edges + 1, 0);
  for (int64_t i = 0; i < 6 * T; ++i) hm.et_ptr[hm.tet_edges[i] + 1]++;
  for (int64_t e = 0; e < hm.n_edges; ++e) hm.et_ptr[e + 1] += hm.et_ptr[e];
  hm.et_tet.resize(6 * T);
  {
    std::vector<int32_t> pos(hm.et_ptr.begin(), hm.et_ptr.end() - 1);
    hm.erow.resize(6 * T);
    for (int64_t i = 0; i < T; ++i)
      for (int k = 0; k < 6; ++k) {
        const int32_t r = pos[hm.tet_edges[6 * i + k]]++;
        hm.et_tet[r] = int32_t(i);
        hm.erow[6 * i + k] = r;   // edge rows follow the edge -> tet lists
      }
  }
  // Order in which the gather visits edges and nodes: within windows of 1,024,
  // by descending row count (stable), so the lanes of a warp sum rows of equal
  // count and few of them idle in the FP64 adds; the windows keep the rows read
  // by neighbouring warps close in memory.
  auto count_order = [](const std::vector<int32_t>& ptr, std::vector<int32_t>& order) {
    const int64_t n = int64_t(ptr.size()) - 1;
    order.resize(n);
    std::iota(order.begin(), order.end(), 0);
    constexpr int64_t kWin = 1024;
    for (int64_t w0 = 0; w0 < n; w0 += kWin)
      std::stable_sort(order.begin() + w0, order.begin() + std::min(n, w0 + kWin), [&](int32_t x, int32_t y) {
        return ptr[x + 1] - ptr[x] > ptr[y + 1] - ptr[y];
      });
  };
  count_order(hm.et_ptr, hm.edge_order);
  count_order(hm.np_ptr, hm.node_order);

  // ---- Eq. 20 neighbour lists on rest centroids, w = V_j (1 - r^2/R^2)^2 normalised ----
  const double R = mat.radius;
  std::vector<double> cen(3 * T);
  for (int64_t i = 0; i < T; ++i)
    for (int c = 0; c < 3; ++c)
      cen[3 * i + c] = 0.25 * (X[3 * hm.tets[4 * i] + c] + X[3 * hm.tets[4 * i + 1] + c] +
                               X[3 * hm.tets[4 * i + 2] + c] + X[3 * hm.tets[4 * i + 3] + c]);
  std::vector<std::vector<int32_t>> nb_list(T);
  std::vector<std::vector<double>> nb_wt(T);
  if (!(R > 0.0)) {
    for (int64_t i = 0; i < T; ++i) {
      nb_list[i] = {int32_t(i)};
      nb_wt[i] = {1.0};
    }
  } else {
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t i = 0; i < T; ++i)
      for (int c = 0; c < 3; ++c) {
        lo[c] = std::min(lo[c], cen[3 * i + c]);
        hi[c] = std::max(hi[c], cen[3 * i + c]);
      }
    int64_t dim[3];
    for (int c = 0; c < 3; ++c) dim[c] = std::max<int64_t>(1, int64_t((hi[c] - lo[c]) / R) + 1);
    if (dim[0] * dim[1] * dim[2] > 64 * T + 64) {   // radius tiny against the extent: coarsen the grid
      double f = std::cbrt(double(dim[0] * dim[1] * dim[2]) / double(64 * T + 64));
      for (int c = 0; c < 3; ++c) dim[c] = std::max<int64_t>(1, int64_t(dim[c] / f));
    }
    double cs[3];
    for (int c = 0; c < 3; ++c) cs[c] = std::max(R, (hi[c] - lo[c]) / double(dim[c]) * (1 + 1e-12));
    auto cell_of = [&](int64_t i, int c) {
      return std::min<int64_t>(dim[c] - 1, int64_t((cen[3 * i + c] - lo[c]) / cs[c]));
    };
    int64_t ncell = dim[0] * dim[1] * dim[2];
    std::vector<int64_t> cstart(ncell + 1, 0);
    std::vector<int64_t> tcell(T);
    for (int64_t i = 0; i < T; ++i) {
      tcell[i] = (cell_of(i, 0) * dim[1] + cell_of(i, 1)) * dim[2] + cell_of(i, 2);
      cstart[tcell[i] + 1]++;
    }
    for (int64_t c = 0; c < ncell; ++c) cstart[c + 1] += cstart[c];
    std::vector<int32_t> cell_tets(T);
    {
      std::vector<int64_t> pos(cstart.begin(), cstart.end() - 1);
      for (int64_t i = 0; i < T; ++i) cell_tets[pos[tcell[i]]++] = int32_t(i);
    }
    const double R2 = R * R;
    parallel_for(T, [&](int64_t b, int64_t e) {
      for (int64_t i = b; i < e; ++i) {
        int64_t ci[3] = {cell_of(i, 0), cell_of(i, 1), cell_of(i, 2)};
        auto& L = nb_list[i];
        for (int64_t x = std::max<int64_t>(0, ci[0] - 1); x <= std::min(dim[0] - 1, ci[0] + 1); ++x)
          for (int64_t y = std::max<int64_t>(0, ci[1] - 1); y <= std::min(dim[1] - 1, ci[1] + 1); ++y)
            for (int64_t z = std::max<int64_t>(0, ci[2] - 1); z <= std::min(dim[2] - 1, ci[2] + 1); ++z) {
              int64_t c = (x * dim[1] + y) * dim[2] + z;
              for (int64_t p = cstart[c]; p < cstart[c + 1]; ++p) {
                int32_t j = cell_tets[p];
                double d0 = cen[3 * j] - cen[3 * i], d1 = cen[3 * j + 1] - cen[3 * i + 1],
                       d2 = cen[3 * j + 2] - cen[3 * i + 2];
                if (d0 * d0 + d1 * d1 + d2 * d2 <= R2) L.push_back(j);
              }
            }
        std::sort(L.begin(), L.end());
        auto& W = nb_wt[i];
        W.resize(L.size());
        double sum = 0;
        for (size_t p = 0; p < L.size(); ++p) {
          int32_t j = L[p];
          double d0 = cen[3 * j] - cen[3 * i], d1 = cen[3 * j + 1] - cen[3 * i + 1], d2 = cen[3 * j + 2] - cen[3 * i + 2];
          double q = 1.0 - (d0 * d0 + d1 * d1 + d2 * d2) / R2;
          W[p] = vol[j] * q * q;
          sum += W[p];
        }
        for (auto& w : W) w /= sum;
      }
    });
  }
  // SELL-32 layout: 32 tets per group, entry k of lane l at off + 32 k + l.
  // Within each window of 1024 consecutive tets the tets are ordered by list
  // length (longest first), so that the 32 lanes of a group have nearly equal
  // lists and the group's padding (to its longest list) is small; the window
  // keeps a group's tets close together on the mesh.
  NeighbourSell& S = hm.nbr;
  int64_t G = (T + 31) / 32;
  S.perm.resize(T);
  S.slot.resize(T);
  for (int64_t i = 0; i < T; ++i) S.perm[i] = int32_t(i);
  constexpr int64_t kWin = 1024;
  for (int64_t w0 = 0; w0 < T; w0 += kWin)
    std::stable_sort(S.perm.begin() + w0, S.perm.begin() + std::min(T, w0 + kWin),
                     [&](int32_t x, int32_t y) { return nb_list[x].size() > nb_list[y].size(); });
  for (int64_t q = 0; q < T; ++q) S.slot[S.perm[q]] = int32_t(q);
  S.group_off.resize(G);
  S.group_len.resize(G);
  int64_t total = 0;
  for (int64_t g = 0; g < G; ++g) {
    size_t mx = 0;
    for (int64_t q = 32 * g; q < std::min(T, 32 * g + 32); ++q) mx = std::max(mx, nb_list[S.perm[q]].size());
    S.group_off[g] = total;
    S.group_len[g] = int32_t(mx);
    total += 32 * int64_t(mx);
  }
  S.idx.assign(total, 0);
  S.w.assign(total, 0.0);
  S.pairs = 0;
  for (int64_t g = 0; g < G; ++g)
    for (int l = 0; l < 32; ++l) {
      const int64_t q = 32 * g + l;
      const int64_t i = q < T ? S.perm[q] : 0;
      for (int32_t k = 0; k < S.group_len[g]; ++k) {
        int64_t o = S.group_off[g] + 32 * int64_t(k) + l;
        if (q < T && size_t(k) < nb_list[i].size()) {
          S.idx[o] = nb_list[i][k];
          S.w[o] = nb_wt[i][k];
          S.pairs++;
        } else {
          S.idx[o] = int32_t(i);
          S.w[o] = 0.0;
        }
      }
    }
  return GF_OK;
}

// Order of the joint list of pair q for the mixed Eq. 20 kernel.  The list is
// padded to a multiple of four entries (a pad repeats a real position of the
// list with zero weights, so it adds +0 and reads a row the pair already
// reads) and read in groups of four consecutive entries: eight lanes take a
// pair, lane s the groups s, s + 8, s + 16, ..., each with one 8-byte load of
// its four positions and two 16-byte loads of their weights.  Within the block
// of 32 entries of round r (groups 8r .. 8r + 7) the eight lanes sum their
// k-th entries together, entries 32r + 4s + k: one chunk per (r, k), eight
// entries (m in a last block of 4m entries).  A lane reads the six floats of
// union row loc as three 8-byte words at bank pair (3 loc + h) mod 16; a
// half-warp (two pairs, q even and q + 1) is one shared-memory wavefront per
// word.  So each chunk takes distinct residues loc mod 16 from one half of the
// residues, the low half when q + c is even and the high half otherwise (c the
// chunk's ordinal 4r + k: the two pairs of a half-warp take opposite halves),
// the residues with the most entries left first; what a half cannot supply
// comes from the other half.  Only the order of the terms changes.
struct JointEntry {
  uint16_t loc;
  float w[2];
};
void deal_entries(std::vector<JointEntry>& e, int64_t q) {
  const int64_t n = int64_t(e.size());
  if (n == 0) return;
  const int64_t n4 = (n + 3) / 4 * 4;
  std::vector<JointEntry> bucket[16];
  for (const auto& x : e) bucket[x.loc % 16].push_back(x);
  size_t next[16] = {};
  auto left = [&](int r) { return bucket[r].size() - next[r]; };
  std::vector<JointEntry> out(static_cast<size_t>(n4));
  int64_t placed = 0;
  uint16_t last_loc = e[0].loc;
  for (int64_t r = 0; 32 * r < n4; ++r) {
    const int64_t m = std::min<int64_t>(8, (n4 - 32 * r) / 4);   // lanes with a group in this block
    for (int k = 0; k < 4; ++k) {
      const int64_t c = 4 * r + k;
      const int half = ((q + c) & 1) ? 8 : 0;
      bool used[16] = {};
      int64_t got = 0;
      const int64_t want = std::min<int64_t>(m, n - placed);
      auto put = [&](const JointEntry& x) {
        out[size_t(32 * r + 4 * got + k)] = x;
        last_loc = x.loc;
        ++got;
        ++placed;
      };
      auto take_from = [&](int lo, bool distinct) {
        while (got < want) {
          int best = -1;
          for (int b = lo; b < lo + 8; ++b)
            if (left(b) > 0 && !(distinct && used[b]) && (best < 0 || left(b) > left(best))) best = b;
          if (best < 0) return;
          used[best] = true;
          put(bucket[best][next[best]++]);
        }
      };
      take_from(half, true);
      take_from(8 - half, true);
      take_from(half, false);
      take_from(8 - half, false);
      for (; got < m; ++got) out[size_t(32 * r + 4 * got + k)] = {last_loc, {0.f, 0.f}};   // pads
    }
  }
  e.swap(out);
}

gf_status build_mixed_host(const double* X, const HostMesh& hm, MixedHost& mx, std::string& err) {
  const int64_t N = hm.n_nodes, T = hm.n_tets, NE = hm.n_edges;
  mx.restA.assign(size_t(kRAStride) * T, 0.f);
  mx.restB.assign(size_t(kRBStride) * T, 0.f);
  for (int64_t i = 0; i < T; ++i) {
    const int32_t* n = &hm.tets[4 * i];
    float* A = &mx.restA[size_t(kRAStride) * i];
    for (int k = 0; k < 3; ++k)
      for (int c = 0; c < 3; ++c) A[kRAE0 + 3 * k + c] = float(X[3 * n[k + 1] + c] - X[3 * n[0] + c]);
    for (int f = 0; f < 21; ++f) A[kRAH + f] = float(hm.rest[size_t(kRestH + f) * T + i]);
    A[kRAV] = float(hm.rest[size_t(kRestV) * T + i]);
    for (int f = 0; f < 9; ++f) mx.restB[size_t(kRBStride) * i + f] = float(hm.rest[size_t(kRestB + f) * T + i]);
  }
  mx.edge_e0.resize(3 * NE);
  for (int64_t e = 0; e < NE; ++e)
    for (int c = 0; c < 3; ++c)
      mx.edge_e0[3 * e + c] = float(X[3 * hm.edges[2 * e + 1] + c] - X[3 * hm.edges[2 * e] + c]);
  // Neighbour lists per tet (from the SELL-32 layout: real entries have w > 0),
  // then the tile unions and the joint lists of tet pairs (2q, 2q+1)
  {
    const NeighbourSell& S = hm.nbr;
    std::vector<int64_t> tp(T + 1, 0);
    for (int64_t i = 0; i < T; ++i) {
      int64_t g = S.slot[i] / 32, l = S.slot[i] % 32;
      int32_t cnt = 0;
      for (int32_t k = 0; k < S.group_len[g]; ++k)
        if (S.w[S.group_off[g] + 32 * int64_t(k) + l] > 0.0) cnt++;
      tp[i + 1] = tp[i] + cnt;
    }
    std::vector<int32_t> nb_id(tp[T]);
    std::vector<float> nb_w(tp[T]);
    for (int64_t i = 0; i < T; ++i) {
      int64_t g = S.slot[i] / 32, l = S.slot[i] % 32, p = tp[i];
      for (int32_t k = 0; k < S.group_len[g]; ++k) {
        int64_t o = S.group_off[g] + 32 * int64_t(k) + l;
        if (S.w[o] > 0.0) {
          nb_id[p] = S.idx[o];
          nb_w[p] = float(S.w[o]);
          ++p;
        }
      }
    }
    // Tiles of kNlTile tets, or of kNlTileSmall where the largest union of the
    // large tile leaves fewer than kNlCtasWanted CTAs per SM room in shared
    // memory (a wide radius): smaller unions let more CTAs hide the list latency
    auto build_tiles = [&](int tile) -> gf_status {
      const int64_t NT = (T + tile - 1) / tile, NQ = (T + 1) / 2;
      std::vector<std::vector<int32_t>> U(NT);
      std::vector<std::vector<JointEntry>> J(NQ);
      std::atomic<int64_t> too_big{-1}, n_real{0};
      parallel_for(NT, [&](int64_t b, int64_t e) {
        int64_t real = 0;
        for (int64_t g = b; g < e; ++g) {
          const int64_t t0 = tile * g, t1 = std::min(T, tile * (g + 1));
          std::vector<int32_t>& u = U[g];
          u.assign(nb_id.begin() + tp[t0], nb_id.begin() + tp[t1]);
          std::sort(u.begin(), u.end());
          u.erase(std::unique(u.begin(), u.end()), u.end());
          if (int64_t(u.size()) > kNlMaxUnion) {
            too_big = g;
            continue;
          }
          auto pos = [&](int32_t j) { return uint16_t(std::lower_bound(u.begin(), u.end(), j) - u.begin()); };
          for (int64_t a = t0; a < t1; a += 2) {   // merge the two sorted lists
            std::vector<JointEntry>& jq = J[a / 2];
            int64_t p = tp[a], pe = tp[a + 1], r = a + 1 < T ? tp[a + 1] : 0, re = a + 1 < T ? tp[a + 2] : 0;
            while (p < pe || r < re) {
              JointEntry x{};
              if (r >= re || (p < pe && nb_id[p] < nb_id[r])) {
                x = {pos(nb_id[p]), {nb_w[p], 0.f}};
                ++p;
              } else if (p >= pe || nb_id[r] < nb_id[p]) {
                x = {pos(nb_id[r]), {0.f, nb_w[r]}};
                ++r;
              } else {
                x = {pos(nb_id[p]), {nb_w[p], nb_w[r]}};
                ++p;
                ++r;
              }
              jq.push_back(x);
            }
            real += int64_t(jq.size());
            deal_entries(jq, a / 2);
          }
        }
        n_real += real;
      });
      if (too_big >= 0) {
        err = "Eq. 20 neighbour sets too large for the mixed-precision path (a tile of " + std::to_string(tile) +
              " tets reaches more than " + std::to_string(kNlMaxUnion) + " tets; reduce the radius)";
        return GF_UNSUPPORTED;
      }
      mx.nl_tile = tile;
      mx.nb_real = n_real;
      mx.nl_uptr.assign(NT + 1, 0);
      int64_t largest = 0;
      for (int64_t g = 0; g < NT; ++g) {
        mx.nl_uptr[g + 1] = mx.nl_uptr[g] + int64_t(U[g].size());
        largest = std::max<int64_t>(largest, int64_t(U[g].size()));
      }
      mx.nl_cap = int32_t(std::min<int64_t>(largest, kNlCapMax));
      mx.nl_uidx.resize(mx.nl_uptr[NT]);
      for (int64_t g = 0; g < NT; ++g) std::copy(U[g].begin(), U[g].end(), mx.nl_uidx.begin() + mx.nl_uptr[g]);
      mx.nb_ptr.assign(NQ + 1, 0);
      for (int64_t q = 0; q < NQ; ++q) mx.nb_ptr[q + 1] = mx.nb_ptr[q] + int64_t(J[q].size());
      mx.nb_loc.resize(mx.nb_ptr[NQ]);
      mx.nb_w2.resize(2 * mx.nb_ptr[NQ]);
      // weights of a block of 32 entries (m lanes' groups) in two planes: lane
      // s's entries 4s, 4s + 1 at 4 s floats, its entries 4s + 2, 4s + 3 after
      // the first plane (at 4 m + 4 s)
      parallel_for(NQ, [&](int64_t b, int64_t e) {
        for (int64_t q = b; q < e; ++q) {
          const int64_t n = int64_t(J[q].size());
          for (int64_t k = 0; k < n; ++k) {
            const int64_t o = mx.nb_ptr[q] + k, r = k / 32, sl = (k % 32) / 4, c = k % 4;
            const int64_t m = std::min<int64_t>(8, (n - 32 * r) / 4);
            const int64_t w = 2 * (mx.nb_ptr[q] + 32 * r) + (c < 2 ? 4 * sl : 4 * m + 4 * sl) + 2 * (c & 1);
            mx.nb_loc[o] = J[q][size_t(k)].loc;
            mx.nb_w2[w] = J[q][size_t(k)].w[0];
            mx.nb_w2[w + 1] = J[q][size_t(k)].w[1];
          }
        }
      });
      return GF_OK;
    };
    gf_status st = build_tiles(kNlTile);
    if (st == GF_OK && int64_t(mx.nl_cap) * 24 * kNlCtasWanted > kNlSmemPerSm) st = build_tiles(kNlTileSmall);
    if (st != GF_OK) return st;
  }
  return GF_OK;
}

}  // namespace gf
