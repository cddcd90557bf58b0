// Host check of the mixed-precision Eq. 20 joint lists (no GPU).  Reads a mesh
// (int64 N, int64 T, double R_d, N*3 doubles, T*4 int32), runs the host
// precompute of gf_mesh_create, then:
//  * reads every pair's list the way k_nonlocal32 does (groups of four
//    entries; per block of 32 entries the weights of each lane's first two
//    entries, then of its last two) and sums a test field over it, which must
//    equal the sum over each tet's own neighbour list (the FP32 weights the
//    lists carry, summed in double);
//  * checks the padding: list starts on multiples of four, pads of zero weight
//    at positions the list already holds, and the count of real entries equal
//    to the sum of the sizes of the pairs' neighbour-set unions;
//  * counts the bank chunks (the eight entries a pair's lanes sum together)
//    whose positions take distinct residues mod 16.
// Prints one JSON line; exit status 1 on a failed check.
#include "host_mesh.cpp"

#include <cstdio>
#include <set>

namespace gf {
void set_last_error(const std::string&) {}
}

int main(int argc, char** argv) {
  if (argc < 2) return 2;
  FILE* f = std::fopen(argv[1], "rb");
  if (!f) return 2;
  int64_t N = 0, T = 0;
  double R = 0.0;
  if (std::fread(&N, 8, 1, f) != 1 || std::fread(&T, 8, 1, f) != 1 || std::fread(&R, 8, 1, f) != 1) return 2;
  std::vector<double> X(3 * N);
  std::vector<int32_t> tets(4 * T);
  if (std::fread(X.data(), 8, X.size(), f) != X.size() || std::fread(tets.data(), 4, tets.size(), f) != tets.size())
    return 2;
  std::fclose(f);
  gf_material mat{};
  mat.young = 1e6;
  mat.poisson = 0.3;
  mat.density = 1000.0;
  mat.threshold = 1.0;
  mat.radius = R;
  mat.shear_coef = 2;
  mat.average_degraded = 1;
  gf::HostMesh hm;
  gf::MixedHost mx;
  std::string err;
  if (gf::build_host_mesh(X.data(), N, tets.data(), T, mat, hm, err) != GF_OK ||
      gf::build_mixed_host(X.data(), hm, mx, err) != GF_OK) {
    std::printf("{\"error\": \"%s\"}\n", err.c_str());
    return 1;
  }
  // the tets' own lists (real entries: w > 0), FP32 weights as the lists carry them
  const gf::NeighbourSell& S = hm.nbr;
  std::vector<std::vector<std::pair<int32_t, float>>> own(T);
  for (int64_t i = 0; i < T; ++i) {
    const int64_t g = S.slot[i] / 32, l = S.slot[i] % 32;
    for (int32_t k = 0; k < S.group_len[g]; ++k) {
      const int64_t o = S.group_off[g] + 32 * int64_t(k) + l;
      if (S.w[o] > 0.0) own[i].push_back({S.idx[o], float(S.w[o])});
    }
  }
  auto field = [](int64_t j, int c) { return 1.0 + 0.37 * c + 0.01 * double((j * 7919 + 13 * c) % 1009); };
  const int64_t NQ = (T + 1) / 2, tile = mx.nl_tile;
  int64_t bad = 0, n_real = 0, union_total = 0, chunks = 0, distinct = 0, pads = 0;
  double worst = 0.0;
  for (int64_t q = 0; q < NQ; ++q) {
    const int64_t beg = mx.nb_ptr[q], n = mx.nb_ptr[q + 1] - beg;
    if (beg % 4 != 0 || n % 4 != 0) ++bad;
    const int64_t g = (2 * q) / tile, u0 = mx.nl_uptr[g], un = mx.nl_uptr[g + 1] - u0;
    double acc[2][6] = {};
    std::set<int> real_locs;
    std::vector<int> pad_locs;
    for (int64_t e = 0; e < n; ++e) {
      const int64_t blk = e & ~int64_t(31), sl = (e & 31) >> 2, k = e & 3;
      const int64_t m = std::min<int64_t>(8, (n - blk) / 4);
      const int64_t w = 2 * (beg + blk) + (k < 2 ? 4 * sl : 4 * m + 4 * sl) + 2 * (k & 1);
      const int loc = mx.nb_loc[beg + e];
      const float wa = mx.nb_w2[w], wb = mx.nb_w2[w + 1];
      if (loc >= un) {
        ++bad;
        continue;
      }
      if (wa == 0.f && wb == 0.f) {
        pad_locs.push_back(loc);
        ++pads;
        continue;
      }
      real_locs.insert(loc);
      ++n_real;
      const int32_t j = mx.nl_uidx[u0 + loc];
      for (int c = 0; c < 6; ++c) {
        acc[0][c] += double(wa) * field(j, c);
        acc[1][c] += double(wb) * field(j, c);
      }
    }
    for (int loc : pad_locs)
      if (!real_locs.count(loc)) ++bad;
    if (n - int64_t(real_locs.size()) > 3) ++bad;
    std::set<int32_t> un_set;
    for (int t = 0; t < 2; ++t) {
      const int64_t i = 2 * q + t;
      if (i >= T) continue;
      for (const auto& p : own[i]) un_set.insert(p.first);
      for (int c = 0; c < 6; ++c) {
        double want = 0.0;
        for (const auto& p : own[i]) want += double(p.second) * field(p.first, c);
        const double err_rel = std::abs(acc[t][c] - want) / std::max(1e-300, std::abs(want));
        worst = std::max(worst, err_rel);
        if (!(err_rel <= 1e-12)) ++bad;
      }
    }
    union_total += int64_t(un_set.size());
    for (int64_t r = 0; 32 * r < n; ++r) {
      const int64_t m = std::min<int64_t>(8, (n - 32 * r) / 4);
      for (int k = 0; k < 4; ++k) {
        bool seen[16] = {}, ok = true;
        for (int64_t s = 0; s < m; ++s) {
          const int b = mx.nb_loc[beg + 32 * r + 4 * s + k] % 16;
          ok = ok && !seen[b];
          seen[b] = true;
        }
        ++chunks;
        distinct += ok ? 1 : 0;
      }
    }
  }
  if (n_real != mx.nb_real || n_real != union_total) ++bad;
  std::printf("{\"tets\": %lld, \"tile\": %d, \"entries\": %lld, \"real\": %lld, \"union_sizes\": %lld, \"pads\": %lld, "
              "\"chunks\": %lld, \"distinct_chunks\": %lld, \"worst_rel\": %.3e, \"bad\": %lld}\n",
              (long long)T, int(tile), (long long)mx.nb_ptr[NQ], (long long)n_real, (long long)union_total,
              (long long)pads, (long long)chunks, (long long)distinct, worst, (long long)bad);
  return bad == 0 ? 0 : 1;
}
