// Internal declarations shared by the graph-FEM library translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "graphfem.h"

#ifdef __CUDACC__
#define GF_HD __host__ __device__
#else
#define GF_HD
#endif

namespace gf {

// Local edge order of a tet (Eq. 15): (0,1) (0,2) (0,3) (1,2) (1,3) (2,3).
// Edge k joins local nodes edge_a(k) -> edge_b(k).
GF_HD constexpr int edge_a(int k) { return k < 3 ? 0 : (k < 5 ? 1 : 2); }
GF_HD constexpr int edge_b(int k) { return k < 3 ? k + 1 : (k == 3 ? 2 : 3); }

// Field offsets of the per-tet rest data (field-major, field f of tet t at f*T + t).
enum RestField : int {
  kRestB = 0,    // B = Dm^-1, 9 values row-major (Dm columns X1-X0, X2-X0, X3-X0)
  kRestS0 = 9,   // rest squared edge lengths, 6
  kRestH = 15,   // V * d2Psi/ds ds (Eq. 37 in edge lengths), 21 upper-triangle values row-major
  kRestV = 36,   // rest volume
  kRestFields = 37
};

// Index of (k, l), k <= l, in the packed upper triangle of a 6x6 matrix.
GF_HD constexpr int tri6(int k, int l) { return k * 6 - k * (k - 1) / 2 + (l - k); }

struct NeighbourSell {            // Eq. 20 neighbour lists, 32 tets per group, entry-major in a group
  std::vector<int64_t> group_off; // [G] first entry of the group
  std::vector<int32_t> group_len; // [G] entries per lane (max count in the group)
  std::vector<int32_t> perm;      // [T] lane slot 32 g + l -> tet (tets sorted by list length within windows)
  std::vector<int32_t> slot;      // [T] tet -> lane slot
  std::vector<int32_t> idx;       // [sum 32*len] neighbour tet (internal order); padding -> own tet
  std::vector<double> w;          // normalised weights; padding -> 0
  int64_t pairs = 0;              // real (unpadded) pairs
};

// FP32 rest data of the mixed-precision path, tet-major (one 128-byte line per
// tet for the gathers of the row-gather assembly):
//   restA [T][32]: rest edge vectors X1-X0, X2-X0, X3-X0 (9), Hs packed (21), V, pad
//   restB [T][12]: B = Dm^-1 row-major (9), pad
enum Rest32Field : int { kRAE0 = 0, kRAH = 9, kRAV = 30, kRAStride = 32, kRBStride = 12 };

// Tiles of the mixed Eq. 20 kernel: a tile of consecutive tets (kNlTile, or
// kNlTileSmall for a wide radius, chosen per mesh) shares one CTA, which
// stages the union of their neighbour sets (at most kNlCap rows in a batched
// launch) in shared memory; each pair names its neighbour by its position in
// that union.  The small tile is taken when kNlCtasWanted CTAs per SM with the
// large tile's largest union would not fit the SM's shared memory.
constexpr int kNlTile = 128, kNlTileSmall = 64;
constexpr int kNlCtasWanted = 4;
constexpr int64_t kNlSmemPerSm = 227 * 1024;
constexpr int kNlCap = 1792;      // staged rows of a batched launch (one shared-memory size for all meshes)
constexpr int kNlCapMax = 9216;   // staged rows of a single-mesh launch at most (216 KB)
constexpr int64_t kNlMaxUnion = 65536;   // 16-bit positions

// Extra host data of the mixed-precision path (two-phase assembly).
struct MixedHost {
  std::vector<float> restA;         // [T][kRAStride]
  std::vector<float> restB;         // [T][kRBStride]
  std::vector<float> edge_e0;       // [NE][3] rest edge vectors (b - a)
  // Eq. 20 lists of the mixed kernel, per pair of consecutive tets (2q, 2q+1):
  // the union of the two neighbour sets, entries [nb_ptr[q], nb_ptr[q+1]),
  // each with the neighbour's position in its tile's union (nb_loc) and the
  // two FP32 weights (nb_w2, zero where a tet lacks that neighbour), padded to
  // a multiple of four entries (pads: a position of the list, zero weights);
  // per tile the union's global tet ids nl_uidx[nl_uptr[g], nl_uptr[g+1]),
  // ascending
  std::vector<int64_t> nb_ptr;      // [ceil(T/2) + 1], multiples of 4
  std::vector<uint16_t> nb_loc;
  std::vector<float> nb_w2;         // [entries][2], per block of 32 entries in two planes (see build_mixed_host)
  int64_t nb_real = 0;              // entries without the pads
  std::vector<int64_t> nl_uptr;
  std::vector<int32_t> nl_uidx;
  int32_t nl_cap = 0;               // rows a single-mesh launch stages: the largest union, at most kNlCapMax
  int32_t nl_tile = kNlTile;        // tets per tile
};



gf_status build_mixed_host(const double* X, const struct HostMesh& hm, MixedHost& mx, std::string& err);

// Everything mesh_create computes on the host before upload.
struct HostMesh {
  int64_t n_nodes = 0, n_tets = 0, n_edges = 0, n_blocks = 0;
  std::vector<int32_t> tets;       // [T][4] internal order (the caller's order)
  std::vector<int32_t> perm;       // internal tet -> caller tet (identity)
  std::vector<int32_t> colour_ptr; // [C+1] ranges of colour_tets
  std::vector<int32_t> colour_tets;// [T] tets grouped by colour (no two share a node within a colour)
  // two-phase assembly: node i's rows [np_ptr[i], np_ptr[i+1]) and edge e's
  // rows [et_ptr[e], et_ptr[e+1]), one per incident tet in ascending order
  std::vector<int32_t> np_ptr;     // [N+1]
  std::vector<int32_t> nrow;       // [T][4] node row of (tet, local node)
  std::vector<int32_t> erow;       // [T][6] edge row of (tet, local edge)
  std::vector<int32_t> edge_slot;  // [NE][2] block slots of (i, j) and (j, i), i < j
  std::vector<int32_t> edges;      // [NE][2]
  std::vector<int32_t> tet_edges;  // [T][6] internal order
  std::vector<int32_t> row_ptr;    // [N+1] block-CSR pattern
  std::vector<int32_t> col;        // [NB]
  std::vector<int32_t> diag_blk;   // [N] block index of (i, i)
  std::vector<int32_t> slot;       // [T][16] block index of local (a, b), internal order
  std::vector<int32_t> et_ptr;     // [NE+1] edge -> incident tets (and edge rows)
  std::vector<int32_t> et_tet;     // internal tet ids
  std::vector<int32_t> edge_order; // [NE] gather order of the edges (row counts grouped)
  std::vector<int32_t> node_order; // [N] gather order of the nodes (row counts grouped)
  std::vector<double> rest;        // [kRestFields][T]
  std::vector<double> mass;        // [N] lumped
  NeighbourSell nbr;
};

// Host precompute; returns GF_OK or GF_BAD_ARG with `err` set.
gf_status build_host_mesh(const double* nodes, int64_t n_nodes, const int32_t* tets, int64_t n_tets,
                          const gf_material& mat, HostMesh& hm, std::string& err);

// 64-bit table: bit m set when the broken-edge mask m (bit k = local edge k)
// leaves the tet's four nodes in two or more pieces (Eq. 25's disjoint rule).
uint64_t disconnect_table();

void set_last_error(const std::string& msg);

}  // namespace gf
