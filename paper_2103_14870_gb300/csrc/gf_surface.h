// Device view of the split visualisation mesh (Sec. 4.1) and its launchers.
#pragma once

#include <algorithm>

#include "gf_device.h"

namespace gf {

struct SurfDev {
  int64_t NF = 0;                       // unique faces
  const double* X = nullptr;            // [3N] rest positions
  const int3* faces = nullptr;          // [NF] sorted node triples
  const int3* face_edges = nullptr;     // [NF] edge ids of (f0,f1), (f0,f2), (f1,f2)
  const int4* tet_faces = nullptr;      // [T] face opposite each local node
  unsigned* bsum = nullptr;             // [blocks + 1] quad counts per block of tets, then their prefix
};

int64_t surf_blocks(const DevMesh& m);
// quad counts: exclusive prefix per block of tets in sd.bsum, the total in sd.bsum[blocks]
int launch_surface_count(const DevMesh& m, const SurfDev& sd, cudaStream_t s);
// V [N + 2 NE + 3 NF + 4 T][3]: nodes, edge, face and tet children
int launch_surface_vertices(const DevMesh& m, const SurfDev& sd, double* V, cudaStream_t s);
// Q [n_quads][4] after launch_surface_count (writes only quads below max_quads)
int launch_surface_quads(const DevMesh& m, const SurfDev& sd, int32_t* Q, int64_t max_quads, cudaStream_t s);

}  // namespace gf
