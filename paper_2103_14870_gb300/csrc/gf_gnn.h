// Device view of the learned warm start / preconditioner network.
#pragma once

#include <cuda_bf16.h>

#include "gf_device.h"

namespace gf {

constexpr int kHid = 64, kNin = 16, kEin = 16, kNout = 9;
constexpr float kEps = 1e-3f;

// parameter tensors in storage order; per message-passing layer l the five
// tensors Wa, We, bm, Wu, bu follow at +5 l
enum GnnParam { kPW0 = 0, kPb0, kPWa, kPWe, kPbm, kPWu, kPbu, kPWd = 17, kPbd = 18, kGnnTensors = 19 };

struct GnnDev {
  int64_t N = 0, E = 0, P = 0;          // nodes, directed graph edges, parameters
  // graph: off-diagonal pattern of the block system, message j -> i stored in row i
  const int32_t* row_ptr = nullptr;     // [N+1]
  const int32_t* col = nullptr;         // [E] j
  const int32_t* dst = nullptr;         // [E] i
  const int32_t* amap = nullptr;        // [E] block index of A_ij
  const int32_t* tpos = nullptr;        // [E] position of the reverse edge (i -> j) in row j
  const float* relpos = nullptr;        // [E][3] (X_j - X_i) / mean rest edge length
  const float* nstat = nullptr;         // [N][2] log(m_i / mean m), degree / 16
  // per-forward data
  float* efeat = nullptr;               // [E][16]
  float* T = nullptr;                   // [N] trace(A_ii) / 3
  float* C = nullptr;                   // [N][6] Cholesky factor of A_ii^-1 (row-major lower)
  float* Y = nullptr;                   // [N][3] A_ii^-1 b_i on free nodes
  float* B = nullptr;                   // [N][3] b
  uint8_t* freem = nullptr;             // [N]
  float* X0 = nullptr;                  // [N][16] node inputs
  float* Z0 = nullptr;                  // [N][64] encoder pre-activation
  float* H = nullptr;                   // [4][N][64] hidden states
  float* Aa = nullptr;                  // [3][N][64] a = Wa h
  float* M = nullptr;                   // [3][N][64] aggregated messages
  float* ZU = nullptr;                  // [3][N][64] update pre-activations
  float* OUT = nullptr;                 // [N][16] decoder outputs (9 used)
  float* Po = nullptr;                  // [N][9] exported P_i
  float* xo = nullptr;                  // [N][3] exported x0_i
  double* xprev = nullptr;              // [3N] previous step's solution (start of the correction)
  double* ebuf = nullptr;               // [3N] training: x0 - target on free nodes
  double* qbuf = nullptr;               // [3N] training: A_ff (x0 - target)
  // backward
  float* dOUT = nullptr;                // [N][16]
  float* dH = nullptr;                  // [N][64]
  float* dZ = nullptr;
  float* dM = nullptr;
  float* dA = nullptr;
  float* gpart = nullptr;               // [n_gpart][part_stride] per-CTA weight-gradient partials
  int64_t part_stride = 0;
  int n_gpart = 0;
  // parameters
  float* grad = nullptr;                // [P]
  float* w32 = nullptr;                 // [P] master weights
  __nv_bfloat16* w16 = nullptr;         // [P] compute copy
  float* m1 = nullptr;                  // [P] Adam moments
  float* m2 = nullptr;
  int64_t off[kGnnTensors] = {};
  // scalars
  float* scal = nullptr;                // [0] s, [1] loss denominator, [2] mean t
  double* dscal = nullptr;              // [0] loss denominator (FP64)
  double* loss = nullptr;               // [1]
  double* red = nullptr;                // reduction partials
  unsigned* ticket = nullptr;           // [4]
  // tensor-core path
  int use_tc = 1;                       // 1: tcgen05 dense layers and edge messages, 0: FP32 FMA kernels
  int64_t n_etiles = 0;                 // edge-message tiles: whole destination nodes, <= 128 messages and nodes
  const int4* etile = nullptr;          // [n_etiles] (first node, nodes, first message, messages)
  unsigned long long* err = nullptr;    // the mesh's counter of tensor-core waits that gave up
};

// tcgen05 kernels (kernels_tc.cu); each returns the launches issued, or -1 when
// the shape has no tensor-core form
int dense_tc(int64_t N, const float* X1, int K1, int ld1, const float* X2, int K2, int ld2, const __nv_bfloat16* W,
             int ldw, int k0, int trans, const __nv_bfloat16* bias, int NO, float* Z, int ldz, const float* Hres,
             float* Hout, int mode, int accumulate, unsigned long long* err, cudaStream_t s);
int gnn_edge_fwd_tc(const GnnDev& g, const float* a, const __nv_bfloat16* We, const __nv_bfloat16* bm, float* M,
                    cudaStream_t s);
constexpr int kEdgeTileRows = 128;

// forward pass on system A (m.val), right-hand side b (FP64, device); returns launches
int gnn_forward(const GnnDev& g, const DevMesh& m, const double* b, cudaStream_t s);
// start dv = x_prev + x0 (flags bit 0) and learned blocks into m.pinv (bit 1)
int gnn_apply_inference(const GnnDev& g, const DevMesh& m, int flags, cudaStream_t s);
// P_i and x0_i into g.Po and g.xo (nothing of the mesh changes)
int gnn_apply_export(const GnnDev& g, cudaStream_t s);
// energy-norm loss of the pair (b, target) and its gradient, added to g.loss and g.grad (after gnn_forward)
int gnn_backward_pair(const GnnDev& g, const DevMesh& m, const double* target, cudaStream_t s);
int gnn_adam(const GnnDev& g, float scale, float lr, int t, cudaStream_t s);
int gnn_refresh_bf16(const GnnDev& g, cudaStream_t s);
// b = b_sys - A w (w = dv pinned, x_prev free) on free rows; target = dv - x_prev on free nodes (may be NULL)
int gnn_pair(const DevMesh& m, const double* xprev, double* b, double* target, cudaStream_t s);
int gnn_max_parts();
int gnn_reduce_slots();

}  // namespace gf
