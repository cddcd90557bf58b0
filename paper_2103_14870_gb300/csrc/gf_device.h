// Device-side data of one mesh and the kernel launchers (FP64 path).
#pragma once

#include "gf_internal.h"

namespace gf {

// Scalars of one PCG solve, resident in device memory so the iteration loop
// needs no host round trip; kernels read them and the last CTA of each
// reduction writes them.
struct PcgState {
  double bb;      // ||b_free||^2 (reference of the relative tolerance)
  double rz;      // r . z
  double pq;      // p . A p
  double rr;      // r . r
  double alpha, beta;
  double tol2;    // rtol^2
  double true_rr; // ||b - A dv||^2 after the solve
  double rr0;     // ||b - A dv||^2 at the start (a Newton iterate's residual when warm-started)
  int32_t iters, maxit, done, status;
  int32_t cg_k;   // Chronopoulos-Gear form (quasi-static solve): reductions taken so far
};

// counters[3] flags an out-of-range pinned id, counters[4] a tensor-core wait that gave up
enum Counter : int { kCntBroken = 0, kCntNewBroken = 1, kCntChiZero = 2, kCntBadPin = 3, kCntTcTimeout = 4, kCntMax = 8 };

// Scalars of the mixed-precision solve: FP64 iterative refinement (outer)
// around an FP32 PCG (inner) whose dot products accumulate in FP64.
struct IrState {
  double bb;        // ||b_free - A dv_fixed||^2 (reference)
  double rr;        // ||r64||^2 of the last FP64 residual
  double tol2;      // outer rtol^2
  double in_tol2;   // inner rtol^2
  double rz, pq, alpha, beta, in_rr, in_rr0;
  float alpha32, beta32;
  int32_t done;     // outer converged (or failed)
  int32_t in_done;  // inner converged for this sweep
  int32_t sweeps, in_iters, total_iters, in_maxit, maxit, status;
  int32_t applied;  // the last inner correction was applied and a new residual is due
};

// Device arrays of the mixed-precision path.
struct MixDev {
  const float* restA = nullptr;       // [T][kRAStride] (128-byte aligned rows)
  const float* restB = nullptr;       // [T][kRBStride]
  const float* edge_e0 = nullptr;     // [NE][3]
  const int64_t* nb_ptr = nullptr;    // [ceil(T/2)+1] Eq. 20 joint lists of tet pairs (2q, 2q+1)
  const uint16_t* nb_loc = nullptr;   // per entry: the neighbour's position in its tile's union
  const float2* nb_w2 = nullptr;      // per entry: the FP32 weights of tets 2q and 2q+1 (0 if not a neighbour), per block of 32 entries in two planes
  const int64_t* nl_uptr = nullptr;   // [ceil(T / nl_tile) + 1] tile unions
  const int32_t* nl_uidx = nullptr;   // union members (global tet ids, ascending per tile)
  int32_t nl_cap = 0;                 // rows a single-mesh launch stages (its shared memory: 24 B a row)
  int32_t nl_tile = 128;              // tets per tile (128, or 64 for a wide radius)
  const float* mass32 = nullptr;      // [N]
  const float* mass_blk32 = nullptr;  // [NB] consistent mass per block slot (NULL: lumped)
  const double* X = nullptr;          // [3N] rest positions
  float* u32 = nullptr;               // [3N] displacement x - X
  float* v32 = nullptr;               // [3N] velocity
  float* chi32 = nullptr;             // [T]
  float* sig_in32 = nullptr;          // [T][8] (6 used; 32-byte rows for single-sector gathers)
  float* sig_bar32 = nullptr;         // [T][8]
  float* val32 = nullptr;             // [NB][9]
  float* ebuf = nullptr;              // [4T][4] node rows (rhs), then [6T][9] edge rows (two-phase assembly)
  float* rhs32 = nullptr;             // [3N]
  float* rres = nullptr;              // [3N] leading float of the refinement residual
  float* pinv32 = nullptr;            // [N][9]
  float *r32 = nullptr, *z32 = nullptr, *p32 = nullptr, *q32 = nullptr, *d32 = nullptr;   // [3N]
  float* p32b = nullptr;              // [3N] second search-direction buffer of the persistent solve
  float* w32 = nullptr;               // [3N] A z of the two-kernel inner PCG
  float4* z4 = nullptr;               // [N] z of the two-kernel inner PCG, one 16-byte row per node (w unused)
  float *dv_hi = nullptr, *dv_lo = nullptr;   // [3N] double-float split of dv
  IrState* ir = nullptr;
};

struct DevMesh {
  int64_t N = 0, T = 0, NE = 0, NB = 0, G = 0;    // nodes, tets, edges, blocks, neighbour groups
  // fixed mesh data
  const int4* tets = nullptr;          // [T] internal order
  const int32_t* tet_edges = nullptr;  // [T][6]
  const int32_t* slot = nullptr;       // [T][16]
  const double* rest = nullptr;        // [kRestFields][T]
  const double* mass = nullptr;        // [N] lumped (row sums of Eq. 5)
  const double* mass_blk = nullptr;    // [NB] consistent mass m_ij of Eq. 5 per block slot (NULL: lumped)
  const int32_t* row_ptr = nullptr;    // [N+1]
  const int32_t* col = nullptr;        // [NB]
  const int32_t* diag_blk = nullptr;   // [N]
  const int2* edges = nullptr;         // [NE]
  const int32_t* et_ptr = nullptr;     // [NE+1]
  const int32_t* et_tet = nullptr;
  const int32_t* colour_tets = nullptr;  // [T] tets grouped by colour
  // assembly rows: node i owns rows [np_ptr[i], np_ptr[i+1]) and edge e rows
  // [et_ptr[e], et_ptr[e+1]), one per incident tet in ascending tet order
  const int32_t* np_ptr = nullptr;     // [N+1]
  const int32_t* nrow = nullptr;       // [T][4] node row of (tet, local node)
  const int32_t* erow = nullptr;       // [T][6] edge row of (tet, local edge)
  const int2* edge_slot = nullptr;     // [NE] block slots of (i, j) and (j, i), i < j
  const int32_t* edge_order = nullptr; // [NE] FP64 gather and edge driver: slot -> edge, row counts grouped
  const int32_t* node_order = nullptr; // [N] FP64 gather and diagonal: slot -> node, row counts grouped
  const int64_t* nb_off = nullptr;     // [G]
  const int32_t* nb_len = nullptr;     // [G]
  const int32_t* nb_idx = nullptr;
  const int32_t* nb_perm = nullptr;    // [T] lane slot -> tet (the SELL order)
  const double* nb_w = nullptr;
  // state
  double* x = nullptr;                 // [3N]
  double* v = nullptr;                 // [3N]
  uint8_t* labels = nullptr;           // [NE]
  double* chi = nullptr;               // [T] internal order
  double* driver = nullptr;            // [NE]
  // per-step work
  double* sig_in = nullptr;            // [T][6] averaged field (chi S or S)
  double* sig_bar = nullptr;           // [T][6] Eq. 20 averages
  double* sigf = nullptr;              // [T][6] local edge-normal stresses
  double* val = nullptr;               // [NB][9] system matrix A
  double* ebuf = nullptr;              // [4T][4] node rows (rhs), then [6T][9] edge rows (two-phase assembly)
  double* rhs = nullptr;               // [3N] b
  double* dv = nullptr;                // [3N] unknown
  double* r = nullptr;
  double* z = nullptr;
  double* p = nullptr;
  double* q = nullptr;
  double* w = nullptr;                 // [3N] A z of the quasi-static Chronopoulos-Gear PCG
  double* pinv = nullptr;              // [N][9] block-Jacobi inverses
  uint8_t* pinned = nullptr;           // [N] 1 = velocity prescribed
  double* f_ext = nullptr;             // [3N] staging
  int32_t* pin_ids = nullptr;          // [N] staging
  double* pin_vel = nullptr;           // [3N] staging
  PcgState* pcg = nullptr;
  MixDev mx;                           // mixed-precision arrays (GF_MIXED only)
  double* partials = nullptr;          // reduction partials
  unsigned* tickets = nullptr;         // reduction tickets (one per reduction site)
  unsigned long long* counters = nullptr;  // [kCntMax]
};

struct Material {
  double lam, mu, young, alpha, beta, threshold, radius;
  double kappa;       // shear coefficient of Eq. 16
  int driver_stress;  // 0: driver = sigma*/E, 1: sigma*
  int average_degraded;
  uint64_t lut;       // disconnection table of Eq. 25
  float lam32, mu32, kappa32, young32, inv_young32;
  int energy;         // GF_ENERGY_STVK (Eq. 37) or GF_ENERGY_SNH (Eq. 35)
  double snh_a;       // a = 1 + mu/lam - mu/(4 lam) of Eq. 35
};

// Per-step scalars of one mesh, formed on the host (no FP64 scalar work per
// thread on the device).
struct StepScalars {
  double dt;
  float dtf, sKv, cv, alphaf, cmf;   // dt, dt beta + dt^2, beta + dt, alpha, 1 + dt alpha
  int has_fext, has_pvel;
  int learned;                        // pcg_init keeps the preconditioner, start and |b_free|^2 already set
  int warm;                           // pcg_init starts from the dv in place (Newton iterations after the first)
  double mscale;                      // factor on the mass in the matrix (1; 0 for the quasi-static system)
  int64_t n_pinned;
};

StepScalars step_scalars(const Material& mt, double dt, bool has_fext, int64_t n_pinned, bool has_pvel);

constexpr int kMaxPartials = 4096;     // max CTAs of a reducing launch
constexpr int kTickets = 16;

// ---------------------------------------------------------------------------
// Batched execution: one launch per kernel kind covers every mesh of a batch.
// Block b of a batched launch belongs to the mesh k with off[kind][k] <= b <
// off[kind][k+1]; inside, the kernel body sees that mesh's data and its local
// block index and count (reductions and grid-stride loops stay per mesh).
// ---------------------------------------------------------------------------
// The FP64 kinds come first: every kind below kB_tet_stress32 is launched by
// the FP64 dispatcher, every kind from it on by the mixed one.
enum BatchKind : int {
  kB_tet_stress = 0, kB_nonlocal, kB_edge_driver, kB_tet_chi, kB_node_init, kB_elem64, kB_gather64, kB_diag64, kB_set_pinned,
  kB_pcg_init, kB_pcg_spmv, kB_pcg_update, kB_pcg_p, kB_true_residual, kB_integrate,
  kB_tet_stress32, kB_nonlocal32, kB_edge_driver32, kB_tet_chi32, kB_elem32, kB_gather32,
  kB_ir_residual, kB_ir_inner_init, kB_ir_spmv, kB_ir_update, kB_ir_p, kB_ir_apply, kB_integrate32, kB_refresh32,
  kB_chi_to32, kB_diag32, kB_step_begin, kB_ir_cg_spmv, kB_ir_cg_update, kBKinds
};
constexpr int kMaxBatch = 256;

struct BatchTab {
  int32_t n;
  int32_t off[kBKinds][kMaxBatch + 1];
  DevMesh mesh[kMaxBatch];
  Material mt[kMaxBatch];
  StepScalars sp[kMaxBatch];
};

#ifdef __CUDACC__
__device__ __forceinline__ int batch_locate(const BatchTab* __restrict__ tab, int kind, unsigned b, unsigned& bid,
                                            unsigned& nb) {
  const int32_t* off = tab->off[kind];
  int lo = 0, hi = tab->n;            // off[lo] <= b < off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (unsigned(off[mid]) <= b) lo = mid;
    else hi = mid;
  }
  bid = b - unsigned(off[lo]);
  nb = unsigned(off[lo + 1] - off[lo]);
  return lo;
}
#endif

// Work table of the distributed solver loop of a batch (GF_SOLVE_DISTRIBUTED):
// the meshes that have not converged and, per solver-loop kind, the offsets
// of their blocks (each mesh keeps its own single-mesh grid).  A kernel rebuilds
// it on the device after every loop iteration; the loop kernels then run with a
// fixed grid whose CTAs take the listed blocks in turn, so a converged mesh
// costs nothing and an active one keeps its full grid.
struct BatchAct {
  int32_t n;                             // meshes still iterating
  int32_t mesh[kMaxBatch];               // their ids, ascending
  int32_t off[kBKinds][kMaxBatch + 1];   // per solver-loop kind: block offsets over them
};

#ifdef __CUDACC__
__device__ __forceinline__ int act_locate(const BatchAct* __restrict__ a, int kind, unsigned w, unsigned& bid,
                                          unsigned& nb) {
  const int32_t* off = a->off[kind];
  int lo = 0, hi = a->n;            // off[lo] <= w < off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (unsigned(off[mid]) <= w) lo = mid;
    else hi = mid;
  }
  bid = w - unsigned(off[lo]);
  nb = unsigned(off[lo + 1] - off[lo]);
  return a->mesh[lo];
}
#endif

// Launch geometry of each kind for one mesh: (blocks, threads).
struct LaunchDims {
  unsigned blocks, threads;
};
LaunchDims launch_dims(int kind, const DevMesh& m, const Material& mt, const StepScalars& sp);
// One batched launch of `kind` over all meshes of the device table `tab`
// (`blocks` = total over the meshes, from the host copy of the offsets).
int launch_batch(int kind, const BatchTab* tab, unsigned blocks, cudaStream_t s, int first = 0);
int launch_kind_fp64(int kind, const DevMesh& m, const Material& mt, const StepScalars& sp, cudaStream_t s);
int launch_kind_mixed(int kind, const DevMesh& m, const Material& mt, const StepScalars& sp, cudaStream_t s, int first);
int launch_batch_fp64(int kind, const BatchTab* tab, unsigned blocks, unsigned threads, cudaStream_t s);
int launch_batch_mixed(int kind, const BatchTab* tab, unsigned blocks, unsigned threads, cudaStream_t s, int first);
// Distributed solver-loop launches: `grid` CTAs over the blocks listed in `act`
// (solver-loop kinds only; returns 0 for other kinds).
int launch_dist_fp64(int kind, const BatchTab* tab, const BatchAct* act, unsigned grid, cudaStream_t s);
int launch_dist_mixed(int kind, const BatchTab* tab, const BatchAct* act, unsigned grid, cudaStream_t s);

// Persistent refinement solve (GF_MIXED): one cooperative launch runs the whole
// solver loop of every mesh in `tab` (inner FP32 PCG and double-float
// refinement), with grid barriers between its phases instead of kernel
// boundaries.  Each phase processes the blocks of the meshes that need it, so
// converged meshes take no CTAs.  Every barrier wait is bounded.
// Phases decide which meshes take part from per-mesh flags (done, in_done,
// applied).  A phase's last block may change them while a CTA without work in
// that phase is still reading them, so the flags live in two slots: during the
// phase after barrier g every CTA reads slot g & 1, and the phase writes slot
// (g + 1) & 1 (the last block of a mesh its new flags, block 0 the unchanged
// flags of the meshes that sit the phase out).
struct PersistCtl {
  unsigned arrive;   // grid-barrier arrivals of the running launch (reset before each launch)
  int error;         // 1: a barrier wait ran out and the launch stopped early
  int rounds;        // rounds the launch ran
  int test_skip;     // test hook: block 0 skips its first arrival, so every wait of that barrier runs out
  int flags[2][kMaxBatch][3];   // [slot][mesh]: done, in_done, applied
};
constexpr unsigned long long kPersistWaitNs = 1000000000ull;   // limit of one barrier wait (1 s)
// Grid of the persistent launch on the current device (resident CTAs x SMs).
unsigned persist_grid();
// Enqueue the persistent solve (a small kernel that resets `ctl` and takes the
// meshes' flags, then the cooperative launch); `cap` bounds its rounds,
// test_skip arms the test hook.  Returns the kernels launched (2), or -1 if the
// cooperative launch was refused.
int launch_ir_persist(const BatchTab* tab, int n, PersistCtl* ctl, int cap, int test_skip, cudaStream_t s);

// single-mesh launches (return the number of kernels launched)
int launch_kind(int kind, const DevMesh& m, const Material& mt, const StepScalars& sp, cudaStream_t s, int first = 0);
int launch_assemble_colour(const DevMesh& m, const Material& mt, double dt, int t0, int t1, cudaStream_t s);
// Newton iterate k >= 1 of the FP64 step: xk = x + dt (v + dv), w = v - dt (v + dv) / (beta + dt)
int launch_newton_prep(const DevMesh& m, const Material& mt, double dt, double* xk, double* w, cudaStream_t s);
// Quasi-static step pieces (FP64): total energy and its magnitude at positions x into out[0..1];
// r . d over free DOFs (r = m.rhs, d = m.dv) into out[2]; xt = x + a d; pinned positions
int launch_qs_energy(const DevMesh& m, const Material& mt, const double* x, const double* f_ext, double* out,
                     cudaStream_t s);
int launch_qs_slope(const DevMesh& m, double* out, cudaStream_t s);
int launch_qs_cg_spmv(const DevMesh& m, cudaStream_t s);     // Chronopoulos-Gear PCG: w = A z, dots, coefficients
int launch_qs_cg_update(const DevMesh& m, cudaStream_t s);   // Chronopoulos-Gear PCG: vector updates
int launch_qs_trial(int64_t n, const double* x, const double* d, double a, double* xt, cudaStream_t s);
// Quasi-static solve with an FP32 inner PCG: val32/pinv32 from the FP64 system,
// the first inner start, and per outer flexible-PCG iteration w = A z with its
// coefficients, then the FP64 updates and the next inner start (m.mx holds the
// FP32 buffers and IrState, m.pcg the outer scalars, m.w the vector A z)
int launch_qsr_to32(const DevMesh& m, cudaStream_t s);
int launch_qsr_start(const DevMesh& m, cudaStream_t s);
int launch_nested_finish(const DevMesh& m, cudaStream_t s);   // its outcome into m.pcg
int launch_fcg_spmv(const DevMesh& m, cudaStream_t s);
int launch_fcg_update(const DevMesh& m, cudaStream_t s);
int launch_qs_set_pins(const DevMesh& m, const int32_t* ids, const double* pos, int64_t n_pinned, cudaStream_t s);

}  // namespace gf
