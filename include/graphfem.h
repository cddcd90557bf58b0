/*
 * graphfem.h -- C ABI of the GB300 graph-based FEM fracture step.
 *
 * Method: Mandal, Chaudhuri & Chaudhuri, "Remeshing-Free Graph-Based Finite
 * Element Method for Ductile and Brittle Fracture".  One call to gf_step()
 * performs one implicit time step of Algorithm 1 (Sec. 4.3) on a fixed
 * tetrahedral mesh graph:
 *   1. stresses along the mesh edges at the start-of-step positions (Eq. 14-19),
 *      non-local average (Eq. 20), irreversible edge relabel (Eq. 21) and the
 *      energy degradation chi of every tet (Eq. 22-25);
 *   2. element forces in squared edge lengths (Eq. 12, Thm 3.1 / Eq. 27-31,
 *      StVK Eq. 37) and 12x12 tangents, scaled by chi (Eq. 32-34), scattered
 *      into a block-CSR matrix whose sparsity never changes (Sec. 1, Sec. 5.4);
 *   3. the linearised backward-Euler system of Eq. 2 with Rayleigh damping
 *      (Sec. 3.1, Sec. 3.6) solved by preconditioned conjugate gradients
 *      (Sec. 4.3), then v += dv, x += dt v.
 *
 * Conventions shared by every entry point
 *   - Node arrays are node-major: x[3*i + c], c in {0,1,2}.
 *   - Edges are the unique node pairs of the tets, numbered in ascending
 *     lexicographic order of (min id, max id); gf_edges_get() returns them.
 *   - Tets keep the caller's numbering at the ABI (the library reorders them
 *     internally and maps back).
 *   - `mem` arguments say where the caller's pointers live: GF_MEM_HOST (any
 *     host memory; pinned memory makes the copies faster) or GF_MEM_DEVICE
 *     (device memory of the mesh's device; the pointer must stay valid until
 *     the call returns).
 *   - The library owns every device buffer of a mesh.  The caller owns what it
 *     passes in; arrays are copied during the call and not retained.
 *   - Every call returns a gf_status; nothing is thrown across the ABI.  On
 *     error, gf_last_error() gives a message for the calling thread.
 *   - Calls on one mesh are not thread-safe; distinct meshes are independent.
 *   - All device work runs on the mesh's stream; every call returns after
 *     that work has completed.
 */
#ifndef GRAPHFEM_H
#define GRAPHFEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gf_status {
  GF_OK = 0,
  GF_BAD_ARG = 1,        /* invalid argument (null, out of range, degenerate tet, ...) */
  GF_CUDA_ERR = 2,       /* a CUDA runtime call or kernel launch failed */
  GF_CG_BREAKDOWN = 3,   /* p^T A p <= 0: the tangent is not positive definite (StVK under compression) */
  GF_CG_MAXITER = 4,     /* CG did not reach the tolerance within cg_maxit iterations */
  GF_NAN = 5,            /* a non-finite residual or state appeared */
  GF_TIMEOUT = 6,        /* a bounded device-side wait gave up */
  GF_OOM = 7,            /* device allocation failed */
  GF_UNSUPPORTED = 8     /* option combination not built */
} gf_status;

enum { GF_MEM_HOST = 0, GF_MEM_DEVICE = 1 };
enum { GF_DRIVER_STRAIN = 0, GF_DRIVER_STRESS = 1 };
enum { GF_FP64 = 0, GF_MIXED = 1 };
enum { GF_PRECOND_BJACOBI = 0 };
enum { GF_ASSEMBLY_GATHER = 0, GF_ASSEMBLY_COLOUR = 1 };
enum { GF_MASS_LUMPED = 0, GF_MASS_CONSISTENT = 1 };
enum { GF_ENERGY_STVK = 0, GF_ENERGY_SNH = 1 };

/* Material and damage parameters (Sec. 3.1, 3.3, 5.2). */
typedef struct gf_material {
  double young;          /* Young's modulus E (Pa) */
  double poisson;        /* Poisson ratio nu, in (-1, 0.5) */
  double density;        /* rho (kg/m^3); element mass of Eq. 5, see mass_matrix */
  double alpha;          /* Rayleigh mass damping (b_e = alpha m_e + beta k_e*, Sec. 3.6) */
  double beta;           /* Rayleigh stiffness damping */
  double threshold;      /* sigma_thres of Eq. 21 in driver units; +inf disables fracture */
  double radius;         /* kernel support R_d of Eq. 20 (length units); 0 = local criterion */
  int32_t driver_mode;   /* GF_DRIVER_STRAIN: driver = sigma_star divided by E (dimensionless); GF_DRIVER_STRESS: sigma_star */
  int32_t shear_coef;    /* 2: normal stress n.S.n (default); 1: Eq. 16 as printed */
  int32_t average_degraded; /* 1: Eq. 20 averages chi_j S_j (default); 0: raw S_j */
  int32_t mass_matrix;   /* GF_MASS_LUMPED (0, default): row sums of Eq. 5, rho V_e / 4 per node and
                            tet; GF_MASS_CONSISTENT: Eq. 5 as it stands, rho V_e (1 + delta_ab) / 20
                            between the nodes a, b of a tet (same block pattern as K) */
  int32_t energy;        /* GF_ENERGY_STVK (0, default): Eq. 37; GF_ENERGY_SNH: the stable
                            Neo-Hookean energy of Eq. 35 with (J - a)^2, a = 1 + mu/lam - mu/(4 lam),
                            J the signed det F; needs 0 < nu < 0.5, GF_FP64, two-phase assembly.
                            The damage criterion then uses its S = 2 dPsi/dC (Eq. 14). */
  int32_t reserved;      /* set to 0 */
} gf_material;

typedef void* (*gf_alloc_fn)(size_t bytes, void* ctx);
typedef void (*gf_free_fn)(void* ptr, void* ctx);

/* Solver and runtime options. Zero-initialise and set what you need. */
typedef struct gf_options {
  int32_t precision;     /* GF_FP64 (default) or GF_MIXED */
  int32_t cg_maxit;      /* 0 -> 10000 */
  double cg_rtol;        /* stop when ||r|| <= cg_rtol ||b|| on free DOFs; 0 -> 1e-6 */
  int32_t precond;       /* GF_PRECOND_BJACOBI */
  int32_t device;        /* CUDA device ordinal; -1 -> the current device */
  void* stream;          /* cudaStream_t for all work; NULL -> a stream the library creates */
  gf_alloc_fn alloc;     /* optional device allocator (e.g. a caching allocator); NULL -> cudaMalloc.
                            It must return 16-byte-aligned device memory (else GF_BAD_ARG) */
  gf_free_fn free;       /* matching free; required when alloc is set */
  void* alloc_ctx;       /* passed to alloc/free */
} gf_options;

/* Per-step diagnostics (all counts after the step). */
typedef struct gf_step_stats {
  int32_t status;        /* gf_status of the step */
  int32_t cg_iters;      /* CG iterations of the step (all refinement sweeps in GF_MIXED) */
  double rel_res;        /* final ||b - A dv|| / ||b|| on free DOFs, FP64 */
  int64_t n_broken;      /* edges with zeta = 1 */
  int64_t n_new_broken;  /* edges that broke in this step */
  int64_t n_chi_zero;    /* tets split into disjoint pieces (chi = 0) */
  int32_t refine_sweeps; /* GF_MIXED: FP64 refinement sweeps; 0 in GF_FP64 */
  int32_t newton_iters;  /* Newton iterations the step ran (gf_newton_set) */
} gf_step_stats;

typedef struct gf_mesh_info {
  int64_t n_nodes;
  int64_t n_tets;
  int64_t n_edges;
  int64_t n_blocks;      /* 3x3 blocks of the fixed block-CSR pattern (node adjacency incl. diagonal) */
  int64_t n_colours;     /* tet colours of the conflict-free assembly scatter */
  int64_t n_nbr_pairs;   /* (tet, neighbour) pairs of Eq. 20 within R_d */
  int64_t device_bytes;  /* device memory held by the mesh */
  int64_t n_joint_entries; /* GF_MIXED: entries of the Eq. 20 joint lists of tet pairs, not counting the
                              padding of each list to a multiple of four (0 otherwise) */
  int64_t n_union_rows;  /* GF_MIXED: tet ids in the per-tile neighbour unions of Eq. 20 (0 otherwise) */
  int64_t eq20_tile;     /* GF_MIXED: tets per tile of the Eq. 20 kernel, 128 or 64 for a wide radius (0 otherwise) */
} gf_mesh_info;

typedef struct gf_mesh gf_mesh;

/* Build a mesh from rest nodes (host, float64 [3*n_nodes]) and tets (host,
 * int32 [4*n_tets], node ids in [0, n_nodes)).  Precomputes edges, rest data,
 * lumped mass, the fixed block-CSR pattern, the tet colouring and the Eq. 20
 * neighbour lists, then uploads them.  The state starts at rest: x = nodes,
 * v = 0, no broken edge, chi = 1.  Degenerate (zero-volume) tets -> GF_BAD_ARG.
 * `opt` may be NULL (defaults).  On success *out owns device memory until
 * gf_mesh_destroy(). */
gf_status gf_mesh_create(const double* nodes, int64_t n_nodes, const int32_t* tets, int64_t n_tets,
                         const gf_material* mat, const gf_options* opt, gf_mesh** out);

/* Host-only planning: runs the mesh_create precompute on the CPU without
 * touching a GPU and reports its sizes in *info (device_bytes is an estimate).
 * Optional outputs (host memory, NULL to skip): edges int32 [2*n_edges] (call
 * once with NULL to learn n_edges), colour int32 [n_tets] (the colour of each
 * caller tet in the conflict-free scatter), nbr_count int32 [n_tets] (Eq. 20
 * neighbours within R_d of each caller tet, itself included). */
gf_status gf_mesh_plan(const double* nodes, int64_t n_nodes, const int32_t* tets, int64_t n_tets,
                       const gf_material* mat, gf_mesh_info* info, int32_t* edges, int32_t* colour,
                       int32_t* nbr_count);

/* Release a mesh (NULL is ignored). */
void gf_mesh_destroy(gf_mesh* mesh);

gf_status gf_mesh_info_get(const gf_mesh* mesh, gf_mesh_info* info);

/* Overwrite the state.  x, v: float64 [3*n_nodes]; labels: uint8 [n_edges]
 * (0 unbroken, 1 broken, Eq. 21); chi: float64 [n_tets] in caller tet order.
 * Any pointer may be NULL to keep that part.  When labels are given and chi is
 * NULL, chi is recomputed from the labels at the (new) positions by Eq. 25. */
gf_status gf_state_set(gf_mesh* mesh, const double* x, const double* v, const uint8_t* labels,
                       const double* chi, int32_t mem);

/* One implicit time step (Algorithm 1).  dt > 0.  f_ext: float64 [3*n_nodes]
 * external nodal forces (NULL = none).  pinned: int32 [n_pinned] node ids whose
 * velocity is prescribed: pinned_vel float64 [3*n_pinned] (NULL = zero).
 * Pointers follow `mem`.  stats may be NULL.  A CG failure leaves the step
 * applied with the last iterate and returns GF_CG_BREAKDOWN / GF_CG_MAXITER. */
gf_status gf_step(gf_mesh* mesh, double dt, const double* f_ext, const int32_t* pinned, int64_t n_pinned,
                  const double* pinned_vel, int32_t mem, gf_step_stats* stats);

/* Execution schedule of a mesh (no effect on results beyond rounding order).
 * assembly: GF_ASSEMBLY_GATHER (default) computes every tet's blocks once into
 * an element buffer and gathers each matrix row in a fixed order (one launch
 * per phase); GF_ASSEMBLY_COLOUR scatters tet by tet in colour order (no two
 * tets of a colour share a node), one launch per colour (GF_FP64 only).
 * step_launch: GF_STEP_GRAPH (default) runs a plain step (one Newton
 * iteration, gather assembly, no network attached, profiling off) as one CUDA
 * graph replay: its launches are captured on the first such step and again
 * whenever dt, the presence of f_ext / pinned velocities, the pinned count or
 * the iteration limit change (device inputs are copied into the mesh's own
 * buffers first, so a new caller buffer per step costs no capture); the solver loop is
 * a device-side WHILE node, so the host waits once per step.  The results are
 * the same bits as GF_STEP_STREAM, which launches kernel by kernel with a host
 * check per chunk of solver iterations (and is what the other steps use). */
enum { GF_STEP_GRAPH = 0, GF_STEP_STREAM = 1 };
/* solve_loop: the form of the solver loop.  A new mesh starts with
 * GF_SOLVE_KERNELS (GF_FP64) or GF_SOLVE_CG (GF_MIXED), the faster form of
 * each on the measured workloads.
 * GF_SOLVE_KERNELS: kernel by kernel, three per PCG iteration (GF_FP64, or the
 * inner FP32 PCG of GF_MIXED) with the refinement's phase kernels around the
 * inner solves, as a WHILE node of the step graph or with host checks in the
 * stream form.
 * GF_SOLVE_CG: two kernels per iteration.  GF_FP64: the PCG in the
 * Chronopoulos-Gear form (Chronopoulos and Gear, 1989): w = A z and the three
 * dot products in one kernel, the vector updates in another, one grid
 * reduction per iteration.  GF_MIXED: the inner FP32 PCG with q = A p carried
 * by recurrence (w = A z and z.w in one kernel; p, q, d, r, z and r.z, r.r in
 * the other).  The iterates equal the three-kernel form's in exact arithmetic.
 * GF_SOLVE_PERSISTENT (GF_MIXED only): the whole refinement loop as one
 * cooperative launch (one CTA set resident on every SM), with grid barriers
 * between its phases and the direction update fused into the SpMV.  Each barrier
 * wait gives up after 1 s and the step then returns GF_TIMEOUT (the mesh state
 * is then unspecified: set it again with gf_state_set).
 * GF_SOLVE_NESTED (GF_FP64 only): the step's linear solve as flexible PCG in
 * FP64 around an inner PCG in FP32 on the matrix and block inverses rounded to
 * FP32, the quasi-static step's GF_QS_SOLVE_NESTED (inner tolerance: the one
 * gf_quasistatic_solver_set sets, default 1e-2).  It stops at the FP64 PCG's
 * residual test, so it solves the same FP64 system; it pays on stiff systems
 * with many PCG iterations.  Steps in this form launch kernel by kernel (the
 * solve loop itself is one graph); stats report the inner iterations.
 * GF_SOLVE_DISTRIBUTED is a batch form (gf_batch_tuning).
 * Another form than the precision supports -> GF_UNSUPPORTED.
 * wait_test: a test hook; 1 makes one CTA of the next persistent solve skip its
 * first barrier arrival, so that every wait of that barrier runs out (the
 * step returns GF_TIMEOUT after about 1 s).  Leave it 0. */
enum { GF_SOLVE_KERNELS = 0, GF_SOLVE_PERSISTENT = 1, GF_SOLVE_CG = 2, GF_SOLVE_DISTRIBUTED = 3, GF_SOLVE_NESTED = 4 };
typedef struct gf_tuning {
  int32_t assembly;
  int32_t step_launch;   /* GF_STEP_GRAPH (0, default) or GF_STEP_STREAM */
  int32_t solve_loop;    /* GF_SOLVE_KERNELS, GF_SOLVE_CG, GF_SOLVE_PERSISTENT or GF_SOLVE_NESTED (default: see above) */
  int32_t wait_test;     /* test hook, 0 */
  int32_t reserved[4];   /* set to 0 */
} gf_tuning;
gf_status gf_tuning_set(gf_mesh* mesh, const gf_tuning* tuning);
gf_status gf_tuning_get(const gf_mesh* mesh, gf_tuning* tuning);

/* Autotuner of one mesh: times `trial_steps` steps (1..64) under each candidate
 * schedule on the mesh's current state, restoring the state (positions,
 * velocities, labels, chi and the FP32 copies) after each, and keeps the
 * fastest.  Candidates: GF_FP64: the two-phase gather and, for the StVK
 * energy, the colour-ordered assembly, each with the solver-loop forms
 * GF_SOLVE_KERNELS, GF_SOLVE_CG and GF_SOLVE_NESTED; GF_MIXED: GF_SOLVE_CG,
 * GF_SOLVE_KERNELS and GF_SOLVE_PERSISTENT; graph launches where the form has
 * them.  Inputs as in gf_step.  best (nullable) receives the chosen tuning, ms
 * (nullable) its time per step.  GF_UNSUPPORTED while a network is attached or
 * with Newton iterations > 1 (their steps carry state between iterations). */
gf_status gf_mesh_autotune(gf_mesh* mesh, double dt, const double* f_ext, const int32_t* pinned, int64_t n_pinned,
                           const double* pinned_vel, int32_t mem, int32_t trial_steps, gf_tuning* best, double* ms);

/* GF_MIXED: relative tolerance of each inner FP32 PCG solve of the FP64
 * iterative refinement (default 1e-5; 0 < inner_rtol < 1; each inner solve also
 * stops after 32 iterations).  The outer FP64 tolerance stays cg_rtol.  At the
 * default, a well-conditioned system at cg_rtol 1e-6 needs one sweep. */
gf_status gf_refine_set(gf_mesh* mesh, double inner_rtol);

/* Change the break threshold sigma_thres of Eq. 21 between steps (same units
 * as gf_material.threshold; +inf breaks nothing).  For a threshold calibrated
 * on the mesh's own run (e.g. a quantile of its drivers).  Labels already
 * broken stay broken.  A batch copies its meshes' materials when it is
 * created, so set the threshold before gf_batch_create.  NaN -> GF_BAD_ARG. */
gf_status gf_threshold_set(gf_mesh* mesh, double threshold);

/* Change the solver tolerance and iteration cap between steps (rtol > 0). */
gf_status gf_solver_set(gf_mesh* mesh, double cg_rtol, int32_t cg_maxit);

/* Newton iterations per step (default 1: the backward-Euler update of Eq. 2
 * linearised at x_n).  With max_iters > 1 the step solves the backward-Euler
 * residual r(v) = M (v - v_n) + dt (B v - f_ext - f*(x_n + dt v)),
 * B = alpha M + beta K*(x_n + dt v), by Newton's method from v = 0, with chi
 * frozen for the step.  Each iteration re-assembles the system at
 * x^k = x_n + dt v^k and solves it to cg_rtol (PCG warm-started from the
 * previous iterate).  It stops after max_iters (1..64) or once
 * |r(v^k)| <= rtol |b^0| on free DOFs (b^0 the first right-hand side; rtol 0
 * runs all iterations).  GF_FP64 meshes only (GF_UNSUPPORTED for GF_MIXED and
 * for batches). */
gf_status gf_newton_set(gf_mesh* mesh, int32_t max_iters, double rtol);

/* Quasi-static load step (Eq. 36; the paper's quasi-static runs solve it by
 * Newton's method with a line search, Sec. 4.3).  No mass or damping.  Order:
 * the damage update at the current positions (stress, Eq. 20 average,
 * relabel, chi, as in gf_step), then the pinned nodes move to pinned_pos
 * (host or device float64 [3 * n_pinned] following `mem`; NULL keeps them
 * where they are), then Newton iterations on f*(x) + f_ext = 0 over the free
 * DOFs with chi frozen: K* d = f_ext + f* solved by the PCG to cg_rtol, step
 * length halved from 1 until the total energy
 * E = sum_e chi_e V_e Psi_e - f_ext . x meets the Armijo condition with
 * c = 1e-4 (or the decrease asked for is below 1e-12 of the magnitude of E's
 * terms, where E cannot resolve it).  Stops when |f_ext + f*| on free DOFs is
 * <= rtol times its value at the first iteration, or after max_newton
 * (1..1000) iterations (GF_CG_MAXITER).  Velocities are zero afterwards.
 * stats (nullable): newton_iters, cg_iters summed, rel_res = the last
 * residual ratio, damage counts.  GF_FP64 meshes only.  With no mass, a
 * node whose tets all have chi = 0 has no stiffness: it keeps its position
 * (its block-Jacobi block is zero).  A separated fragment of several tets is a
 * free rigid body; the PCG finds the solution without rigid motion of it. */
gf_status gf_quasistatic_step(gf_mesh* mesh, const double* f_ext, const int32_t* pinned, int64_t n_pinned,
                              const double* pinned_pos, int32_t mem, int32_t max_newton, double rtol,
                              gf_step_stats* stats);

/* Linear solver of the quasi-static Newton iterations (GF_FP64 meshes).
 * GF_QS_SOLVE_FP64 (default): the PCG in FP64 (Chronopoulos-Gear form).
 * GF_QS_SOLVE_NESTED: flexible PCG in FP64 (Notay, 2000; one previous
 * direction kept) whose preconditioner is an inner PCG in FP32 on the matrix
 * and the block-Jacobi inverses rounded to FP32 (two kernels per iteration),
 * run until its residual falls by inner_rtol (0 < inner_rtol < 1; a value <= 0
 * keeps the current one, default 1e-2).  The outer residual, iterate and
 * coefficients are FP64 and the outer test is the FP64 PCG's
 * (|r| <= cg_rtol |b|), so the Newton iterations solve the same FP64 systems;
 * the outer Krylov iteration keeps converging where the FP32 matrix's rounding
 * would stall plain refinement.  cg_maxit bounds the inner iterations summed
 * over the outer ones, and stats report them as cg_iters.  GF_BAD_ARG for
 * another solver value, GF_UNSUPPORTED on GF_MIXED meshes.  The FP32 copies
 * (36 B per block, 108 B per node) are allocated on the first such load step. */
enum { GF_QS_SOLVE_FP64 = 0, GF_QS_SOLVE_NESTED = 1 };
gf_status gf_quasistatic_solver_set(gf_mesh* mesh, int32_t solver, double inner_rtol);

/* Split visualisation mesh for output (Sec. 4.1, Fig. 6; nothing of it feeds
 * the dynamics).  Every tet is cut into four node-associated pieces; a broken
 * edge (Eq. 21 labels) splits into two child nodes at its midpoint, a face
 * into three at its centroid, a tet into four at its centroid, one child per
 * parent node.  A child sits at its entity's rest centroid plus the mean
 * displacement x - X of the parents still joined to it through unbroken
 * edges of that entity (with no broken edge: the current centroid).
 * Vertices (float64 [n_vertices][3]): [0, N) the current positions, then
 * N + 2 e + s (edge e, child of its node edges[e][s], gf_edges_get order),
 * N + 2 NE + 3 f + c (face f, child of its c-th node; faces are the sorted
 * node triples in lexicographic order), N + 2 NE + 3 NF + 4 t + a (tet t,
 * child of local node a).  Quads (int32 [n_quads][4], vertex ids): for each
 * tet t and each of its broken local edges k = (a, b), c < d the other local
 * nodes, [E(a), F(abc, a), T(a), F(abd, a)] then [E(b), F(abd, b), T(b),
 * F(abc, b)]: the crack surface between the pieces of a and b; in order of
 * tet, local edge (Eq. 15 order), a-side first.
 * gf_surface_sizes gives the counts for the current labels; gf_surface_get
 * fills caller buffers (host or device per `mem`) and fails with GF_BAD_ARG,
 * n_quads set, when max_quads is too small.  The first call builds the face
 * tables on the host (kept with the mesh). */
gf_status gf_surface_sizes(gf_mesh* mesh, int64_t* n_vertices, int64_t* n_faces, int64_t* n_quads);
gf_status gf_surface_get(gf_mesh* mesh, double* vertices, int32_t* quads, int64_t max_quads, int32_t mem,
                         int64_t* n_quads);

/* Current positions / velocities, float64 [3*n_nodes]. */
gf_status gf_positions_get(gf_mesh* mesh, double* x, int32_t mem);
gf_status gf_velocities_get(gf_mesh* mesh, double* v, int32_t mem);

/* Damage of the last step: driver float64 [n_edges] (max over incident tets of
 * the Eq. 20 edge stress, divided by E in strain mode; -inf before any step),
 * labels uint8 [n_edges].  Either pointer may be NULL. */
gf_status gf_damage_get(gf_mesh* mesh, double* driver, uint8_t* labels, int32_t mem);

/* chi of every tet (Eq. 25) in caller tet order, float64 [n_tets]. */
gf_status gf_chi_get(gf_mesh* mesh, double* chi, int32_t mem);

/* Edge list, int32 [2*n_edges] host memory, (min, max) pairs in edge order. */
gf_status gf_edges_get(const gf_mesh* mesh, int32_t* edges);

/* The last assembled linear system A dv = b (host memory): block-CSR pattern
 * row_ptr int32 [n_nodes+1], col int32 [n_blocks], values float64
 * [9*n_blocks] (row-major 3x3 blocks; in GF_MIXED the FP32 tangent widened),
 * rhs float64 [3*n_nodes].  Any pointer may be NULL.  For tests and tools. */
gf_status gf_system_get(gf_mesh* mesh, int32_t* row_ptr, int32_t* col, double* values, double* rhs);

/* Kernel timing: when enabled, every kernel group of gf_step() is bracketed by
 * CUDA events on the mesh's stream.  gf_profile_get() fills up to `n` entries
 * of total milliseconds and launch counts since the last reset, in the order
 * of gf_profile_names(); returns the number of groups. */
gf_status gf_profile_enable(gf_mesh* mesh, int32_t on);
int32_t gf_profile_get(gf_mesh* mesh, double* total_ms, int64_t* launches, int32_t n);
const char* gf_profile_name(int32_t i);
gf_status gf_profile_reset(gf_mesh* mesh);

/* Kernel launches this mesh has issued since creation (all entry points). */
int64_t gf_launch_count(const gf_mesh* mesh);

/* Allocation-free solve of a caller's block-CSR system A x = b by projected
 * block-Jacobi PCG.  The paper has no counterpart of this entry point: it is
 * for callers that cannot allocate device memory while they solve (cudaMalloc
 * and cudaFree can synchronise the device and stall other streams; some host
 * programs give all device memory to one pool up front).  It calls no
 * allocator: its scratch is a fixed array of about 5.5 MB in the library's
 * device memory, held by every GPU that loads the library until exit, which
 * limits n_rows to 32768 block rows (98,304 unknowns); larger systems return
 * GF_BAD_ARG.  All pointers are device memory of the current device:
 * row_ptr int32 [n_rows+1], col int32 [row_ptr[n_rows]] (each in [0, n_rows),
 * else GF_BAD_ARG), values float64 [9 * row_ptr[n_rows]] row-major 3x3 blocks of
 * a symmetric positive definite matrix, b float64 [3 * n_rows], x float64
 * [3 * n_rows] (in: prescribed values on fixed rows; free rows are never read,
 * so they may hold anything, and the solve starts from 0 there; out: the
 * solution), fixed uint8 [n_rows] (1 = row held at x, NULL = none).  Every
 * free row needs an invertible diagonal block (block-Jacobi preconditioner);
 * a missing or singular one returns GF_BAD_ARG before any iteration.  Stops
 * when ||b - A x|| <= rtol ||b - A x_fixed|| on free rows.  stream:
 * cudaStream_t (NULL = legacy default); returns after the solve completes.
 * iters and rel_res (host, may be NULL) receive the CG iterations and the final
 * relative residual.  The scratch array is shared by all calls on a device and
 * keeps the last call's contents (each call clears what must start at zero);
 * calls whose work overlaps on the GPU race on it.  The first call on a device
 * looks up the array's device address and keeps it for the life of the
 * process, so that call should come before any stream capture, and this entry
 * point must not be used after a cudaDeviceReset of that device. */
gf_status gf_bsr_pcg_solve_static(const int32_t* row_ptr, const int32_t* col, const double* values, int64_t n_rows,
                                  const double* b, double* x, const uint8_t* fixed, double rtol, int32_t maxit,
                                  void* stream, int32_t* iters, double* rel_res);

/* ---------------------------------------------------------------------------
 * Batched stepping (many independent meshes per launch).
 *
 * A batch groups meshes created on one device with one precision; each mesh
 * keeps its own state, options and getters.  gf_batch_step() advances every
 * mesh by one step of Algorithm 1 with one launch per kernel kind for the whole
 * batch (each CTA maps to one mesh), and, by default, replays the step as a
 * single CUDA graph whose solver loop is a device-side conditional node: the
 * meshes converge independently and the host is not consulted between
 * iterations.  All work runs on the first mesh's stream; do not step the
 * member meshes individually while the batch is stepping.
 * ------------------------------------------------------------------------- */
typedef struct gf_batch gf_batch;

typedef struct gf_batch_tuning {
  int32_t graph;        /* 1: whole step as one CUDA graph with a device-side solve loop (default)
                           0: stream launches, host checks convergence every `chunk` iterations */
  int32_t chunk;        /* iterations between host checks when graph = 0 (0 -> 8) */
  int32_t grid_budget;  /* CTAs of one launch of a solver-loop kernel, summed over the meshes.
                           0 (default): every mesh keeps its single-mesh grid, and members step
                           bit-identically to single-mesh steps.  > 0: the budget is split over the
                           meshes by node count (at least 1 CTA each, at most the single-mesh grid);
                           converged meshes then cost few early-exit CTAs per iteration, and the
                           per-mesh reductions sum in a different (still fixed) order. */
  int32_t solve_loop;   /* A new batch starts with its members' default form (GF_SOLVE_KERNELS for
                           GF_FP64, GF_SOLVE_CG for GF_MIXED).
                           GF_SOLVE_KERNELS: per-kind launches of the solver loop
                           (graph WHILE node or stream, as `graph` says), each mesh with its
                           single-mesh grid or its share of grid_budget.
                           GF_SOLVE_DISTRIBUTED: per-kind launches of grid_budget CTAs (0: four per
                           SM) over a work table the device rebuilds after every loop iteration:
                           the grid is split over the meshes not yet converged by node count (at
                           least one block each, at most the single-mesh grid), so a converged
                           mesh costs nothing and the last ones to converge get the whole grid.
                           The reductions then group rows by the current split (a fixed order for
                           a given batch and state). 
                           GF_SOLVE_PERSISTENT (GF_MIXED batches): the whole solve of every member
                           as one cooperative launch whose phases take only the blocks of the
                           meshes still iterating (members step bit-identically to single-mesh
                           persistent steps).
                           GF_SOLVE_CG (GF_MIXED batches): the per-kind form with the inner FP32
                           PCG in two kernels per iteration (gf_tuning's GF_SOLVE_CG; members
                           step bit-identically to single-mesh steps in that form). */
  int32_t inner;        /* GF_MIXED, per-kind and distributed forms: inner iterations per pass of
                           the solver loop (a pass is: inner start, `inner` iterations, apply,
                           residual; a member whose inner solve ends early waits for the pass to
                           end).  0 -> 8.  Any value gives the same results. */
  int32_t reserved[3];  /* set to 0 */
} gf_batch_tuning;

/* meshes: n handles (1 <= n <= 256), same device and precision.  The batch
 * does not own the meshes: destroy it before them. */
gf_status gf_batch_create(gf_mesh* const* meshes, int32_t n, gf_batch** out);
void gf_batch_destroy(gf_batch* batch);

/* One step of every mesh with a common dt.  Per-mesh inputs are arrays of n
 * pointers (the array itself may be NULL for none, entries may be NULL):
 * f_ext[k] float64 [3 * n_nodes_k], pinned[k] int32 [n_pinned[k]], pinned_vel[k]
 * float64 [3 * n_pinned[k]] (NULL = zero); n_pinned may be NULL (no pins).  The
 * pointed-to arrays follow `mem`.  stats: n entries or NULL.  Returns the first
 * non-OK status of any mesh (every mesh is stepped). */
gf_status gf_batch_step(gf_batch* batch, double dt, const double* const* f_ext, const int32_t* const* pinned,
                        const int64_t* n_pinned, const double* const* pinned_vel, int32_t mem, gf_step_stats* stats);

gf_status gf_batch_tuning_set(gf_batch* batch, const gf_batch_tuning* tuning);
gf_status gf_batch_tuning_get(const gf_batch* batch, gf_batch_tuning* tuning);

/* Autotuner: times `trial_steps` batch steps under each candidate schedule
 * (graph replay vs stream launches with several host-check intervals, with
 * the single-mesh grids and with grid budgets of 1, 2 and 4 waves; the
 * persistent, distributed and two-kernel solver-loop forms; 2 to 16 inner
 * iterations per loop pass) on a copy of the current state, restores the
 * state, keeps the fastest schedule and returns it in *best (may be NULL) and
 * its time per step in *ms (may be NULL).  Inputs as in gf_batch_step. */
gf_status gf_batch_autotune(gf_batch* batch, double dt, const double* const* f_ext, const int32_t* const* pinned,
                            const int64_t* n_pinned, const double* const* pinned_vel, int32_t mem,
                            int32_t trial_steps, gf_batch_tuning* best, double* ms);

/* Kernel launches issued by the batch (graph replays count the kernels run). */
int64_t gf_batch_launch_count(const gf_batch* batch);

/* ------------------------------------------------------------------------
 * Learned warm start and block preconditioner for the linear solve of each
 * step (the system of Eq. 2 after the backward-Euler linearisation).  The
 * paper solves it with a plain Krylov method; this is an optional extension:
 * a message-passing network over the mesh graph (3 layers, hidden width 64,
 * bfloat16 weights, FP32 activations) reads the assembled system and the
 * right-hand side and outputs, per node i, a 3x3 SPD block
 *   P_i = C_i (L_i L_i^T + 1e-3 I) C_i^T,   C_i C_i^T = A_ii^-1,
 * and a start x0_i = P_i b_i + s delta_i (s = rms of |A_ii^-1 b_i| over free
 * nodes).  With zero decoder weights it is block Jacobi scaled by 1.001.
 * Parameters: gf_gnn_n_params() floats in the order W0[16][64], b0[64], then
 * per layer l = 0..2: Wa[64][64], We[16][64], bm[64], Wu[128][64], bu[64],
 * then Wd[64][9], bd[9] (row-major [in][out]).
 * Only FP64 meshes (GF_FP64) are supported; the network lives on the mesh's
 * device and stream.  Destroy it before its mesh.
 * ------------------------------------------------------------------------ */
typedef struct gf_gnn gf_gnn;

int64_t gf_gnn_n_params(void);

/* Allocates the network's buffers for `mesh` (graph = off-diagonal block
 * pattern, static node/edge inputs from the rest positions and masses).
 * Weights start at zero: set them with gf_gnn_params_set.  One network per
 * mesh; GF_UNSUPPORTED for a GF_MIXED mesh.  While it exists, every gf_step
 * keeps the previous step's solution for it (3 n_nodes doubles, device copy). */
gf_status gf_gnn_create(gf_mesh* mesh, gf_gnn** out);
void gf_gnn_destroy(gf_gnn* gnn);

/* Host float32 arrays of gf_gnn_n_params() entries (n must equal it).  _set
 * also resets the optimiser state. */
gf_status gf_gnn_params_set(gf_gnn* gnn, const float* w, int64_t n);
gf_status gf_gnn_params_get(gf_gnn* gnn, float* w, int64_t n);

/* Forward pass on the system assembled by the mesh's last gf_step (its
 * matrix and pinned set) with right-hand side b (float64 [3 * n_nodes],
 * following `mem`).  Host outputs, each may be NULL: out float32 [n_nodes][9]
 * (delta, ell), P float32 [n_nodes][9], x0 float32 [n_nodes][3], node_in
 * float32 [n_nodes][16], edge_in float32 [n_graph_edges][16] (graph rows as in
 * gf_system_get's pattern without the diagonal).  The mesh is not changed. */
gf_status gf_gnn_forward(gf_gnn* gnn, const double* b, int32_t mem, float* out, float* P, float* x0, float* node_in,
                         float* edge_in);

/* Energy-norm loss (x0 - target)^T A_ff (x0 - target) / target^T A_ff target
 * (A_ff: free block of the mesh's last system) for the pair (b, target), and
 * its gradient (host float32 [n_params], may be NULL).  b, target: float64
 * [3 * n_nodes] following `mem`; entries on pinned nodes are ignored. */
gf_status gf_gnn_loss_grad(gf_gnn* gnn, const double* b, const double* target, int32_t mem, double* loss,
                           float* grad);

/* Online training on the mesh's last solved step.  With x_prev the solution
 * of the step before it and w = dv on pinned nodes, x_prev on free ones, the
 * pair is b = b_sys - A w on free rows and target = dv - x_prev on free nodes;
 * the loss is the energy-norm error (x0 - target)^T A_ff (x0 - target) /
 * target^T A_ff target.  Runs `iters` (1..1024) Adam steps (beta 0.9 / 0.999,
 * learning rate lr) and returns the loss before the first and before the last
 * update (each may be NULL). */
gf_status gf_gnn_train(gf_gnn* gnn, int32_t iters, float lr, double* loss_first, double* loss_last);

/* The pair gf_gnn_train uses, for the mesh's last solved step: host float64
 * [3 * n_nodes] each. */
gf_status gf_gnn_pair_get(gf_gnn* gnn, double* b, double* target);

/* Use of the network in gf_step (flags = 0 turns it off; the default after
 * gf_gnn_create).  GF_GNN_START: the solve starts from x_prev + x0, where
 * x_prev is the previous step's solution and x0 the network's answer for the
 * right-hand side b_free - A_ff x_prev.  GF_GNN_PRECOND: the learned blocks
 * P_i replace block Jacobi.  Convergence is still
 * |b_free - A dv| <= rtol |b_free| either way. */
enum { GF_GNN_START = 1, GF_GNN_PRECOND = 2 };
gf_status gf_gnn_attach(gf_mesh* mesh, gf_gnn* gnn, int32_t flags);

/* Kernels of the network's dense contractions (the eight node-wise dense
 * layers, the per-edge message layer We e_ij of each message-passing layer and
 * the input gradients of the backward pass).  GF_GNN_TENSOR_CORES (default):
 * tcgen05 MMAs with the FP32 activations split into three bf16 parts (exact
 * products, FP32 accumulation, so FP32-accurate); GF_GNN_FP32_FMA: FP32 FMA
 * kernels.  Both give the same results up to FP32 rounding order.  A device
 * wait of the tensor-core kernels that gives up (after one second) makes the
 * call (or gf_step) return GF_TIMEOUT. */
enum { GF_GNN_TENSOR_CORES = 0, GF_GNN_FP32_FMA = 1 };
gf_status gf_gnn_kernels_set(gf_gnn* gnn, int32_t kernels);

const char* gf_status_string(gf_status s);
const char* gf_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GRAPHFEM_H */
