// C ABI of the graph-FEM fracture step: mesh lifetime, state, one implicit step.
#include <algorithm>
#include <utility>
#include <cmath>
#include <cstring>
#include <new>
#include <memory>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "gf_device.h"
#include "gf_gnn.h"
#include "gf_surface.h"

namespace gf {

thread_local std::string g_last_error;
void set_last_error(const std::string& msg) { g_last_error = msg; }

StepScalars step_scalars(const Material& mt, double dt, bool has_fext, int64_t n_pinned, bool has_pvel) {
  StepScalars sp{};
  sp.dt = dt;
  sp.dtf = float(dt);
  sp.sKv = float(dt * mt.beta + dt * dt);
  sp.cv = float(mt.beta + dt);
  sp.alphaf = float(mt.alpha);
  sp.cmf = float(1.0 + dt * mt.alpha);
  sp.has_fext = has_fext ? 1 : 0;
  sp.has_pvel = has_pvel ? 1 : 0;
  sp.n_pinned = n_pinned;
  sp.mscale = 1.0;
  return sp;
}

namespace {
inline unsigned cdiv(int64_t n, int d) { return unsigned((n + d - 1) / d); }
inline unsigned red_grid(int64_t n) {   // FP64 reducing kernels: one thread per row, <= kMaxPartials CTAs
  const int64_t b = (n + 255) / 256;
  return unsigned(b < 1 ? 1 : (b > kMaxPartials ? kMaxPartials : b));
}
inline unsigned ir_grid(int64_t n, int per_sm = 4) {    // refinement kernels: <= per_sm CTAs per SM, grid-stride
  const int64_t b = (n + 255) / 256;
  return unsigned(b < 1 ? 1 : (b > per_sm * 152 ? per_sm * 152 : b));
}

// Solver-loop condition of the single-mesh step graph: continue while the
// solve is not done (and below the cap on WHILE iterations).
__global__ void k_step_cond(const PcgState* pcg, const IrState* ir, int* loops, int cap,
                            cudaGraphConditionalHandle h) {
  if (threadIdx.x != 0) return;
  const int it = ++*loops;
  const bool go = ir ? !ir->done : !pcg->done;
  cudaGraphSetConditional(h, (go && it < cap) ? 1u : 0u);
}

}  // namespace

LaunchDims launch_dims(int kind, const DevMesh& m, const Material& mt, const StepScalars& sp) {
  const int64_t N = m.N, T = m.T, NE = m.NE;
  switch (kind) {
    case kB_tet_stress: case kB_tet_chi: case kB_tet_stress32: case kB_tet_chi32: case kB_chi_to32:
      return {cdiv(T, 256), 256};
    case kB_nonlocal: return {mt.radius > 0.0 ? cdiv(T, 256) : 0u, 256};
    case kB_nonlocal32: return {mt.radius > 0.0 ? cdiv(T, m.mx.nl_tile) : 0u, 256};
    case kB_edge_driver: case kB_edge_driver32: return {cdiv(NE, 256), 256};
    case kB_node_init: return {cdiv(N, 256), 256};
    case kB_elem64: case kB_elem32: return {cdiv(T, 128), 128};
    case kB_gather64: return {cdiv(9 * m.NE + 3 * N, 256), 256};
    case kB_diag64: return {cdiv(9 * N, 256), 256};
    case kB_gather32: return {cdiv(9 * m.NE + 3 * N, 256), 256};
    case kB_diag32: return {cdiv(9 * N, 288), 288};   // 32 nodes x 9 entries per CTA
    case kB_set_pinned: return {cdiv(sp.n_pinned, 256), 256};
    case kB_pcg_init: case kB_pcg_spmv: case kB_pcg_update: case kB_true_residual: return {red_grid(N), 256};
    case kB_pcg_p: return {red_grid(3 * N), 256};
    case kB_integrate: case kB_integrate32: case kB_refresh32: return {cdiv(3 * N, 256), 256};
    case kB_ir_residual: return {ir_grid(8 * N, 5), 256};
    case kB_ir_spmv: case kB_ir_cg_spmv: return {ir_grid(16 * N, 6), 256};
    case kB_ir_inner_init: case kB_ir_update: case kB_ir_cg_update: return {ir_grid(N), 256};
    case kB_ir_p: case kB_ir_apply: return {ir_grid(3 * N), 256};
    case kB_step_begin: return {cdiv(3 * N, 256), 256};
  }
  return {0u, 256};
}

int launch_kind(int kind, const DevMesh& m, const Material& mt, const StepScalars& sp, cudaStream_t s, int first) {
  return kind < kB_tet_stress32 ? launch_kind_fp64(kind, m, mt, sp, s) : launch_kind_mixed(kind, m, mt, sp, s, first);
}

int launch_batch(int kind, const BatchTab* tab, unsigned blocks, cudaStream_t s, int first) {
  const unsigned threads = (kind == kB_elem64 || kind == kB_elem32) ? 128u : kind == kB_diag32 ? 288u : 256u;
  return kind < kB_tet_stress32 ? launch_batch_fp64(kind, tab, blocks, threads, s)
                                : launch_batch_mixed(kind, tab, blocks, threads, s, first);
}

namespace {

enum ProfGroup : int {
  kPStress = 0, kPNonlocal, kPEdge, kPChi, kPAssemble, kPPcgInit, kPSpmv, kPPcgUpdate, kPPcgP, kPResidual,
  kPIntegrate, kPIrResidual, kPIrInit, kPIrApply, kPGnn, kPGather, kPSolve, kPCount
};
const char* kProfNames[kPCount] = {"tet_stress",  "nonlocal_avg", "edge_driver", "tet_chi",     "assemble",
                                   "pcg_init",    "pcg_spmv",     "pcg_update",  "pcg_p",       "true_residual",
                                   "integrate",   "ir_residual",  "ir_inner_init", "ir_apply",
                                   "gnn",         "assemble_gather", "solve_persistent"};

__global__ void k_fill(double* p, int64_t n, double v) {
  int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i < n) p[i] = v;
}
// internal[i] = caller[perm[i]]
__global__ void k_gather(const double* src, const int32_t* perm, double* dst, int64_t n) {
  int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i < n) dst[i] = src[perm[i]];
}
// caller[perm[i]] = internal[i]
__global__ void k_scatter(const double* src, const int32_t* perm, double* dst, int64_t n) {
  int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i < n) dst[perm[i]] = src[i];
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (dev != prev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace
}  // namespace gf

using namespace gf;

struct gf_mesh {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  gf_alloc_fn alloc = nullptr;
  gf_free_fn free_fn = nullptr;
  void* alloc_ctx = nullptr;
  std::vector<void*> blocks;
  int64_t bytes = 0;

  gf_material mat{};
  gf_options opt{};
  gf::Material mt{};
  uint64_t lut = 0;
  HostMesh hm;          // host copies kept for getters (pattern, edges, perm, colours)
  std::vector<double> X0;     // rest positions [N][3]
  gf_gnn* gnn = nullptr;      // learned start / preconditioner created for this mesh
  int gnn_flags = 0;          // GF_GNN_START | GF_GNN_PRECOND while attached
  bool assembled = false;     // a step has assembled the system
  DevMesh dm;
  int32_t* perm_dev = nullptr;
  int last_iters = 4;
  gf_tuning tune{};           // assembly schedule etc. (defaults: two-phase gather)
  bool mixed = false;
  int last_inner = 3;
  double in_rtol = 1e-5;
  int newton_iters = 1;       // Newton iterations per step (FP64 path)
  double newton_rtol = 0.0;   // stop early when |r(v^k)| <= newton_rtol |b^0| on free DOFs
  int newton_done = 1;        // iterations of the last step
  double newton_res = 0.0;    // |r(v^k)| / |b^0| at the start of the last iteration (0 after one)
  int newton_cg_total = 0;    // CG iterations of the last step over its Newton iterations
  double* qs_x = nullptr;     // quasi-static: trial positions [3N]
  double* qs_zero = nullptr;  // quasi-static: zero velocities [3N]
  double* qs_out = nullptr;   // quasi-static: E, |E| scale, slope [4]
  double* qs_w = nullptr;     // quasi-static: A z of the Chronopoulos-Gear PCG [3N]
  int qs_solver = GF_QS_SOLVE_FP64;
  double qs_in_rtol = 1e-2;   // inner tolerance of the nested solve (quasi-static step, GF_SOLVE_NESTED)
  MixDev qsr{};               // its FP32 matrix, inverses, vectors and state (first use)
  cudaGraph_t qs_graph = nullptr;          // its solver loop as a WHILE node (first use)
  cudaGraphExec_t qs_graph_exec = nullptr;
  int* qs_loops = nullptr;                 // the loop's body count
  SurfDev surf{};             // split visualisation mesh tables (built on first use)
  bool surf_ready = false;
  void* surf_stage = nullptr; // host-output staging of the surface buffers (cudaMalloc, grown on demand)
  size_t surf_stage_bytes = 0;
  int64_t launches = 0;
  int64_t nbr_pairs = 0;
  int64_t joint_entries = 0;  // GF_MIXED: entries of the Eq. 20 joint lists of tet pairs
  int64_t union_rows = 0;     // GF_MIXED: tet ids of the per-tile neighbour unions

  PcgState* h_pcg = nullptr;               // pinned host mirror
  IrState* h_ir = nullptr;                 // pinned host mirror (mixed)
  unsigned long long* h_cnt = nullptr;     // pinned host mirror of counters

  // graph form of the plain step (see step_graph)
  struct GraphKey {
    double dt = 0.0;
    int64_t n_pinned = -1;
    int has_fext = -1, has_pvel = -1, maxit = -1, loop = -1;
    const void *f_ext = nullptr, *pin_ids = nullptr, *pin_vel = nullptr;
    bool operator==(const GraphKey& o) const {
      return dt == o.dt && n_pinned == o.n_pinned && has_fext == o.has_fext && has_pvel == o.has_pvel &&
             maxit == o.maxit && loop == o.loop && f_ext == o.f_ext && pin_ids == o.pin_ids && pin_vel == o.pin_vel;
    }
  };
  GraphKey gkey;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  cudaStream_t body_stream = nullptr;      // capture stream of the WHILE body
  int* d_loops = nullptr;                  // WHILE iterations of the last replay
  int* h_loops = nullptr;                  // pinned mirror
  void* h_init = nullptr;                  // pinned solver-state initialiser read by the graph
  int64_t g_prefix = 0, g_body = 0, g_suffix = 0;

  // persistent solve (GF_MIXED, GF_SOLVE_PERSISTENT): a one-mesh table and its control block
  BatchTab* ptab = nullptr;
  PersistCtl* pctl = nullptr;
  PersistCtl* h_pctl = nullptr;            // pinned host mirror of the control block's head

  bool prof = false;
  double prof_ms[kPCount] = {};
  int64_t prof_n[kPCount] = {};
  std::vector<cudaEvent_t> ev_pool;
  struct Rec { int group; int ev0; int ev1; int iter; };
  std::vector<Rec> recs;
  int ev_next = 0;
};

void gnn_orphan(gf_gnn* g);

namespace {

#define GF_CK(call)                                                                         \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) {                                                                \
      set_last_error(std::string(#call) + ": " + cudaGetErrorString(e_));                  \
      return e_ == cudaErrorMemoryAllocation ? GF_OOM : GF_CUDA_ERR;                        \
    }                                                                                       \
  } while (0)

gf_status dev_alloc(gf_mesh* m, size_t bytes, void** out) {
  bytes = (bytes + 255) & ~size_t(255);
  if (bytes == 0) bytes = 256;
  void* p = nullptr;
  if (m->alloc) {
    p = m->alloc(bytes, m->alloc_ctx);
    if (!p) {
      set_last_error("device allocator returned NULL for " + std::to_string(bytes) + " bytes");
      return GF_OOM;
    }
    if (reinterpret_cast<uintptr_t>(p) % 16 != 0) {   // the kernels use 16-byte vector accesses
      m->free_fn(p, m->alloc_ctx);
      set_last_error("device allocator returned a pointer that is not 16-byte aligned");
      return GF_BAD_ARG;
    }
  } else {
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      set_last_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
      return GF_OOM;
    }
  }
  m->blocks.push_back(p);
  m->bytes += int64_t(bytes);
  *out = p;
  return GF_OK;
}

template <class T>
gf_status upload(gf_mesh* m, const std::vector<T>& h, const T** out) {
  void* p = nullptr;
  gf_status st = dev_alloc(m, h.size() * sizeof(T), &p);
  if (st != GF_OK) return st;
  if (!h.empty()) GF_CK(cudaMemcpyAsync(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, m->stream));
  *out = static_cast<const T*>(p);
  return GF_OK;
}

template <class T>
gf_status scratch(gf_mesh* m, size_t n, T** out) {
  void* p = nullptr;
  gf_status st = dev_alloc(m, n * sizeof(T), &p);
  if (st != GF_OK) return st;
  *out = static_cast<T*>(p);
  return GF_OK;
}

void release(gf_mesh* m) {
  if (!m) return;
  for (void* p : m->blocks) {
    if (m->free_fn) m->free_fn(p, m->alloc_ctx);
    else cudaFree(p);
  }
  m->blocks.clear();
  for (auto e : m->ev_pool) cudaEventDestroy(e);
  if (m->h_pcg) cudaFreeHost(m->h_pcg);
  if (m->h_ir) cudaFreeHost(m->h_ir);
  if (m->h_cnt) cudaFreeHost(m->h_cnt);
  if (m->graph_exec) cudaGraphExecDestroy(m->graph_exec);
  if (m->graph) cudaGraphDestroy(m->graph);
  if (m->qs_graph_exec) cudaGraphExecDestroy(m->qs_graph_exec);
  if (m->qs_graph) cudaGraphDestroy(m->qs_graph);
  if (m->body_stream) cudaStreamDestroy(m->body_stream);
  if (m->h_loops) cudaFreeHost(m->h_loops);
  if (m->h_init) cudaFreeHost(m->h_init);
  if (m->surf_stage) cudaFree(m->surf_stage);
  if (m->own_stream && m->stream) cudaStreamDestroy(m->stream);
}

// profiling helpers: an event pair around each launch of a group
int prof_mark(gf_mesh* m) {
  if (m->ev_next == int(m->ev_pool.size())) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    m->ev_pool.push_back(e);
  }
  int i = m->ev_next++;
  cudaEventRecord(m->ev_pool[i], m->stream);
  return i;
}
// An NVTX range on the host thread (header-only NVTX 3: it costs a pointer
// test when no tool is attached): tools such as Nsight Systems show the phases
// of a call and which kernels each phase enqueued.
struct Nvtx {
  explicit Nvtx(const char* name) { nvtxRangePushA(name); }
  ~Nvtx() { nvtxRangePop(); }
  Nvtx(const Nvtx&) = delete;
  Nvtx& operator=(const Nvtx&) = delete;
};

// A kernel group of a step: an NVTX range named after the group and, when
// profiling is on, CUDA events on the mesh's stream around its launches.
struct Prof {
  gf_mesh* m;
  int group, ev0 = -1, iter;
  Nvtx range;
  Prof(gf_mesh* mm, int g, int it = -1) : m(mm), group(g), iter(it), range(kProfNames[g]) {
    if (m->prof) ev0 = prof_mark(m);
  }
  ~Prof() {
    if (m->prof) m->recs.push_back({group, ev0, prof_mark(m), iter});
  }
};

void prof_collect(gf_mesh* m, int cg_iters, bool converged) {
  if (!m->prof) return;
  for (auto& r : m->recs) {
    // early-exit PCG launches after convergence did no work: do not count them
    if (r.iter >= 0 && cg_iters < (1 << 30)) {
      bool worked = (r.group == kPSpmv || r.group == kPPcgUpdate) ? r.iter < cg_iters
                                                                    : r.iter < (converged ? cg_iters - 1 : cg_iters);
      if (!worked) continue;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, m->ev_pool[r.ev0], m->ev_pool[r.ev1]);
    m->prof_ms[r.group] += ms;
    m->prof_n[r.group] += 1;
  }
  m->recs.clear();
  m->ev_next = 0;
}

bool material_ok(const gf_material& M) {
  if (!(M.young > 0) || !(M.poisson > -1.0 && M.poisson < 0.5) || !(M.density > 0) || !(M.radius >= 0) ||
      std::isnan(M.threshold) || !(M.alpha >= 0) || !(M.beta >= 0) || (M.shear_coef != 1 && M.shear_coef != 2) ||
      (M.driver_mode != GF_DRIVER_STRAIN && M.driver_mode != GF_DRIVER_STRESS) ||
      (M.mass_matrix != GF_MASS_LUMPED && M.mass_matrix != GF_MASS_CONSISTENT) ||
      (M.energy != GF_ENERGY_STVK && M.energy != GF_ENERGY_SNH) || (M.energy == GF_ENERGY_SNH && !(M.poisson > 0.0))) {
    set_last_error("invalid material (need E > 0, -1 < nu < 0.5, rho > 0, R_d >= 0, alpha, beta >= 0, shear_coef 1|2, "
                   "mass_matrix lumped|consistent, energy StVK|SNH (SNH: nu > 0))");
    return false;
  }
  return true;
}

bool valid_mem(int32_t mem) { return mem == GF_MEM_HOST || mem == GF_MEM_DEVICE; }

cudaMemcpyKind to_dev(int32_t mem) { return mem == GF_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice; }
cudaMemcpyKind from_dev(int32_t mem) { return mem == GF_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice; }

gf_status recompute_chi(gf_mesh* m) {
  if (m->mixed) {
    const StepScalars sp = step_scalars(m->mt, 1.0, false, 0, false);
    m->launches += launch_kind(kB_tet_stress32, m->dm, m->mt, sp, m->stream);
    m->launches += launch_kind(kB_tet_chi32, m->dm, m->mt, sp, m->stream);
  } else {
    const StepScalars sp = step_scalars(m->mt, 1.0, false, 0, false);
    m->launches += launch_kind(kB_tet_stress, m->dm, m->mt, sp, m->stream);
    m->launches += launch_kind(kB_tet_chi, m->dm, m->mt, sp, m->stream);
  }
  GF_CK(cudaGetLastError());
  return GF_OK;
}

// The autotuners' choice: every candidate timed once, then the three fastest
// timed again, each kept at the lower of its two times (a host stall only ever
// lengthens a trial), and the fastest of those.  Stops at the first failing
// trial (status in st).  Returns the index (n if none) and its ms per step.
template <typename Trial>
std::pair<size_t, double> pick_fastest(size_t n, Trial&& trial, gf_status& st) {
  std::vector<double> t(n, 1e300);
  for (size_t i = 0; i < n && st == GF_OK; ++i) t[i] = trial(i);
  if (st != GF_OK || n == 0) return {n, 1e300};
  std::vector<size_t> order(n);
  for (size_t i = 0; i < n; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](size_t a, size_t b) { return t[a] < t[b]; });
  for (size_t k = 0; k < std::min<size_t>(3, n) && st == GF_OK; ++k) t[order[k]] = std::min(t[order[k]], trial(order[k]));
  if (st != GF_OK) return {n, 1e300};
  const size_t best = size_t(std::min_element(t.begin(), t.end()) - t.begin());
  return {best, t[best]};
}

}  // namespace

extern "C" {

const char* gf_status_string(gf_status s) {
  switch (s) {
    case GF_OK: return "ok";
    case GF_BAD_ARG: return "bad argument";
    case GF_CUDA_ERR: return "CUDA error";
    case GF_CG_BREAKDOWN: return "CG breakdown (p^T A p <= 0)";
    case GF_CG_MAXITER: return "CG reached the iteration cap";
    case GF_NAN: return "non-finite value";
    case GF_TIMEOUT: return "device wait timed out";
    case GF_OOM: return "out of device memory";
    case GF_UNSUPPORTED: return "unsupported option";
  }
  return "unknown status";
}

const char* gf_last_error(void) { return gf::g_last_error.c_str(); }

gf_status gf_mesh_create(const double* nodes, int64_t n_nodes, const int32_t* tets, int64_t n_tets,
                         const gf_material* mat, const gf_options* opt_in, gf_mesh** out) {
  if (!out) {
    set_last_error("out is NULL");
    return GF_BAD_ARG;
  }
  *out = nullptr;
  if (!nodes || !tets || !mat) {
    set_last_error("nodes, tets and mat must not be NULL");
    return GF_BAD_ARG;
  }
  gf_options opt{};
  if (opt_in) opt = *opt_in;
  if (opt.cg_maxit <= 0) opt.cg_maxit = 10000;
  if (!(opt.cg_rtol > 0)) opt.cg_rtol = 1e-6;
  if (opt.precision != GF_FP64 && opt.precision != GF_MIXED) {
    set_last_error("precision must be GF_FP64 or GF_MIXED");
    return GF_UNSUPPORTED;
  }
  if (opt.precond != GF_PRECOND_BJACOBI) {
    set_last_error("unknown preconditioner");
    return GF_UNSUPPORTED;
  }
  if ((opt.alloc == nullptr) != (opt.free == nullptr)) {
    set_last_error("alloc and free must be given together");
    return GF_BAD_ARG;
  }
  const gf_material& M = *mat;
  if (!material_ok(M)) return GF_BAD_ARG;
  if (M.energy == GF_ENERGY_SNH && opt.precision == GF_MIXED) {
    set_last_error("the stable Neo-Hookean energy is built for GF_FP64 meshes only");
    return GF_UNSUPPORTED;
  }
  int dev = opt.device;
  if (dev < 0) {
    if (cudaGetDevice(&dev) != cudaSuccess) {
      set_last_error("no CUDA device");
      return GF_CUDA_ERR;
    }
  }
  DeviceGuard guard(dev);

  gf_mesh* m = new gf_mesh();
  m->device = dev;
  m->mat = M;
  m->opt = opt;
  m->alloc = opt.alloc;
  m->free_fn = opt.free;
  m->alloc_ctx = opt.alloc_ctx;
  auto fail = [&](gf_status st) {
    release(m);
    delete m;
    return st;
  };
  if (opt.stream) {
    m->stream = static_cast<cudaStream_t>(opt.stream);
  } else {
    if (cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking) != cudaSuccess) {
      set_last_error("cudaStreamCreate failed");
      return fail(GF_CUDA_ERR);
    }
    m->own_stream = true;
  }
  std::string err;
  gf_status st = build_host_mesh(nodes, n_nodes, tets, n_tets, M, m->hm, err);
  if (st == GF_OK) m->X0.assign(nodes, nodes + 3 * n_nodes);
  if (st != GF_OK) {
    set_last_error(err);
    return fail(st);
  }
  const double lam = M.young * M.poisson / ((1.0 + M.poisson) * (1.0 - 2.0 * M.poisson));
  const double mu = M.young / (2.0 * (1.0 + M.poisson));
  m->mt = gf::Material{lam, mu, M.young, M.alpha, M.beta, M.threshold, M.radius, double(M.shear_coef),
                       M.driver_mode == GF_DRIVER_STRESS ? 1 : 0, M.average_degraded ? 1 : 0};
  m->lut = disconnect_table();
  m->mt.lut = m->lut;
  m->mt.lam32 = float(m->mt.lam);
  m->mt.mu32 = float(m->mt.mu);
  m->mt.kappa32 = float(m->mt.kappa);
  m->mt.young32 = float(m->mt.young);
  m->mt.inv_young32 = float(1.0 / m->mt.young);
  m->mt.energy = M.energy;
  m->mt.snh_a = 1.0 + mu / lam - mu / (4.0 * lam);

  HostMesh& hm = m->hm;
  DevMesh& d = m->dm;
  const bool mixed = opt.precision == GF_MIXED;
  m->mixed = mixed;
  // the mixed step's default solver loop: the inner FP32 PCG in two kernels per iteration
  m->tune.solve_loop = mixed ? GF_SOLVE_CG : GF_SOLVE_KERNELS;
  MixedHost mxh;
  if (mixed) {
    st = build_mixed_host(nodes, hm, mxh, err);
    if (st != GF_OK) {
      set_last_error(err);
      return fail(st);
    }
  }
  d.N = hm.n_nodes;
  d.T = hm.n_tets;
  d.NE = hm.n_edges;
  d.NB = hm.n_blocks;
  d.G = int64_t(hm.nbr.group_off.size());
#define UP(field, vec, type)                                                     \
  do {                                                                           \
    const type* p_ = nullptr;                                                    \
    if ((st = upload(m, vec, &p_)) != GF_OK) return fail(st);                    \
    field = reinterpret_cast<decltype(field)>(p_);                               \
  } while (0)
  UP(d.tets, hm.tets, int32_t);
  UP(d.tet_edges, hm.tet_edges, int32_t);
  UP(d.mass, hm.mass, double);
  UP(d.row_ptr, hm.row_ptr, int32_t);
  UP(d.col, hm.col, int32_t);
  UP(d.diag_blk, hm.diag_blk, int32_t);
  UP(d.edges, hm.edges, int32_t);
  UP(d.et_ptr, hm.et_ptr, int32_t);
  UP(d.et_tet, hm.et_tet, int32_t);
  UP(d.colour_tets, hm.colour_tets, int32_t);
  UP(d.np_ptr, hm.np_ptr, int32_t);
  UP(d.nrow, hm.nrow, int32_t);
  UP(d.erow, hm.erow, int32_t);
  UP(d.edge_slot, hm.edge_slot, int32_t);
  UP(d.edge_order, hm.edge_order, int32_t);
  UP(d.node_order, hm.node_order, int32_t);
  std::vector<double> mass_blk;
  if (M.mass_matrix == GF_MASS_CONSISTENT) {
    // Eq. 5 for a linear tet: m_ab = rho V (1 + delta_ab) / 20, summed into the block slots
    mass_blk.assign(hm.n_blocks, 0.0);
    for (int64_t t = 0; t < hm.n_tets; ++t) {
      const double mv = M.density * hm.rest[size_t(kRestV) * hm.n_tets + t] / 20.0;
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) mass_blk[hm.slot[16 * t + 4 * a + b]] += (a == b ? 2.0 : 1.0) * mv;
    }
    UP(d.mass_blk, mass_blk, double);
  }
  if (!mixed) {
    UP(d.nb_off, hm.nbr.group_off, int64_t);
    UP(d.nb_len, hm.nbr.group_len, int32_t);
    UP(d.nb_idx, hm.nbr.idx, int32_t);
    UP(d.nb_perm, hm.nbr.perm, int32_t);
    UP(d.slot, hm.slot, int32_t);
    UP(d.rest, hm.rest, double);
    UP(d.nb_w, hm.nbr.w, double);
  } else {
    UP(d.mx.restA, mxh.restA, float);
    UP(d.mx.restB, mxh.restB, float);
    UP(d.mx.edge_e0, mxh.edge_e0, float);
    UP(d.mx.nb_ptr, mxh.nb_ptr, int64_t);
    UP(d.mx.nb_loc, mxh.nb_loc, uint16_t);
    UP(d.mx.nb_w2, mxh.nb_w2, float);
    UP(d.mx.nl_uptr, mxh.nl_uptr, int64_t);
    UP(d.mx.nl_uidx, mxh.nl_uidx, int32_t);
    d.mx.nl_cap = mxh.nl_cap;
    d.mx.nl_tile = mxh.nl_tile;
    m->joint_entries = mxh.nb_real;
    m->union_rows = int64_t(mxh.nl_uidx.size());
    std::vector<float> m32(hm.mass.begin(), hm.mass.end());
    UP(d.mx.mass32, m32, float);
    if (!mass_blk.empty()) {
      std::vector<float> mb32(mass_blk.begin(), mass_blk.end());
      UP(d.mx.mass_blk32, mb32, float);
    }
    std::vector<double> Xv(nodes, nodes + 3 * n_nodes);
    UP(d.mx.X, Xv, double);
  }
#undef UP
  {
    const int32_t* pp = nullptr;
    if ((st = upload(m, hm.perm, &pp)) != GF_OK) return fail(st);
    m->perm_dev = const_cast<int32_t*>(pp);
  }
  const int64_t N = d.N, T = d.T, NE = d.NE, NB = d.NB;
  if ((st = scratch(m, 3 * N, &d.x)) || (st = scratch(m, 3 * N, &d.v)) || (st = scratch(m, NE, &d.labels)) ||
      (st = scratch(m, T, &d.chi)) || (st = scratch(m, NE, &d.driver)) || (st = scratch(m, 3 * N, &d.rhs)) ||
      (st = scratch(m, 3 * N, &d.dv)) || (st = scratch(m, N, &d.pinned)) || (st = scratch(m, 3 * N, &d.f_ext)) ||
      (st = scratch(m, N, &d.pin_ids)) || (st = scratch(m, 3 * N, &d.pin_vel)) || (st = scratch(m, 1, &d.pcg)) ||
      (st = scratch(m, 4 * kMaxPartials, &d.partials)) || (st = scratch(m, kTickets, &d.tickets)) ||
      (st = scratch(m, kCntMax, &d.counters)) || (st = scratch(m, 6 * T, &d.sigf)))
    return fail(st);
  if (!mixed) {
    if ((st = scratch(m, 6 * T, &d.sig_in)) || (st = scratch(m, 6 * T, &d.sig_bar)) ||
        (st = scratch(m, 9 * NB, &d.val)) || (st = scratch(m, 70 * T, &d.ebuf)) ||
        (st = scratch(m, 3 * N, &d.r)) || (st = scratch(m, 3 * N, &d.z)) ||
        (st = scratch(m, 3 * N, &d.p)) || (st = scratch(m, 3 * N, &d.q)) || (st = scratch(m, 9 * N, &d.pinv)))
      return fail(st);
  } else {
    MixDev& x = d.mx;
    if ((st = scratch(m, 3 * N, &x.u32)) || (st = scratch(m, 3 * N, &x.v32)) || (st = scratch(m, T, &x.chi32)) ||
        (st = scratch(m, 8 * T, &x.sig_in32)) || (st = scratch(m, 8 * T, &x.sig_bar32)) ||
        (st = scratch(m, 9 * NB, &x.val32)) ||
        (st = scratch(m, 70 * T, &x.ebuf)) || (st = scratch(m, 3 * N, &x.rhs32)) ||
        (st = scratch(m, 3 * N, &x.rres)) ||
        (st = scratch(m, 9 * N, &x.pinv32)) || (st = scratch(m, 3 * N, &x.r32)) || (st = scratch(m, 3 * N, &x.z32)) ||
        (st = scratch(m, 3 * N, &x.p32)) || (st = scratch(m, 3 * N, &x.p32b)) || (st = scratch(m, 3 * N, &x.w32)) || (st = scratch(m, N, &x.z4)) || (st = scratch(m, 3 * N, &x.q32)) || (st = scratch(m, 3 * N, &x.d32)) ||
        (st = scratch(m, 3 * N, &x.dv_hi)) || (st = scratch(m, 3 * N, &x.dv_lo)) ||
        (st = scratch(m, 1, &x.ir)))
      return fail(st);
  }
  if (cudaMallocHost(&m->h_pcg, sizeof(PcgState)) != cudaSuccess ||
      cudaMallocHost(&m->h_ir, sizeof(IrState)) != cudaSuccess ||
      cudaMallocHost(&m->h_cnt, sizeof(unsigned long long) * kCntMax) != cudaSuccess) {
    set_last_error("cudaMallocHost failed");
    return fail(GF_OOM);
  }
  // rest state: x = nodes, v = 0, no broken edge, chi = 1, driver = -inf
  GF_CK(cudaMemcpyAsync(d.x, nodes, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, m->stream));
  GF_CK(cudaMemsetAsync(d.v, 0, sizeof(double) * 3 * N, m->stream));
  GF_CK(cudaMemsetAsync(d.labels, 0, NE, m->stream));
  GF_CK(cudaMemsetAsync(d.tickets, 0, sizeof(unsigned) * kTickets, m->stream));
  GF_CK(cudaMemsetAsync(d.dv, 0, sizeof(double) * 3 * N, m->stream));
  if (!mixed) GF_CK(cudaMemsetAsync(d.val, 0, sizeof(double) * 9 * NB, m->stream));
  else GF_CK(cudaMemsetAsync(d.mx.val32, 0, sizeof(float) * 9 * NB, m->stream));
  GF_CK(cudaMemsetAsync(d.rhs, 0, sizeof(double) * 3 * N, m->stream));
  k_fill<<<unsigned((T + 255) / 256), 256, 0, m->stream>>>(d.chi, T, 1.0);
  k_fill<<<unsigned((NE + 255) / 256), 256, 0, m->stream>>>(d.driver, NE, -INFINITY);
  m->launches += 2;
  if (mixed) {
    const StepScalars sp0 = step_scalars(m->mt, 1.0, false, 0, false);
    m->launches += launch_kind(kB_refresh32, d, m->mt, sp0, m->stream);
    m->launches += launch_kind(kB_chi_to32, d, m->mt, sp0, m->stream);
  }
  GF_CK(cudaGetLastError());
  GF_CK(cudaStreamSynchronize(m->stream));
  // drop host copies not needed after upload
  m->nbr_pairs = hm.nbr.pairs;
  hm.rest = {};
  hm.slot = {};
  hm.nbr = {};
  hm.et_tet = {};
  hm.tets = {};
  hm.tet_edges = {};
  *out = m;
  return GF_OK;
}

gf_status gf_mesh_plan(const double* nodes, int64_t n_nodes, const int32_t* tets, int64_t n_tets,
                       const gf_material* mat, gf_mesh_info* info, int32_t* edges, int32_t* colour,
                       int32_t* nbr_count) {
  if (!nodes || !tets || !mat || !info) {
    set_last_error("nodes, tets, mat and info must not be NULL");
    return GF_BAD_ARG;
  }
  if (!material_ok(*mat)) return GF_BAD_ARG;
  HostMesh hm;
  std::string err;
  gf_status st = build_host_mesh(nodes, n_nodes, tets, n_tets, *mat, hm, err);
  if (st != GF_OK) {
    set_last_error(err);
    return st;
  }
  info->n_nodes = hm.n_nodes;
  info->n_tets = hm.n_tets;
  info->n_edges = hm.n_edges;
  info->n_blocks = hm.n_blocks;
  info->n_colours = int64_t(hm.colour_ptr.size()) - 1;
  info->n_nbr_pairs = hm.nbr.pairs;
  info->n_joint_entries = 0;
  info->n_union_rows = 0;
  info->eq20_tile = 0;
  const int64_t N = hm.n_nodes, T = hm.n_tets;
  info->device_bytes = int64_t(hm.tets.size() * 4 + hm.tet_edges.size() * 4 + hm.slot.size() * 4 +
                               hm.rest.size() * 8 + hm.row_ptr.size() * 4 + hm.col.size() * 4 +
                               hm.edges.size() * 4 + hm.et_ptr.size() * 4 + hm.et_tet.size() * 4 +
                               hm.edge_order.size() * 4 + hm.node_order.size() * 4 +
                               hm.nbr.idx.size() * 12 + hm.nbr.group_off.size() * 12 + hm.nbr.perm.size() * 4) +
                       N * (8 + 8 * 3 * 12 + 9 * 8 + 8) + T * (8 + 18 * 8 + 4) + hm.n_edges * 9 + hm.n_blocks * 72;
  if (edges) std::memcpy(edges, hm.edges.data(), sizeof(int32_t) * hm.edges.size());
  if (colour)
    for (size_t c = 0; c + 1 < hm.colour_ptr.size(); ++c)
      for (int32_t i = hm.colour_ptr[c]; i < hm.colour_ptr[c + 1]; ++i) colour[hm.colour_tets[i]] = int32_t(c);
  if (nbr_count) {
    const NeighbourSell& S = hm.nbr;
    for (int64_t i = 0; i < T; ++i) {
      int64_t g = S.slot[i] / 32, l = S.slot[i] % 32;
      int32_t cnt = 0;
      for (int32_t k = 0; k < S.group_len[g]; ++k) cnt += S.w[S.group_off[g] + 32 * k + l] > 0.0 ? 1 : 0;
      nbr_count[hm.perm[i]] = cnt;
    }
  }
  return GF_OK;
}

void gf_mesh_destroy(gf_mesh* mesh) {
  if (!mesh) return;
  DeviceGuard guard(mesh->device);
  cudaStreamSynchronize(mesh->stream);
  if (mesh->gnn) gnn_orphan(mesh->gnn);   // the network outlives its mesh: it can only be destroyed now
  release(mesh);
  delete mesh;
}

gf_status gf_mesh_info_get(const gf_mesh* m, gf_mesh_info* info) {
  if (!m || !info) {
    set_last_error("NULL argument");
    return GF_BAD_ARG;
  }
  info->n_nodes = m->dm.N;
  info->n_tets = m->dm.T;
  info->n_edges = m->dm.NE;
  info->n_blocks = m->dm.NB;
  info->n_colours = int64_t(m->hm.colour_ptr.size()) - 1;
  info->n_nbr_pairs = m->nbr_pairs;
  info->device_bytes = m->bytes;
  info->n_joint_entries = m->joint_entries;
  info->n_union_rows = m->union_rows;
  info->eq20_tile = m->mixed && m->mt.radius > 0.0 ? m->dm.mx.nl_tile : 0;
  return GF_OK;
}

gf_status gf_state_set(gf_mesh* m, const double* x, const double* v, const uint8_t* labels, const double* chi,
                       int32_t mem) {
  if (!m || !valid_mem(mem)) {
    set_last_error("NULL mesh or bad mem kind");
    return GF_BAD_ARG;
  }
  DeviceGuard guard(m->device);
  DevMesh& d = m->dm;
  if (x) GF_CK(cudaMemcpyAsync(d.x, x, sizeof(double) * 3 * d.N, to_dev(mem), m->stream));
  if (v) GF_CK(cudaMemcpyAsync(d.v, v, sizeof(double) * 3 * d.N, to_dev(mem), m->stream));
  if (labels) GF_CK(cudaMemcpyAsync(d.labels, labels, d.NE, to_dev(mem), m->stream));
  const StepScalars sp0 = step_scalars(m->mt, 1.0, false, 0, false);
  if (m->mixed && (x || v)) m->launches += launch_kind(kB_refresh32, d, m->mt, sp0, m->stream);
  if (chi) {
    const double* src = chi;
    if (mem == GF_MEM_HOST) {
      GF_CK(cudaMemcpyAsync(d.sigf, chi, sizeof(double) * d.T, cudaMemcpyHostToDevice, m->stream));
      src = d.sigf;
    }
    k_gather<<<unsigned((d.T + 255) / 256), 256, 0, m->stream>>>(src, m->perm_dev, d.chi, d.T);
    m->launches += 1;
    if (m->mixed) m->launches += launch_kind(kB_chi_to32, d, m->mt, sp0, m->stream);
    GF_CK(cudaGetLastError());
  } else if (labels) {
    gf_status st = recompute_chi(m);
    if (st != GF_OK) return st;
  }
  GF_CK(cudaStreamSynchronize(m->stream));
  return GF_OK;
}

gf_status gf_tuning_set(gf_mesh* m, const gf_tuning* t) {
  if (!m || !t || (t->assembly != GF_ASSEMBLY_GATHER && t->assembly != GF_ASSEMBLY_COLOUR)) {
    set_last_error("bad tuning (assembly must be GF_ASSEMBLY_GATHER or GF_ASSEMBLY_COLOUR)");
    return GF_BAD_ARG;
  }
  if (m->mixed && t->assembly != GF_ASSEMBLY_GATHER) {
    set_last_error("GF_MIXED assembles by gather only");
    return GF_UNSUPPORTED;
  }
  if (t->step_launch != GF_STEP_GRAPH && t->step_launch != GF_STEP_STREAM) {
    set_last_error("bad tuning (step_launch must be GF_STEP_GRAPH or GF_STEP_STREAM)");
    return GF_BAD_ARG;
  }
  if ((t->solve_loop != GF_SOLVE_KERNELS && t->solve_loop != GF_SOLVE_PERSISTENT && t->solve_loop != GF_SOLVE_CG &&
       t->solve_loop != GF_SOLVE_NESTED) ||
      (t->wait_test != 0 && t->wait_test != 1)) {
    set_last_error("bad tuning (solve_loop must be GF_SOLVE_KERNELS, GF_SOLVE_PERSISTENT, GF_SOLVE_CG or "
                   "GF_SOLVE_NESTED, wait_test 0 or 1)");
    return GF_BAD_ARG;
  }
  if (t->solve_loop == GF_SOLVE_PERSISTENT && !m->mixed) {
    set_last_error("GF_SOLVE_PERSISTENT is built for GF_MIXED meshes");
    return GF_UNSUPPORTED;
  }
  if (t->solve_loop == GF_SOLVE_NESTED && m->mixed) {
    set_last_error("GF_SOLVE_NESTED is built for GF_FP64 meshes");
    return GF_UNSUPPORTED;
  }
  m->tune = *t;
  m->gkey = gf_mesh::GraphKey{};   // capture again on the next step
  return GF_OK;
}

gf_status gf_tuning_get(const gf_mesh* m, gf_tuning* t) {
  if (!m || !t) return GF_BAD_ARG;
  *t = m->tune;
  return GF_OK;
}

gf_status gf_mesh_autotune(gf_mesh* m, double dt, const double* f_ext, const int32_t* pinned, int64_t n_pinned,
                           const double* pinned_vel, int32_t mem, int32_t trial_steps, gf_tuning* best, double* best_ms) {
  if (!m || trial_steps < 1 || trial_steps > 64) {
    set_last_error("autotune: need a mesh and 1 <= trial_steps <= 64");
    return GF_BAD_ARG;
  }
  if (m->gnn || m->newton_iters > 1) {
    set_last_error("autotune: not with a network attached or Newton iterations > 1");
    return GF_UNSUPPORTED;
  }
  DeviceGuard guard(m->device);
  cudaStream_t s = m->stream;
  const DevMesh& d = m->dm;
  // the state a step reads and writes, saved on the device and put back after each trial
  struct Saved {
    void* p;
    void* dst;
    size_t bytes;
  };
  std::vector<Saved> saved;
  gf_status st = GF_OK;
  auto keep = [&](void* src, size_t bytes) {
    if (st != GF_OK || bytes == 0) return;
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      set_last_error("autotune: cannot save the state");
      st = GF_OOM;
      return;
    }
    saved.push_back({p, src, bytes});
    if (cudaMemcpyAsync(p, src, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) st = GF_CUDA_ERR;
  };
  keep(d.x, sizeof(double) * 3 * d.N);
  keep(d.v, sizeof(double) * 3 * d.N);
  keep(d.labels, size_t(d.NE));
  keep(d.chi, sizeof(double) * d.T);
  if (m->mixed) {
    keep(d.mx.u32, sizeof(float) * 3 * d.N);
    keep(d.mx.v32, sizeof(float) * 3 * d.N);
    keep(d.mx.chi32, sizeof(float) * d.T);
  }
  auto restore = [&]() {
    for (auto& sv : saved) cudaMemcpyAsync(sv.dst, sv.p, sv.bytes, cudaMemcpyDeviceToDevice, s);
    cudaStreamSynchronize(s);
  };
  const gf_tuning orig = m->tune;
  std::vector<gf_tuning> cands;
  auto cand = [&](int assembly, int form) {
    gf_tuning t = orig;
    t.assembly = assembly;
    t.solve_loop = form;
    t.step_launch = GF_STEP_GRAPH;
    t.wait_test = 0;
    cands.push_back(t);
  };
  if (m->mixed) {
    for (int form : {GF_SOLVE_CG, GF_SOLVE_KERNELS, GF_SOLVE_PERSISTENT}) cand(GF_ASSEMBLY_GATHER, form);
  } else {
    for (int form : {GF_SOLVE_KERNELS, GF_SOLVE_CG, GF_SOLVE_NESTED}) {
      cand(GF_ASSEMBLY_GATHER, form);
      if (m->mat.energy != GF_ENERGY_SNH) cand(GF_ASSEMBLY_COLOUR, form);
    }
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // ms per step of candidate ci: one untimed step (graph capture, first-use
  // allocations), then the timed trial; the state is put back after each
  auto trial = [&](size_t ci) -> double {
    if ((st = gf_tuning_set(m, &cands[ci])) != GF_OK) return 1e300;
    st = gf_step(m, dt, f_ext, pinned, n_pinned, pinned_vel, mem, nullptr);
    restore();
    if (st != GF_OK) return 1e300;
    cudaEventRecord(e0, s);
    for (int r = 0; r < trial_steps && st == GF_OK; ++r)
      st = gf_step(m, dt, f_ext, pinned, n_pinned, pinned_vel, mem, nullptr);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    restore();
    return st == GF_OK ? double(ms) / trial_steps : 1e300;
  };
  const std::pair<size_t, double> pick = pick_fastest(cands.size(), trial, st);
  const gf_tuning best_c = pick.first < cands.size() ? cands[pick.first] : orig;
  const double best_t = pick.second;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (auto& sv : saved) cudaFree(sv.p);
  const gf_tuning keep_t = st == GF_OK ? best_c : orig;
  gf_status st2 = gf_tuning_set(m, &keep_t);
  if (st == GF_OK) st = st2;
  if (best) *best = m->tune;
  if (best_ms) *best_ms = best_t;
  return st;
}

gf_status gf_refine_set(gf_mesh* m, double inner_rtol) {
  if (!m || !(inner_rtol > 0) || !(inner_rtol < 1)) {
    set_last_error("need 0 < inner_rtol < 1");
    return GF_BAD_ARG;
  }
  m->in_rtol = inner_rtol;
  return GF_OK;
}

gf_status gf_quasistatic_solver_set(gf_mesh* m, int32_t solver, double inner_rtol) {
  if (!m || (solver != GF_QS_SOLVE_FP64 && solver != GF_QS_SOLVE_NESTED) || !(inner_rtol < 1) ||
      std::isnan(inner_rtol)) {
    set_last_error("need solver GF_QS_SOLVE_FP64 or GF_QS_SOLVE_NESTED and inner_rtol < 1");
    return GF_BAD_ARG;
  }
  if (m->mixed) {
    set_last_error("the quasi-static step is built for GF_FP64 meshes only");
    return GF_UNSUPPORTED;
  }
  m->qs_solver = solver;
  if (inner_rtol > 0) m->qs_in_rtol = inner_rtol;
  return GF_OK;
}

gf_status gf_newton_set(gf_mesh* m, int32_t max_iters, double rtol) {
  if (!m || max_iters < 1 || max_iters > 64 || !(rtol >= 0) || !std::isfinite(rtol)) {
    set_last_error("need 1 <= max_iters <= 64 and rtol >= 0");
    return GF_BAD_ARG;
  }
  if (m->mixed && max_iters > 1) {
    set_last_error("more than one Newton iteration per step is built for GF_FP64 meshes only");
    return GF_UNSUPPORTED;
  }
  m->newton_iters = max_iters;
  m->newton_rtol = rtol;
  return GF_OK;
}

gf_status gf_threshold_set(gf_mesh* m, double threshold) {
  if (!m || std::isnan(threshold)) {
    set_last_error("need a mesh and a threshold that is not NaN");
    return GF_BAD_ARG;
  }
  m->mat.threshold = threshold;
  m->mt.threshold = threshold;
  m->gkey = gf_mesh::GraphKey{};   // the captured step holds the material by value: capture again
  return GF_OK;
}

gf_status gf_solver_set(gf_mesh* m, double rtol, int32_t maxit) {
  if (!m || !(rtol > 0) || maxit <= 0) {
    set_last_error("need rtol > 0 and maxit > 0");
    return GF_BAD_ARG;
  }
  m->opt.cg_rtol = rtol;
  m->opt.cg_maxit = maxit;
  return GF_OK;
}

}  // extern "C"

namespace {

int64_t gnn_step_start(gf_gnn* g, const DevMesh& d, int flags, cudaStream_t s);
cudaError_t gnn_keep_previous(gf_gnn* g, const DevMesh& d, cudaStream_t s);

// The one-mesh table and control block of the persistent solve (allocated and
// uploaded on first use, outside any stream capture: the table's pointers and
// block counts do not change for the life of the mesh).
// Blocks of a mesh in one phase of the persistent solve: the kernel form's
// grid, at most one CTA set of the persistent launch (so a lone mesh's phase
// is one balanced wave).  The same for a mesh alone and in a batch.
unsigned persist_blocks(int kind, unsigned blocks) {
  const bool solve_kind = kind == kB_ir_inner_init || kind == kB_ir_spmv || kind == kB_ir_update ||
                          kind == kB_ir_apply || kind == kB_ir_residual;
  const unsigned g = persist_grid();
  return (solve_kind && g > 0 && blocks > g) ? g : blocks;
}

gf_status persist_setup(gf_mesh* m) {
  if (m->ptab) return GF_OK;
  gf_status st = GF_OK;
  void* p = nullptr;
  if ((st = dev_alloc(m, sizeof(BatchTab), &p)) != GF_OK) return st;
  BatchTab* dt = static_cast<BatchTab*>(p);
  if ((st = dev_alloc(m, sizeof(PersistCtl), &p)) != GF_OK) return st;
  PersistCtl* ctl = static_cast<PersistCtl*>(p);
  if (!m->h_pctl) GF_CK(cudaMallocHost(&m->h_pctl, sizeof(PersistCtl)));
  std::unique_ptr<BatchTab> h(new BatchTab());
  h->n = 1;
  h->mesh[0] = m->dm;
  h->mt[0] = m->mt;
  h->sp[0] = step_scalars(m->mt, 1.0, false, 0, false);
  for (int kind = 0; kind < kBKinds; ++kind) {
    h->off[kind][0] = 0;
    h->off[kind][1] = int32_t(persist_blocks(kind, launch_dims(kind, h->mesh[0], h->mt[0], h->sp[0]).blocks));
  }
  GF_CK(cudaMemcpyAsync(dt, h.get(), sizeof(BatchTab), cudaMemcpyHostToDevice, m->stream));
  GF_CK(cudaStreamSynchronize(m->stream));
  m->ptab = dt;
  m->pctl = ctl;
  return GF_OK;
}

bool persist_on(const gf_mesh* m) { return m->mixed && m->tune.solve_loop == GF_SOLVE_PERSISTENT; }

// GF_SOLVE_CG: the Chronopoulos-Gear PCG needs the vector w = A z (FP64: allocated
// on first use; GF_MIXED: its FP32 w32 is allocated with the mesh)
bool cg_form_on(const gf_mesh* m) { return !m->mixed && m->tune.solve_loop == GF_SOLVE_CG; }
bool mixed_cg_on(const gf_mesh* m) { return m->mixed && m->tune.solve_loop == GF_SOLVE_CG; }
// GF_SOLVE_NESTED (GF_FP64): flexible FP64 PCG around an FP32 inner PCG (the
// quasi-static nested solve), stream form
bool nested_on(const gf_mesh* m) { return !m->mixed && m->tune.solve_loop == GF_SOLVE_NESTED; }
gf_status qs_nested_solve(gf_mesh* m, DevMesh dq, const gf::Material& mq, const StepScalars& sq, int64_t& L,
                          int& iters, int& status);
gf_status cg_form_setup(gf_mesh* m, DevMesh& d) {
  if (!m->qs_w) {
    gf_status st = scratch(m, 3 * size_t(d.N), &m->qs_w);
    if (st != GF_OK) return st;
  }
  d.w = m->qs_w;
  return GF_OK;
}

// FP64 path: damage, two-phase (or colour-ordered) assembly, projected PCG (all FP64).
// Newton iterations after the first re-assemble at x^k = x + dt v^k with the
// same kernels (see k_newton_prep) and warm-start the PCG from the previous dv.
gf_status step_fp64(gf_mesh* m, DevMesh& d, double dt, bool has_fext, int64_t n_pinned, bool has_pvel,
                    int64_t& L) {
  cudaStream_t s = m->stream;
  const gf::Material& mt = m->mt;
  const StepScalars sp = step_scalars(mt, dt, has_fext, n_pinned, has_pvel);
  const int64_t N = d.N;
  if (mt.energy == GF_ENERGY_SNH && m->tune.assembly == GF_ASSEMBLY_COLOUR) {
    set_last_error("the colour-ordered assembly is built for the StVK energy only");
    return GF_UNSUPPORTED;
  }
  if (!(mt.radius > 0.0)) d.sig_bar = d.sig_in;   // R_d = 0: the tet alone (local criterion)
  { Prof p(m, kPStress); L += launch_kind(kB_tet_stress, d, mt, sp, s); }
  if (mt.radius > 0.0) {
    Prof p(m, kPNonlocal);
    L += launch_kind(kB_nonlocal, d, mt, sp, s);
  }
  { Prof p(m, kPEdge); L += launch_kind(kB_edge_driver, d, mt, sp, s); }
  { Prof p(m, kPChi); L += launch_kind(kB_tet_chi, d, mt, sp, s); }
  // system at positions/velocities of the view de (element kernels) and d (mass terms)
  auto assemble = [&](const DevMesh& de) -> gf_status {
    {
      Prof p(m, kPAssemble);
      if (m->tune.assembly == GF_ASSEMBLY_COLOUR) {
        GF_CK(cudaMemsetAsync(d.val, 0, sizeof(double) * 9 * d.NB, s));
        L += launch_kind(kB_node_init, d, mt, sp, s);
        const auto& cp = m->hm.colour_ptr;
        for (size_t c = 0; c + 1 < cp.size(); ++c) L += launch_assemble_colour(de, mt, dt, cp[c], cp[c + 1], s);
      } else {
        L += launch_kind(kB_elem64, de, mt, sp, s);
      }
    }
    if (m->tune.assembly != GF_ASSEMBLY_COLOUR) {
      Prof p(m, kPGather);
      L += launch_kind(kB_gather64, d, mt, sp, s);
      L += launch_kind(kB_diag64, d, mt, sp, s);
    }
    return GF_OK;
  };
  // PCG on the assembled system from the dv in place; returns after convergence or maxit
  const bool cg_form = cg_form_on(m), nested = nested_on(m);
  if (cg_form || nested) {   // both keep w = A z
    gf_status st = cg_form_setup(m, d);
    if (st != GF_OK) return st;
  }
  auto run_pcg = [&]() -> gf_status {
    if (nested) {   // its outcome lands in d.pcg like the PCG's
      int its = 0, nst = GF_OK;
      gf_status st = qs_nested_solve(m, d, mt, sp, L, its, nst);
      if (st != GF_OK) return st;
      GF_CK(cudaMemcpyAsync(m->h_pcg, d.pcg, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
      GF_CK(cudaStreamSynchronize(s));
      return GF_OK;
    }
    int launched_iters = 0;
    int chunk = std::max(1, std::min(m->last_iters + 1, 64));
    if (cg_form) { Prof p(m, kPSpmv, 0); L += launch_qs_cg_spmv(d, s); }   // w = A z, coefficients
    for (;;) {
      for (int j = 0; j < chunk; ++j, ++launched_iters) {
        if (cg_form) {   // Chronopoulos-Gear: updates, then the next w = A z with the coefficients
          { Prof p(m, kPPcgUpdate, launched_iters); L += launch_qs_cg_update(d, s); }
          { Prof p(m, kPSpmv, launched_iters + 1); L += launch_qs_cg_spmv(d, s); }
          continue;
        }
        { Prof p(m, kPSpmv, launched_iters); L += launch_kind(kB_pcg_spmv, d, mt, sp, s); }
        { Prof p(m, kPPcgUpdate, launched_iters); L += launch_kind(kB_pcg_update, d, mt, sp, s); }
        { Prof p(m, kPPcgP, launched_iters); L += launch_kind(kB_pcg_p, d, mt, sp, s); }
      }
      GF_CK(cudaGetLastError());
      GF_CK(cudaMemcpyAsync(m->h_pcg, d.pcg, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
      GF_CK(cudaStreamSynchronize(s));
      if (m->h_pcg->done || launched_iters >= m->opt.cg_maxit) break;
      chunk = 8;
    }
    return GF_OK;
  };
  gf_status st = assemble(d);
  if (st != GF_OK) return st;
  PcgState init{};
  init.tol2 = m->opt.cg_rtol * m->opt.cg_rtol;
  init.maxit = m->opt.cg_maxit;
  *m->h_pcg = init;
  GF_CK(cudaMemcpyAsync(d.pcg, m->h_pcg, sizeof(PcgState), cudaMemcpyHostToDevice, s));
  GF_CK(cudaMemsetAsync(d.pinned, 0, N, s));
  if (m->gnn) GF_CK(gnn_keep_previous(m->gnn, d, s));   // the previous solution starts the learned correction
  GF_CK(cudaMemsetAsync(d.dv, 0, sizeof(double) * 3 * N, s));
  L += launch_kind(kB_set_pinned, d, mt, sp, s);
  { Prof p(m, kPPcgInit); L += launch_kind(kB_pcg_init, d, mt, sp, s); }
  if (m->gnn && m->gnn_flags) {   // learned start and preconditioner
    { Prof p(m, kPGnn); L += gnn_step_start(m->gnn, d, m->gnn_flags, s); }
    StepScalars sl = sp;
    sl.learned = 1;
    { Prof p(m, kPPcgInit); L += launch_kind(kB_pcg_init, d, mt, sl, s); }
  }
  if ((st = run_pcg()) != GF_OK) return st;
  m->newton_done = 1;
  m->newton_res = 0.0;
  int cg_total = m->h_pcg->iters;
  const double bb0 = m->h_pcg->bb;
  for (int k = 1; k < m->newton_iters && m->h_pcg->status == GF_OK; ++k) {
    // iterate k: assemble at x^k (element view: positions d.q, K v velocity d.z; PCG vectors are free here)
    L += launch_newton_prep(d, mt, dt, d.q, d.z, s);
    DevMesh de = d;
    de.x = d.q;
    de.v = d.z;
    if ((st = assemble(de)) != GF_OK) return st;
    PcgState again = init;
    *m->h_pcg = again;
    GF_CK(cudaMemcpyAsync(d.pcg, m->h_pcg, sizeof(PcgState), cudaMemcpyHostToDevice, s));
    StepScalars sw = sp;
    sw.warm = 1;
    { Prof p(m, kPPcgInit); L += launch_kind(kB_pcg_init, d, mt, sw, s); }
    if ((st = run_pcg()) != GF_OK) return st;
    cg_total += m->h_pcg->iters;
    m->newton_done = k + 1;
    m->newton_res = bb0 > 0 ? std::sqrt(m->h_pcg->rr0 / bb0) : 0.0;   // |r(v^k)| / |b^0| on free DOFs
    if (m->newton_res <= m->newton_rtol) break;
  }
  { Prof p(m, kPResidual); L += launch_kind(kB_true_residual, d, mt, sp, s); }
  { Prof p(m, kPIntegrate); L += launch_kind(kB_integrate, d, mt, sp, s); }
  GF_CK(cudaGetLastError());
  GF_CK(cudaMemcpyAsync(m->h_pcg, d.pcg, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
  m->newton_cg_total = cg_total;
  return GF_OK;
}

// Mixed path: FP32 damage and tangents, row-gather assembly, FP64 iterative
// refinement around FP32 PCG with FP64 dot products.
gf_status step_mixed(gf_mesh* m, DevMesh& d, double dt, bool has_fext, int64_t n_pinned, bool has_pvel, int64_t& L) {
  cudaStream_t s = m->stream;
  const gf::Material& mt = m->mt;
  const StepScalars sp = step_scalars(mt, dt, has_fext, n_pinned, has_pvel);
  const int64_t N = d.N;
  if (!(mt.radius > 0.0)) d.mx.sig_bar32 = d.mx.sig_in32;
  { Prof p(m, kPStress); L += launch_kind(kB_tet_stress32, d, mt, sp, s); }
  if (mt.radius > 0.0) {
    Prof p(m, kPNonlocal);
    L += launch_kind(kB_nonlocal32, d, mt, sp, s);
  }
  { Prof p(m, kPEdge); L += launch_kind(kB_edge_driver32, d, mt, sp, s); }
  { Prof p(m, kPChi); L += launch_kind(kB_tet_chi32, d, mt, sp, s); }
  {
    Prof p(m, kPAssemble);
    L += launch_kind(kB_elem32, d, mt, sp, s);
  }
  {
    Prof p(m, kPGather);
    L += launch_kind(kB_gather32, d, mt, sp, s);
    L += launch_kind(kB_diag32, d, mt, sp, s);
  }
  IrState init{};
  init.tol2 = m->opt.cg_rtol * m->opt.cg_rtol;
  init.in_tol2 = m->in_rtol * m->in_rtol;
  init.maxit = m->opt.cg_maxit;
  init.in_maxit = 32;         // numerics: each inner solve stops at in_rtol or 32 iterations
  init.applied = 1;
  init.in_done = 1;
  // launches per block only: an unfinished inner solve continues in the next block
  const int K = std::max(2, std::min(m->last_inner + 1, 32));
  *m->h_ir = init;
  GF_CK(cudaMemcpyAsync(d.mx.ir, m->h_ir, sizeof(IrState), cudaMemcpyHostToDevice, s));
  GF_CK(cudaMemsetAsync(d.pinned, 0, N, s));
  GF_CK(cudaMemsetAsync(d.dv, 0, sizeof(double) * 3 * N, s));
  L += launch_kind(kB_set_pinned, d, mt, sp, s);
  L += launch_kind(kB_refresh32, d, mt, sp, s);
  { Prof p(m, kPIrResidual); L += launch_kind(kB_ir_residual, d, mt, sp, s, 1); }
  if (persist_on(m)) {
    int n;
    {
      Prof p(m, kPSolve);
      n = launch_ir_persist(m->ptab, 1, m->pctl, 2 * m->opt.cg_maxit + 64, m->tune.wait_test, s);
    }
    if (n < 0) {
      set_last_error("the cooperative launch of the persistent solve was refused");
      return GF_CUDA_ERR;
    }
    L += n;
    GF_CK(cudaMemcpyAsync(m->h_pctl, m->pctl, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
    { Prof p(m, kPIntegrate); L += launch_kind(kB_integrate32, d, mt, sp, s); }
    GF_CK(cudaGetLastError());
    GF_CK(cudaMemcpyAsync(m->h_ir, d.mx.ir, sizeof(IrState), cudaMemcpyDeviceToHost, s));
    return GF_OK;
  }
  int max_inner = 0;
  for (int round = 0;; ++round) {
    for (int sw = 0; sw < 2; ++sw) {
      { Prof p(m, kPIrInit); L += launch_kind(kB_ir_inner_init, d, mt, sp, s); }
      for (int j = 0; j < K; ++j) {
        if (mixed_cg_on(m)) {
          { Prof p(m, kPSpmv, -2); L += launch_kind(kB_ir_cg_spmv, d, mt, sp, s); }
          { Prof p(m, kPPcgUpdate, -2); L += launch_kind(kB_ir_cg_update, d, mt, sp, s); }
          continue;
        }
        { Prof p(m, kPSpmv, -2); L += launch_kind(kB_ir_spmv, d, mt, sp, s); }
        { Prof p(m, kPPcgUpdate, -2); L += launch_kind(kB_ir_update, d, mt, sp, s); }
        { Prof p(m, kPPcgP, -2); L += launch_kind(kB_ir_p, d, mt, sp, s); }
      }
      { Prof p(m, kPIrApply); L += launch_kind(kB_ir_apply, d, mt, sp, s); }
      { Prof p(m, kPIrResidual); L += launch_kind(kB_ir_residual, d, mt, sp, s, 0); }
    }
    GF_CK(cudaGetLastError());
    GF_CK(cudaMemcpyAsync(m->h_ir, d.mx.ir, sizeof(IrState), cudaMemcpyDeviceToHost, s));
    GF_CK(cudaStreamSynchronize(s));
    max_inner = std::max(max_inner, m->h_ir->in_iters);
    if (m->h_ir->done || m->h_ir->total_iters >= m->opt.cg_maxit || round >= 4096) break;
  }
  m->last_inner = std::max(1, std::min(max_inner, 32));
  { Prof p(m, kPIntegrate); L += launch_kind(kB_integrate32, d, mt, sp, s); }
  GF_CK(cudaGetLastError());
  GF_CK(cudaMemcpyAsync(m->h_ir, d.mx.ir, sizeof(IrState), cudaMemcpyDeviceToHost, s));
  return GF_OK;
}

// Whether a step can run as the captured graph: the plain step (one Newton
// iteration, two-phase assembly, no network, no per-launch profiling).
bool graph_step_ok(const gf_mesh* m) {
  return m->tune.step_launch == GF_STEP_GRAPH && !m->prof && !m->gnn && !nested_on(m) &&
         (m->mixed || (m->newton_iters == 1 && m->tune.assembly == GF_ASSEMBLY_GATHER));
}

// Capture the plain step: the launches of step_fp64 / step_mixed in the same
// order (so the results are the same bits), with the solver loop as a WHILE
// node whose body is `loop` PCG iterations (FP64) or one round of two
// refinement sweeps with `loop` inner iterations each (mixed).
gf_status build_step_graph(gf_mesh* m, DevMesh d, const StepScalars& sp, int loop) {
  cudaStream_t s = m->stream;
  const gf::Material& mt = m->mt;
  if (m->graph_exec) cudaGraphExecDestroy(m->graph_exec);
  if (m->graph) cudaGraphDestroy(m->graph);
  m->graph_exec = nullptr;
  m->graph = nullptr;
  if (!m->body_stream) GF_CK(cudaStreamCreateWithFlags(&m->body_stream, cudaStreamNonBlocking));
  cudaGraph_t g;
  GF_CK(cudaGraphCreate(&g, 0));
  // the persistent solve needs no WHILE node, and a graph may hold no unused conditional handle
  const bool persist = m->mixed && persist_on(m);
  cudaGraphConditionalHandle h{};
  if (!persist) GF_CK(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
  GF_CK(cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  int64_t L = 0;
  GF_CK(cudaMemsetAsync(m->d_loops, 0, sizeof(int), s));
  if (m->mixed) {
    if (!(mt.radius > 0.0)) d.mx.sig_bar32 = d.mx.sig_in32;
    L += launch_kind(kB_tet_stress32, d, mt, sp, s);
    if (mt.radius > 0.0) L += launch_kind(kB_nonlocal32, d, mt, sp, s);
    for (int kind : {kB_edge_driver32, kB_tet_chi32, kB_elem32, kB_gather32, kB_diag32})
      L += launch_kind(kind, d, mt, sp, s);
    GF_CK(cudaMemcpyAsync(d.mx.ir, m->h_init, sizeof(IrState), cudaMemcpyHostToDevice, s));
  } else {
    if (!(mt.radius > 0.0)) d.sig_bar = d.sig_in;
    L += launch_kind(kB_tet_stress, d, mt, sp, s);
    if (mt.radius > 0.0) L += launch_kind(kB_nonlocal, d, mt, sp, s);
    for (int kind : {kB_edge_driver, kB_tet_chi, kB_elem64, kB_gather64, kB_diag64}) L += launch_kind(kind, d, mt, sp, s);
    GF_CK(cudaMemcpyAsync(d.pcg, m->h_init, sizeof(PcgState), cudaMemcpyHostToDevice, s));
  }
  GF_CK(cudaMemsetAsync(d.pinned, 0, d.N, s));
  GF_CK(cudaMemsetAsync(d.dv, 0, sizeof(double) * 3 * d.N, s));
  L += launch_kind(kB_set_pinned, d, mt, sp, s);
  if (m->mixed) {
    L += launch_kind(kB_refresh32, d, mt, sp, s);
    L += launch_kind(kB_ir_residual, d, mt, sp, s, 1);
  } else {
    L += launch_kind(kB_pcg_init, d, mt, sp, s);
    if (cg_form_on(m)) L += launch_qs_cg_spmv(d, s);   // w = A z and the first coefficients
  }
  if (persist) {   // the whole solve as one cooperative launch: no WHILE node
    const int n = launch_ir_persist(m->ptab, 1, m->pctl, 2 * m->opt.cg_maxit + 64, m->tune.wait_test, s);
    if (n < 0) {
      cudaGraph_t dead = nullptr;
      cudaStreamEndCapture(s, &dead);
      if (dead) cudaGraphDestroy(dead);
      cudaGraphDestroy(g);
      set_last_error("the cooperative launch of the persistent solve could not be captured");
      return GF_CUDA_ERR;
    }
    L += n;
    GF_CK(cudaMemcpyAsync(m->h_pctl, m->pctl, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
    L += launch_kind(kB_integrate32, d, mt, sp, s);
    m->g_prefix = L;
    m->g_body = 0;
    m->g_suffix = 0;
    GF_CK(cudaStreamEndCapture(s, &g));
    m->graph = g;
    GF_CK(cudaGraphInstantiate(&m->graph_exec, g, 0));
    return GF_OK;
  }
  m->g_prefix = L;
  cudaStreamCaptureStatus cs;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* ed = nullptr;
  size_t nd = 0;
  GF_CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, nullptr, &deps, &ed, &nd));
  cudaGraphNodeParams p{};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t wn;
  GF_CK(cudaGraphAddNode(&wn, g, deps, ed, nd, &p));
  cudaGraph_t body = p.conditional.phGraph_out[0];
  cudaStream_t bs = m->body_stream;
  GF_CK(cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  L = 0;
  int cap;
  if (m->mixed) {
    for (int sw = 0; sw < 2; ++sw) {
      L += launch_kind(kB_ir_inner_init, d, mt, sp, bs);
      for (int j = 0; j < loop; ++j) {
        if (mixed_cg_on(m)) {
          for (int kind : {kB_ir_cg_spmv, kB_ir_cg_update}) L += launch_kind(kind, d, mt, sp, bs);
          continue;
        }
        for (int kind : {kB_ir_spmv, kB_ir_update, kB_ir_p}) L += launch_kind(kind, d, mt, sp, bs);
      }
      L += launch_kind(kB_ir_apply, d, mt, sp, bs);
      L += launch_kind(kB_ir_residual, d, mt, sp, bs, 0);
    }
    cap = 4096;
    k_step_cond<<<1, 32, 0, bs>>>(nullptr, d.mx.ir, m->d_loops, cap, h);
  } else if (cg_form_on(m)) {
    for (int j = 0; j < loop; ++j) {
      L += launch_qs_cg_update(d, bs);
      L += launch_qs_cg_spmv(d, bs);
    }
    cap = m->opt.cg_maxit / loop + 2;
    k_step_cond<<<1, 32, 0, bs>>>(d.pcg, nullptr, m->d_loops, cap, h);
  } else {
    for (int j = 0; j < loop; ++j)
      for (int kind : {kB_pcg_spmv, kB_pcg_update, kB_pcg_p}) L += launch_kind(kind, d, mt, sp, bs);
    cap = m->opt.cg_maxit / loop + 2;
    k_step_cond<<<1, 32, 0, bs>>>(d.pcg, nullptr, m->d_loops, cap, h);
  }
  m->g_body = L + 1;
  GF_CK(cudaStreamEndCapture(bs, &body));
  GF_CK(cudaStreamUpdateCaptureDependencies(s, &wn, nullptr, 1, cudaStreamSetCaptureDependencies));
  L = 0;
  if (m->mixed) {
    L += launch_kind(kB_integrate32, d, mt, sp, s);
  } else {
    L += launch_kind(kB_true_residual, d, mt, sp, s);
    L += launch_kind(kB_integrate, d, mt, sp, s);
  }
  m->g_suffix = L;
  GF_CK(cudaStreamEndCapture(s, &g));
  m->graph = g;
  GF_CK(cudaGraphInstantiate(&m->graph_exec, g, 0));
  return GF_OK;
}

// The plain step as one graph replay: stage the solver initialiser, capture
// the graph when the key changed, launch it and queue the state read-back.
gf_status step_graph(gf_mesh* m, DevMesh& d, double dt, bool has_fext, int64_t n_pinned, bool has_pvel) {
  cudaStream_t s = m->stream;
  const StepScalars sp = step_scalars(m->mt, dt, has_fext, n_pinned, has_pvel);
  if (!m->h_loops) GF_CK(cudaMallocHost(&m->h_loops, sizeof(int)));
  if (!m->h_init) GF_CK(cudaMallocHost(&m->h_init, std::max(sizeof(IrState), sizeof(PcgState))));
  if (!m->d_loops) {
    gf_status st = scratch(m, 1, &m->d_loops);
    if (st != GF_OK) return st;
  }
  gf_mesh::GraphKey key;
  key.dt = dt;
  key.n_pinned = n_pinned;
  key.has_fext = has_fext ? 1 : 0;
  key.has_pvel = has_pvel ? 1 : 0;
  key.maxit = m->opt.cg_maxit;
  key.f_ext = d.f_ext;
  key.pin_ids = d.pin_ids;
  key.pin_vel = d.pin_vel;
  // the loop body: 2 PCG iterations (FP64); inner iterations of a sweep as the
  // stream form picks them from the previous step (mixed)
  key.loop = m->mixed ? std::max(2, std::min(m->last_inner + 1, 32)) : 2;
  if (m->mixed) {
    IrState init{};
    init.tol2 = m->opt.cg_rtol * m->opt.cg_rtol;
    init.in_tol2 = m->in_rtol * m->in_rtol;
    init.maxit = m->opt.cg_maxit;
    init.in_maxit = 32;
    init.applied = 1;
    init.in_done = 1;
    std::memcpy(m->h_init, &init, sizeof(IrState));
  } else {
    PcgState init{};
    init.tol2 = m->opt.cg_rtol * m->opt.cg_rtol;
    init.maxit = m->opt.cg_maxit;
    std::memcpy(m->h_init, &init, sizeof(PcgState));
  }
  // a key that differs from the captured one only in the mixed loop length keeps the graph
  gf_mesh::GraphKey cmp = key;
  if (m->mixed && m->graph_exec) cmp.loop = m->gkey.loop;
  if (persist_on(m)) {
    gf_status st = persist_setup(m);
    if (st != GF_OK) return st;
  }
  if (cg_form_on(m)) {
    gf_status st = cg_form_setup(m, d);
    if (st != GF_OK) return st;
  }
  if (!m->graph_exec || !(cmp == m->gkey)) {
    gf_status st = build_step_graph(m, d, sp, key.loop);
    if (st != GF_OK) {
      m->gkey = gf_mesh::GraphKey{};
      return st;
    }
    m->gkey = key;
  }
  GF_CK(cudaGraphLaunch(m->graph_exec, s));
  GF_CK(cudaGetLastError());
  if (m->mixed) GF_CK(cudaMemcpyAsync(m->h_ir, d.mx.ir, sizeof(IrState), cudaMemcpyDeviceToHost, s));
  else GF_CK(cudaMemcpyAsync(m->h_pcg, d.pcg, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
  GF_CK(cudaMemcpyAsync(m->h_loops, m->d_loops, sizeof(int), cudaMemcpyDeviceToHost, s));
  return GF_OK;
}

// The quasi-static solve of K dv = b with an FP32 inner solve
// (GF_QS_SOLVE_NESTED), after k_pcg_init has formed the FP64 block-Jacobi
// inverses, r = b and |b|^2 (bb) with dv = 0: flexible PCG in FP64 whose
// preconditioner is the mixed step's two-kernel inner PCG on the FP32 copies,
// until |r|^2 <= cg_rtol^2 bb.  The loop runs as one graph: a WHILE node whose
// body is kQsPairs inner iterations and the outer pair (which acts only once
// the inner solve has finished); with per-launch profiling on, the same
// launches go from the host.  iters: inner iterations; status: the solve's.
constexpr int kQsPairs = 8;

gf_status qs_nested_graph(gf_mesh* m, const DevMesh& dq, const gf::Material& mq, const StepScalars& sq) {
  if (m->qs_graph_exec) return GF_OK;
  if (!m->body_stream) GF_CK(cudaStreamCreateWithFlags(&m->body_stream, cudaStreamNonBlocking));
  cudaGraph_t g;
  GF_CK(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle h{};
  GF_CK(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams p{};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t wn;
  GF_CK(cudaGraphAddNode(&wn, g, nullptr, nullptr, 0, &p));
  cudaGraph_t body = p.conditional.phGraph_out[0];
  cudaStream_t bs = m->body_stream;
  GF_CK(cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  for (int j = 0; j < kQsPairs; ++j) {
    launch_kind(kB_ir_cg_spmv, dq, mq, sq, bs);
    launch_kind(kB_ir_cg_update, dq, mq, sq, bs);
  }
  launch_fcg_spmv(dq, bs);
  launch_fcg_update(dq, bs);
  const int cap = m->opt.cg_maxit / kQsPairs + 4096;
  k_step_cond<<<1, 32, 0, bs>>>(nullptr, dq.mx.ir, m->qs_loops, cap, h);
  GF_CK(cudaStreamEndCapture(bs, &body));
  m->qs_graph = g;
  GF_CK(cudaGraphInstantiate(&m->qs_graph_exec, g, 0));
  return GF_OK;
}

gf_status qs_nested_solve(gf_mesh* m, DevMesh dq, const gf::Material& mq, const StepScalars& sq, int64_t& L,
                          int& iters, int& status) {
  cudaStream_t s = m->stream;
  const int64_t N = dq.N;
  MixDev& x = m->qsr;
  if (!x.ir) {
    gf_status st;
    if ((st = scratch(m, 9 * size_t(dq.NB), &x.val32)) || (st = scratch(m, 9 * size_t(N), &x.pinv32)) ||
        (st = scratch(m, 3 * size_t(N), &x.r32)) || (st = scratch(m, 3 * size_t(N), &x.z32)) ||
        (st = scratch(m, 3 * size_t(N), &x.p32)) || (st = scratch(m, 3 * size_t(N), &x.q32)) ||
        (st = scratch(m, 3 * size_t(N), &x.w32)) || (st = scratch(m, 3 * size_t(N), &x.d32)) ||
        (st = scratch(m, size_t(N), &x.z4)) || (st = scratch(m, 1, &x.ir)) || (st = scratch(m, 1, &m->qs_loops)))
      return st;
  }
  dq.mx = x;
  L += launch_qsr_to32(dq, s);
  IrState init{};   // bb: k_qsr_start takes the reference k_pcg_init left in m.pcg
  init.tol2 = m->opt.cg_rtol * m->opt.cg_rtol;
  init.in_tol2 = m->qs_in_rtol * m->qs_in_rtol;
  init.maxit = m->opt.cg_maxit;
  init.in_maxit = m->opt.cg_maxit;
  *m->h_ir = init;
  GF_CK(cudaMemcpyAsync(x.ir, m->h_ir, sizeof(IrState), cudaMemcpyHostToDevice, s));
  { Prof p(m, kPIrInit); L += launch_qsr_start(dq, s); }
  if (!m->prof) {
    if (!m->h_loops) GF_CK(cudaMallocHost(&m->h_loops, sizeof(int)));
    gf_status st = qs_nested_graph(m, dq, mq, sq);
    if (st != GF_OK) return st;
    GF_CK(cudaMemsetAsync(m->qs_loops, 0, sizeof(int), s));
    GF_CK(cudaGraphLaunch(m->qs_graph_exec, s));
    int loops = 0;
    GF_CK(cudaMemcpyAsync(m->h_ir, x.ir, sizeof(IrState), cudaMemcpyDeviceToHost, s));
    GF_CK(cudaMemcpyAsync(m->h_loops, m->qs_loops, sizeof(int), cudaMemcpyDeviceToHost, s));
    GF_CK(cudaStreamSynchronize(s));
    loops = *m->h_loops;
    L += int64_t(loops) * (2 * kQsPairs + 3);
  } else {
    int chunk = std::max(2, std::min(m->last_iters + 1, 64));
    for (int outer = 0; outer < 100000; ++outer) {
      for (;;) {
        for (int j = 0; j < chunk; ++j) {
          { Prof p(m, kPSpmv, -2); L += launch_kind(kB_ir_cg_spmv, dq, mq, sq, s); }
          { Prof p(m, kPPcgUpdate, -2); L += launch_kind(kB_ir_cg_update, dq, mq, sq, s); }
        }
        GF_CK(cudaGetLastError());
        GF_CK(cudaMemcpyAsync(m->h_ir, x.ir, sizeof(IrState), cudaMemcpyDeviceToHost, s));
        GF_CK(cudaStreamSynchronize(s));
        if (m->h_ir->done || m->h_ir->in_done) break;
        chunk = 8;
      }
      if (m->h_ir->done) break;
      chunk = std::max(2, std::min(m->h_ir->in_iters + 1, 64));
      { Prof p(m, kPIrResidual); L += launch_fcg_spmv(dq, s); }
      { Prof p(m, kPIrApply); L += launch_fcg_update(dq, s); }
    }
  }
  L += launch_nested_finish(dq, s);
  GF_CK(cudaGetLastError());
  iters = m->h_ir->total_iters;
  status = m->h_ir->done ? m->h_ir->status : GF_CG_MAXITER;
  return GF_OK;
}

}  // namespace

extern "C" {

gf_status gf_step(gf_mesh* m, double dt, const double* f_ext, const int32_t* pinned, int64_t n_pinned,
                  const double* pinned_vel, int32_t mem, gf_step_stats* stats) {
  if (!m || !valid_mem(mem) || !(dt > 0) || !std::isfinite(dt) || n_pinned < 0 || n_pinned > m->dm.N ||
      (n_pinned > 0 && !pinned)) {
    set_last_error("bad step arguments (need dt > 0, 0 <= n_pinned <= n_nodes, pinned when n_pinned > 0)");
    return GF_BAD_ARG;
  }
  if (mem == GF_MEM_HOST)
    for (int64_t i = 0; i < n_pinned; ++i)
      if (pinned[i] < 0 || pinned[i] >= m->dm.N) {
        set_last_error("pinned node id out of range");
        return GF_BAD_ARG;
      }
  DeviceGuard guard(m->device);
  Nvtx range(graph_step_ok(m) ? "gf_step (graph replay)" : "gf_step");
  cudaStream_t s = m->stream;
  DevMesh d = m->dm;   // per-step view (input pointers may be overridden)
  const int64_t N = d.N;
  const bool graph = graph_step_ok(m);
  GF_CK(cudaMemsetAsync(d.counters, 0, sizeof(unsigned long long) * kCntMax, s));
  // inputs: host arrays are copied into the library's buffers; device arrays are
  // read in place, except by the graph form, which copies them too (a few us) so
  // that a new caller buffer per step does not force a new capture
  const cudaMemcpyKind in_kind = mem == GF_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  const bool copy_in = mem == GF_MEM_HOST || graph;
  if (f_ext && copy_in) {
    GF_CK(cudaMemcpyAsync(d.f_ext, f_ext, sizeof(double) * 3 * N, in_kind, s));
  } else if (f_ext) {
    d.f_ext = const_cast<double*>(f_ext);
  }
  if (n_pinned > 0) {
    if (copy_in) {
      GF_CK(cudaMemcpyAsync(d.pin_ids, pinned, sizeof(int32_t) * n_pinned, in_kind, s));
      if (pinned_vel) GF_CK(cudaMemcpyAsync(d.pin_vel, pinned_vel, sizeof(double) * 3 * n_pinned, in_kind, s));
    } else {
      d.pin_ids = const_cast<int32_t*>(pinned);
      if (pinned_vel) d.pin_vel = const_cast<double*>(pinned_vel);
    }
  }
  int64_t L = 0;
  const bool persist = persist_on(m);
  if (persist && !graph) {
    gf_status ps = persist_setup(m);
    if (ps != GF_OK) return ps;
  }
  gf_status st = graph ? step_graph(m, d, dt, f_ext != nullptr, n_pinned, pinned_vel != nullptr)
                 : m->mixed ? step_mixed(m, d, dt, f_ext != nullptr, n_pinned, pinned_vel != nullptr, L)
                            : step_fp64(m, d, dt, f_ext != nullptr, n_pinned, pinned_vel != nullptr, L);
  if (st != GF_OK) return st;
  m->assembled = true;
  GF_CK(cudaMemcpyAsync(m->h_cnt, d.counters, sizeof(unsigned long long) * kCntMax, cudaMemcpyDeviceToHost, s));
  GF_CK(cudaStreamSynchronize(s));
  if (graph) {
    L = m->g_prefix + m->g_suffix + int64_t(*m->h_loops) * m->g_body;
    if (m->mixed) {
      m->last_inner = std::max(1, std::min(m->h_ir->in_iters, 32));
    } else {
      m->newton_done = 1;
      m->newton_res = 0.0;
      m->newton_cg_total = m->h_pcg->iters;
    }
  }
  m->launches += L;
  gf_status status;
  int iters, sweeps = 0;
  double rel;
  if (m->mixed) {
    const IrState& ir = *m->h_ir;
    status = gf_status(ir.status);
    iters = ir.total_iters;
    sweeps = ir.sweeps;
    rel = ir.bb > 0 ? std::sqrt(ir.rr / ir.bb) : 0.0;
    if (status == GF_OK && !ir.done) status = GF_CG_MAXITER;
    prof_collect(m, 1 << 30, false);
  } else {
    const PcgState& ps = *m->h_pcg;
    m->last_iters = ps.iters;
    prof_collect(m, ps.iters, ps.status == GF_OK);
    status = gf_status(ps.status);
    iters = m->newton_cg_total;
    rel = ps.bb > 0 ? std::sqrt(ps.true_rr / ps.bb) : 0.0;
  }
  if (status == GF_OK && !std::isfinite(rel)) status = GF_NAN;
  if (persist && m->h_pctl->error != 0) {
    // a phase cut short may leave reduction tickets counted: clear them for the next step
    GF_CK(cudaMemsetAsync(d.tickets, 0, sizeof(unsigned) * kTickets, s));
    GF_CK(cudaStreamSynchronize(s));
    status = GF_TIMEOUT;
  }
  if (status == GF_OK && m->h_cnt[kCntTcTimeout] != 0) {
    set_last_error("a tensor-core wait of the network gave up (device timeout)");
    status = GF_TIMEOUT;
  }
  if (m->h_cnt[kCntBadPin] != 0) {
    set_last_error("pinned node id out of range (skipped)");
    status = GF_BAD_ARG;
  }
  if (stats) {
    stats->status = status;
    stats->cg_iters = iters;
    stats->rel_res = rel;
    stats->n_broken = int64_t(m->h_cnt[kCntBroken]);
    stats->n_new_broken = int64_t(m->h_cnt[kCntNewBroken]);
    stats->n_chi_zero = int64_t(m->h_cnt[kCntChiZero]);
    stats->refine_sweeps = sweeps;
    stats->newton_iters = m->mixed ? 1 : m->newton_done;
  }
  if (status != GF_OK && status != GF_BAD_ARG)
    set_last_error(std::string("step: ") + gf_status_string(status));
  return status;
}

gf_status gf_quasistatic_step(gf_mesh* m, const double* f_ext, const int32_t* pinned, int64_t n_pinned,
                              const double* pinned_pos, int32_t mem, int32_t max_newton, double rtol,
                              gf_step_stats* stats) {
  if (!m || !valid_mem(mem) || n_pinned < 0 || n_pinned > m->dm.N || (n_pinned > 0 && !pinned) ||
      max_newton < 1 || max_newton > 1000 || !(rtol >= 0) || !std::isfinite(rtol) || (pinned_pos && n_pinned == 0)) {
    set_last_error("bad quasi-static step arguments (need 1 <= max_newton <= 1000, rtol >= 0, pinned when "
                   "n_pinned > 0, pinned_pos only with pinned nodes)");
    return GF_BAD_ARG;
  }
  if (m->mixed) {
    set_last_error("the quasi-static step is built for GF_FP64 meshes only");
    return GF_UNSUPPORTED;
  }
  if (mem == GF_MEM_HOST)
    for (int64_t i = 0; i < n_pinned; ++i)
      if (pinned[i] < 0 || pinned[i] >= m->dm.N) {
        set_last_error("pinned node id out of range");
        return GF_BAD_ARG;
      }
  DeviceGuard guard(m->device);
  Nvtx range("gf_quasistatic_step");
  cudaStream_t s = m->stream;
  DevMesh d = m->dm;
  const int64_t N = d.N;
  gf_status st = GF_OK;
  if (!m->qs_x) {
    if ((st = scratch(m, 3 * N, &m->qs_x)) || (st = scratch(m, 3 * N, &m->qs_zero)) || (st = scratch(m, 4, &m->qs_out)) ||
        (st = scratch(m, 3 * N, &m->qs_w)))
      return st;
    GF_CK(cudaMemsetAsync(m->qs_zero, 0, sizeof(double) * 3 * N, s));
  }
  GF_CK(cudaMemsetAsync(d.counters, 0, sizeof(unsigned long long) * kCntMax, s));
  if (f_ext && mem == GF_MEM_HOST) GF_CK(cudaMemcpyAsync(d.f_ext, f_ext, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, s));
  else if (f_ext) d.f_ext = const_cast<double*>(f_ext);
  const double* pos = nullptr;
  if (n_pinned > 0) {
    if (mem == GF_MEM_HOST) {
      GF_CK(cudaMemcpyAsync(d.pin_ids, pinned, sizeof(int32_t) * n_pinned, cudaMemcpyHostToDevice, s));
      if (pinned_pos) {
        GF_CK(cudaMemcpyAsync(d.pin_vel, pinned_pos, sizeof(double) * 3 * n_pinned, cudaMemcpyHostToDevice, s));
        pos = d.pin_vel;
      }
    } else {
      d.pin_ids = const_cast<int32_t*>(pinned);
      pos = pinned_pos;
    }
  }
  int64_t L = 0;
  // 1. damage at the start-of-step positions (Algorithm 1 order), chi frozen afterwards
  const gf::Material& mt = m->mt;
  const StepScalars sp0 = step_scalars(mt, 1.0, false, 0, false);
  if (!(mt.radius > 0.0)) d.sig_bar = d.sig_in;
  { Prof p(m, kPStress); L += launch_kind(kB_tet_stress, d, mt, sp0, s); }
  if (mt.radius > 0.0) {
    Prof p(m, kPNonlocal);
    L += launch_kind(kB_nonlocal, d, mt, sp0, s);
  }
  { Prof p(m, kPEdge); L += launch_kind(kB_edge_driver, d, mt, sp0, s); }
  { Prof p(m, kPChi); L += launch_kind(kB_tet_chi, d, mt, sp0, s); }
  // 2. the pinned nodes move to their prescribed positions
  if (pos) L += launch_qs_set_pins(d, d.pin_ids, pos, n_pinned, s);
  // 3. Newton on f* + f_ext = 0 (free DOFs): the dynamic system with no mass, no damping, dt = 1, v = 0
  gf::Material mq = mt;
  mq.alpha = 0.0;
  mq.beta = 0.0;
  StepScalars sq = step_scalars(mq, 1.0, f_ext != nullptr, n_pinned, false);
  sq.mscale = 0.0;
  DevMesh dq = d;
  dq.v = m->qs_zero;
  dq.w = m->qs_w;
  GF_CK(cudaMemsetAsync(d.pinned, 0, N, s));
  double r0 = -1.0, rel = 0.0, h_out[4];
  int cg_total = 0, k = 0, status = GF_OK;
  const double c_armijo = 1e-4;
  for (k = 0; k < max_newton; ++k) {
    { Prof p(m, kPAssemble); L += launch_kind(kB_elem64, dq, mq, sq, s); }
    {
      Prof p(m, kPGather);
      L += launch_kind(kB_gather64, dq, mq, sq, s);
      L += launch_kind(kB_diag64, dq, mq, sq, s);
    }
    PcgState init{};
    init.tol2 = m->opt.cg_rtol * m->opt.cg_rtol;
    init.maxit = m->opt.cg_maxit;
    *m->h_pcg = init;
    GF_CK(cudaMemcpyAsync(d.pcg, m->h_pcg, sizeof(PcgState), cudaMemcpyHostToDevice, s));
    GF_CK(cudaMemsetAsync(d.dv, 0, sizeof(double) * 3 * N, s));
    L += launch_kind(kB_set_pinned, dq, mq, sq, s);
    { Prof p(m, kPPcgInit); L += launch_kind(kB_pcg_init, dq, mq, sq, s); }
    GF_CK(cudaMemcpyAsync(m->h_pcg, d.pcg, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
    GF_CK(cudaStreamSynchronize(s));
    const double rn = std::sqrt(m->h_pcg->bb);   // |f_ext + f*| on free DOFs
    if (r0 < 0) r0 = rn;
    rel = r0 > 0 ? rn / r0 : 0.0;
    if (!std::isfinite(rn)) {
      status = GF_NAN;
      break;
    }
    if (rn == 0.0 || rn <= rtol * r0) break;
    if (m->qs_solver == GF_QS_SOLVE_NESTED) {
      int its = 0, qst = GF_OK;
      if ((st = qs_nested_solve(m, dq, mq, sq, L, its, qst)) != GF_OK) return st;
      cg_total += its;
      m->last_iters = its;
      if (qst != GF_OK) {
        status = qst;
        break;
      }
    } else {
    // PCG in the Chronopoulos-Gear form: w = A z and the coefficients, then
    // per iteration the vector updates and the next w = A z
    int launched = 0;
    int chunk = std::max(1, std::min(m->last_iters + 1, 64));
    { Prof p(m, kPSpmv, launched); L += launch_qs_cg_spmv(dq, s); }
    for (;;) {
      for (int j = 0; j < chunk; ++j, ++launched) {
        { Prof p(m, kPPcgUpdate, launched); L += launch_qs_cg_update(dq, s); }
        { Prof p(m, kPSpmv, launched); L += launch_qs_cg_spmv(dq, s); }
      }
      GF_CK(cudaGetLastError());
      GF_CK(cudaMemcpyAsync(m->h_pcg, d.pcg, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
      GF_CK(cudaStreamSynchronize(s));
      if (m->h_pcg->done || launched >= m->opt.cg_maxit) break;
      chunk = 8;
    }
    cg_total += m->h_pcg->iters;
    m->last_iters = m->h_pcg->iters;
    if (m->h_pcg->status != GF_OK) {
      status = m->h_pcg->status;
      break;
    }
    }
    // line search on E(x) = sum chi V Psi - f_ext . x
    L += launch_qs_slope(dq, m->qs_out, s);
    L += launch_qs_energy(dq, mq, d.x, f_ext ? d.f_ext : nullptr, m->qs_out, s);
    GF_CK(cudaMemcpyAsync(h_out, m->qs_out, sizeof(double) * 3, cudaMemcpyDeviceToHost, s));
    GF_CK(cudaStreamSynchronize(s));
    const double e0 = h_out[0], scale = h_out[1], slope = h_out[2];
    double a = 1.0;
    while (a > std::ldexp(1.0, -30)) {
      if (c_armijo * a * slope <= 1e-12 * scale) break;   // below what E resolves: take the step
      L += launch_qs_trial(3 * N, d.x, d.dv, a, m->qs_x, s);
      L += launch_qs_energy(dq, mq, m->qs_x, f_ext ? d.f_ext : nullptr, m->qs_out, s);
      GF_CK(cudaMemcpyAsync(h_out, m->qs_out, sizeof(double), cudaMemcpyDeviceToHost, s));
      GF_CK(cudaStreamSynchronize(s));
      if (h_out[0] <= e0 - c_armijo * a * slope) break;
      a *= 0.5;
    }
    L += launch_qs_trial(3 * N, d.x, d.dv, a, m->qs_x, s);
    GF_CK(cudaMemcpyAsync(d.x, m->qs_x, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, s));
  }
  GF_CK(cudaMemsetAsync(d.v, 0, sizeof(double) * 3 * N, s));   // quasi-static: at rest after the step
  GF_CK(cudaGetLastError());
  GF_CK(cudaMemcpyAsync(m->h_cnt, d.counters, sizeof(unsigned long long) * kCntMax, cudaMemcpyDeviceToHost, s));
  GF_CK(cudaStreamSynchronize(s));
  m->assembled = true;
  m->launches += L;
  prof_collect(m, 1 << 30, false);
  bool newton_short = false;
  if (status == GF_OK && k >= max_newton && rel > rtol) {
    status = GF_CG_MAXITER;
    newton_short = true;
  }
  if (m->h_cnt[kCntBadPin] != 0) {
    set_last_error("pinned node id out of range (skipped)");
    status = GF_BAD_ARG;
  }
  if (stats) {
    stats->status = status;
    stats->cg_iters = cg_total;
    stats->rel_res = rel;
    stats->n_broken = int64_t(m->h_cnt[kCntBroken]);
    stats->n_new_broken = int64_t(m->h_cnt[kCntNewBroken]);
    stats->n_chi_zero = int64_t(m->h_cnt[kCntChiZero]);
    stats->refine_sweeps = 0;
    stats->newton_iters = k;
  }
  if (newton_short)
    set_last_error("quasi-static step: Newton did not reach rtol within max_newton iterations");
  else if (status != GF_OK && status != GF_BAD_ARG)
    set_last_error(std::string("quasi-static step: ") + gf_status_string(gf_status(status)));
  return gf_status(status);
}

}  // extern "C"

namespace {

// Faces (sorted node triples, lexicographic), the face opposite each local node
// of every tet and each face's edge ids; rest positions; the scan buffer.
gf_status surface_setup(gf_mesh* m) {
  if (m->surf_ready) return GF_OK;
  DevMesh& d = m->dm;
  const int64_t T = d.T;
  std::vector<int32_t> tets(4 * T);
  GF_CK(cudaMemcpyAsync(tets.data(), d.tets, sizeof(int32_t) * 4 * T, cudaMemcpyDeviceToHost, m->stream));
  GF_CK(cudaStreamSynchronize(m->stream));
  struct Tri { int32_t a, b, c; int64_t slot; };
  std::vector<Tri> tri(4 * T);
  const int opp[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
  for (int64_t t = 0; t < T; ++t)
    for (int i = 0; i < 4; ++i) {
      int32_t v[3] = {tets[4 * t + opp[i][0]], tets[4 * t + opp[i][1]], tets[4 * t + opp[i][2]]};
      std::sort(v, v + 3);
      tri[4 * t + i] = {v[0], v[1], v[2], 4 * t + i};
    }
  std::sort(tri.begin(), tri.end(), [](const Tri& x, const Tri& y) {
    return x.a != y.a ? x.a < y.a : (x.b != y.b ? x.b < y.b : (x.c != y.c ? x.c < y.c : x.slot < y.slot));
  });
  std::vector<int32_t> faces, tet_faces(4 * T), face_edges;
  const std::vector<int32_t>& E = m->hm.edges;
  const int64_t NE = m->hm.n_edges;
  auto edge_id = [&](int32_t u, int32_t v) -> int32_t {
    int64_t lo = 0, hi = NE;
    while (lo < hi) {
      const int64_t mid = (lo + hi) / 2;
      if (E[2 * mid] < u || (E[2 * mid] == u && E[2 * mid + 1] < v)) lo = mid + 1;
      else hi = mid;
    }
    return int32_t(lo);
  };
  for (size_t i = 0; i < tri.size(); ++i) {
    if (i == 0 || tri[i].a != tri[i - 1].a || tri[i].b != tri[i - 1].b || tri[i].c != tri[i - 1].c) {
      faces.insert(faces.end(), {tri[i].a, tri[i].b, tri[i].c});
      face_edges.insert(face_edges.end(), {edge_id(tri[i].a, tri[i].b), edge_id(tri[i].a, tri[i].c),
                                           edge_id(tri[i].b, tri[i].c)});
    }
    tet_faces[tri[i].slot] = int32_t(faces.size() / 3 - 1);
  }
  SurfDev& sd = m->surf;
  sd.NF = int64_t(faces.size() / 3);
  gf_status st = GF_OK;
  const double* X = nullptr;
  const int32_t *pf = nullptr, *pfe = nullptr, *ptf = nullptr;
  if ((st = upload(m, m->X0, &X)) || (st = upload(m, faces, &pf)) || (st = upload(m, face_edges, &pfe)) ||
      (st = upload(m, tet_faces, &ptf)) || (st = scratch(m, size_t(surf_blocks(d) + 1), &sd.bsum)))
    return st;
  sd.X = X;
  sd.faces = reinterpret_cast<const int3*>(pf);
  sd.face_edges = reinterpret_cast<const int3*>(pfe);
  sd.tet_faces = reinterpret_cast<const int4*>(ptf);
  m->surf_ready = true;
  return GF_OK;
}

gf_status surface_count(gf_mesh* m, int64_t* n_quads) {
  gf_status st = surface_setup(m);
  if (st != GF_OK) return st;
  m->launches += launch_surface_count(m->dm, m->surf, m->stream);
  GF_CK(cudaGetLastError());
  unsigned total = 0;
  GF_CK(cudaMemcpyAsync(&total, m->surf.bsum + surf_blocks(m->dm), sizeof(unsigned), cudaMemcpyDeviceToHost,
                        m->stream));
  GF_CK(cudaStreamSynchronize(m->stream));
  *n_quads = int64_t(total);
  return GF_OK;
}

}  // namespace

extern "C" {

gf_status gf_surface_sizes(gf_mesh* m, int64_t* n_vertices, int64_t* n_faces, int64_t* n_quads) {
  if (!m || !n_vertices || !n_faces || !n_quads) {
    set_last_error("surface_sizes: need the mesh and three outputs");
    return GF_BAD_ARG;
  }
  DeviceGuard guard(m->device);
  gf_status st = surface_count(m, n_quads);
  if (st != GF_OK) return st;
  *n_faces = m->surf.NF;
  *n_vertices = m->dm.N + 2 * m->dm.NE + 3 * m->surf.NF + 4 * m->dm.T;
  return GF_OK;
}

gf_status gf_surface_get(gf_mesh* m, double* vertices, int32_t* quads, int64_t max_quads, int32_t mem,
                         int64_t* n_quads) {
  if (!m || !vertices || !n_quads || max_quads < 0 || (max_quads > 0 && !quads) || !valid_mem(mem)) {
    set_last_error("surface_get: need the mesh, vertices, n_quads, quads when max_quads > 0, a memory kind");
    return GF_BAD_ARG;
  }
  DeviceGuard guard(m->device);
  int64_t nq = 0;
  gf_status st = surface_count(m, &nq);
  if (st != GF_OK) return st;
  *n_quads = nq;
  if (nq > max_quads) {
    set_last_error("surface_get: max_quads is below the quad count (returned in n_quads)");
    return GF_BAD_ARG;
  }
  const DevMesh& d = m->dm;
  const int64_t nv = d.N + 2 * d.NE + 3 * m->surf.NF + 4 * d.T;
  double* V = vertices;
  int32_t* Q = quads;
  if (mem == GF_MEM_HOST) {
    const size_t need = sizeof(double) * 3 * nv + sizeof(int32_t) * 4 * size_t(nq) + 256;
    if (need > m->surf_stage_bytes) {
      if (m->surf_stage) cudaFree(m->surf_stage);
      m->surf_stage = nullptr;
      m->surf_stage_bytes = 0;
      if (cudaMalloc(&m->surf_stage, need) != cudaSuccess) {
        cudaGetLastError();
        set_last_error("surface_get: staging allocation failed");
        return GF_OOM;
      }
      m->surf_stage_bytes = need;
    }
    V = static_cast<double*>(m->surf_stage);
    Q = reinterpret_cast<int32_t*>(static_cast<char*>(m->surf_stage) + ((sizeof(double) * 3 * nv + 255) & ~size_t(255)));
  }
  m->launches += launch_surface_vertices(d, m->surf, V, m->stream);
  if (nq > 0) m->launches += launch_surface_quads(d, m->surf, Q, nq, m->stream);
  GF_CK(cudaGetLastError());
  if (mem == GF_MEM_HOST) {
    GF_CK(cudaMemcpyAsync(vertices, V, sizeof(double) * 3 * nv, cudaMemcpyDeviceToHost, m->stream));
    if (nq > 0) GF_CK(cudaMemcpyAsync(quads, Q, sizeof(int32_t) * 4 * nq, cudaMemcpyDeviceToHost, m->stream));
  }
  GF_CK(cudaStreamSynchronize(m->stream));
  return GF_OK;
}

gf_status gf_positions_get(gf_mesh* m, double* x, int32_t mem) {
  if (!m || !x || !valid_mem(mem)) {
    set_last_error("bad arguments");
    return GF_BAD_ARG;
  }
  DeviceGuard guard(m->device);
  GF_CK(cudaMemcpyAsync(x, m->dm.x, sizeof(double) * 3 * m->dm.N, from_dev(mem), m->stream));
  GF_CK(cudaStreamSynchronize(m->stream));
  return GF_OK;
}

gf_status gf_velocities_get(gf_mesh* m, double* v, int32_t mem) {
  if (!m || !v || !valid_mem(mem)) {
    set_last_error("bad arguments");
    return GF_BAD_ARG;
  }
  DeviceGuard guard(m->device);
  GF_CK(cudaMemcpyAsync(v, m->dm.v, sizeof(double) * 3 * m->dm.N, from_dev(mem), m->stream));
  GF_CK(cudaStreamSynchronize(m->stream));
  return GF_OK;
}

gf_status gf_damage_get(gf_mesh* m, double* driver, uint8_t* labels, int32_t mem) {
  if (!m || !valid_mem(mem)) {
    set_last_error("bad arguments");
    return GF_BAD_ARG;
  }
  DeviceGuard guard(m->device);
  if (driver) GF_CK(cudaMemcpyAsync(driver, m->dm.driver, sizeof(double) * m->dm.NE, from_dev(mem), m->stream));
  if (labels) GF_CK(cudaMemcpyAsync(labels, m->dm.labels, m->dm.NE, from_dev(mem), m->stream));
  GF_CK(cudaStreamSynchronize(m->stream));
  return GF_OK;
}

gf_status gf_chi_get(gf_mesh* m, double* chi, int32_t mem) {
  if (!m || !chi || !valid_mem(mem)) {
    set_last_error("bad arguments");
    return GF_BAD_ARG;
  }
  DeviceGuard guard(m->device);
  DevMesh& d = m->dm;
  // scatter to caller order through a scratch buffer
  k_scatter<<<unsigned((d.T + 255) / 256), 256, 0, m->stream>>>(d.chi, m->perm_dev, d.sigf, d.T);
  m->launches += 1;
  GF_CK(cudaGetLastError());
  GF_CK(cudaMemcpyAsync(chi, d.sigf, sizeof(double) * d.T, from_dev(mem), m->stream));
  GF_CK(cudaStreamSynchronize(m->stream));
  return GF_OK;
}

gf_status gf_edges_get(const gf_mesh* m, int32_t* edges) {
  if (!m || !edges) {
    set_last_error("bad arguments");
    return GF_BAD_ARG;
  }
  std::memcpy(edges, m->hm.edges.data(), sizeof(int32_t) * m->hm.edges.size());
  return GF_OK;
}

gf_status gf_system_get(gf_mesh* m, int32_t* row_ptr, int32_t* col, double* values, double* rhs) {
  if (!m) {
    set_last_error("NULL mesh");
    return GF_BAD_ARG;
  }
  DeviceGuard guard(m->device);
  if (row_ptr) std::memcpy(row_ptr, m->hm.row_ptr.data(), sizeof(int32_t) * m->hm.row_ptr.size());
  if (col) std::memcpy(col, m->hm.col.data(), sizeof(int32_t) * m->hm.col.size());
  std::vector<float> v32;
  if (values && !m->mixed)
    GF_CK(cudaMemcpyAsync(values, m->dm.val, sizeof(double) * 9 * m->dm.NB, cudaMemcpyDeviceToHost, m->stream));
  if (values && m->mixed) {
    v32.resize(9 * m->dm.NB);
    GF_CK(cudaMemcpyAsync(v32.data(), m->dm.mx.val32, sizeof(float) * 9 * m->dm.NB, cudaMemcpyDeviceToHost, m->stream));
  }
  std::vector<float> r32;
  if (rhs && !m->mixed)
    GF_CK(cudaMemcpyAsync(rhs, m->dm.rhs, sizeof(double) * 3 * m->dm.N, cudaMemcpyDeviceToHost, m->stream));
  if (rhs && m->mixed) {
    r32.resize(3 * m->dm.N);
    GF_CK(cudaMemcpyAsync(r32.data(), m->dm.mx.rhs32, sizeof(float) * 3 * m->dm.N, cudaMemcpyDeviceToHost, m->stream));
  }
  GF_CK(cudaStreamSynchronize(m->stream));
  for (size_t i = 0; i < v32.size(); ++i) values[i] = double(v32[i]);
  for (size_t i = 0; i < r32.size(); ++i) rhs[i] = double(r32[i]);
  return GF_OK;
}

gf_status gf_profile_enable(gf_mesh* m, int32_t on) {
  if (!m) return GF_BAD_ARG;
  m->prof = on != 0;
  return GF_OK;
}

int32_t gf_profile_get(gf_mesh* m, double* total_ms, int64_t* launches, int32_t n) {
  if (!m) return 0;
  for (int i = 0; i < std::min<int32_t>(n, kPCount); ++i) {
    if (total_ms) total_ms[i] = m->prof_ms[i];
    if (launches) launches[i] = m->prof_n[i];
  }
  return kPCount;
}

const char* gf_profile_name(int32_t i) { return (i >= 0 && i < kPCount) ? kProfNames[i] : ""; }

gf_status gf_profile_reset(gf_mesh* m) {
  if (!m) return GF_BAD_ARG;
  std::fill(std::begin(m->prof_ms), std::end(m->prof_ms), 0.0);
  std::fill(std::begin(m->prof_n), std::end(m->prof_n), int64_t(0));
  return GF_OK;
}

int64_t gf_launch_count(const gf_mesh* m) { return m ? m->launches : 0; }

}  // extern "C"

// ===========================================================================
// Batched stepping
// ===========================================================================
namespace gf {
namespace {

// Solver scalars every mesh starts a step from.
struct BatchInit {
  PcgState pcg;
  IrState ir;
};

// What the host reads back after a batch step, per mesh.
struct BatchOut {
  PcgState pcg;
  IrState ir;
  unsigned long long cnt[kCntMax];
};

// Per-step reset of every mesh's solver scalars, counters, pinned flags and dv.
__global__ void __launch_bounds__(256) kb_step_begin(const BatchTab* __restrict__ tab, const BatchInit* init,
                                                      int mixed, int* iter) {
  unsigned bid, nb;
  const int k = batch_locate(tab, kB_step_begin, blockIdx.x, bid, nb);
  const DevMesh& m = tab->mesh[k];
  const int64_t i0 = bid * int64_t(blockDim.x) + threadIdx.x;
  if (i0 == 0) {
    if (mixed) *m.mx.ir = init[k].ir;
    else *m.pcg = init[k].pcg;
#pragma unroll
    for (int c = 0; c < kCntMax; ++c) m.counters[c] = 0ull;
    if (k == 0) *iter = 0;
  }
  for (int64_t i = i0; i < 3 * m.N; i += int64_t(nb) * blockDim.x) {
    m.dv[i] = 0.0;
    if (i < m.N) m.pinned[i] = 0;
  }
}

// Exclusive block-wide prefix sum (blockDim.x = 256 >= the batch size);
// s[t] receives thread t's offset and the function returns the total.
__device__ int block_scan256(int v, int* s, int* sw) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  __syncthreads();   // s and sw may still be read from the previous call
  if (lane == 31) sw[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int w = lane < 8 ? sw[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += u;
    }
    if (lane < 8) sw[lane] = w;
  }
  __syncthreads();
  const int base = wid ? sw[wid - 1] : 0;
  s[threadIdx.x] = base + incl - v;
  __syncthreads();
  return sw[7];
}

// The work table of the distributed loop: the unconverged meshes and, per
// solver-loop kind, the offsets of their blocks.  The launch grid `grid` is
// split over the active meshes by node count (at least one block each, at most
// its single-mesh grid), so as meshes converge the others get more of it.
// Returns whether any mesh is left.
__device__ bool build_act(const BatchTab* __restrict__ tab, BatchAct* act, int mixed, int grid) {
  __shared__ int s_pos[256], s_off[256], s_w[8];
  __shared__ unsigned long long s_nodes;
  const int k = threadIdx.x, n = tab->n;
  const int active = k < n && (mixed ? !tab->mesh[k].mx.ir->done : !tab->mesh[k].pcg->done);
  if (k == 0) s_nodes = 0ull;
  __syncthreads();
  if (active) atomicAdd(&s_nodes, (unsigned long long)tab->mesh[k].N);
  const int n_act = block_scan256(active, s_pos, s_w);
  const unsigned long long nodes = s_nodes;
  if (active) act->mesh[s_pos[k]] = k;
  const int nk = mixed ? 6 : 3;
  for (int j = 0; j < nk; ++j) {
    int kind;
    if (mixed) {
      switch (j) {
        case 0: kind = kB_ir_inner_init; break;
        case 1: kind = kB_ir_spmv; break;
        case 2: kind = kB_ir_update; break;
        case 3: kind = kB_ir_p; break;
        case 4: kind = kB_ir_apply; break;
        default: kind = kB_ir_residual; break;
      }
    } else {
      kind = j == 0 ? kB_pcg_spmv : (j == 1 ? kB_pcg_update : kB_pcg_p);
    }
    int cnt = 0;
    if (active) {
      const long long natural = tab->off[kind][k + 1] - tab->off[kind][k];
      const long long share = (static_cast<long long>(grid) * tab->mesh[k].N + (long long)nodes - 1) / (long long)nodes;
      cnt = int(share < 1 ? 1 : (share > natural ? natural : share));
    }
    const int total = block_scan256(cnt, s_off, s_w);
    if (active) act->off[kind][s_pos[k]] = s_off[k];
    if (k == 0) act->off[kind][n_act] = total;
  }
  if (k == 0) act->n = n_act;
  return n_act > 0;
}

__global__ void __launch_bounds__(256) kb_activate(const BatchTab* __restrict__ tab, BatchAct* act, int mixed,
                                                    int grid) {
  build_act(tab, act, mixed, grid);
}

// Solve-loop condition: continue while any mesh is unconverged (and below the
// cap); with a work table, rebuild it for the next iteration.
__global__ void __launch_bounds__(256) kb_any_active(const BatchTab* __restrict__ tab, int mixed, int* iter, int cap,
                                                      cudaGraphConditionalHandle h, BatchAct* act, int grid) {
  int active = 0;
  if (act) {
    active = build_act(tab, act, mixed, grid);
  } else {
    for (int k = threadIdx.x; k < tab->n; k += blockDim.x)
      active |= mixed ? !tab->mesh[k].mx.ir->done : !tab->mesh[k].pcg->done;
    active = __syncthreads_or(active);
  }
  if (threadIdx.x == 0) {
    const int it = ++(*iter);
    cudaGraphSetConditional(h, (active && it < cap) ? 1u : 0u);
  }
}

__global__ void kb_collect(const BatchTab* __restrict__ tab, int mixed, BatchOut* out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= tab->n) return;
  const DevMesh& m = tab->mesh[k];
  if (mixed) out[k].ir = *m.mx.ir;
  else out[k].pcg = *m.pcg;
#pragma unroll
  for (int c = 0; c < kCntMax; ++c) out[k].cnt[c] = m.counters[c];
}

}  // namespace
}  // namespace gf

struct gf_batch {
  std::vector<gf_mesh*> ms;
  int n = 0;
  bool mixed = false;
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t body_stream = nullptr;
  BatchTab* htab = nullptr;          // pinned host mirror
  BatchTab* dtab = nullptr;
  BatchInit* dinit = nullptr;
  BatchOut* hout = nullptr;
  BatchOut* dout = nullptr;
  int* d_iter = nullptr;
  int* h_iter = nullptr;
  unsigned blocks[kBKinds] = {};
  std::vector<int32_t> shape;        // offsets the graph was captured with
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  gf_batch_tuning tune{};
  int cap = 0;
  BatchAct* dact = nullptr;          // work table of the distributed solve loop
  PersistCtl* pctl = nullptr;        // control block of the persistent solve
  PersistCtl* h_pctl = nullptr;      // pinned mirror of its head
  int64_t launches = 0;
  int64_t prefix_kernels = 0, body_kernels = 0, suffix_kernels = 0;
};

namespace {

void batch_free(gf_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->dtab) cudaFree(b->dtab);
  if (b->dinit) cudaFree(b->dinit);
  if (b->dout) cudaFree(b->dout);
  if (b->d_iter) cudaFree(b->d_iter);
  if (b->htab) cudaFreeHost(b->htab);
  if (b->hout) cudaFreeHost(b->hout);
  if (b->h_iter) cudaFreeHost(b->h_iter);
  if (b->body_stream) cudaStreamDestroy(b->body_stream);
  if (b->pctl) cudaFree(b->pctl);
  if (b->dact) cudaFree(b->dact);
  if (b->h_pctl) cudaFreeHost(b->h_pctl);
}

bool batch_dist(const gf_batch* b) { return b->tune.solve_loop == GF_SOLVE_DISTRIBUTED; }
// grid of a distributed loop launch: the tuning's budget, else four CTAs per SM
unsigned dist_grid(const gf_batch* b) {
  if (b->tune.grid_budget > 0) return unsigned(b->tune.grid_budget);
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return unsigned(4 * sms);
}

const int kPrefixFp64[] = {kB_tet_stress, kB_nonlocal, kB_edge_driver, kB_tet_chi, kB_elem64, kB_gather64, kB_diag64,
                           kB_set_pinned, kB_pcg_init};
const int kBodyFp64[] = {kB_pcg_spmv, kB_pcg_update, kB_pcg_p};
const int kSuffixFp64[] = {kB_true_residual, kB_integrate};
const int kPrefixMixed[] = {kB_tet_stress32, kB_nonlocal32, kB_edge_driver32, kB_tet_chi32, kB_elem32,
                            kB_gather32, kB_diag32, kB_set_pinned, kB_refresh32};
const int kSuffixMixed[] = {kB_integrate32};

template <size_t K>
int64_t enqueue_kinds(gf_batch* b, const int (&kinds)[K], cudaStream_t s) {
  int64_t L = 0;
  for (int kind : kinds) L += launch_batch(kind, b->dtab, b->blocks[kind], s, 0);
  return L;
}

int64_t enqueue_prefix(gf_batch* b, cudaStream_t s) {
  int64_t L = 0;
  kb_step_begin<<<b->blocks[kB_step_begin], 256, 0, s>>>(b->dtab, b->dinit, b->mixed ? 1 : 0, b->d_iter);
  ++L;
  if (b->mixed) {
    L += enqueue_kinds(b, kPrefixMixed, s);
    L += launch_batch(kB_ir_residual, b->dtab, b->blocks[kB_ir_residual], s, 1);
  } else {
    L += enqueue_kinds(b, kPrefixFp64, s);
  }
  if (batch_dist(b)) {   // the first work table: the meshes the first residual left unconverged
    kb_activate<<<1, 256, 0, s>>>(b->dtab, b->dact, b->mixed ? 1 : 0, int(dist_grid(b)));
    ++L;
  }
  return L;
}

// One pass of the solver loop.  GF_MIXED: inner start, `inner` inner iterations
// (three kernels each, or two in the GF_SOLVE_CG form), apply, residual: a
// member's kernels act only in the phase its own flags call for, so a member
// whose inner solve ends early idles to the end of the pass.  FP64: one PCG
// iteration.
int64_t enqueue_body(gf_batch* b, cudaStream_t s) {
  const bool dist = batch_dist(b);
  const unsigned g = dist ? dist_grid(b) : 0u;
  int64_t L = 0;
  if (!b->mixed) {
    if (dist)
      for (int kind : kBodyFp64) L += launch_dist_fp64(kind, b->dtab, b->dact, g, s);
    else
      L += enqueue_kinds(b, kBodyFp64, s);
    return L;
  }
  auto one = [&](int kind) {
    L += dist ? launch_dist_mixed(kind, b->dtab, b->dact, g, s) : launch_batch(kind, b->dtab, b->blocks[kind], s, 0);
  };
  const int inner = b->tune.inner > 0 ? b->tune.inner : 8;
  one(kB_ir_inner_init);
  for (int j = 0; j < inner; ++j) {
    if (b->tune.solve_loop == GF_SOLVE_CG) {
      one(kB_ir_cg_spmv);
      one(kB_ir_cg_update);
    } else {
      one(kB_ir_spmv);
      one(kB_ir_update);
      one(kB_ir_p);
    }
  }
  one(kB_ir_apply);
  one(kB_ir_residual);
  return L;
}

bool batch_persist(const gf_batch* b) { return b->mixed && b->tune.solve_loop == GF_SOLVE_PERSISTENT; }

// the whole solve of every member as one cooperative launch (after the prefix)
int64_t enqueue_persist(gf_batch* b, cudaStream_t s) {
  const int n = launch_ir_persist(b->dtab, b->n, b->pctl, b->cap, 0, s);
  if (n < 0) return -1;
  if (cudaMemcpyAsync(b->h_pctl, b->pctl, 4 * sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return -1;
  return n;
}

int64_t enqueue_suffix(gf_batch* b, cudaStream_t s) {
  int64_t L = b->mixed ? enqueue_kinds(b, kSuffixMixed, s) : enqueue_kinds(b, kSuffixFp64, s);
  kb_collect<<<unsigned((b->n + 127) / 128), 128, 0, s>>>(b->dtab, b->mixed ? 1 : 0, b->dout);
  return L + 1;
}

#define GB_CK(call)                                                                         \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) {                                                                \
      set_last_error(std::string(#call) + ": " + cudaGetErrorString(e_));                  \
      return GF_CUDA_ERR;                                                                   \
    }                                                                                       \
  } while (0)

gf_status build_graph(gf_batch* b) {
  cudaStream_t s = b->stream;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  cudaGraph_t g;
  GB_CK(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle h{};
  if (!batch_persist(b)) GB_CK(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
  GB_CK(cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  b->prefix_kernels = enqueue_prefix(b, s);
  if (batch_persist(b)) {   // no WHILE node: the solve loop runs inside one cooperative launch
    const int64_t np = enqueue_persist(b, s);
    if (np < 0) {
      cudaGraph_t dead = nullptr;
      cudaStreamEndCapture(s, &dead);
      if (dead) cudaGraphDestroy(dead);
      cudaGraphDestroy(g);
      set_last_error("the cooperative launch of the persistent solve could not be captured");
      return GF_CUDA_ERR;
    }
    b->prefix_kernels += np;
    b->body_kernels = 0;
    GB_CK(cudaMemsetAsync(b->d_iter, 0, sizeof(int), s));
    b->suffix_kernels = enqueue_suffix(b, s);
    GB_CK(cudaMemcpyAsync(b->h_iter, b->d_iter, sizeof(int), cudaMemcpyDeviceToHost, s));
    GB_CK(cudaStreamEndCapture(s, &g));
    GB_CK(cudaGraphInstantiate(&b->exec, g, 0));
    b->graph = g;
    return GF_OK;
  }
  cudaStreamCaptureStatus cs;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* ed = nullptr;
  size_t nd = 0;
  GB_CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, nullptr, &deps, &ed, &nd));
  cudaGraphNodeParams p{};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t wn;
  GB_CK(cudaGraphAddNode(&wn, g, deps, ed, nd, &p));
  cudaGraph_t body = p.conditional.phGraph_out[0];
  GB_CK(cudaStreamBeginCaptureToGraph(b->body_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  b->body_kernels = enqueue_body(b, b->body_stream);
  kb_any_active<<<1, 256, 0, b->body_stream>>>(b->dtab, b->mixed ? 1 : 0, b->d_iter, b->cap, h,
                                                 batch_dist(b) ? b->dact : nullptr, int(dist_grid(b)));
  ++b->body_kernels;
  GB_CK(cudaStreamEndCapture(b->body_stream, &body));
  GB_CK(cudaStreamUpdateCaptureDependencies(s, &wn, nullptr, 1, cudaStreamSetCaptureDependencies));
  b->suffix_kernels = enqueue_suffix(b, s);
  GB_CK(cudaMemcpyAsync(b->h_iter, b->d_iter, sizeof(int), cudaMemcpyDeviceToHost, s));
  GB_CK(cudaStreamEndCapture(s, &g));
  GB_CK(cudaGraphInstantiate(&b->exec, g, 0));
  b->graph = g;
  return GF_OK;
}

// stage the per-mesh inputs, step scalars and launch shape; rebuild the graph if the shape changed
gf_status batch_prepare(gf_batch* b, double dt, const double* const* f_ext, const int32_t* const* pinned,
                        const int64_t* n_pinned, const double* const* pinned_vel, int32_t mem) {
  cudaStream_t s = b->stream;
  const cudaMemcpyKind kind = mem == GF_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  for (int k = 0; k < b->n; ++k) {
    gf_mesh* m = b->ms[k];
    const int64_t np = n_pinned ? n_pinned[k] : 0;
    const int32_t* pk = pinned ? pinned[k] : nullptr;
    if (np < 0 || np > m->dm.N || (np > 0 && !pk)) {
      set_last_error("batch step: bad pinned list of mesh " + std::to_string(k));
      return GF_BAD_ARG;
    }
    if (mem == GF_MEM_HOST)
      for (int64_t i = 0; i < np; ++i)
        if (pk[i] < 0 || pk[i] >= m->dm.N) {
          set_last_error("batch step: pinned node id out of range in mesh " + std::to_string(k));
          return GF_BAD_ARG;
        }
    const double* fk = f_ext ? f_ext[k] : nullptr;
    const double* vk = (pinned_vel && np > 0) ? pinned_vel[k] : nullptr;
    if (fk) GB_CK(cudaMemcpyAsync(m->dm.f_ext, fk, sizeof(double) * 3 * m->dm.N, kind, s));
    if (np > 0) GB_CK(cudaMemcpyAsync(m->dm.pin_ids, pk, sizeof(int32_t) * np, kind, s));
    if (vk) GB_CK(cudaMemcpyAsync(m->dm.pin_vel, vk, sizeof(double) * 3 * np, kind, s));
    b->htab->sp[k] = step_scalars(m->mt, dt, fk != nullptr, np, vk != nullptr);
  }
  std::vector<int32_t> shape;
  shape.reserve(size_t(kBKinds) * (b->n + 1));
  int64_t n_sum = 0;
  for (int k = 0; k < b->n; ++k) n_sum += b->htab->mesh[k].N;
  const int64_t budget = b->tune.grid_budget;
  for (int kind = 0; kind < kBKinds; ++kind) {
    // the solver-loop kernels are grid-stride: any per-mesh grid covers the mesh
    const bool loop_kind = kind == kB_ir_inner_init || kind == kB_ir_spmv || kind == kB_ir_update || kind == kB_ir_p ||
                           kind == kB_ir_apply || kind == kB_ir_residual || kind == kB_ir_cg_spmv ||
                           kind == kB_ir_cg_update || kind == kB_pcg_spmv || kind == kB_pcg_update || kind == kB_pcg_p;
    int32_t acc = 0;
    b->htab->off[kind][0] = 0;
    for (int k = 0; k < b->n; ++k) {
      int64_t blocks = launch_dims(kind, b->htab->mesh[k], b->htab->mt[k], b->htab->sp[k]).blocks;
      if (batch_persist(b)) blocks = persist_blocks(kind, unsigned(blocks));
      if (loop_kind && budget > 0 && blocks > 0 && !batch_dist(b))
        blocks = std::min(blocks, std::max<int64_t>(1, (budget * b->htab->mesh[k].N + n_sum - 1) / n_sum));
      acc += int32_t(blocks);
      b->htab->off[kind][k + 1] = acc;
    }
    b->blocks[kind] = unsigned(acc);
    shape.insert(shape.end(), b->htab->off[kind], b->htab->off[kind] + b->n + 1);
  }
  const size_t sp_off = offsetof(BatchTab, sp);
  GB_CK(cudaMemcpyAsync(reinterpret_cast<char*>(b->dtab) + sp_off, &b->htab->sp[0], sizeof(StepScalars) * b->n,
                        cudaMemcpyHostToDevice, s));
  if (shape != b->shape) {
    GB_CK(cudaMemcpyAsync(reinterpret_cast<char*>(b->dtab) + offsetof(BatchTab, off), &b->htab->off[0][0],
                          sizeof(b->htab->off), cudaMemcpyHostToDevice, s));
    b->shape = shape;
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
  }
  return GF_OK;
}

gf_status batch_run(gf_batch* b, gf_step_stats* stats) {
  cudaStream_t s = b->stream;
  int64_t L = 0;
  if (b->tune.graph) {
    if (!b->exec) {
      gf_status st = build_graph(b);
      if (st != GF_OK) return st;
    }
    GB_CK(cudaGraphLaunch(b->exec, s));
    GB_CK(cudaMemcpyAsync(b->hout, b->dout, sizeof(BatchOut) * b->n, cudaMemcpyDeviceToHost, s));
    GB_CK(cudaStreamSynchronize(s));
    L = b->prefix_kernels + b->suffix_kernels + int64_t(*b->h_iter) * b->body_kernels;
  } else if (batch_persist(b)) {
    L += enqueue_prefix(b, s);
    const int64_t np = enqueue_persist(b, s);
    if (np < 0) {
      set_last_error("the cooperative launch of the persistent solve was refused");
      return GF_CUDA_ERR;
    }
    L += np;
    L += enqueue_suffix(b, s);
    GB_CK(cudaGetLastError());
    GB_CK(cudaMemcpyAsync(b->hout, b->dout, sizeof(BatchOut) * b->n, cudaMemcpyDeviceToHost, s));
    GB_CK(cudaStreamSynchronize(s));
  } else {
    L += enqueue_prefix(b, s);
    const int chunk = b->tune.chunk > 0 ? b->tune.chunk : 8;
    int it = 0;
    for (;;) {
      for (int j = 0; j < chunk; ++j, ++it) {
        L += enqueue_body(b, s);
        if (batch_dist(b)) {   // the next iteration's work table
          kb_activate<<<1, 256, 0, s>>>(b->dtab, b->dact, b->mixed ? 1 : 0, int(dist_grid(b)));
          ++L;
        }
      }
      kb_collect<<<unsigned((b->n + 127) / 128), 128, 0, s>>>(b->dtab, b->mixed ? 1 : 0, b->dout);
      ++L;
      GB_CK(cudaGetLastError());
      GB_CK(cudaMemcpyAsync(b->hout, b->dout, sizeof(BatchOut) * b->n, cudaMemcpyDeviceToHost, s));
      GB_CK(cudaStreamSynchronize(s));
      bool active = false;
      for (int k = 0; k < b->n; ++k) active |= b->mixed ? !b->hout[k].ir.done : !b->hout[k].pcg.done;
      if (!active || it >= b->cap) break;
    }
    L += enqueue_suffix(b, s);
    GB_CK(cudaGetLastError());
    GB_CK(cudaMemcpyAsync(b->hout, b->dout, sizeof(BatchOut) * b->n, cudaMemcpyDeviceToHost, s));
    GB_CK(cudaStreamSynchronize(s));
  }
  b->launches += L;
  const bool timed_out = batch_persist(b) && b->h_pctl->error != 0;
  if (timed_out) {   // a phase cut short may leave reduction tickets counted: clear them
    for (int k = 0; k < b->n; ++k) GB_CK(cudaMemsetAsync(b->ms[k]->dm.tickets, 0, sizeof(unsigned) * kTickets, s));
    GB_CK(cudaStreamSynchronize(s));
  }
  gf_status first_bad = GF_OK;
  for (int k = 0; k < b->n; ++k) {
    const BatchOut& o = b->hout[k];
    gf_step_stats st{};
    if (b->mixed) {
      st.status = o.ir.status;
      if (st.status == GF_OK && !o.ir.done) st.status = GF_CG_MAXITER;
      st.cg_iters = o.ir.total_iters;
      st.refine_sweeps = o.ir.sweeps;
      st.rel_res = o.ir.bb > 0 ? std::sqrt(o.ir.rr / o.ir.bb) : 0.0;
    } else {
      st.status = o.pcg.status;
      if (st.status == GF_OK && !o.pcg.done) st.status = GF_CG_MAXITER;
      st.cg_iters = o.pcg.iters;
      st.rel_res = o.pcg.bb > 0 ? std::sqrt(o.pcg.true_rr / o.pcg.bb) : 0.0;
    }
    if (st.status == GF_OK && !std::isfinite(st.rel_res)) st.status = GF_NAN;
    if (timed_out) st.status = GF_TIMEOUT;
    if (o.cnt[3] != 0) st.status = GF_BAD_ARG;
    st.n_broken = int64_t(o.cnt[kCntBroken]);
    st.n_new_broken = int64_t(o.cnt[kCntNewBroken]);
    st.n_chi_zero = int64_t(o.cnt[kCntChiZero]);
    st.newton_iters = 1;
    if (stats) stats[k] = st;
    if (st.status != GF_OK && first_bad == GF_OK) first_bad = gf_status(st.status);
  }
  if (first_bad != GF_OK) set_last_error(std::string("batch step: ") + gf_status_string(first_bad));
  return first_bad;
}

}  // namespace

extern "C" {

gf_status gf_batch_create(gf_mesh* const* meshes, int32_t n, gf_batch** out) {
  if (!out || !meshes || n < 1 || n > kMaxBatch) {
    set_last_error("batch: need 1 <= n <= 256 meshes and an output pointer");
    return GF_BAD_ARG;
  }
  *out = nullptr;
  for (int k = 0; k < n; ++k)
    if (!meshes[k] || meshes[k]->device != meshes[0]->device || meshes[k]->mixed != meshes[0]->mixed) {
      set_last_error("batch: meshes must be non-NULL, on one device, with one precision");
      return GF_BAD_ARG;
    }
  for (int k = 0; k < n; ++k)
    if (meshes[k]->mt.energy != GF_ENERGY_STVK) {
      set_last_error("batches run the StVK energy (Eq. 37) only");
      return GF_UNSUPPORTED;
    }
  DeviceGuard guard(meshes[0]->device);
  gf_batch* b = new gf_batch();
  b->ms.assign(meshes, meshes + n);
  b->n = n;
  b->mixed = meshes[0]->mixed;
  b->device = meshes[0]->device;
  b->stream = meshes[0]->stream;
  b->tune.graph = 1;
  b->tune.chunk = 8;
  b->tune.solve_loop = b->mixed ? GF_SOLVE_CG : GF_SOLVE_KERNELS;   // as a member mesh's default
  auto fail = [&](const char* what) {
    set_last_error(std::string("batch create: ") + what);
    batch_free(b);
    delete b;
    return GF_CUDA_ERR;
  };
  if (cudaStreamCreateWithFlags(&b->body_stream, cudaStreamNonBlocking) != cudaSuccess) return fail("stream");
  if (cudaMallocHost(&b->htab, sizeof(BatchTab)) != cudaSuccess || cudaMalloc(&b->dtab, sizeof(BatchTab)) != cudaSuccess ||
      cudaMalloc(&b->dinit, sizeof(BatchInit) * n) != cudaSuccess ||
      cudaMallocHost(&b->hout, sizeof(BatchOut) * n) != cudaSuccess ||
      cudaMalloc(&b->dout, sizeof(BatchOut) * n) != cudaSuccess || cudaMalloc(&b->d_iter, sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&b->h_iter, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&b->pctl, sizeof(PersistCtl)) != cudaSuccess || cudaMallocHost(&b->h_pctl, sizeof(PersistCtl)) != cudaSuccess ||
      cudaMalloc(&b->dact, sizeof(BatchAct)) != cudaSuccess)
    return fail("allocation");
  std::memset(b->h_pctl, 0, sizeof(PersistCtl));
  new (b->htab) BatchTab();   // pinned host memory from cudaMallocHost: construct the table in place
  b->htab->n = n;
  std::vector<BatchInit> init(n);
  int maxit = 1;
  for (int k = 0; k < n; ++k) {
    gf_mesh* m = meshes[k];
    DevMesh d = m->dm;
    if (!(m->mt.radius > 0.0)) {
      d.sig_bar = d.sig_in;
      d.mx.sig_bar32 = d.mx.sig_in32;
    }
    b->htab->mesh[k] = d;
    b->htab->mt[k] = m->mt;
    BatchInit& bi = init[k];
    std::memset(&bi, 0, sizeof(bi));
    bi.pcg.tol2 = m->opt.cg_rtol * m->opt.cg_rtol;
    bi.pcg.maxit = m->opt.cg_maxit;
    bi.ir.tol2 = m->opt.cg_rtol * m->opt.cg_rtol;
    bi.ir.in_tol2 = m->in_rtol * m->in_rtol;
    bi.ir.maxit = m->opt.cg_maxit;
    bi.ir.in_maxit = 32;
    bi.ir.applied = 1;
    bi.ir.in_done = 1;
    maxit = std::max(maxit, m->opt.cg_maxit);
  }
  // body iterations: one PCG iteration (FP64) or one inner iteration / sweep transition (mixed)
  b->cap = 2 * maxit + 64;
  if (cudaMemcpy(b->dtab, b->htab, sizeof(BatchTab), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->dinit, init.data(), sizeof(BatchInit) * n, cudaMemcpyHostToDevice) != cudaSuccess)
    return fail("upload");
  *out = b;
  return GF_OK;
}

void gf_batch_destroy(gf_batch* b) {
  if (!b) return;
  DeviceGuard guard(b->device);
  cudaStreamSynchronize(b->stream);
  batch_free(b);
  delete b;
}

gf_status gf_batch_step(gf_batch* b, double dt, const double* const* f_ext, const int32_t* const* pinned,
                        const int64_t* n_pinned, const double* const* pinned_vel, int32_t mem, gf_step_stats* stats) {
  if (!b || !(dt > 0) || !std::isfinite(dt) || !valid_mem(mem)) {
    set_last_error("batch step: need a batch, dt > 0 and a memory kind");
    return GF_BAD_ARG;
  }
  for (gf_mesh* mm : b->ms)
    if (mm->newton_iters > 1) {
      set_last_error("batch step: members run one Newton iteration per step (gf_newton_set 1)");
      return GF_UNSUPPORTED;
    }
  DeviceGuard guard(b->device);
  Nvtx range("gf_batch_step");
  gf_status st = batch_prepare(b, dt, f_ext, pinned, n_pinned, pinned_vel, mem);
  if (st != GF_OK) return st;
  return batch_run(b, stats);
}

gf_status gf_batch_tuning_set(gf_batch* b, const gf_batch_tuning* t) {
  if (!b || !t || (t->graph != 0 && t->graph != 1) || t->chunk < 0 || t->grid_budget < 0 || t->inner < 0 ||
      t->inner > 64 ||
      (t->solve_loop != GF_SOLVE_PERSISTENT && t->solve_loop != GF_SOLVE_KERNELS &&
       t->solve_loop != GF_SOLVE_DISTRIBUTED && t->solve_loop != GF_SOLVE_CG)) {
    set_last_error("batch tuning: graph must be 0 or 1, chunk >= 0, grid_budget >= 0, 0 <= inner <= 64, "
                   "solve_loop GF_SOLVE_KERNELS, GF_SOLVE_PERSISTENT, GF_SOLVE_CG or GF_SOLVE_DISTRIBUTED");
    return GF_BAD_ARG;
  }
  if (t->solve_loop == GF_SOLVE_CG && !b->mixed) {
    set_last_error("batch tuning: GF_SOLVE_CG is built for GF_MIXED batches");
    return GF_UNSUPPORTED;
  }
  const bool rebuild = t->solve_loop != b->tune.solve_loop || t->inner != b->tune.inner;
  b->tune = *t;
  if (rebuild && b->exec) {   // the captured graph holds the other solve form
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  return GF_OK;
}

gf_status gf_batch_tuning_get(const gf_batch* b, gf_batch_tuning* t) {
  if (!b || !t) return GF_BAD_ARG;
  *t = b->tune;
  return GF_OK;
}

int64_t gf_batch_launch_count(const gf_batch* b) { return b ? b->launches : 0; }

gf_status gf_batch_autotune(gf_batch* b, double dt, const double* const* f_ext, const int32_t* const* pinned,
                            const int64_t* n_pinned, const double* const* pinned_vel, int32_t mem, int32_t trial_steps,
                            gf_batch_tuning* best, double* best_ms) {
  if (!b || trial_steps < 1) {
    set_last_error("autotune: need a batch and trial_steps >= 1");
    return GF_BAD_ARG;
  }
  DeviceGuard guard(b->device);
  cudaStream_t s = b->stream;
  // save every mesh's state (x, v, labels, chi, FP32 copies) on the device
  struct Saved {
    void* p;
    const void* src;
    size_t bytes;
  };
  std::vector<Saved> saved;
  auto keep = [&](const void* src, size_t bytes) -> gf_status {
    void* p = nullptr;
    if (bytes == 0) return GF_OK;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      set_last_error("autotune: cannot save state");
      return GF_OOM;
    }
    saved.push_back({p, src, bytes});
    return cudaMemcpyAsync(p, src, bytes, cudaMemcpyDeviceToDevice, s) == cudaSuccess ? GF_OK : GF_CUDA_ERR;
  };
  gf_status st = GF_OK;
  for (int k = 0; k < b->n && st == GF_OK; ++k) {
    const DevMesh& d = b->ms[k]->dm;
    if ((st = keep(d.x, sizeof(double) * 3 * d.N)) || (st = keep(d.v, sizeof(double) * 3 * d.N)) ||
        (st = keep(d.labels, d.NE)) || (st = keep(d.chi, sizeof(double) * d.T)))
      break;
    if (b->mixed && ((st = keep(d.mx.u32, sizeof(float) * 3 * d.N)) || (st = keep(d.mx.v32, sizeof(float) * 3 * d.N)) ||
                     (st = keep(d.mx.chi32, sizeof(float) * d.T))))
      break;
  }
  auto restore = [&]() {
    for (auto& sv : saved) cudaMemcpyAsync(const_cast<void*>(sv.src), sv.p, sv.bytes, cudaMemcpyDeviceToDevice, s);
    cudaStreamSynchronize(s);
  };
  const gf_batch_tuning orig = b->tune;
  std::vector<gf_batch_tuning> cands;
  {
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    const int wave = 4 * sms;   // one wave of a loop kernel at 4 CTAs per SM
    for (int budget : {0, wave, 2 * wave, 4 * wave}) {
      gf_batch_tuning t{};
      t.graph = 1;
      t.chunk = 8;
      t.grid_budget = budget;
      t.solve_loop = GF_SOLVE_KERNELS;
      cands.push_back(t);
      if (budget > 2 * wave) continue;
      for (int c : {2, 8}) {
        t.graph = 0;
        t.chunk = c;
        cands.push_back(t);
      }
    }
    if (b->mixed) {   // the persistent solve: every member's own blocks, or a budget of one or two waves
      for (int budget : {0, wave, 2 * wave}) {
        gf_batch_tuning t{};
        t.graph = 1;
        t.chunk = 8;
        t.grid_budget = budget;
        t.solve_loop = GF_SOLVE_PERSISTENT;
        cands.push_back(t);
      }
      // the two-kernel inner form, and both forms with shorter and longer passes
      // at budgets of two and four waves
      for (int budget : {0, wave, 2 * wave, 4 * wave}) {
        gf_batch_tuning t{};
        t.graph = 1;
        t.chunk = 8;
        t.grid_budget = budget;
        t.solve_loop = GF_SOLVE_CG;
        cands.push_back(t);
      }
      for (int budget : {2 * wave, 4 * wave})
        for (int form : {GF_SOLVE_KERNELS, GF_SOLVE_CG})
          for (int inner : {2, 4, 16}) {
            gf_batch_tuning t{};
            t.graph = 1;
            t.chunk = 8;
            t.grid_budget = budget;
            t.solve_loop = form;
            t.inner = inner;
            cands.push_back(t);
          }
    }
    for (int g : {wave / 2, wave, 2 * wave, 4 * wave}) {   // the distributed loop: its launch grid
      gf_batch_tuning t{};
      t.graph = 1;
      t.chunk = 8;
      t.grid_budget = g;
      t.solve_loop = GF_SOLVE_DISTRIBUTED;
      cands.push_back(t);
    }
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // ms per step of candidate ci: one untimed step (graph build, caches), then
  // the timed trial; the state is put back after each
  auto trial = [&](size_t ci) -> double {
    b->tune = cands[ci];
    st = gf_batch_step(b, dt, f_ext, pinned, n_pinned, pinned_vel, mem, nullptr);
    restore();
    if (st != GF_OK) return 1e300;
    cudaEventRecord(e0, s);
    for (int r = 0; r < trial_steps && st == GF_OK; ++r)
      st = gf_batch_step(b, dt, f_ext, pinned, n_pinned, pinned_vel, mem, nullptr);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    restore();
    return st == GF_OK ? double(ms) / trial_steps : 1e300;
  };
  const std::pair<size_t, double> pick = pick_fastest(cands.size(), trial, st);
  const gf_batch_tuning best_c = pick.first < cands.size() ? cands[pick.first] : orig;
  const double best_t = pick.second;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (auto& sv : saved) cudaFree(sv.p);
  b->tune = st == GF_OK ? best_c : orig;
  if (best) *best = b->tune;
  if (best_ms) *best_ms = best_t;
  return st;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Learned warm start and block preconditioner
// ---------------------------------------------------------------------------

struct gf_gnn {
  gf_mesh* mesh = nullptr;       // NULL once the mesh is destroyed
  int device = 0;
  std::vector<void*> blocks;
  GnnDev g;
  int adam_t = 0;
  double* stage_b = nullptr;     // [3N] staged right-hand side
  double* stage_t = nullptr;     // [3N] staged target
  double* loss_hist = nullptr;   // [kGnnMaxIters]
};

namespace {

constexpr int kGnnMaxIters = 1024;

void gnn_free(gf_gnn* g) {
  for (void* p : g->blocks) cudaFree(p);
  g->blocks.clear();
}

template <class T>
gf_status gnn_alloc(gf_gnn* g, size_t n, T** out) {
  void* p = nullptr;
  const size_t bytes = std::max<size_t>(256, (n * sizeof(T) + 255) & ~size_t(255));
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_last_error("network buffers: cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    return e == cudaErrorMemoryAllocation ? GF_OOM : GF_CUDA_ERR;
  }
  g->blocks.push_back(p);
  *out = static_cast<T*>(p);
  return GF_OK;
}

template <class T>
gf_status gnn_upload(gf_gnn* g, const std::vector<T>& h, const T** out, cudaStream_t s) {
  T* p = nullptr;
  gf_status st = gnn_alloc(g, h.size(), &p);
  if (st != GF_OK) return st;
  if (!h.empty()) GF_CK(cudaMemcpyAsync(p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, s));
  *out = p;
  return GF_OK;
}

int64_t gnn_param_offsets(int64_t (&off)[kGnnTensors]) {
  int64_t sz[kGnnTensors];
  sz[kPW0] = kNin * kHid;
  sz[kPb0] = kHid;
  for (int l = 0; l < 3; ++l) {
    sz[kPWa + 5 * l] = kHid * kHid;
    sz[kPWe + 5 * l] = kEin * kHid;
    sz[kPbm + 5 * l] = kHid;
    sz[kPWu + 5 * l] = 2 * kHid * kHid;
    sz[kPbu + 5 * l] = kHid;
  }
  sz[kPWd] = kHid * kNout;
  sz[kPbd] = kNout;
  int64_t o = 0;
  for (int k = 0; k < kGnnTensors; ++k) {
    off[k] = o;
    o += sz[k];
  }
  return o;
}

gf_status gnn_check(gf_gnn* g) {
  if (!g || !g->mesh) {
    set_last_error(g ? "the network's mesh was destroyed" : "NULL network");
    return GF_BAD_ARG;
  }
  if (!g->mesh->assembled) {
    set_last_error("the mesh has no assembled system yet: call gf_step first");
    return GF_BAD_ARG;
  }
  return GF_OK;
}

// b (host or device) -> device pointer
gf_status gnn_stage(gf_gnn* g, const double* src, int32_t mem, double* stage, const double** out) {
  if (mem == GF_MEM_DEVICE) {
    *out = src;
    return GF_OK;
  }
  GF_CK(cudaMemcpyAsync(stage, src, sizeof(double) * 3 * g->g.N, cudaMemcpyHostToDevice, g->mesh->stream));
  *out = stage;
  return GF_OK;
}

// network right-hand side b - A w (w = pinned values, previous solution on free
// nodes), forward pass, start and blocks into the mesh
int64_t gnn_step_start(gf_gnn* g, const DevMesh& d, int flags, cudaStream_t s) {
  int64_t L = gnn_pair(d, g->g.xprev, g->stage_b, nullptr, s);
  L += gnn_forward(g->g, d, g->stage_b, s);
  L += gnn_apply_inference(g->g, d, flags, s);
  return L;
}

cudaError_t gnn_keep_previous(gf_gnn* g, const DevMesh& d, cudaStream_t s) {
  return cudaMemcpyAsync(g->g.xprev, d.dv, sizeof(double) * 3 * d.N, cudaMemcpyDeviceToDevice, s);
}

// the mesh counter of tensor-core waits that gave up: cleared before a network
// call, read after it (the stream is synchronised by the caller)
cudaError_t gnn_tc_clear(gf_gnn* g) { return cudaMemsetAsync(g->g.err, 0, sizeof(unsigned long long), g->mesh->stream); }
gf_status gnn_tc_status(gf_gnn* g) {
  unsigned long long n = 0;
  GF_CK(cudaMemcpy(&n, g->g.err, sizeof(n), cudaMemcpyDeviceToHost));
  if (n != 0) {
    set_last_error("a tensor-core wait of the network gave up (device timeout)");
    return GF_TIMEOUT;
  }
  return GF_OK;
}

}  // namespace

extern "C" {

int64_t gf_gnn_n_params(void) {
  int64_t off[kGnnTensors];
  return gnn_param_offsets(off);
}

gf_status gf_gnn_create(gf_mesh* mesh, gf_gnn** out) {
  if (!out || !mesh) {
    set_last_error("mesh and out must not be NULL");
    return GF_BAD_ARG;
  }
  *out = nullptr;
  if (mesh->mixed) {
    set_last_error("the learned preconditioner runs with GF_FP64 meshes only");
    return GF_UNSUPPORTED;
  }
  if (mesh->gnn) {
    set_last_error("the mesh already has a network");
    return GF_BAD_ARG;
  }
  DeviceGuard guard(mesh->device);
  cudaStream_t s = mesh->stream;
  const HostMesh& hm = mesh->hm;
  const int64_t N = hm.n_nodes;
  // graph: the block pattern without its diagonal (rows sorted)
  std::vector<int32_t> rp(N + 1, 0), col, dst, amap;
  col.reserve(hm.col.size());
  for (int64_t i = 0; i < N; ++i) {
    for (int32_t p = hm.row_ptr[i]; p < hm.row_ptr[i + 1]; ++p) {
      if (hm.col[p] == i) continue;
      col.push_back(hm.col[p]);
      dst.push_back(int32_t(i));
      amap.push_back(p);
    }
    rp[i + 1] = int32_t(col.size());
  }
  const int64_t E = int64_t(col.size());
  std::vector<int32_t> tpos(E);
  for (int64_t q = 0; q < E; ++q) {
    const int32_t i = dst[q], j = col[q];
    const int32_t* b = col.data() + rp[j];
    const int32_t* e = col.data() + rp[j + 1];
    const int32_t* it = std::lower_bound(b, e, i);
    if (it == e || *it != i) {
      set_last_error("block pattern is not symmetric");
      return GF_BAD_ARG;
    }
    tpos[q] = int32_t(it - col.data());
  }
  // static inputs
  const std::vector<double>& X = mesh->X0;
  double hsum = 0.0;
  for (int64_t k = 0; k < hm.n_edges; ++k) {
    const int32_t a = hm.edges[2 * k], b = hm.edges[2 * k + 1];
    double l2 = 0.0;
    for (int c = 0; c < 3; ++c) l2 += (X[3 * b + c] - X[3 * a + c]) * (X[3 * b + c] - X[3 * a + c]);
    hsum += std::sqrt(l2);
  }
  const double hbar = hm.n_edges > 0 ? hsum / double(hm.n_edges) : 1.0;
  std::vector<float> relpos(3 * E), nstat(2 * N);
  for (int64_t q = 0; q < E; ++q)
    for (int c = 0; c < 3; ++c) relpos[3 * q + c] = float((X[3 * col[q] + c] - X[3 * dst[q] + c]) / hbar);
  double msum = 0.0;
  for (int64_t i = 0; i < N; ++i) msum += hm.mass[i];
  const double mmean = msum / double(N);
  for (int64_t i = 0; i < N; ++i) {
    nstat[2 * i] = float(std::log(hm.mass[i] / mmean));
    nstat[2 * i + 1] = float(rp[i + 1] - rp[i]) / 16.f;
  }

  // edge-message tiles of the tensor-core kernel: runs of whole destination
  // nodes with at most kEdgeTileRows messages and nodes each (none when a node
  // alone has more messages: the FP32 kernel then serves every layer)
  // (each tile: first node, node count, first message, message count)
  std::vector<int32_t> etile;
  for (int64_t i = 0; i < N;) {
    int64_t j = i;
    while (j < N && j - i < kEdgeTileRows && rp[j + 1] - rp[i] <= kEdgeTileRows) ++j;
    if (j == i) {
      etile.clear();
      break;
    }
    etile.insert(etile.end(), {int32_t(i), int32_t(j - i), rp[i], rp[j] - rp[i]});
    i = j;
  }

  gf_gnn* g = new gf_gnn();
  g->mesh = mesh;
  g->device = mesh->device;
  GnnDev& G = g->g;
  G.N = N;
  G.E = E;
  G.n_etiles = int64_t(etile.size()) / 4;
  G.err = mesh->dm.counters + kCntTcTimeout;
  G.P = gnn_param_offsets(G.off);
  auto fail = [&](gf_status st) {
    cudaStreamSynchronize(s);
    gnn_free(g);
    delete g;
    return st;
  };
  gf_status st = GF_OK;
#define GNN_TRY(call)            \
  do {                           \
    st = (call);                 \
    if (st != GF_OK) return fail(st); \
  } while (0)
  GNN_TRY(gnn_upload(g, rp, &G.row_ptr, s));
  GNN_TRY(gnn_upload(g, col, &G.col, s));
  GNN_TRY(gnn_upload(g, dst, &G.dst, s));
  GNN_TRY(gnn_upload(g, amap, &G.amap, s));
  GNN_TRY(gnn_upload(g, tpos, &G.tpos, s));
  GNN_TRY(gnn_upload(g, relpos, &G.relpos, s));
  GNN_TRY(gnn_upload(g, nstat, &G.nstat, s));
  GNN_TRY(gnn_upload(g, etile, reinterpret_cast<const int32_t**>(&G.etile), s));
  const size_t NH = size_t(N) * kHid;
  GNN_TRY(gnn_alloc(g, size_t(E) * kEin, &G.efeat));
  GNN_TRY(gnn_alloc(g, size_t(N), &G.T));
  GNN_TRY(gnn_alloc(g, size_t(N) * 6, &G.C));
  GNN_TRY(gnn_alloc(g, size_t(N) * 3, &G.Y));
  GNN_TRY(gnn_alloc(g, size_t(N) * 3, &G.B));
  GNN_TRY(gnn_alloc(g, size_t(N), &G.freem));
  GNN_TRY(gnn_alloc(g, size_t(N) * kNin, &G.X0));
  GNN_TRY(gnn_alloc(g, NH, &G.Z0));
  GNN_TRY(gnn_alloc(g, 4 * NH, &G.H));
  GNN_TRY(gnn_alloc(g, 3 * NH, &G.Aa));
  GNN_TRY(gnn_alloc(g, 3 * NH, &G.M));
  GNN_TRY(gnn_alloc(g, 3 * NH, &G.ZU));
  GNN_TRY(gnn_alloc(g, size_t(N) * 16, &G.OUT));
  GNN_TRY(gnn_alloc(g, size_t(N) * 9, &G.Po));
  GNN_TRY(gnn_alloc(g, size_t(N) * 3, &G.xo));
  GNN_TRY(gnn_alloc(g, size_t(N) * 3, &G.xprev));
  GNN_TRY(gnn_alloc(g, size_t(N) * 3, &G.ebuf));
  GNN_TRY(gnn_alloc(g, size_t(N) * 3, &G.qbuf));
  GNN_TRY(gnn_alloc(g, 1, &G.dscal));
  GNN_TRY(gnn_alloc(g, size_t(N) * 16, &G.dOUT));
  GNN_TRY(gnn_alloc(g, NH, &G.dH));
  GNN_TRY(gnn_alloc(g, NH, &G.dZ));
  GNN_TRY(gnn_alloc(g, NH, &G.dM));
  GNN_TRY(gnn_alloc(g, NH, &G.dA));
  G.part_stride = (2 * kHid + 1) * kHid;
  G.n_gpart = gnn_max_parts();
  GNN_TRY(gnn_alloc(g, size_t(G.n_gpart) * G.part_stride, &G.gpart));
  GNN_TRY(gnn_alloc(g, size_t(G.P), &G.grad));
  GNN_TRY(gnn_alloc(g, size_t(G.P), &G.w32));
  GNN_TRY(gnn_alloc(g, size_t(G.P), &G.w16));
  GNN_TRY(gnn_alloc(g, size_t(G.P), &G.m1));
  GNN_TRY(gnn_alloc(g, size_t(G.P), &G.m2));
  GNN_TRY(gnn_alloc(g, 4, &G.scal));
  GNN_TRY(gnn_alloc(g, kGnnMaxIters, &g->loss_hist));
  G.loss = g->loss_hist;
  GNN_TRY(gnn_alloc(g, size_t(3) * gnn_reduce_slots(), &G.red));
  GNN_TRY(gnn_alloc(g, 4, &G.ticket));
  GNN_TRY(gnn_alloc(g, size_t(N) * 3, &g->stage_b));
  GNN_TRY(gnn_alloc(g, size_t(N) * 3, &g->stage_t));
#undef GNN_TRY
  cudaError_t e = cudaSuccess;
  e = e ? e : cudaMemsetAsync(G.ticket, 0, 4 * sizeof(unsigned), s);
  e = e ? e : cudaMemsetAsync(G.xprev, 0, sizeof(double) * 3 * N, s);
  e = e ? e : cudaMemsetAsync(G.w32, 0, sizeof(float) * G.P, s);
  e = e ? e : cudaMemsetAsync(G.w16, 0, sizeof(__nv_bfloat16) * G.P, s);
  e = e ? e : cudaMemsetAsync(G.m1, 0, sizeof(float) * G.P, s);
  e = e ? e : cudaMemsetAsync(G.m2, 0, sizeof(float) * G.P, s);
  e = e ? e : cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_last_error(std::string("network setup: ") + cudaGetErrorString(e));
    return fail(GF_CUDA_ERR);
  }
  mesh->gnn = g;
  mesh->gnn_flags = 0;
  *out = g;
  return GF_OK;
}

void gf_gnn_destroy(gf_gnn* g) {
  if (!g) return;
  DeviceGuard guard(g->device);
  if (g->mesh) {
    cudaStreamSynchronize(g->mesh->stream);
    if (g->mesh->gnn == g) {
      g->mesh->gnn = nullptr;
      g->mesh->gnn_flags = 0;
    }
  } else {
    cudaDeviceSynchronize();
  }
  gnn_free(g);
  delete g;
}

gf_status gf_gnn_params_set(gf_gnn* g, const float* w, int64_t n) {
  if (!g || !g->mesh || !w || n != g->g.P) {
    set_last_error("params_set: need the network, a host array and n == gf_gnn_n_params()");
    return GF_BAD_ARG;
  }
  DeviceGuard guard(g->mesh->device);
  cudaStream_t s = g->mesh->stream;
  GF_CK(cudaMemcpyAsync(g->g.w32, w, sizeof(float) * n, cudaMemcpyHostToDevice, s));
  GF_CK(cudaMemsetAsync(g->g.m1, 0, sizeof(float) * n, s));
  GF_CK(cudaMemsetAsync(g->g.m2, 0, sizeof(float) * n, s));
  g->mesh->launches += gnn_refresh_bf16(g->g, s);
  GF_CK(cudaGetLastError());
  GF_CK(cudaStreamSynchronize(s));
  g->adam_t = 0;
  return GF_OK;
}

gf_status gf_gnn_params_get(gf_gnn* g, float* w, int64_t n) {
  if (!g || !g->mesh || !w || n != g->g.P) {
    set_last_error("params_get: need the network, a host array and n == gf_gnn_n_params()");
    return GF_BAD_ARG;
  }
  DeviceGuard guard(g->mesh->device);
  GF_CK(cudaMemcpyAsync(w, g->g.w32, sizeof(float) * n, cudaMemcpyDeviceToHost, g->mesh->stream));
  GF_CK(cudaStreamSynchronize(g->mesh->stream));
  return GF_OK;
}

gf_status gf_gnn_forward(gf_gnn* g, const double* b, int32_t mem, float* out, float* P, float* x0, float* node_in,
                         float* edge_in) {
  gf_status st = gnn_check(g);
  if (st != GF_OK) return st;
  if (!b || !valid_mem(mem)) {
    set_last_error("forward: b must not be NULL, mem GF_MEM_HOST or GF_MEM_DEVICE");
    return GF_BAD_ARG;
  }
  DeviceGuard guard(g->mesh->device);
  cudaStream_t s = g->mesh->stream;
  const GnnDev& G = g->g;
  const double* bd = nullptr;
  if ((st = gnn_stage(g, b, mem, g->stage_b, &bd)) != GF_OK) return st;
  GF_CK(gnn_tc_clear(g));
  int64_t L = gnn_forward(G, g->mesh->dm, bd, s);
  L += gnn_apply_export(G, s);
  g->mesh->launches += L;
  GF_CK(cudaGetLastError());
  std::vector<float> o16;
  if (out) {
    o16.resize(size_t(G.N) * 16);
    GF_CK(cudaMemcpyAsync(o16.data(), G.OUT, sizeof(float) * o16.size(), cudaMemcpyDeviceToHost, s));
  }
  if (P) GF_CK(cudaMemcpyAsync(P, G.Po, sizeof(float) * 9 * G.N, cudaMemcpyDeviceToHost, s));
  if (x0) GF_CK(cudaMemcpyAsync(x0, G.xo, sizeof(float) * 3 * G.N, cudaMemcpyDeviceToHost, s));
  if (node_in) GF_CK(cudaMemcpyAsync(node_in, G.X0, sizeof(float) * kNin * G.N, cudaMemcpyDeviceToHost, s));
  if (edge_in && G.E > 0)
    GF_CK(cudaMemcpyAsync(edge_in, G.efeat, sizeof(float) * kEin * G.E, cudaMemcpyDeviceToHost, s));
  GF_CK(cudaStreamSynchronize(s));
  if ((st = gnn_tc_status(g)) != GF_OK) return st;
  if (out)
    for (int64_t i = 0; i < G.N; ++i)
      for (int k = 0; k < kNout; ++k) out[kNout * i + k] = o16[16 * i + k];
  return GF_OK;
}

gf_status gf_gnn_loss_grad(gf_gnn* g, const double* b, const double* target, int32_t mem, double* loss,
                           float* grad) {
  gf_status st = gnn_check(g);
  if (st != GF_OK) return st;
  if (!b || !target || !valid_mem(mem)) {
    set_last_error("loss_grad: b and target must not be NULL, mem GF_MEM_HOST or GF_MEM_DEVICE");
    return GF_BAD_ARG;
  }
  DeviceGuard guard(g->mesh->device);
  cudaStream_t s = g->mesh->stream;
  const GnnDev& G = g->g;
  const double *bd = nullptr, *td = nullptr;
  if ((st = gnn_stage(g, b, mem, g->stage_b, &bd)) != GF_OK) return st;
  if ((st = gnn_stage(g, target, mem, g->stage_t, &td)) != GF_OK) return st;
  GF_CK(cudaMemsetAsync(G.grad, 0, sizeof(float) * G.P, s));
  GF_CK(cudaMemsetAsync(G.loss, 0, sizeof(double), s));
  GF_CK(gnn_tc_clear(g));
  int64_t L = gnn_forward(G, g->mesh->dm, bd, s);
  L += gnn_backward_pair(G, g->mesh->dm, td, s);
  g->mesh->launches += L;
  GF_CK(cudaGetLastError());
  double h_loss = 0.0;
  GF_CK(cudaMemcpyAsync(&h_loss, G.loss, sizeof(double), cudaMemcpyDeviceToHost, s));
  if (grad) GF_CK(cudaMemcpyAsync(grad, G.grad, sizeof(float) * G.P, cudaMemcpyDeviceToHost, s));
  GF_CK(cudaStreamSynchronize(s));
  if ((st = gnn_tc_status(g)) != GF_OK) return st;
  if (loss) *loss = h_loss;
  return GF_OK;
}

gf_status gf_gnn_train(gf_gnn* g, int32_t iters, float lr, double* loss_first, double* loss_last) {
  gf_status st = gnn_check(g);
  if (st != GF_OK) return st;
  if (iters < 1 || iters > kGnnMaxIters || !(lr > 0.f) || !std::isfinite(lr)) {
    set_last_error("train: need 1 <= iters <= 1024 and lr > 0");
    return GF_BAD_ARG;
  }
  DeviceGuard guard(g->mesh->device);
  cudaStream_t s = g->mesh->stream;
  const DevMesh& d = g->mesh->dm;
  int64_t L = gnn_pair(d, g->g.xprev, g->stage_b, g->stage_t, s);
  GF_CK(cudaMemsetAsync(g->loss_hist, 0, sizeof(double) * iters, s));
  GF_CK(gnn_tc_clear(g));
  for (int k = 0; k < iters; ++k) {
    GnnDev G = g->g;
    G.loss = g->loss_hist + k;
    GF_CK(cudaMemsetAsync(G.grad, 0, sizeof(float) * G.P, s));
    L += gnn_forward(G, d, g->stage_b, s);
    L += gnn_backward_pair(G, d, g->stage_t, s);
    L += gnn_adam(G, 1.f, lr, ++g->adam_t, s);
  }
  g->mesh->launches += L;
  GF_CK(cudaGetLastError());
  double h[2] = {0.0, 0.0};
  GF_CK(cudaMemcpyAsync(&h[0], g->loss_hist, sizeof(double), cudaMemcpyDeviceToHost, s));
  GF_CK(cudaMemcpyAsync(&h[1], g->loss_hist + (iters - 1), sizeof(double), cudaMemcpyDeviceToHost, s));
  GF_CK(cudaStreamSynchronize(s));
  if ((st = gnn_tc_status(g)) != GF_OK) return st;
  if (loss_first) *loss_first = h[0];
  if (loss_last) *loss_last = h[1];
  return GF_OK;
}

gf_status gf_gnn_pair_get(gf_gnn* g, double* b, double* target) {
  gf_status st = gnn_check(g);
  if (st != GF_OK) return st;
  if (!b || !target) {
    set_last_error("pair_get: b and target must not be NULL");
    return GF_BAD_ARG;
  }
  DeviceGuard guard(g->mesh->device);
  cudaStream_t s = g->mesh->stream;
  g->mesh->launches += gnn_pair(g->mesh->dm, g->g.xprev, g->stage_b, g->stage_t, s);
  GF_CK(cudaGetLastError());
  GF_CK(cudaMemcpyAsync(b, g->stage_b, sizeof(double) * 3 * g->g.N, cudaMemcpyDeviceToHost, s));
  GF_CK(cudaMemcpyAsync(target, g->stage_t, sizeof(double) * 3 * g->g.N, cudaMemcpyDeviceToHost, s));
  GF_CK(cudaStreamSynchronize(s));
  return GF_OK;
}

gf_status gf_gnn_kernels_set(gf_gnn* g, int32_t kernels) {
  if (!g || (kernels != GF_GNN_TENSOR_CORES && kernels != GF_GNN_FP32_FMA)) {
    set_last_error("kernels_set: need the network and GF_GNN_TENSOR_CORES or GF_GNN_FP32_FMA");
    return GF_BAD_ARG;
  }
  g->g.use_tc = kernels == GF_GNN_TENSOR_CORES ? 1 : 0;
  return GF_OK;
}

gf_status gf_gnn_attach(gf_mesh* mesh, gf_gnn* g, int32_t flags) {
  if (!mesh || !g || g->mesh != mesh || (flags & ~(GF_GNN_START | GF_GNN_PRECOND))) {
    set_last_error("attach: the network must belong to this mesh; flags GF_GNN_START | GF_GNN_PRECOND or 0");
    return GF_BAD_ARG;
  }
  mesh->gnn_flags = flags;
  return GF_OK;
}

}  // extern "C"

void gnn_orphan(gf_gnn* g) { g->mesh = nullptr; }
