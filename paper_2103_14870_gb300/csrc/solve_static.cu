// Allocation-free block-Jacobi PCG on a caller-owned block-CSR system.
//
// Some callers cannot allocate device memory while they solve: cudaMalloc and
// cudaFree can synchronise the whole device and stall work on other streams,
// and some host programs hand all device memory to one pool up front and allow
// no allocation afterwards.  gf_bsr_pcg_solve_static() serves them: its
// scratch vectors live in the file-scope array below, of a fixed maximum size,
// which every GPU that loads this library holds until the process exits.
//
// The array is shared by every call on a device and keeps the last call's
// contents; each call clears the parts that must start at zero (reduction
// tickets and solver scalars).  Calls whose work overlaps on the GPU (for
// example on two streams at once) race on the array: serialise them.
//
// Host code cannot use the array's name as a device address (it names a host
// stand-in), so the device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, on the first call there.
// That first call on a device should therefore come before any stream capture.
#include <cmath>
#include <mutex>
#include <string>

#include "gf_internal.h"

namespace gf {
namespace {

constexpr int64_t kStaticMaxRows = 32768;   // block rows (3 unknowns each)
constexpr int kSThreads = 256;
constexpr int kSMaxGrid = int((kStaticMaxRows + kSThreads - 1) / kSThreads);
constexpr int kMaxDevices = 64;

struct StaticState {
  double bb, rz, pq, rr, alpha, beta, tol2, true_rr;
  double bad_cols, bad_diag;   // column ids out of range; free rows without an invertible diagonal block
  int32_t iters, maxit, done, status;
  unsigned tickets[4];
};

// scratch layout in doubles: r, z, p, q [3 * rows each], block-Jacobi [9 * rows],
// reduction partials [5 * grid] (at most 5 values per CTA), solver state
constexpr int64_t kOffR = 0;
constexpr int64_t kOffZ = kOffR + 3 * kStaticMaxRows;
constexpr int64_t kOffP = kOffZ + 3 * kStaticMaxRows;
constexpr int64_t kOffQ = kOffP + 3 * kStaticMaxRows;
constexpr int64_t kOffPinv = kOffQ + 3 * kStaticMaxRows;
constexpr int64_t kOffPart = kOffPinv + 9 * kStaticMaxRows;
constexpr int64_t kOffState = kOffPart + 5 * kSMaxGrid;
constexpr int64_t kScratchDoubles = kOffState + (sizeof(StaticState) + 7) / 8;

static __device__ __align__(256) double g_pcg_scratch[kScratchDoubles];

struct SView {
  const int32_t* row_ptr;
  const int32_t* col;
  const double* val;
  const double* b;
  double* x;
  const uint8_t* fixed;
  int64_t n;
  double *r, *z, *p, *q, *pinv, *part;
  StaticState* st;
};

__device__ __forceinline__ double swarp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// per-CTA partials, then the last CTA sums them in CTA order (no waiting)
template <int NV>
__device__ bool sreduce(double (&v)[NV], double* part, unsigned* ticket, double (&out)[NV]) {
  __shared__ double sh[NV][32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double t = swarp_sum(v[i]);
    if (lane == 0) sh[i][wid] = t;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double t = swarp_sum(lane < nw ? sh[i][lane] : 0.0);
      if (lane == 0) part[blockIdx.x * NV + i] = t;
    }
  }
  if (threadIdx.x == 0) {
    __threadfence();
    last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double t = 0.0;
    for (unsigned j = threadIdx.x; j < gridDim.x; j += blockDim.x) t += __ldcg(&part[j * NV + i]);
    t = swarp_sum(t);
    __syncthreads();
    if (lane == 0) sh[i][wid] = t;
    __syncthreads();
    if (wid == 0) {
      t = swarp_sum(lane < nw ? sh[i][lane] : 0.0);
      if (lane == 0) out[i] = t;
    }
  }
  if (threadIdx.x == 0) *ticket = 0u;
  return true;
}

__device__ __forceinline__ bool is_fixed(const SView& v, int64_t i) { return v.fixed && v.fixed[i]; }

// Free rows of x are not read: the solve starts from x = 0 there (written
// below), so the caller may pass uninitialised values.  r = t = b - A x_fixed
// on free rows; block-Jacobi inverses; z = P r; p = z.  Counts column ids out
// of range and free rows whose diagonal block is missing or not invertible.
__global__ void __launch_bounds__(kSThreads) ks_init(SView v) {
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};   // r.z, r.r, t.t, bad columns, bad diagonals
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < v.n; i += int64_t(gridDim.x) * blockDim.x) {
    double r[3] = {0, 0, 0}, z[3] = {0, 0, 0};
    if (!is_fixed(v, i)) {
      double t[3] = {v.b[3 * i], v.b[3 * i + 1], v.b[3 * i + 2]};
      const double* d = nullptr;
      for (int k = v.row_ptr[i]; k < v.row_ptr[i + 1]; ++k) {
        const int64_t j = v.col[k];
        if (j < 0 || j >= v.n) {
          acc[3] += 1.0;
          continue;
        }
        const double* a = v.val + 9 * int64_t(k);
        if (j == i) d = a;
        if (!is_fixed(v, j)) continue;   // free columns multiply the zero start
        const double x0 = v.x[3 * j], x1 = v.x[3 * j + 1], x2 = v.x[3 * j + 2];
        t[0] -= a[0] * x0 + a[1] * x1 + a[2] * x2;
        t[1] -= a[3] * x0 + a[4] * x1 + a[5] * x2;
        t[2] -= a[6] * x0 + a[7] * x1 + a[8] * x2;
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) r[c] = t[c];
      double inv[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
      bool ok = false;
      if (d) {
        const double c00 = d[4] * d[8] - d[5] * d[7], c01 = d[2] * d[7] - d[1] * d[8], c02 = d[1] * d[5] - d[2] * d[4];
        const double c10 = d[5] * d[6] - d[3] * d[8], c11 = d[0] * d[8] - d[2] * d[6], c12 = d[2] * d[3] - d[0] * d[5];
        const double c20 = d[3] * d[7] - d[4] * d[6], c21 = d[1] * d[6] - d[0] * d[7], c22 = d[0] * d[4] - d[1] * d[3];
        const double det = d[0] * c00 + d[1] * c10 + d[2] * c20;
        const double id = 1.0 / det;
        ok = det != 0.0 && isfinite(id);
        if (ok) {
          const double w[9] = {c00 * id, c01 * id, c02 * id, c10 * id, c11 * id, c12 * id, c20 * id, c21 * id, c22 * id};
#pragma unroll
          for (int k = 0; k < 9; ++k) inv[k] = w[k];
        }
      }
      if (!ok) acc[4] += 1.0;
#pragma unroll
      for (int k = 0; k < 9; ++k) v.pinv[9 * i + k] = inv[k];
#pragma unroll
      for (int c = 0; c < 3; ++c) z[c] = inv[3 * c] * r[0] + inv[3 * c + 1] * r[1] + inv[3 * c + 2] * r[2];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        acc[2] += t[c] * t[c];
        v.x[3 * i + c] = 0.0;
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      v.r[3 * i + c] = r[c];
      v.z[3 * i + c] = z[c];
      v.p[3 * i + c] = z[c];
      acc[0] += r[c] * z[c];
      acc[1] += r[c] * r[c];
    }
  }
  double out[5];
  if (sreduce<5>(acc, v.part, &v.st->tickets[0], out) && threadIdx.x == 0) {
    StaticState* s = v.st;
    s->rz = out[0];
    s->rr = out[1];
    s->bb = out[2];
    s->bad_cols = out[3];
    s->bad_diag = out[4];
    s->iters = 0;
    s->status = GF_OK;
    s->done = (out[1] == 0.0 || out[1] <= s->tol2 * out[2]) ? 1 : 0;
    if (!isfinite(out[1]) || !isfinite(out[2])) {
      s->status = GF_NAN;
      s->done = 1;
    }
    if (out[3] > 0.0 || out[4] > 0.0) {
      s->status = GF_BAD_ARG;
      s->done = 1;
    }
  }
}

__device__ __forceinline__ void srow(const SView& v, int64_t i, const double* x, double y[3]) {
  double y0 = 0, y1 = 0, y2 = 0;
  for (int k = v.row_ptr[i]; k < v.row_ptr[i + 1]; ++k) {
    const int64_t j = v.col[k];
    if (j < 0 || j >= v.n) continue;   // rejected in ks_init; never read out of range
    const double* a = v.val + 9 * int64_t(k);
    const double x0 = x[3 * j], x1 = x[3 * j + 1], x2 = x[3 * j + 2];
    y0 += a[0] * x0 + a[1] * x1 + a[2] * x2;
    y1 += a[3] * x0 + a[4] * x1 + a[5] * x2;
    y2 += a[6] * x0 + a[7] * x1 + a[8] * x2;
  }
  y[0] = y0;
  y[1] = y1;
  y[2] = y2;
}

__global__ void __launch_bounds__(kSThreads) ks_spmv(SView v) {
  if (v.st->done) return;
  double acc[1] = {0.0};
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < v.n; i += int64_t(gridDim.x) * blockDim.x) {
    double y[3];
    srow(v, i, v.p, y);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      v.q[3 * i + c] = y[c];
      acc[0] += v.p[3 * i + c] * y[c];
    }
  }
  double out[1];
  if (sreduce<1>(acc, v.part, &v.st->tickets[1], out) && threadIdx.x == 0) {
    StaticState* s = v.st;
    s->pq = out[0];
    if (!(out[0] > 0.0)) {
      s->status = isfinite(out[0]) ? GF_CG_BREAKDOWN : GF_NAN;
      s->done = 1;
    } else {
      s->alpha = s->rz / out[0];
    }
  }
}

__global__ void __launch_bounds__(kSThreads) ks_update(SView v) {
  if (v.st->done) return;
  const double alpha = v.st->alpha;
  double acc[2] = {0.0, 0.0};
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < v.n; i += int64_t(gridDim.x) * blockDim.x) {
    if (is_fixed(v, i)) continue;
    double r[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      v.x[3 * i + c] += alpha * v.p[3 * i + c];
      r[c] = v.r[3 * i + c] - alpha * v.q[3 * i + c];
      v.r[3 * i + c] = r[c];
    }
    const double* pi = v.pinv + 9 * i;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double z = pi[3 * c] * r[0] + pi[3 * c + 1] * r[1] + pi[3 * c + 2] * r[2];
      v.z[3 * i + c] = z;
      acc[0] += r[c] * z;
      acc[1] += r[c] * r[c];
    }
  }
  double out[2];
  if (sreduce<2>(acc, v.part, &v.st->tickets[2], out) && threadIdx.x == 0) {
    StaticState* s = v.st;
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

__global__ void __launch_bounds__(kSThreads) ks_p(SView v) {
  if (v.st->done) return;
  const double beta = v.st->beta;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < 3 * v.n; i += int64_t(gridDim.x) * blockDim.x)
    v.p[i] = v.z[i] + beta * v.p[i];
}

// ||b - A x||^2 over free rows (x complete)
__global__ void __launch_bounds__(kSThreads) ks_residual(SView v) {
  if (v.st->status == GF_BAD_ARG) return;
  double acc[1] = {0.0};
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < v.n; i += int64_t(gridDim.x) * blockDim.x) {
    if (is_fixed(v, i)) continue;
    double y[3];
    srow(v, i, v.x, y);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double r = v.b[3 * i + c] - y[c];
      acc[0] += r * r;
    }
  }
  double out[1];
  if (sreduce<1>(acc, v.part, &v.st->tickets[3], out) && threadIdx.x == 0) v.st->true_rr = out[0];
}

std::mutex g_sym_mutex;
double* g_sym_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
gf_status scratch_on_current_device(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_last_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    return GF_CUDA_ERR;
  }
  std::lock_guard<std::mutex> lock(g_sym_mutex);
  if (!g_sym_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_pcg_scratch);
    if (e != cudaSuccess || !p) {
      set_last_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return GF_CUDA_ERR;
    }
    g_sym_addr[dev] = static_cast<double*>(p);
  }
  *out = g_sym_addr[dev];
  return GF_OK;
}

#define GS_CK(call)                                                             \
  do {                                                                          \
    cudaError_t e_ = (call);                                                    \
    if (e_ != cudaSuccess) {                                                    \
      set_last_error(std::string(#call) + ": " + cudaGetErrorString(e_));      \
      return GF_CUDA_ERR;                                                       \
    }                                                                           \
  } while (0)

}  // namespace
}  // namespace gf

using namespace gf;

extern "C" gf_status gf_bsr_pcg_solve_static(const int32_t* row_ptr, const int32_t* col, const double* values,
                                             int64_t n_rows, const double* b, double* x, const uint8_t* fixed,
                                             double rtol, int32_t maxit, void* stream, int32_t* iters,
                                             double* rel_res) {
  if (!row_ptr || !col || !values || !b || !x) {
    set_last_error("row_ptr, col, values, b and x must be device pointers, not NULL");
    return GF_BAD_ARG;
  }
  if (n_rows <= 0 || n_rows > kStaticMaxRows) {
    set_last_error("n_rows must be in [1, " + std::to_string(kStaticMaxRows) +
                   "]: the static scratch of this entry point holds at most that many block rows");
    return GF_BAD_ARG;
  }
  if (!(rtol > 0.0) || maxit <= 0) {
    set_last_error("need rtol > 0 and maxit > 0");
    return GF_BAD_ARG;
  }
  double* base = nullptr;
  gf_status st = scratch_on_current_device(&base);
  if (st != GF_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  SView v{row_ptr, col, values, b, x, fixed, n_rows,
          base + kOffR, base + kOffZ, base + kOffP, base + kOffQ, base + kOffPinv, base + kOffPart,
          reinterpret_cast<StaticState*>(base + kOffState)};
  // scalars and tickets must start from zero; the array keeps the last call's values
  StaticState init{};
  init.tol2 = rtol * rtol;
  init.maxit = maxit;
  GS_CK(cudaMemcpyAsync(v.st, &init, sizeof(StaticState), cudaMemcpyHostToDevice, s));
  const unsigned grid = unsigned(std::min<int64_t>((n_rows + kSThreads - 1) / kSThreads, kSMaxGrid));
  const unsigned grid3 = unsigned(std::min<int64_t>((3 * n_rows + kSThreads - 1) / kSThreads, kSMaxGrid));
  ks_init<<<grid, kSThreads, 0, s>>>(v);
  GS_CK(cudaGetLastError());
  StaticState host{};
  int launched = 0;
  for (;;) {
    for (int j = 0; j < 8; ++j, ++launched) {
      ks_spmv<<<grid, kSThreads, 0, s>>>(v);
      ks_update<<<grid, kSThreads, 0, s>>>(v);
      ks_p<<<grid3, kSThreads, 0, s>>>(v);
    }
    GS_CK(cudaGetLastError());
    GS_CK(cudaMemcpyAsync(&host, v.st, sizeof(StaticState), cudaMemcpyDeviceToHost, s));
    GS_CK(cudaStreamSynchronize(s));
    if (host.done || launched >= maxit) break;
  }
  ks_residual<<<grid, kSThreads, 0, s>>>(v);
  GS_CK(cudaGetLastError());
  GS_CK(cudaMemcpyAsync(&host, v.st, sizeof(StaticState), cudaMemcpyDeviceToHost, s));
  GS_CK(cudaStreamSynchronize(s));
  if (iters) *iters = host.iters;
  if (rel_res) *rel_res = host.bb > 0 ? std::sqrt(host.true_rr / host.bb) : 0.0;
  gf_status status = gf_status(host.status);
  if (status == GF_OK && !host.done) status = GF_CG_MAXITER;
  if (status == GF_BAD_ARG) {
    std::string msg = "static solve:";
    if (host.bad_cols > 0) msg += " " + std::to_string(int64_t(host.bad_cols)) + " column ids lie outside [0, n_rows);";
    if (host.bad_diag > 0)
      msg += " " + std::to_string(int64_t(host.bad_diag)) +
             " free rows have no diagonal block or a singular one (block Jacobi needs its inverse);";
    msg.pop_back();
    set_last_error(msg);
  }
  else if (status != GF_OK) set_last_error(std::string("static solve: ") + gf_status_string(status));
  return status;
}
