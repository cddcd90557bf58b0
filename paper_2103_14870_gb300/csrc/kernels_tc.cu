// Tensor-core (tcgen05) kernels of the learned warm start's network: the dense
// layers Z = [X1 | X2] W' (+ bias) and the edge messages relu(a_j + We e_ij + bm)
// with their per-node mean.  Both are dense contractions with K <= 128 and at
// most 64 outputs, so one 128-row tile is one M=128 MMA chain into 64 tensor
// memory columns.
//
// Precision.  The weights are bf16 (exact as tensor-core operands).  The FP32
// activations are split into three bf16 parts, x = hi + mid + lo exactly, and
// the three products W hi, W mid, W lo accumulate into one FP32 accumulator:
// every product is exact and only the accumulation rounds, as in an FP32 FMA
// chain.  So the tensor-core layers agree with FP32 arithmetic to rounding order.
//
// One CTA = 4 warps (128 threads), persistent over tiles.  Per tile:
//   1. all threads load the FP32 tile with coalesced 16-byte loads, split it
//      and store the three bf16 parts into shared memory (K-major core matrices);
//   2. one thread issues 3 K/16 MMAs (A and B from shared memory, D in tensor
//      memory) and commits them to an mbarrier;
//   3. every warp reads its 32 accumulator rows back (tcgen05.ld), and the
//      epilogue (bias, residual, relu, per-node mean) runs through a shared
//      staging tile so that every global store is coalesced.
// Every wait is bounded (one second); on a timeout the kernel sets *err and
// every CTA leaves its loop, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>

#include "gf_gnn.h"
#include "gf_tc.cuh"

namespace gf {
namespace {

constexpr int kTcThreads = 128;
constexpr int kTcRows = 128;            // MMA M
constexpr uint32_t kTmemCols = 64;      // accumulator columns (N <= 64)
constexpr uint64_t kWaitNs = 1000000000ull;

__device__ __forceinline__ void flag_error(unsigned long long* err) {
  if (err) atomicAdd(err, 1ull);
}

// Split 4 FP32 values and store hi / mid / lo (8 bytes each) at the three
// K offsets 0, KP, 2 KP of row `row`, column `k` (k % 4 == 0).
template <int KP>
__device__ __forceinline__ void store_split4(uint8_t* A, int row, int k, const float4 v, uint32_t lbo, uint32_t sbo) {
  uint32_t h[4], m[4], l[4];
  tc::split3(v.x, h[0], m[0], l[0]);
  tc::split3(v.y, h[1], m[1], l[1]);
  tc::split3(v.z, h[2], m[2], l[2]);
  tc::split3(v.w, h[3], m[3], l[3]);
  const uint2 ph = make_uint2(tc::pack_hi16(h[0], h[1]), tc::pack_hi16(h[2], h[3]));
  const uint2 pm = make_uint2(tc::pack_hi16(m[0], m[1]), tc::pack_hi16(m[2], m[3]));
  const uint2 pl = make_uint2(tc::pack_hi16(l[0], l[1]), tc::pack_hi16(l[2], l[3]));
  *reinterpret_cast<uint2*>(A + tc::kmajor_off(row, k, lbo, sbo)) = ph;
  *reinterpret_cast<uint2*>(A + tc::kmajor_off(row, KP + k, lbo, sbo)) = pm;
  *reinterpret_cast<uint2*>(A + tc::kmajor_off(row, 2 * KP + k, lbo, sbo)) = pl;
}

// One MMA chain D (+)= sum_s A_s B over the three split parts, issued by one
// thread (the first MMA overwrites D unless accumulate_first).
template <int KP, int NP>
__device__ __forceinline__ void issue_split_mma(uint32_t tmem, uint32_t a_base, uint32_t b_base, uint64_t* bar,
                                                bool accumulate_first) {
  constexpr uint32_t lboA = (kTcRows / 8) * 128, sboA = 128;
  constexpr uint32_t lboB = (NP / 8) * 128, sboB = 128;
  constexpr uint32_t idesc = tc::idesc_bf16_f32(kTcRows, NP);
  tc::fence_after_sync();
#pragma unroll
  for (int s = 0; s < 3; ++s)
#pragma unroll
    for (int q = 0; q < KP / 16; ++q) {
      const uint64_t ad = tc::smem_desc(a_base + uint32_t(s * (KP / 8) + 2 * q) * lboA, lboA, sboA);
      const uint64_t bd = tc::smem_desc(b_base + uint32_t(2 * q) * lboB, lboB, sboB);
      tc::mma_bf16(tmem, ad, bd, idesc, accumulate_first || (s | q) != 0);
    }
  tc::mma_commit(bar);
}

// ---------------------------------------------------------------------------
// Weights.  B'_c = W'[:, c KC .. c KC + KC) for every K chunk c, as NP x KC
// K-major operands one after the other.  W'(k, o) = W[k ldw + o], or
// W[(k0 + o) ldw + k] when trans.  With ldw and k0 multiples of 8 and W
// 16-byte aligned, 8 weights move per 16-byte load (along o, or along k when
// trans, where they land as one 16-byte core-matrix row); otherwise one by one.
// ---------------------------------------------------------------------------
template <int KC, int NP>
__device__ __forceinline__ void stage_weights(uint8_t* B, const __nv_bfloat16* __restrict__ W, int ldw, int k0,
                                              int trans, int NO, int K, int nch) {
  constexpr uint32_t lboB = (NP / 8) * 128, sboB = 128, chunk_bytes = NP * KC * 2;
  const int KT = nch * KC;
  auto put = [&](int o, int k, __nv_bfloat16 v) {
    const int c = k / KC;
    *reinterpret_cast<__nv_bfloat16*>(B + c * chunk_bytes + tc::kmajor_off(o, k - c * KC, lboB, sboB)) = v;
  };
  const bool vec = ((reinterpret_cast<uintptr_t>(W) & 15) == 0) && (ldw % 8 == 0) && (k0 % 8 == 0);
  if (vec && !trans) {
    // 8 outputs of one input row per load
    for (int idx = threadIdx.x; idx < KT * (NP / 8); idx += kTcThreads) {
      const int k = idx / (NP / 8), o0 = 8 * (idx - k * (NP / 8));
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (k < K && o0 + 8 <= NO) v = *reinterpret_cast<const uint4*>(W + int64_t(k) * ldw + o0);
      const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&v);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        __nv_bfloat16 w = e[q];
        if (o0 + 8 > NO) w = (k < K && o0 + q < NO) ? W[int64_t(k) * ldw + o0 + q] : __float2bfloat16_rn(0.f);
        put(o0 + q, k, w);
      }
    }
  } else if (vec) {
    // 8 inputs of one output per load: one 16-byte row of a core matrix
    for (int idx = threadIdx.x; idx < NP * (KT / 8); idx += kTcThreads) {
      const int o = idx / (KT / 8), kk = 8 * (idx - o * (KT / 8));
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (o < NO && kk + 8 <= K) {
        v = *reinterpret_cast<const uint4*>(W + int64_t(k0 + o) * ldw + kk);
      } else if (o < NO) {
        __nv_bfloat16* e = reinterpret_cast<__nv_bfloat16*>(&v);
        for (int q = 0; q < 8; ++q) e[q] = kk + q < K ? W[int64_t(k0 + o) * ldw + kk + q] : __float2bfloat16_rn(0.f);
      }
      const int c = kk / KC;
      *reinterpret_cast<uint4*>(B + c * chunk_bytes + tc::kmajor_off(o, kk - c * KC, lboB, sboB)) = v;
    }
  } else {
    for (int idx = threadIdx.x; idx < NP * KT; idx += kTcThreads) {
      int o, k;
      if (trans) { o = idx / KT; k = idx - o * KT; }
      else { k = idx / NP; o = idx - k * NP; }
      __nv_bfloat16 w = __float2bfloat16_rn(0.f);
      if (o < NO && k < K) w = trans ? W[int64_t(k0 + o) * ldw + k] : W[int64_t(k) * ldw + o];
      put(o, k, w);
    }
  }
}

// ---------------------------------------------------------------------------
// Dense layer.  Z = [X1 | X2] W' (+ bias) for the NO outputs.  K is taken in
// chunks of KC columns (KC = 64, or 16 for K <= 16); the accumulator collects
// every chunk of a 128-row tile before its epilogue.  NP = NO rounded up to 16.
// Epilogue: mode 0 Z = acc (+ Z when accumulate), mode 1 also Hout = relu(Z),
// mode 2 also Hout = Hres + relu(Z) (Hout, Hres rows of 64).  X rows are read
// as float4 (ld1, ld2 multiples of 4; K1 a multiple of KC when K2 > 0).  The
// next chunk (of this tile or the next) is loaded into registers while the
// tensor core works on the current one.
// ---------------------------------------------------------------------------
template <int KC, int NP>
struct DenseSmem {
  static constexpr int kMaxChunks = KC == 64 ? 2 : 1;
  static constexpr uint32_t kA = kTcRows * 3 * KC * 2;             // split activations of one chunk
  static constexpr uint32_t kOut = kTcRows * (NP + 4) * 4;         // FP32 output staging (aliases A)
  static constexpr uint32_t kU = kA > kOut ? kA : kOut;
  static constexpr uint32_t kB = kMaxChunks * NP * KC * 2;
  static constexpr uint32_t kBytes = kU + kB + 128;               // + alignment slack
};

template <int KC, int NP>
__global__ void __launch_bounds__(kTcThreads, KC == 64 ? 3 : 4) k_dense_tc(int64_t N, const float* __restrict__ X1, int K1, int ld1,
                                                          const float* __restrict__ X2, int K2, int ld2,
                                                          const __nv_bfloat16* __restrict__ W, int ldw, int k0,
                                                          int trans, const __nv_bfloat16* __restrict__ bias, int NO,
                                                          float* Z, int ldz, const float* Hres, float* Hout, int mode,
                                                          int accumulate, unsigned long long* err) {
  using S = DenseSmem<KC, NP>;
  extern __shared__ uint8_t dyn[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_slot;
  __shared__ float bsh[NP];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dyn) + 127) & ~uintptr_t(127));
  uint8_t* A = base;
  float* OUT = reinterpret_cast<float*>(base);
  uint8_t* B = base + S::kU;
  constexpr uint32_t lboA = (kTcRows / 8) * 128, sboA = 128;
  constexpr int OS = NP + 4;
  // patch = 8 rows x 16 columns of a chunk; lane -> (row l % 8, 4 columns at 4 (l / 8)); warp w takes patches w, w + 4, ...
  constexpr int kPer = (kTcRows / 8) * (KC / 16) / (kTcThreads / 32);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int K = K1 + K2;
  const int nch = (K + KC - 1) / KC;

  if (warp == 0) {
    tc::tmem_alloc(&tmem_slot, kTmemCols);
    tc::tmem_relinquish();
  }
  if (tid == 0) tc::mbar_init(&bar, 1);
  stage_weights<KC, NP>(B, W, ldw, k0, trans, NO, K, nch);
  for (int o = tid; o < NP; o += kTcThreads) bsh[o] = (bias && o < NO) ? __bfloat162float(bias[o]) : 0.f;
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_slot;
  const uint32_t a_base = tc::smem_u32(A), b_base = tc::smem_u32(B);

  const int64_t n_tiles = (N + kTcRows - 1) / kTcRows;
  const int64_t my_tiles = int64_t(blockIdx.x) < n_tiles ? (n_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t n_units = my_tiles * nch;
  float4 xv[kPer];
  auto load_unit = [&](int64_t u) {
    const int64_t r0 = (int64_t(blockIdx.x) + (u / nch) * gridDim.x) * kTcRows;
    const int c = int(u % nch);
    if (r0 + kTcRows <= N && (c + 1) * KC <= K && (c + 1) * KC <= K1 + (c * KC >= K1 ? K2 : 0) &&
        (c * KC >= K1 || (c + 1) * KC <= K1)) {
      // whole chunk inside one source and inside the rows: no per-element checks
      const float* src = c * KC < K1 ? X1 + int64_t(ld1) * r0 + c * KC : X2 + int64_t(ld2) * r0 + (c * KC - K1);
      const int ld = c * KC < K1 ? ld1 : ld2;
#pragma unroll
      for (int i = 0; i < kPer; ++i) {
        const int pi = warp + (kTcThreads / 32) * i;
        const int row = 8 * (pi % (kTcRows / 8)) + (lane & 7), k = 16 * (pi / (kTcRows / 8)) + 4 * (lane >> 3);
        xv[i] = *reinterpret_cast<const float4*>(src + int64_t(ld) * row + k);
      }
      return;
    }
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int pi = warp + (kTcThreads / 32) * i;
      const int row = 8 * (pi % (kTcRows / 8)) + (lane & 7);
      const int k = c * KC + 16 * (pi / (kTcRows / 8)) + 4 * (lane >> 3);
      const int64_t gr = r0 + row;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (gr < N && k < K) {
        v = k < K1 ? *reinterpret_cast<const float4*>(X1 + int64_t(ld1) * gr + k)
                   : *reinterpret_cast<const float4*>(X2 + int64_t(ld2) * gr + (k - K1));
        if (k + 1 >= K) v.y = 0.f;
        if (k + 2 >= K) v.z = 0.f;
        if (k + 3 >= K) v.w = 0.f;
      }
      xv[i] = v;
    }
  };
  if (n_units > 0) load_unit(0);
  uint32_t phase = 0;
  for (int64_t u = 0; u < n_units; ++u) {
    const int64_t r0 = (int64_t(blockIdx.x) + (u / nch) * gridDim.x) * kTcRows;
    const int c = int(u % nch);
    // 1. split and stage this chunk
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int pi = warp + (kTcThreads / 32) * i;
      store_split4<KC>(A, 8 * (pi % (kTcRows / 8)) + (lane & 7), 16 * (pi / (kTcRows / 8)) + 4 * (lane >> 3), xv[i],
                       lboA, sboA);
    }
    tc::fence_async_smem();
    __syncthreads();
    // 2. MMA chain of the chunk; the next chunk's loads overlap it
    if (tid == 0) issue_split_mma<KC, NP>(tmem, a_base, b_base + uint32_t(c) * (NP * KC * 2), &bar, c > 0);
    if (u + 1 < n_units) load_unit(u + 1);
    const bool ok = tc::mbar_wait(&bar, phase, kWaitNs);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      if (tid == 0) flag_error(err);
      break;
    }
    tc::fence_after_sync();
    if (c + 1 < nch) continue;   // the operand space is free again; the accumulator keeps collecting
    // 3. accumulator rows -> staging
    {
      const int row = 32 * warp + lane;
      const uint32_t taddr = tmem + (uint32_t(32 * warp) << 16);
#pragma unroll
      for (int cc = 0; cc < NP / 16; ++cc) {
        uint32_t r[16];
        tc::tmem_ld16_wait(taddr + 16 * cc, r);
#pragma unroll
        for (int j = 0; j < 16; j += 4)
          *reinterpret_cast<float4*>(OUT + row * OS + 16 * cc + j) =
              make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]), __uint_as_float(r[j + 2]),
                          __uint_as_float(r[j + 3]));
      }
    }
    tc::fence_before_sync();
    __syncthreads();
    // 4. coalesced write-out (+ bias, accumulate, relu, residual)
    if (NO == NP) {
      // every thread keeps one 4-column group: rows tid / NP4 + (128 / NP4) q
      constexpr int NP4 = NP / 4, kItems = kTcRows * NP4 / kTcThreads, kBatch = kItems < 8 ? kItems : 8;
      const int o = 4 * (tid % NP4), rb = tid / NP4;
      const float4 bv = make_float4(bsh[o], bsh[o + 1], bsh[o + 2], bsh[o + 3]);
#pragma unroll
      for (int q0 = 0; q0 < kItems; q0 += kBatch) {
        float4 z[kBatch], e[kBatch];
#pragma unroll
        for (int q = 0; q < kBatch; ++q) {      // loads of the batch first
          const int row = rb + (kTcThreads / NP4) * (q0 + q);
          const int64_t gr = r0 + row;
          z[q] = *reinterpret_cast<const float4*>(OUT + row * OS + o);
          e[q] = make_float4(0.f, 0.f, 0.f, 0.f);
          if (gr < N) {
            if (accumulate) e[q] = *reinterpret_cast<const float4*>(Z + int64_t(ldz) * gr + o);
            else if (mode == 2) e[q] = *reinterpret_cast<const float4*>(Hres + 64 * gr + o);
          }
        }
#pragma unroll
        for (int q = 0; q < kBatch; ++q) {
          const int row = rb + (kTcThreads / NP4) * (q0 + q);
          const int64_t gr = r0 + row;
          if (gr >= N) continue;
          float4 v = make_float4(z[q].x + bv.x, z[q].y + bv.y, z[q].z + bv.z, z[q].w + bv.w);
          if (accumulate) {
            v.x += e[q].x; v.y += e[q].y; v.z += e[q].z; v.w += e[q].w;
          }
          *reinterpret_cast<float4*>(Z + int64_t(ldz) * gr + o) = v;
          if (mode == 1) {
            *reinterpret_cast<float4*>(Hout + 64 * gr + o) =
                make_float4(fmaxf(v.x, 0.f), fmaxf(v.y, 0.f), fmaxf(v.z, 0.f), fmaxf(v.w, 0.f));
          } else if (mode == 2) {
            const float4 h = accumulate ? *reinterpret_cast<const float4*>(Hres + 64 * gr + o) : e[q];
            *reinterpret_cast<float4*>(Hout + 64 * gr + o) = make_float4(
                h.x + fmaxf(v.x, 0.f), h.y + fmaxf(v.y, 0.f), h.z + fmaxf(v.z, 0.f), h.w + fmaxf(v.w, 0.f));
          }
        }
      }
    } else {
      for (int idx = tid; idx < kTcRows * NO; idx += kTcThreads) {
        const int row = idx / NO, o = idx - row * NO;
        const int64_t gr = r0 + row;
        if (gr >= N) continue;
        float z = OUT[row * OS + o] + bsh[o];
        float* zp = Z + int64_t(ldz) * gr + o;
        if (accumulate) z += *zp;
        *zp = z;
        if (mode == 1) Hout[64 * gr + o] = fmaxf(z, 0.f);
        else if (mode == 2) Hout[64 * gr + o] = Hres[64 * gr + o] + fmaxf(z, 0.f);
      }
    }
    __syncthreads();   // the staging tile is the next chunk's operand space
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

// ---------------------------------------------------------------------------
// Edge messages.  Tile = a run of whole destination nodes with at most 128
// incoming messages and 128 nodes: etile[t] = (first node n0, nodes, first
// message p0, messages).  Row r of the tile is message p = p0 + r, j -> i; the
// MMA gives We e_p for all rows, the epilogue adds a_j and bm, applies relu,
// and sums each node's rows in message order: M_i = (1 / deg_i) sum_p relu(.).
// While a tile is in the tensor core, its neighbour rows a_j are copied into
// shared memory (cp.async, 16 bytes per lane, two rows per warp instruction)
// and the next tile's descriptor, edge inputs and neighbour ids are loaded
// into registers.
// ---------------------------------------------------------------------------
constexpr int kEdgeKP = 16, kEdgeNP = 64, kEdgeOS = 68;   // row stride 272 B: 16-byte aligned, conflict-free float4
struct EdgeSmem {
  static constexpr uint32_t kA = kTcRows * 3 * kEdgeKP * 2;
  static constexpr uint32_t kS = kTcRows * kEdgeOS * 4;   // a_j rows, then the messages in place
  static constexpr uint32_t kB = kEdgeNP * kEdgeKP * 2;
  static constexpr uint32_t kBytes = kA + kS + kB + 128;
};

struct EdgeTileRegs {
  int4 d;               // (n0, nodes, p0, messages)
  int rp, rp_last;      // row_ptr[n0 + tid] - p0 (tid <= nodes); thread 0: row_ptr[n0 + 128] - p0
  int j;                // neighbour of this thread's message row, -1 past the tile
  float4 ev[kTcRows / 8 / (kTcThreads / 32)];
};

__device__ __forceinline__ void fetch_edge_tile(const GnnDev& g, int64_t tile, EdgeTileRegs& t) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  t.d = g.etile[tile];
  t.rp = tid <= t.d.y ? g.row_ptr[t.d.x + tid] - t.d.z : 0;
  t.rp_last = (tid == 0 && t.d.y == kTcRows) ? g.row_ptr[t.d.x + kTcRows] - t.d.z : 0;
  const int row = 32 * warp + lane;
  t.j = row < t.d.w ? g.col[t.d.z + row] : -1;
#pragma unroll
  for (int i = 0; i < kTcRows / 8 / (kTcThreads / 32); ++i) {
    const int r = 8 * (warp + (kTcThreads / 32) * i) + (lane & 7), k = 4 * (lane >> 3);
    t.ev[i] = r < t.d.w ? *reinterpret_cast<const float4*>(g.efeat + int64_t(kEin) * (t.d.z + r) + k)
                        : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
}

__global__ void __launch_bounds__(kTcThreads, 4) k_gnn_edge_fwd_tc(GnnDev g, const float* __restrict__ a,
                                                                 const __nv_bfloat16* __restrict__ We,
                                                                 const __nv_bfloat16* __restrict__ bm, float* M,
                                                                 unsigned long long* err) {
  extern __shared__ uint8_t dyn[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_slot;
  __shared__ float bsh[kEdgeNP];
  __shared__ int32_t rp_sh[kTcRows + 1];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dyn) + 127) & ~uintptr_t(127));
  uint8_t* A = base;
  float* S = reinterpret_cast<float*>(base + EdgeSmem::kA);
  uint8_t* B = base + EdgeSmem::kA + EdgeSmem::kS;
  constexpr uint32_t lboA = (kTcRows / 8) * 128, sboA = 128;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    tc::tmem_alloc(&tmem_slot, kTmemCols);
    tc::tmem_relinquish();
  }
  if (tid == 0) tc::mbar_init(&bar, 1);
  stage_weights<kEdgeKP, kEdgeNP>(B, We, 64, 0, 0, kEdgeNP, kEin, 1);
  for (int o = tid; o < kEdgeNP; o += kTcThreads) bsh[o] = __bfloat162float(bm[o]);
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_slot;
  const uint32_t a_base = tc::smem_u32(A), b_base = tc::smem_u32(B), s_base = tc::smem_u32(S);

  EdgeTileRegs t;
  if (int64_t(blockIdx.x) < g.n_etiles) fetch_edge_tile(g, blockIdx.x, t);
  uint32_t phase = 0;
  for (int64_t tile = blockIdx.x; tile < g.n_etiles; tile += gridDim.x) {
    const int n0 = t.d.x, nn = t.d.y;
    // 1. stage this tile: node offsets, split edge inputs; neighbour rows start moving
    if (tid <= nn) rp_sh[tid] = t.rp;
    if (tid == 0 && nn == kTcRows) rp_sh[kTcRows] = t.rp_last;
#pragma unroll
    for (int i = 0; i < kTcRows / 8 / (kTcThreads / 32); ++i) {
      const int r = 8 * (warp + (kTcThreads / 32) * i) + (lane & 7), k = 4 * (lane >> 3);
      store_split4<kEdgeKP>(A, r, k, t.ev[i], lboA, sboA);
    }
#pragma unroll 4
    for (int i = 0; i < 16; ++i) {     // rows 32 warp + 2 i + lane / 16, 16-byte piece lane % 16
      const int rl = 2 * i + (lane >> 4);
      const int jr = __shfl_sync(0xffffffffu, t.j, rl);
      if (jr >= 0)
        cp_async16(s_base + uint32_t((32 * warp + rl) * kEdgeOS + 4 * (lane & 15)) * 4u,
                   a + 64 * int64_t(jr) + 4 * (lane & 15));
    }
    tc::fence_async_smem();
    __syncthreads();
    if (tid == 0) issue_split_mma<kEdgeKP, kEdgeNP>(tmem, a_base, b_base, &bar, false);
    // 2. the next tile's registers
    if (tile + gridDim.x < g.n_etiles) fetch_edge_tile(g, tile + gridDim.x, t);
    cp_async_wait_all();
    const bool ok = tc::mbar_wait(&bar, phase, kWaitNs);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      if (tid == 0) flag_error(err);
      break;
    }
    tc::fence_after_sync();
    // 3. relu(We e + a_j + bm) over the a_j rows in place
    {
      const int row = 32 * warp + lane;
      const uint32_t taddr = tmem + (uint32_t(32 * warp) << 16);
#pragma unroll
      for (int c = 0; c < kEdgeNP / 16; ++c) {
        uint32_t r[16];
        tc::tmem_ld16_wait(taddr + 16 * c, r);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int o = 16 * c + 4 * q;
          float4* sp = reinterpret_cast<float4*>(S + row * kEdgeOS + o);
          const float4 v = *sp;
          *sp = make_float4(fmaxf(__uint_as_float(r[4 * q]) + v.x + bsh[o], 0.f),
                            fmaxf(__uint_as_float(r[4 * q + 1]) + v.y + bsh[o + 1], 0.f),
                            fmaxf(__uint_as_float(r[4 * q + 2]) + v.z + bsh[o + 2], 0.f),
                            fmaxf(__uint_as_float(r[4 * q + 3]) + v.w + bsh[o + 3], 0.f));
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();
    // 4. per-node mean, rows in message order; lanes own consecutive outputs (coalesced stores)
    for (int idx = tid; idx < nn * kEdgeNP; idx += kTcThreads) {
      const int il = idx >> 6, o = idx & 63;
      const int b = rp_sh[il], e = rp_sh[il + 1];
      float s = 0.f;
      for (int r = b; r < e; ++r) s += S[r * kEdgeOS + o];
      M[64 * int64_t(n0 + il) + o] = s * (1.f / float(max(e - b, 1)));
    }
    __syncthreads();
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

// Persistent grid: resident CTAs per SM times the SM count, per device.  The
// residency is computed from the kernel's registers and shared memory and the
// tensor-memory columns each CTA holds (512 per SM), not from the runtime's
// occupancy query (which assumes one CTA per SM for kernels that allocate
// tensor memory).  Launching more CTAs than fit would only queue them.
constexpr int kMaxDevices = 64;
template <class F>
int64_t persistent_ctas(F kernel, uint32_t smem, int (&cache)[kMaxDevices]) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 0;
  if (cache[dev] == 0) {
    cudaFuncAttributes fa{};
    int sms = 0, smem_sm = 0, smem_rsv = 0, regs_sm = 0, thr_sm = 0;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess ||
        cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, kernel) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess) {
      cudaGetLastError();
      cache[dev] = -1;
    } else {
      const int by_smem = smem_sm / int(smem + fa.sharedSizeBytes + smem_rsv);
      const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;   // allocation unit: 256 per warp
      const int by_regs = regs_sm / (regs_warp * (kTcThreads / 32));
      const int by_thr = thr_sm / kTcThreads;
      const int by_tmem = 512 / int(kTmemCols);
      const int n = std::min(std::min(by_smem, by_regs), std::min(by_thr, by_tmem));
      cache[dev] = n * sms > 0 ? n * sms : -1;
    }
  }
  return cache[dev] > 0 ? cache[dev] : 0;
}

template <int KC, int NP>
int launch_dense_tc(int64_t N, const float* X1, int K1, int ld1, const float* X2, int K2, int ld2,
                    const __nv_bfloat16* W, int ldw, int k0, int trans, const __nv_bfloat16* bias, int NO, float* Z,
                    int ldz, const float* Hres, float* Hout, int mode, int accumulate, unsigned long long* err,
                    cudaStream_t s) {
  using Sm = DenseSmem<KC, NP>;
  static int cache[kMaxDevices] = {};
  const int64_t cap = persistent_ctas(k_dense_tc<KC, NP>, Sm::kBytes, cache);
  if (cap < 1) return -1;
  const int64_t tiles = (N + kTcRows - 1) / kTcRows;
  if (tiles == 0) return 0;
  const unsigned grid = unsigned(tiles < cap ? tiles : cap);
  k_dense_tc<KC, NP><<<grid, kTcThreads, Sm::kBytes, s>>>(N, X1, K1, ld1, X2, K2, ld2, W, ldw, k0, trans, bias, NO, Z,
                                                          ldz, Hres, Hout, mode, accumulate, err);
  return 1;
}

}  // namespace

// Returns the number of kernels launched, or -1 when the shape has no
// tensor-core form (the caller keeps the FP32 kernel).
int dense_tc(int64_t N, const float* X1, int K1, int ld1, const float* X2, int K2, int ld2, const __nv_bfloat16* W,
             int ldw, int k0, int trans, const __nv_bfloat16* bias, int NO, float* Z, int ldz, const float* Hres,
             float* Hout, int mode, int accumulate, unsigned long long* err, cudaStream_t s) {
  const int K = K1 + K2;
  if (K < 1 || K > 128 || NO < 1 || NO > 64 || (ld1 & 3) || ld1 < ((K1 + 3) & ~3) ||
      (K2 > 0 && ((ld2 & 3) || ld2 < ((K2 + 3) & ~3))) || ((NO & 3) == 0 && (ldz & 3)))
    return -1;
  if (K <= 16) {
    if (NO > 16) return launch_dense_tc<16, 64>(N, X1, K1, ld1, X2, K2, ld2, W, ldw, k0, trans, bias, NO, Z, ldz,
                                                Hres, Hout, mode, accumulate, err, s);
    return -1;
  }
  if (K2 > 0 && (K1 % 64)) return -1;   // a 64-column chunk never straddles X1 and X2
  if (NO <= 16) return launch_dense_tc<64, 16>(N, X1, K1, ld1, X2, K2, ld2, W, ldw, k0, trans, bias, NO, Z, ldz, Hres,
                                               Hout, mode, accumulate, err, s);
  return launch_dense_tc<64, 64>(N, X1, K1, ld1, X2, K2, ld2, W, ldw, k0, trans, bias, NO, Z, ldz, Hres, Hout, mode,
                                 accumulate, err, s);
}

int gnn_edge_fwd_tc(const GnnDev& g, const float* a, const __nv_bfloat16* We, const __nv_bfloat16* bm, float* M,
                    cudaStream_t s) {
  static int cache[kMaxDevices] = {};
  const int64_t cap = persistent_ctas(k_gnn_edge_fwd_tc, EdgeSmem::kBytes, cache);
  if (cap < 1 || g.n_etiles <= 0 || !g.etile) return -1;
  const unsigned grid = unsigned(g.n_etiles < cap ? g.n_etiles : cap);
  k_gnn_edge_fwd_tc<<<grid, kTcThreads, EdgeSmem::kBytes, s>>>(g, a, We, bm, M, g.err);
  return 1;
}

}  // namespace gf
