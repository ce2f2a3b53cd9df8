// Internal declarations of libgridpull: the context and band objects, error
// plumbing, launch helpers and the small device functions every kernel shares
// (exact cell lookup, brick addressing, Philox4x32-10, Box-Muller, Feistel).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "gridpull.h"

// ------------------------------------------------------------------ objects
struct gp_prof_rec {
  const char* name;
  cudaEvent_t start, stop;
};

struct gp_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  std::string err;
  // Tracing: launch counter (always on) and, while profiling, one pair of
  // CUDA events around every kernel launch on the context's stream.
  int64_t launches = 0;
  bool profiling = false;
  std::vector<gp_prof_rec> prof;
  std::vector<cudaEvent_t> event_pool;
  // Bands made from this context that are still alive; gp_destroy defers the
  // release until the last of them is destroyed.
  int64_t live_bands = 0;
  bool destroy_pending = false;
};

// Release a context's memory (called when no band refers to it any more).
void gp_ctx_release(gp_ctx* ctx);

// Record the start event of the next launch (profiling only).
void gp_prof_pre(gp_ctx* ctx);
// Record the stop event and count the launch.
void gp_prof_post(gp_ctx* ctx, const char* name);

// Launch a kernel of this library: counted, traced while profiling, checked.
#define GP_KERNEL(ctx, name, ...)                            \
  do {                                                       \
    gp_prof_pre(ctx);                                        \
    __VA_ARGS__;                                             \
    gp_prof_post(ctx, name);                                 \
    GP_LAUNCH_CHECK(ctx, name);                              \
  } while (0)

// Number of fp64 partial-sum slots the reduction kernels may use per call.
constexpr int GP_MAX_PARTIAL_BLOCKS = 4096;
// Device int slots of gp_band::dev_ints.
enum { GP_DI_NVALID = 0, GP_DI_ERROR = 1, GP_DI_DONE = 2, GP_DI_COUNT = 8 };
// Error bits raised by kernels in dev_ints[GP_DI_ERROR].
enum { GP_EF_NUMERIC = 1, GP_EF_TIMEOUT = 2, GP_EF_RANGE = 4 };

struct gp_band {
  gp_ctx* ctx = nullptr;
  int R = 0, M1 = 0, M2 = 0, nb = 0, knn_k = 0, G = 0;
  uint32_t flags = 0;
  int64_t J = 0, n_bricks = 0, n_active = 0;
  int64_t V_trainable = 0, V_tv = 0, n_pull = 0, n_occ = 0;

  // Brick storage: brick_table[(bz*nb + by)*nb + bx] = slot or -1.
  int32_t* brick_table = nullptr;
  int32_t* brick_coord = nullptr;  // n_bricks x 3 (bx, by, bz)
  int32_t* brick_nbr = nullptr;    // n_bricks x 27: slots of the 3x3x3 bricks around each (x fastest, -1 absent)
  uint32_t* masks = nullptr;       // n_bricks x 48 words: [T 16][trainable 16][pull 16]
  int32_t* active = nullptr;       // slots of bricks with a trainable vertex
  float* D = nullptr;              // values, V_stored
  float* m = nullptr;              // Adam first moment
  float* v = nullptr;              // Adam second moment
  unsigned long long* acc = nullptr;  // deterministic two-word fixed-point gradient (2 x V_stored)
  float* D_alt = nullptr;          // second value buffer: gp_step_update writes the new values here, then swaps
  float* qgrad = nullptr;          // query part of the gradient for gp_step_update, all zero between calls
  float* tv_inv = nullptr;         // 1/TV_i per slot (0 outside T), written by gp_step's first L_TV pass

  // Point cloud: original order copy, cell list sorted copy, sigma, permutation.
  float* pts = nullptr;            // J x 3
  float4* pts_sorted = nullptr;    // J: x, y, z, original index (int bits)
  int32_t* cell_start = nullptr;   // G^3 + 1
  float* sigma = nullptr;          // J
  float* normals = nullptr;        // J x 3: unit normal estimate (PCA of the sigma-ball), seeds gp_nn
  int32_t* perm = nullptr;         // J: Pi_e of the cached epoch
  int32_t* inv_perm = nullptr;     // J: Pi_e^-1 (point -> pool slot within a replica)
  int32_t* order_tiles = nullptr;  // per-tile counts / offsets of the spatial batch order
  int32_t* emit_order = nullptr;   // J: point indices in Morton order of their cell-list cells
  int32_t* emit_slot = nullptr;    // J: Pi_e^-1(emit_order[u]), the epoch's pool slot of the u-th emitted point
  float4* emit_pts = nullptr;      // J: (x, y, z, sigma) of emit_order[u]
  bool perm_valid = false;
  uint64_t perm_seed = 0;
  uint32_t perm_epoch = 0;

  // Launch shape of the fused step kernel (records in flight per thread,
  // resident blocks per SM it is compiled for), set by gp_band_autotune.
  int q_rpt = 1;
  int q_bps = 3;
  // Form of the (atomic-mode) query pass: GP_QUERY_DIRECT, GP_QUERY_WINDOW
  // or GP_QUERY_WINDOW_STAGED, also chosen by gp_band_autotune.
  int q_form = GP_QUERY_DIRECT;

  // Scratch for reductions and counters.
  double* partials = nullptr;      // GP_MAX_PARTIAL_BLOCKS x 8
  int32_t* dev_ints = nullptr;     // GP_DI_COUNT

  int64_t V_stored() const { return n_bricks * 512; }
};

// ------------------------------------------------------------ error helpers
gp_status gp_fail(gp_ctx* ctx, gp_status st, const std::string& msg);
gp_status gp_cuda_fail(gp_ctx* ctx, cudaError_t e, const char* what);

#define GP_CUDA(ctx, call)                                   \
  do {                                                       \
    cudaError_t _e = (call);                                 \
    if (_e != cudaSuccess) return gp_cuda_fail(ctx, _e, #call); \
  } while (0)

#define GP_LAUNCH_CHECK(ctx, what)                           \
  do {                                                       \
    cudaError_t _e = cudaGetLastError();                     \
    if (_e != cudaSuccess) return gp_cuda_fail(ctx, _e, what); \
  } while (0)

template <typename T>
gp_status gp_alloc(gp_ctx* ctx, T** p, size_t count, const char* what) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return gp_fail(ctx, e == cudaErrorMemoryAllocation ? GP_ERR_OOM : GP_ERR_CUDA,
                   std::string("cudaMalloc failed for ") + what + ": " + cudaGetErrorString(e));
  }
  return GP_OK;
}

inline void gp_free(void* p) {
  if (p) cudaFree(p);
}

inline unsigned gp_blocks(int64_t n, int threads, int64_t cap = 1 << 30) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (unsigned)b;
}

// Device-wide exclusive scan of n int32 counts in place; returns the total in
// *total_host (synchronises).  Scratch is allocated and freed inside (set-up
// paths only).
gp_status gp_exclusive_scan_i32(gp_ctx* ctx, int32_t* data, int64_t n, int64_t* total_host);

// Pi_e and its inverse for (seed, epoch), recomputed only when they change.
gp_status gp_build_permutation(gp_band* band, uint64_t seed, uint32_t epoch);

// Tile of sorted points handled by one block of the spatial batch order.
constexpr int GP_ORDER_THREADS = 512;
constexpr int GP_ORDER_PER_THREAD = 4;
constexpr int GP_ORDER_TILE = GP_ORDER_THREADS * GP_ORDER_PER_THREAD;

// ------------------------------------------------------ device: geometry
// Exact cell of one float32 coordinate: t = (x + 1) * R/2.  x + 1 is split
// into s + e without error (TwoSum) and R/2 is a power of two, so t_hi + t_lo
// is the real value; floor is taken on it.  The _rn intrinsics keep the
// compiler from contracting any step into an FMA.
struct gp_cell1 {
  int c;      // floor(t), unclamped
  float t;    // t - c, in [0, 1]
};

__device__ __forceinline__ gp_cell1 gp_cell_exact(float x, float half_r) {
  gp_cell1 out;
  if (!(fabsf(x) < 1.0e30f)) {  // NaN or huge: far outside
    out.c = -(1 << 30);
    out.t = 0.f;
    return out;
  }
  float s = __fadd_rn(x, 1.0f);
  float bb = __fsub_rn(s, x);
  float e = __fadd_rn(__fsub_rn(x, __fsub_rn(s, bb)), __fsub_rn(1.0f, bb));
  float thi = __fmul_rn(s, half_r);
  float tlo = __fmul_rn(e, half_r);
  float fl = floorf(thi);
  if (thi == fl && tlo < 0.f) fl -= 1.0f;
  out.c = (int)fl;
  out.t = __fadd_rn(__fsub_rn(thi, fl), tlo);
  return out;
}

// Brick slot of vertex (i,j,k), or -1 when the brick is not stored or the
// vertex is outside the virtual brick grid.
__device__ __forceinline__ int gp_brick_slot(const int32_t* __restrict__ table, int nb, int i, int j,
                                             int k) {
  int bx = i >> 3, by = j >> 3, bz = k >> 3;
  if ((unsigned)bx >= (unsigned)nb || (unsigned)by >= (unsigned)nb || (unsigned)bz >= (unsigned)nb) return -1;
  return __ldg(table + ((int64_t)bz * nb + by) * nb + bx);
}

__host__ __device__ __forceinline__ int gp_local(int i, int j, int k) {
  return (((k & 7) << 3) | (j & 7)) << 3 | (i & 7);
}

__device__ __forceinline__ int64_t gp_vaddr(int slot, int i, int j, int k) {
  return (int64_t)slot * 512 + gp_local(i, j, k);
}

__device__ __forceinline__ bool gp_mask_bit(const uint32_t* __restrict__ masks, int slot, int which,
                                            int local) {
  uint32_t w = __ldg(masks + (int64_t)slot * 48 + which * 16 + (local >> 5));
  return (w >> (local & 31)) & 1u;
}

// --------------------------------------------------- device: Philox4x32-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3"
// (SC'11): ten rounds of two 32x32->64 products; the key is bumped by the
// Weyl increments between rounds.
struct gp_u4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ gp_u4 gp_philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                           uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t lo0 = 0xD2511F53u * c0;
    uint32_t hi0 = __umulhi(0xD2511F53u, c0);
    uint32_t lo1 = 0xCD9E8D57u * c2;
    uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return {c0, c1, c2, c3};
}

// Box-Muller on two word pairs -> three standard normals (float32).
__device__ __forceinline__ float3 gp_box_muller3(gp_u4 w) {
  const float s24 = 5.9604644775390625e-08f;  // 2^-24
  float u1 = (float)((w.x >> 8) + 1u) * s24;
  float u2 = (float)(w.y >> 8) * s24;
  float u3 = (float)((w.z >> 8) + 1u) * s24;
  float u4 = (float)(w.w >> 8) * s24;
  float r1 = sqrtf(-2.0f * logf(u1));
  float r2 = sqrtf(-2.0f * logf(u3));
  float s1, c1, s2, c2;
  sincospif(2.0f * u2, &s1, &c1);
  sincospif(2.0f * u4, &s2, &c2);
  return make_float3(r1 * c1, r1 * s1, r2 * c2);
}

// 4-round balanced Feistel network on 2*half bits; the round function is word
// 0 of Philox4x32-10 at counter (value, round, epoch, 1).
__device__ __forceinline__ uint32_t gp_feistel(uint32_t x, int half, uint32_t epoch, uint32_t k0,
                                               uint32_t k1) {
  uint32_t mask = (half >= 32) ? 0xFFFFFFFFu : ((1u << half) - 1u);
  uint32_t left = x >> half, right = x & mask;
#pragma unroll
  for (uint32_t r = 0; r < 4; ++r) {
    uint32_t f = gp_philox(right, r, epoch, 1u, k0, k1).x & mask;
    uint32_t nl = right;
    right = left ^ f;
    left = nl;
  }
  return (left << half) | right;
}

// Query at pool position k of an epoch: q = s_j + sigma_j * z, z the three
// Box-Muller normals of Philox4x32-10 at counter (k, epoch, 0, 0).
__device__ __forceinline__ float3 gp_draw_query(const float* __restrict__ pts, const float* __restrict__ sigma, int32_t j,
                                             int64_t k, uint32_t epoch, uint32_t k0, uint32_t k1) {
  float3 z = gp_box_muller3(gp_philox((uint32_t)k, epoch, 0u, 0u, k0, k1));
  float sg = sigma[j];
  return make_float3(pts[3 * (int64_t)j + 0] + sg * z.x, pts[3 * (int64_t)j + 1] + sg * z.y,
                     pts[3 * (int64_t)j + 2] + sg * z.z);
}

// The same query from a point's (x, y, z, sigma) packed in a float4.
__device__ __forceinline__ float3 gp_draw_query4(float4 ps, int64_t k, uint32_t epoch, uint32_t k0, uint32_t k1) {
  float3 z = gp_box_muller3(gp_philox((uint32_t)k, epoch, 0u, 0u, k0, k1));
  return make_float3(ps.x + ps.w * z.x, ps.y + ps.w * z.y, ps.z + ps.w * z.z);
}

__host__ __device__ inline int gp_feistel_bits(int64_t J) {
  int m = 2;
  while ((int64_t(1) << m) < J) ++m;
  return m + (m & 1);
}

// ------------------------------------------ device: spatial batch order
// Replicas r >= 0 of pool slot p whose position k = p + r J lies in
// [first, last): r in [r0, r0 + n).
// All of p < J, first <= last <= Q are below 2^31, so the divisions are
// unsigned 32-bit ones.
__device__ __forceinline__ void owned_range(int64_t p, int64_t J, int64_t first, int64_t last, int64_t& r0, int& n) {
  const int32_t lo = (int32_t)(first - p), hi = (int32_t)(last - 1 - p);
  const uint32_t uj = (uint32_t)J;
  const uint32_t a = lo <= 0 ? 0u : ((uint32_t)lo + uj - 1u) / uj;
  r0 = a;
  if (hi < 0) {
    n = 0;
    return;
  }
  const uint32_t b = (uint32_t)hi / uj;
  n = b >= a ? (int)(b - a + 1u) : 0;
}

// Exclusive scan of one int per thread over a block of GP_ORDER_THREADS
// threads; returns the block total.
__device__ __forceinline__ int block_exclusive_scan(int v, int* excl) {
  __shared__ int wsum[GP_ORDER_THREADS / 32];
  __shared__ int total_s;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int w = lane < GP_ORDER_THREADS / 32 ? wsum[lane] : 0;
    int wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < GP_ORDER_THREADS / 32) wsum[lane] = wi - w;
    if (lane == GP_ORDER_THREADS / 32 - 1) total_s = wi;
  }
  __syncthreads();
  *excl = wsum[wid] + incl - v;
  int t = total_s;
  __syncthreads();  // wsum and total_s may be reused by the next call
  return t;
}

// Exclusive scan, in place, of n ints by one block of GP_ORDER_THREADS threads.
constexpr int GP_SCAN_PER_THREAD = 8;
__device__ __forceinline__ void gp_block_scan_inplace(int32_t* __restrict__ a, int64_t n) {
  int carry = 0;
  for (int64_t base = 0; base < n; base += (int64_t)GP_ORDER_THREADS * GP_SCAN_PER_THREAD) {
    const int64_t i0 = base + (int64_t)threadIdx.x * GP_SCAN_PER_THREAD;
    int v[GP_SCAN_PER_THREAD];
    int sum = 0;
#pragma unroll
    for (int k = 0; k < GP_SCAN_PER_THREAD; ++k) {
      v[k] = i0 + k < n ? a[i0 + k] : 0;
      sum += v[k];
    }
    int excl;
    const int total = block_exclusive_scan(sum, &excl);
    int run = carry + excl;
#pragma unroll
    for (int k = 0; k < GP_SCAN_PER_THREAD; ++k) {
      if (i0 + k < n) a[i0 + k] = run;
      run += v[k];
    }
    carry += total;
  }
}

// ------------------------------------------------------ device: reductions
__device__ __forceinline__ float gp_warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double gp_warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int gp_warp_sum_i(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------ device: step records
// The band as the step kernels see it.
struct Grid {
  const int32_t* __restrict__ table;
  const uint32_t* __restrict__ masks;
  const float* __restrict__ D;
  int nb;
  int R;
  float half_r;  // R/2 = 1/h
};

struct Cells {
  int cq[3], cs[3];
  float tq[3], ts[3];
  int slot_q, slot_s;
};

// The arithmetic half of classify(): q inside the domain, s finite; the cells
// and local coordinates of q and s (cell(s) clamped to the grid, its local
// coordinate extended accordingly).
__device__ __forceinline__ bool classify_cells(const Grid& G, const float q[3], const float s[3], Cells& C) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    gp_cell1 g = gp_cell_exact(q[a], G.half_r);
    if (g.c < 0 || g.c > G.R - 1) return false;
    C.cq[a] = g.c;
    C.tq[a] = g.t;
    gp_cell1 h = gp_cell_exact(s[a], G.half_r);
    if (h.c == -(1 << 30)) return false;
    int cc = min(max(h.c, 0), G.R - 1);
    C.cs[a] = cc;
    C.ts[a] = h.t + (float)(h.c - cc);
  }
  return true;
}

// Validity of a record (Sec. 3 pull band; readings in the header): q inside
// the domain, cell(q) and cell(s) in the M1 band.
__device__ __forceinline__ bool classify(const Grid& G, const float q[3], const float s[3], Cells& C) {
  if (!classify_cells(G, q, s, C)) return false;
  C.slot_q = gp_brick_slot(G.table, G.nb, C.cq[0], C.cq[1], C.cq[2]);
  if (C.slot_q < 0 || !gp_mask_bit(G.masks, C.slot_q, 2, gp_local(C.cq[0], C.cq[1], C.cq[2]))) return false;
  C.slot_s = gp_brick_slot(G.table, G.nb, C.cs[0], C.cs[1], C.cs[2]);
  if (C.slot_s < 0 || !gp_mask_bit(G.masks, C.slot_s, 2, gp_local(C.cs[0], C.cs[1], C.cs[2]))) return false;
  return true;
}

__device__ __forceinline__ void load_rec(const float* __restrict__ rec, int64_t i, float q[3], float s[3]) {
  const float2* r2 = reinterpret_cast<const float2*>(rec + 6 * i);
  float2 a = __ldg(r2), b = __ldg(r2 + 1), c = __ldg(r2 + 2);
  q[0] = a.x;
  q[1] = a.y;
  q[2] = b.x;
  s[0] = b.y;
  s[1] = c.x;
  s[2] = c.y;
}

