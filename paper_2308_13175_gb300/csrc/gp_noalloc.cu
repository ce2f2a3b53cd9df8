// gp_step_dense_noalloc: the query part of the step on a caller-owned dense
// grid, for callers that cannot allocate device memory.
//
// Who needs it: code that must not call cudaMalloc on its own - a plugin whose
// host framework owns every device allocation, a real-time loop that may not
// block on the allocator, or a caller that plans all memory up front.  Such a
// caller cannot build a band (gp_build_band allocates), so this entry point
// takes everything it reads and writes as caller-owned device pointers and
// keeps its own scratch (per-block partial sums and two counters) in a
// fixed-size array compiled into the library.
//
// The scratch array lives in this file; every GPU that loads the library holds
// it (about 128 KiB) until the process exits.  Host code cannot hand the
// array's name to a kernel (on the host it is only a stand-in), so the first
// call on a device, with that device current, looks up its device address with
// cudaGetSymbolAddress and keeps it.  Each call makes the context's device
// current while it runs and restores the caller's current device before it
// returns.  Every call on a device shares the array
// and leaves the last call's sums in it; each call clears the counters it needs
// before use.  Two calls whose work overlaps on the GPU (different streams, or
// different host threads) race on the array and both results are then wrong:
// keep calls on one device in one stream order.
#include <mutex>

#include "gp_internal.cuh"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_MAX_BLOCKS = 4096;                                  // one partial row per block
constexpr int64_t NA_MAX_RECORDS = (int64_t)NA_MAX_BLOCKS * NA_THREADS;  // 1,048,576 records per call
constexpr int NA_MAX_R = 1024;
constexpr int NA_MAX_DEVICES = 64;
constexpr int NA_COUNTER_WORDS = 32;  // tail words of the array hold the integer counters

// Partial sums: NA_MAX_BLOCKS rows of 4 doubles, then the counters.
static __device__ __align__(256) double gp_noalloc_scratch[NA_MAX_BLOCKS * 4 + NA_COUNTER_WORDS];

void* g_scratch_addr[NA_MAX_DEVICES] = {};
std::mutex g_scratch_mutex;

struct NACounters {
  int nvalid;
  int done;
};

__device__ __forceinline__ NACounters* na_counters(double* scratch) {
  return reinterpret_cast<NACounters*>(scratch + NA_MAX_BLOCKS * 4);
}

__global__ void k_na_clear(double* __restrict__ scratch) {
  if (threadIdx.x == 0) {
    NACounters* c = na_counters(scratch);
    c->nvalid = 0;
    c->done = 0;
  }
}

__global__ void k_na_zero(float* __restrict__ g, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    g[i] = 0.f;
}

struct DenseCell {
  int cq[3], cs[3];
  float tq[3], ts[3];
};

// A record is valid when q lies inside the domain and s is finite: every
// cell of a dense grid is in the pull band.
__device__ __forceinline__ bool na_classify(float half_r, int R, const float q[3], const float s[3], DenseCell& C) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    gp_cell1 g = gp_cell_exact(q[a], half_r);
    if (g.c < 0 || g.c > R - 1) return false;
    C.cq[a] = g.c;
    C.tq[a] = g.t;
    gp_cell1 h = gp_cell_exact(s[a], half_r);
    if (h.c == -(1 << 30)) return false;
    int cc = min(max(h.c, 0), R - 1);
    C.cs[a] = cc;
    C.ts[a] = h.t + (float)(h.c - cc);
  }
  return true;
}

__device__ __forceinline__ void na_rec(const float* __restrict__ rec, int64_t i, float q[3], float s[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    q[a] = rec[6 * i + a];
    s[a] = rec[6 * i + 3 + a];
  }
}

__global__ void __launch_bounds__(NA_THREADS) k_na_count(int R, const float* __restrict__ rec, int64_t B,
                                                         double* __restrict__ scratch) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool v = false;
  if (i < B) {
    float q[3], s[3];
    na_rec(rec, i, q, s);
    DenseCell C;
    v = na_classify(0.5f * (float)R, R, q, s, C);
  }
  int n = __syncthreads_count(v);
  if (threadIdx.x == 0 && n) atomicAdd(&na_counters(scratch)->nvalid, n);
}

__device__ __forceinline__ int64_t na_vkey(int R, int i, int j, int k) {
  const int64_t n1 = R + 1;
  return (int64_t)i + n1 * ((int64_t)j + n1 * (int64_t)k);
}

__device__ __forceinline__ float na_lerp(float t, float a, float b) { return fmaf(t, b - a, a); }

// f and df/dt of Eq. 3 from the 8 corner values (corner k = dx + 2 dy + 4 dz):
// f by lerps, each gradient component by a bilinear blend of the exact
// cell-edge differences along its axis.
__device__ __forceinline__ void na_trilerp(const float d[8], const float t[3], float& f, float gt[3]) {
  float e00 = na_lerp(t[0], d[0], d[1]), e10 = na_lerp(t[0], d[2], d[3]);
  float e01 = na_lerp(t[0], d[4], d[5]), e11 = na_lerp(t[0], d[6], d[7]);
  f = na_lerp(t[2], na_lerp(t[1], e00, e10), na_lerp(t[1], e01, e11));
  gt[0] = na_lerp(t[2], na_lerp(t[1], d[1] - d[0], d[3] - d[2]), na_lerp(t[1], d[5] - d[4], d[7] - d[6]));
  gt[1] = na_lerp(t[2], na_lerp(t[0], d[2] - d[0], d[3] - d[1]), na_lerp(t[0], d[6] - d[4], d[7] - d[5]));
  gt[2] = na_lerp(t[1], na_lerp(t[0], d[4] - d[0], d[5] - d[1]), na_lerp(t[0], d[6] - d[2], d[7] - d[3]));
}

__device__ __forceinline__ void na_corners(const float* __restrict__ D, int R, const int c[3], float d[8]) {
#pragma unroll
  for (int k = 0; k < 8; ++k) d[k] = __ldg(D + na_vkey(R, c[0] + (k & 1), c[1] + ((k >> 1) & 1), c[2] + (k >> 2)));
}

__device__ __forceinline__ void na_scatter(float* __restrict__ grad, int R, const int c[3], const float t[3], float A,
                                           const float Gt[3]) {
  float wx[2] = {1.f - t[0], t[0]}, wy[2] = {1.f - t[1], t[1]}, wz[2] = {1.f - t[2], t[2]};
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    int dx = k & 1, dy = (k >> 1) & 1, dz = k >> 2;
    float sx = dx ? 1.f : -1.f, sy = dy ? 1.f : -1.f, sz = dz ? 1.f : -1.f;
    float wyz = wy[dy] * wz[dz];
    float val = A * wx[dx] * wyz + Gt[0] * sx * wyz + Gt[1] * wx[dx] * sy * wz[dz] + Gt[2] * wx[dx] * wy[dy] * sz;
    atomicAdd(grad + na_vkey(R, c[0] + dx, c[1] + dy, c[2] + dz), val);
  }
}

// One thread per record; block sums to the scratch rows; the last block to
// finish writes the loss slots (threadfence reduction) and re-arms the counter.
__global__ void __launch_bounds__(NA_THREADS) k_na_query(int R, const float* __restrict__ D,
                                                         const float* __restrict__ rec, int64_t B, float beta,
                                                         float gamma, float* __restrict__ grad,
                                                         double* __restrict__ scratch, float* __restrict__ loss) {
  const float half_r = 0.5f * (float)R;
  NACounters* cnt = na_counters(scratch);
  const int bv = *(volatile int*)&cnt->nvalid;
  const float w = bv > 0 ? 1.0f / (float)bv : 0.f;
  float sp = 0.f, sg = 0.f, ss = 0.f;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float q[3], s[3];
  DenseCell C;
  if (i < B) na_rec(rec, i, q, s);
  if (i < B && na_classify(half_r, R, q, s, C)) {
    float dq[8], ds[8], f, fs, gtq[3], gts[3];
    na_corners(D, R, C.cq, dq);
    na_corners(D, R, C.cs, ds);
    na_trilerp(dq, C.tq, f, gtq);
    na_trilerp(ds, C.ts, fs, gts);
    float g[3] = {gtq[0] * half_r, gtq[1] * half_r, gtq[2] * half_r};
    float gsv[3] = {gts[0] * half_r, gts[1] * half_r, gts[2] * half_r};
    float gl = sqrtf(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    float gls = sqrtf(gsv[0] * gsv[0] + gsv[1] * gsv[1] + gsv[2] * gsv[2]);
    float inv = 1.0f / fmaxf(gl, 1e-12f), invs = 1.0f / fmaxf(gls, 1e-12f);
    float n[3] = {g[0] * inv, g[1] * inv, g[2] * inv};
    float ns[3] = {gsv[0] * invs, gsv[1] * invs, gsv[2] * invs};
    float r[3] = {(q[0] - s[0]) - f * n[0], (q[1] - s[1]) - f * n[1], (q[2] - s[2]) - f * n[2]};
    float lp = sqrtf(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    // 1 - n . ns as |n - ns|^2 / 2 plus the deficits of non-unit vectors
    // (below the 1e-12 floor): no cancellation near cos = 1.
    const float e0 = n[0] - ns[0], e1 = n[1] - ns[1], e2 = n[2] - ns[2];
    float lgr = 0.5f * (e0 * e0 + e1 * e1 + e2 * e2);
    if (!(gl > 1e-12f)) lgr += 0.5f * (1.0f - (n[0] * n[0] + n[1] * n[1] + n[2] * n[2]));
    if (!(gls > 1e-12f)) lgr += 0.5f * (1.0f - (ns[0] * ns[0] + ns[1] * ns[1] + ns[2] * ns[2]));
    sp = lp;
    sg = lgr;
    ss = fabsf(fs);
    if (grad) {
      float ilp = lp > 0.f ? 1.0f / lp : 0.f;
      float u[3] = {r[0] * ilp, r[1] * ilp, r[2] * ilp};
      float un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
      float dn[3], dns[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        dn[a] = -w * f * u[a] - w * gamma * ns[a];
        dns[a] = -w * gamma * n[a];
      }
      float ndn = n[0] * dn[0] + n[1] * dn[1] + n[2] * dn[2];
      float nsdns = ns[0] * dns[0] + ns[1] * dns[1] + ns[2] * dns[2];
      float Gq[3], Gs[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        Gq[a] = (gl > 1e-12f ? (dn[a] - n[a] * ndn) : dn[a]) * inv * half_r;
        Gs[a] = (gls > 1e-12f ? (dns[a] - ns[a] * nsdns) : dns[a]) * invs * half_r;
      }
      float dfs = fs > 0.f ? w * beta : (fs < 0.f ? -w * beta : 0.f);
      na_scatter(grad, R, C.cq, C.tq, -w * un, Gq);
      na_scatter(grad, R, C.cs, C.ts, dfs, Gs);
    }
  }
  __shared__ float red[3][NA_THREADS / 32];
  sp = gp_warp_sum(sp);
  sg = gp_warp_sum(sg);
  ss = gp_warp_sum(ss);
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = sp;
    red[1][threadIdx.x >> 5] = sg;
    red[2][threadIdx.x >> 5] = ss;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0, c = 0;
    for (int k = 0; k < NA_THREADS / 32; ++k) {
      a += red[0][k];
      b += red[1][k];
      c += red[2][k];
    }
    double* row = scratch + (int64_t)blockIdx.x * 4;
    row[0] = a;
    row[1] = b;
    row[2] = c;
  }
  __shared__ int am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) am_last = (atomicAdd(&cnt->done, 1) == (int)gridDim.x - 1);
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  if (threadIdx.x == 0) {
    double t0 = 0, t1 = 0, t2 = 0;
    for (unsigned k = 0; k < gridDim.x; ++k) {
      t0 += __ldcg(scratch + (int64_t)k * 4 + 0);
      t1 += __ldcg(scratch + (int64_t)k * 4 + 1);
      t2 += __ldcg(scratch + (int64_t)k * 4 + 2);
    }
    double lp = bv > 0 ? t0 / bv : 0.0, lg = bv > 0 ? t1 / bv : 0.0, ls = bv > 0 ? t2 / bv : 0.0;
    loss[GP_LOSS_TOTAL] = (float)(lp + beta * ls + gamma * lg);
    loss[GP_LOSS_PULL] = (float)lp;
    loss[GP_LOSS_GRAD] = (float)lg;
    loss[GP_LOSS_SURF] = (float)ls;
    loss[GP_LOSS_TV] = 0.f;
    loss[GP_LOSS_BV] = (float)bv;
    loss[GP_LOSS_T] = 0.f;
    loss[7] = 0.f;
    cnt->done = 0;
  }
}

// Makes `dev` the calling thread's current device for the scope of the call
// and puts the caller's device back on every return path, so the call never
// leaves the thread on another device than it found it on.
struct DeviceScope {
  int prev = -1;
  cudaError_t err = cudaSuccess;
  explicit DeviceScope(int dev) {
    err = cudaGetDevice(&prev);
    if (err == cudaSuccess && prev != dev) err = cudaSetDevice(dev);
    if (err != cudaSuccess) cudaGetLastError();
  }
  ~DeviceScope() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// Device address of the scratch array on the current device (the context's,
// made current by the caller's DeviceScope); looked up once per device by the
// first call.
gp_status na_scratch(gp_ctx* ctx, double** out) {
  const int dev = ctx->device;
  if (dev < 0 || dev >= NA_MAX_DEVICES) return gp_fail(ctx, GP_ERR_ARG, "gp_step_dense_noalloc: device index >= 64");
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, gp_noalloc_scratch);
    if (e != cudaSuccess || !p) return gp_cuda_fail(ctx, e != cudaSuccess ? e : cudaErrorInvalidSymbol,
                                                    "gp_step_dense_noalloc: cudaGetSymbolAddress");
    g_scratch_addr[dev] = p;
  }
  *out = static_cast<double*>(g_scratch_addr[dev]);
  return GP_OK;
}

}  // namespace

extern "C" gp_status gp_step_dense_noalloc(gp_ctx* ctx, int32_t R, const float* d_dev, const float* rec_dev, int64_t B,
                                           const gp_loss_w* w, float* grad_dev, float* loss_dev) {
  if (!ctx) return GP_ERR_ARG;
  if (R < 8 || R > NA_MAX_R || (R & (R - 1)))
    return gp_fail(ctx, GP_ERR_ARG, "gp_step_dense_noalloc: R must be a power of two in [8, 1024]");
  if (B < 0 || B > NA_MAX_RECORDS)
    return gp_fail(ctx, GP_ERR_ARG,
                   "gp_step_dense_noalloc: B must be in [0, 1048576] (one scratch row per 256 records)");
  if (!d_dev || !loss_dev || !w || (B > 0 && !rec_dev))
    return gp_fail(ctx, GP_ERR_ARG, "gp_step_dense_noalloc: null pointer");
  DeviceScope scope(ctx->device);
  if (scope.err != cudaSuccess) return gp_cuda_fail(ctx, scope.err, "gp_step_dense_noalloc: cudaSetDevice");
  double* scratch = nullptr;
  gp_status st = na_scratch(ctx, &scratch);
  if (st) return st;
  cudaStream_t s = ctx->stream;
  const int64_t nv = (int64_t)(R + 1) * (R + 1) * (R + 1);
  GP_KERNEL(ctx, "k_na_clear", k_na_clear<<<1, 32, 0, s>>>(scratch));
  if (grad_dev) GP_KERNEL(ctx, "k_na_zero", k_na_zero<<<gp_blocks(nv, 256, 4096), 256, 0, s>>>(grad_dev, nv));
  const unsigned blocks = gp_blocks(B, NA_THREADS, NA_MAX_BLOCKS);
  if (B > 0) GP_KERNEL(ctx, "k_na_count", k_na_count<<<blocks, NA_THREADS, 0, s>>>(R, rec_dev, B, scratch));
  GP_KERNEL(ctx, "k_na_query", k_na_query<<<blocks, NA_THREADS, 0, s>>>(R, d_dev, rec_dev, B, w->beta, w->gamma,
                                                                        grad_dev, scratch, loss_dev));
  return GP_OK;
}
