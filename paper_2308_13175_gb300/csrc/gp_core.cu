// Context, errors and the device-wide scan used by the set-up paths.
#include <cstdio>
#include <string>

#include "gp_internal.cuh"

gp_status gp_fail(gp_ctx* ctx, gp_status st, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return st;
}

gp_status gp_cuda_fail(gp_ctx* ctx, cudaError_t e, const char* what) {
  std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();  // clear a sticky launch error where possible
  return gp_fail(ctx, GP_ERR_CUDA, msg);
}

extern "C" gp_status gp_create(gp_ctx** out, int device, void* stream) {
  if (!out) return GP_ERR_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return GP_ERR_ARG;
  }
  gp_ctx* ctx = new (std::nothrow) gp_ctx();
  if (!ctx) return GP_ERR_OOM;
  ctx->device = device;
  ctx->stream = (cudaStream_t)stream;
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return GP_ERR_CUDA;
  }
  *out = ctx;
  return GP_OK;
}

extern "C" gp_status gp_set_stream(gp_ctx* ctx, void* stream) {
  if (!ctx) return GP_ERR_ARG;
  ctx->stream = (cudaStream_t)stream;
  return GP_OK;
}

extern "C" void gp_destroy(gp_ctx* ctx) {
  if (!ctx) return;
  if (ctx->live_bands > 0) {
    ctx->destroy_pending = true;
    return;
  }
  gp_ctx_release(ctx);
}

void gp_ctx_release(gp_ctx* ctx) {
  for (auto& r : ctx->prof) {
    if (r.start) cudaEventDestroy(r.start);
    if (r.stop) cudaEventDestroy(r.stop);
  }
  for (auto e : ctx->event_pool) cudaEventDestroy(e);
  delete ctx;
}

// ---------------------------------------------------------------- tracing
static cudaEvent_t prof_event(gp_ctx* ctx) {
  if (!ctx->event_pool.empty()) {
    cudaEvent_t e = ctx->event_pool.back();
    ctx->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

void gp_prof_pre(gp_ctx* ctx) {
  if (!ctx->profiling) return;
  gp_prof_rec r{nullptr, prof_event(ctx), prof_event(ctx)};
  if (r.start) cudaEventRecord(r.start, ctx->stream);
  ctx->prof.push_back(r);
}

void gp_prof_post(gp_ctx* ctx, const char* name) {
  ++ctx->launches;
  if (!ctx->profiling || ctx->prof.empty()) return;
  gp_prof_rec& r = ctx->prof.back();
  r.name = name;
  if (r.stop) cudaEventRecord(r.stop, ctx->stream);
}

extern "C" gp_status gp_profile(gp_ctx* ctx, int enable) {
  if (!ctx) return GP_ERR_ARG;
  ctx->profiling = enable != 0;
  return GP_OK;
}

extern "C" int64_t gp_launch_count(const gp_ctx* ctx) { return ctx ? ctx->launches : -1; }

extern "C" gp_status gp_profile_read(gp_ctx* ctx, char* names, double* total_ms, int64_t* launches, int32_t max_kernels,
                                     int32_t* n_kernels) {
  if (!ctx) return GP_ERR_ARG;
  if (!n_kernels || (max_kernels > 0 && (!names || !total_ms || !launches)))
    return gp_fail(ctx, GP_ERR_ARG, "gp_profile_read: null pointer");
  GP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  std::vector<std::string> seen;
  std::vector<double> ms;
  std::vector<int64_t> cnt;
  for (auto& r : ctx->prof) {
    float t = 0.f;
    if (r.start && r.stop && r.name && cudaEventElapsedTime(&t, r.start, r.stop) == cudaSuccess) {
      size_t k = 0;
      while (k < seen.size() && seen[k] != r.name) ++k;
      if (k == seen.size()) {
        seen.emplace_back(r.name);
        ms.push_back(0.0);
        cnt.push_back(0);
      }
      ms[k] += t;
      cnt[k] += 1;
    } else {
      cudaGetLastError();
    }
    if (r.start) ctx->event_pool.push_back(r.start);
    if (r.stop) ctx->event_pool.push_back(r.stop);
  }
  ctx->prof.clear();
  *n_kernels = (int32_t)seen.size();
  for (size_t k = 0; k < seen.size() && (int32_t)k < max_kernels; ++k) {
    std::snprintf(names + 32 * k, 32, "%s", seen[k].c_str());
    total_ms[k] = ms[k];
    launches[k] = cnt[k];
  }
  return GP_OK;
}

extern "C" const char* gp_last_error(const gp_ctx* ctx) { return ctx ? ctx->err.c_str() : ""; }

extern "C" const char* gp_version(void) { return "gridpull-gb300 0.1"; }

// ------------------------------------------------------------------- scan
// Three-phase exclusive scan: per-block scans of SCAN_TILE elements, a
// recursive scan of the block totals, then a uniform add.
namespace {
constexpr int SCAN_THREADS = 512;
constexpr int SCAN_PER_THREAD = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_PER_THREAD;

__global__ void k_scan_tiles(int32_t* __restrict__ data, int64_t n, int32_t* __restrict__ tile_sums) {
  __shared__ int32_t warp_tot[SCAN_THREADS / 32];
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_PER_THREAD;
  int32_t v[SCAN_PER_THREAD];
  int32_t run = 0;
#pragma unroll
  for (int i = 0; i < SCAN_PER_THREAD; ++i) {
    int64_t idx = base + i;
    int32_t x = idx < n ? data[idx] : 0;
    v[i] = run;
    run += x;
  }
  // inclusive scan of per-thread totals across the block
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int32_t incl = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int32_t w = lane < SCAN_THREADS / 32 ? warp_tot[lane] : 0;
    int32_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int32_t y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < SCAN_THREADS / 32) warp_tot[lane] = wi - w;  // exclusive warp offsets
    if (lane == SCAN_THREADS / 32 - 1) tile_sums[blockIdx.x] = wi;
  }
  __syncthreads();
  int32_t off = warp_tot[wid] + (incl - run);
#pragma unroll
  for (int i = 0; i < SCAN_PER_THREAD; ++i) {
    int64_t idx = base + i;
    if (idx < n) data[idx] = v[i] + off;
  }
}

__global__ void k_scan_add(int32_t* __restrict__ data, int64_t n, const int32_t* __restrict__ tile_offs) {
  int64_t idx = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x;
  int32_t add = tile_offs[blockIdx.x];
#pragma unroll
  for (int i = 0; i < SCAN_PER_THREAD; ++i, idx += SCAN_THREADS)
    if (idx < n) data[idx] += add;
}

gp_status scan_rec(gp_ctx* ctx, int32_t* data, int64_t n) {
  int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  int32_t* sums = nullptr;
  gp_status st = gp_alloc(ctx, &sums, (size_t)tiles, "scan tile sums");
  if (st) return st;
  k_scan_tiles<<<(unsigned)tiles, SCAN_THREADS, 0, ctx->stream>>>(data, n, sums);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && tiles > 1) {
    st = scan_rec(ctx, sums, tiles);
    if (!st) {
      k_scan_add<<<(unsigned)tiles, SCAN_THREADS, 0, ctx->stream>>>(data, n, sums);
      e = cudaGetLastError();
    }
  }
  cudaStreamSynchronize(ctx->stream);
  cudaFree(sums);
  if (st) return st;
  if (e != cudaSuccess) return gp_cuda_fail(ctx, e, "scan kernels");
  return GP_OK;
}
}  // namespace

gp_status gp_exclusive_scan_i32(gp_ctx* ctx, int32_t* data, int64_t n, int64_t* total_host) {
  if (n <= 0) {
    if (total_host) *total_host = 0;
    return GP_OK;
  }
  int32_t last_in = 0, last_out = 0;
  GP_CUDA(ctx, cudaMemcpyAsync(&last_in, data + n - 1, 4, cudaMemcpyDeviceToHost, ctx->stream));
  GP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  gp_status st = scan_rec(ctx, data, n);
  if (st) return st;
  GP_CUDA(ctx, cudaMemcpyAsync(&last_out, data + n - 1, 4, cudaMemcpyDeviceToHost, ctx->stream));
  GP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (total_host) *total_host = (int64_t)last_out + last_in;
  return GP_OK;
}
