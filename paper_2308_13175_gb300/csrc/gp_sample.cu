// Query sampling (Sec. 3): every epoch visits the points in a fresh random
// order and draws one Gaussian query around each visited point, q = s_j +
// sigma_j * z.  The visiting order Pi_e is a 4-round Feistel bijection of
// [0, J) (cycle walking), keyed by (seed, epoch); z comes from Philox4x32-10
// at counter (k, epoch, 0, 0) through Box-Muller.  Both are counter based, so
// any pool position is generated on its own, in any order.
//
// A batch is the pool positions [first, first + count).  In position order the
// queries of a batch are scattered over the whole surface.  In spatial order
// (GP_SAMPLE_SPATIAL) the same queries are emitted grouped by their source
// point, the points taken in Morton order of their cells: position k
// belongs to point Pi_e(k mod J), so point j owns positions Pi_e^-1(j) + r J,
// and a three-kernel count / scan / emit pass lists them without a sort.
// Neighbouring outputs then lie close together, which is what the nearest-point
// search and the gather / scatter of the step profit from; the loss does not
// depend on the order.
#include <algorithm>

#include "gp_internal.cuh"

namespace {

constexpr int WALK_LIMIT = 4096;  // cycle walks end in < 4 rounds on average

__global__ void k_perm(int64_t J, int half, uint32_t epoch, uint32_t k0, uint32_t k1, int32_t* __restrict__ perm,
                       int32_t* __restrict__ inv, int32_t* __restrict__ err) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= J) return;
  uint32_t x = (uint32_t)p;
  int it = 0;
  do {
    x = gp_feistel(x, half, epoch, k0, k1);
  } while ((int64_t)x >= J && ++it < WALK_LIMIT);
  if ((int64_t)x >= J) {
    atomicOr(err, GP_EF_RANGE);
    x = (uint32_t)(x % (uint64_t)J);
  }
  perm[p] = (int32_t)x;
  inv[x] = (int32_t)p;
}

// Pi_e^-1 composed with the emission order, once per epoch, so that the
// per-step count and emit passes read it in their own order (coalesced)
// instead of gathering inv[order[u]].
__global__ void k_emit_slots(const int32_t* __restrict__ order, const int32_t* __restrict__ inv, int64_t J,
                             int32_t* __restrict__ slot) {
  int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u < J) slot[u] = inv[order[u]];
}

__device__ __forceinline__ void put_query(int64_t i, float3 v, int32_t j, int64_t k, float* __restrict__ q,
                                          int32_t* __restrict__ src, int32_t* __restrict__ pos) {
  q[3 * i + 0] = v.x;
  q[3 * i + 1] = v.y;
  q[3 * i + 2] = v.z;
  if (src) src[i] = j;
  if (pos) pos[i] = (int32_t)k;
}

__global__ void k_sample(const float* __restrict__ pts, const float* __restrict__ sigma,
                         const int32_t* __restrict__ perm, int64_t J, int64_t first, int64_t count, uint32_t epoch,
                         uint32_t k0, uint32_t k1, float* __restrict__ q, int32_t* __restrict__ src,
                         int32_t* __restrict__ pos) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  int64_t k = first + i;
  int32_t j = perm[k % J];
  put_query(i, gp_draw_query(pts, sigma, j, k, epoch, k0, k1), j, k, q, src, pos);
}

// The GP_ORDER_PER_THREAD consecutive emission slots of this thread in tile
// `tile` (an aligned 16-byte load where all are in range), 0 past J.
__device__ __forceinline__ void load_slots(const int32_t* __restrict__ eslot, int64_t J, int64_t t0,
                                           int32_t p[GP_ORDER_PER_THREAD]) {
  static_assert(GP_ORDER_PER_THREAD == 4, "one int4 of slots per thread");
  if (t0 + 3 < J) {
    const int4 v = __ldg(reinterpret_cast<const int4*>(eslot + t0));
    p[0] = v.x;
    p[1] = v.y;
    p[2] = v.z;
    p[3] = v.w;
  } else {
#pragma unroll
    for (int u = 0; u < 4; ++u) p[u] = t0 + u < J ? __ldg(eslot + t0 + u) : 0;
  }
}

// Pass 1: queries owned by each tile of GP_ORDER_TILE sorted points (four
// consecutive points per thread); only the tile totals are needed.
constexpr int COUNT_WARPS = GP_ORDER_THREADS / 32;

__global__ void __launch_bounds__(GP_ORDER_THREADS) k_order_count(const int32_t* __restrict__ eslot, int64_t J,
                                                                  int64_t first, int64_t last,
                                                                  int32_t* __restrict__ tiles, int64_t ntiles) {
  __shared__ int red[COUNT_WARPS];
  const int64_t t0 = (int64_t)blockIdx.x * GP_ORDER_TILE + (int64_t)threadIdx.x * GP_ORDER_PER_THREAD;
  int32_t p[GP_ORDER_PER_THREAD];
  load_slots(eslot, J, t0, p);
  int c = 0;
#pragma unroll
  for (int u = 0; u < GP_ORDER_PER_THREAD; ++u) {
    if (t0 + u < J) {
      int64_t r0;
      int n;
      owned_range(p[u], J, first, last, r0, n);
      c += n;
    }
  }
  c = gp_warp_sum_i(c);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0 && blockIdx.x < ntiles) {
    int total = 0;
    for (int w = 0; w < COUNT_WARPS; ++w) total += red[w];
    tiles[blockIdx.x] = total;
  }
}

// Pass 2: exclusive scan of the tile counts in place (one block, any length,
// GP_SCAN_PER_THREAD consecutive counts per thread and round).
__global__ void __launch_bounds__(GP_ORDER_THREADS) k_order_tiles(int32_t* __restrict__ tiles, int64_t ntiles) {
  gp_block_scan_inplace(tiles, ntiles);
}

// Pass 3: the tile's queries in order (by point, then replica) written from
// its offset.  The points' query counts are scanned into shared memory first;
// the queries are then drawn one per thread over the tile's compacted list
// (each finds its point by a binary search of the offsets), so that a warp's
// lanes all draw even when few of the tile's points own a query.  `splits`
// blocks share a tile (each scans it, then draws every splits-th round of
// its list), so that clouds of few tiles with many queries per point still
// fill the GPU.
__global__ void __launch_bounds__(GP_ORDER_THREADS) k_order_emit(
    const int32_t* __restrict__ order, const int32_t* __restrict__ eslot, const float4* __restrict__ epts,
    int64_t J, int64_t first, int64_t last, const int32_t* __restrict__ tiles, int splits,
    uint32_t epoch, uint32_t k0, uint32_t k1, float* __restrict__ q, int32_t* __restrict__ src,
    int32_t* __restrict__ pos, int32_t* __restrict__ err) {
  __shared__ int s_pre[GP_ORDER_TILE];  // first query of each point within the tile
  __shared__ int s_r0[GP_ORDER_TILE];   // its first replica
  __shared__ int s_p[GP_ORDER_TILE];    // its pool slot
  const int tile = blockIdx.x / splits, split = blockIdx.x % splits;
  const int64_t tile_base = (int64_t)tile * GP_ORDER_TILE;
  const int l0 = threadIdx.x * GP_ORDER_PER_THREAD;
  const int64_t n_out = last - first;
  int32_t p[GP_ORDER_PER_THREAD];
  load_slots(eslot, J, tile_base + l0, p);
  int nn[GP_ORDER_PER_THREAD], rr[GP_ORDER_PER_THREAD];
  int c = 0;
#pragma unroll
  for (int u = 0; u < GP_ORDER_PER_THREAD; ++u) {
    nn[u] = 0;
    rr[u] = 0;
    if (tile_base + l0 + u < J) {
      int64_t r0;
      owned_range(p[u], J, first, last, r0, nn[u]);
      rr[u] = (int)r0;
    }
    c += nn[u];
  }
  int excl;
  const int total = block_exclusive_scan(c, &excl);
#pragma unroll
  for (int u = 0; u < GP_ORDER_PER_THREAD; ++u) {
    s_pre[l0 + u] = excl;
    s_r0[l0 + u] = rr[u];
    s_p[l0 + u] = p[u];
    excl += nn[u];
  }
  __syncthreads();
  const int64_t out0 = tiles[tile];
  for (int i = split * GP_ORDER_THREADS + threadIdx.x; i < total; i += splits * GP_ORDER_THREADS) {
    // The last point t with s_pre[t] <= i (s_pre[0] = 0): the one owning query i.
    int t = 0;
#pragma unroll
    for (int step = GP_ORDER_TILE / 2; step > 0; step >>= 1)
      if (s_pre[t + step] <= i) t += step;
    const int64_t k = (int64_t)s_p[t] + (int64_t)(s_r0[t] + (i - s_pre[t])) * J;
    const int64_t o = out0 + i;
    if (o < 0 || o >= n_out) {  // only if Pi_e were not a bijection
      atomicOr(err, GP_EF_RANGE);
      continue;
    }
    const int64_t g = tile_base + t;
    put_query(o, gp_draw_query4(__ldg(epts + g), k, epoch, k0, k1), __ldg(order + g), k, q, src, pos);
  }
}

}  // namespace

gp_status gp_build_permutation(gp_band* b, uint64_t seed, uint32_t epoch) {
  if (b->perm_valid && b->perm_seed == seed && b->perm_epoch == epoch) return GP_OK;
  gp_ctx* ctx = b->ctx;
  int half = gp_feistel_bits(b->J) / 2;
  GP_KERNEL(ctx, "k_perm",
            k_perm<<<gp_blocks(b->J, 256), 256, 0, ctx->stream>>>(b->J, half, epoch, (uint32_t)seed,
                                                                  (uint32_t)(seed >> 32), b->perm, b->inv_perm,
                                                                  b->dev_ints + GP_DI_ERROR));
  if (b->emit_order)
    GP_KERNEL(ctx, "k_emit_slots",
              k_emit_slots<<<gp_blocks(b->J, 256), 256, 0, ctx->stream>>>(b->emit_order, b->inv_perm, b->J,
                                                                         b->emit_slot));
  b->perm_valid = true;
  b->perm_seed = seed;
  b->perm_epoch = epoch;
  return GP_OK;
}

extern "C" gp_status gp_sample(gp_band* b, uint64_t seed, uint32_t epoch, int64_t Q, int64_t first, int64_t count,
                               uint32_t flags, float* q_dev, int32_t* src_dev, int32_t* pos_dev) {
  if (!b) return GP_ERR_ARG;
  gp_ctx* ctx = b->ctx;
  if (Q < 0 || Q >= (int64_t(1) << 31) || first < 0 || count < 0 || first + count > Q)
    return gp_fail(ctx, GP_ERR_ARG, "gp_sample: need 0 <= first, first + count <= Q < 2^31");
  if (count == 0) return GP_OK;
  if (!q_dev) return gp_fail(ctx, GP_ERR_ARG, "gp_sample: null output");
  if (!b->sigma) return gp_fail(ctx, GP_ERR_STATE, "gp_sample: band built with knn_k = 0 (no sigma)");
  gp_status st = gp_build_permutation(b, seed, epoch);
  if (st) return st;
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  if (!(flags & GP_SAMPLE_SPATIAL)) {
    GP_KERNEL(ctx, "k_sample",
              k_sample<<<gp_blocks(count, 256), 256, 0, ctx->stream>>>(b->pts, b->sigma, b->perm, b->J, first, count,
                                                                      epoch, k0, k1, q_dev, src_dev, pos_dev));
    return GP_OK;
  }
  const int64_t J = b->J, last = first + count;
  const int64_t ntiles = (J + GP_ORDER_TILE - 1) / GP_ORDER_TILE;
  GP_KERNEL(ctx, "k_order_count",
            k_order_count<<<(unsigned)ntiles, GP_ORDER_THREADS, 0, ctx->stream>>>(b->emit_slot, J, first, last,
                                                                                 b->order_tiles, ntiles));
  GP_KERNEL(ctx, "k_order_tiles", k_order_tiles<<<1, GP_ORDER_THREADS, 0, ctx->stream>>>(b->order_tiles, ntiles));
  // Blocks per tile: enough for about four per SM, at most one per round of
  // GP_ORDER_THREADS queries of an average tile.
  const int64_t per_tile = (count + ntiles - 1) / ntiles;
  int64_t splits = (4 * (int64_t)ctx->num_sms + ntiles - 1) / ntiles;
  splits = std::min<int64_t>(splits, (per_tile + GP_ORDER_THREADS - 1) / GP_ORDER_THREADS);
  splits = std::max<int64_t>(1, std::min<int64_t>(splits, 64));
  GP_KERNEL(ctx, "k_order_emit",
            k_order_emit<<<(unsigned)(ntiles * splits), GP_ORDER_THREADS, 0, ctx->stream>>>(
                b->emit_order, b->emit_slot, b->emit_pts, J, first, last, b->order_tiles, (int)splits, epoch, k0,
                k1, q_dev, src_dev, pos_dev, b->dev_ints + GP_DI_ERROR));
  return GP_OK;
}
