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

// Pass 1: queries owned by each tile of sorted points (GP_ORDER_TILE points,
// one per thread), TPB tiles per block; only the tile totals are needed, so
// each is a warp-sum reduction with one barrier for all of them.  Four tiles
// per block pay on large clouds (10 M points: 53 -> 37 us); on small ones the
// grid would be too small, so they take one.
constexpr int COUNT_WARPS = GP_ORDER_THREADS / 32;

template <int COUNT_TILES>
__global__ void __launch_bounds__(GP_ORDER_THREADS) k_order_count(const int32_t* __restrict__ eslot, int64_t J,
                                                                  int64_t first, int64_t last,
                                                                  int32_t* __restrict__ tiles, int64_t ntiles) {
  static_assert(GP_ORDER_PER_THREAD == 1, "one point per thread and tile");
  __shared__ int red[COUNT_TILES][COUNT_WARPS];
  const int64_t tile0 = (int64_t)blockIdx.x * COUNT_TILES;
#pragma unroll
  for (int k = 0; k < COUNT_TILES; ++k) {
    const int64_t t = (tile0 + k) * GP_ORDER_TILE + threadIdx.x;
    int c = 0;
    if (t < J) {
      int64_t r0;
      owned_range(eslot[t], J, first, last, r0, c);
    }
    c = gp_warp_sum_i(c);
    if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = c;
  }
  __syncthreads();
  if (threadIdx.x < COUNT_TILES && tile0 + threadIdx.x < ntiles) {
    int total = 0;
    for (int w = 0; w < COUNT_WARPS; ++w) total += red[threadIdx.x][w];
    tiles[tile0 + threadIdx.x] = total;
  }
}

// Pass 2: exclusive scan of the tile counts in place (one block, any length,
// GP_SCAN_PER_THREAD consecutive counts per thread and round).
__global__ void __launch_bounds__(GP_ORDER_THREADS) k_order_tiles(int32_t* __restrict__ tiles, int64_t ntiles) {
  gp_block_scan_inplace(tiles, ntiles);
}

// Pass 3: every sorted point writes its queries at its offset.
__global__ void __launch_bounds__(GP_ORDER_THREADS) k_order_emit(
    const int32_t* __restrict__ order, const int32_t* __restrict__ eslot, const float4* __restrict__ epts,
    int64_t J, int64_t first, int64_t last, const int32_t* __restrict__ tiles,
    uint32_t epoch, uint32_t k0, uint32_t k1, float* __restrict__ q, int32_t* __restrict__ src,
    int32_t* __restrict__ pos, int32_t* __restrict__ err) {
  int64_t base = (int64_t)blockIdx.x * GP_ORDER_TILE + (int64_t)threadIdx.x * GP_ORDER_PER_THREAD;
  const int64_t n_out = last - first;
  int jj[GP_ORDER_PER_THREAD], nn[GP_ORDER_PER_THREAD];
  int64_t rr[GP_ORDER_PER_THREAD], pp[GP_ORDER_PER_THREAD];
  int c = 0;
#pragma unroll
  for (int u = 0; u < GP_ORDER_PER_THREAD; ++u) {
    int64_t t = base + u;
    nn[u] = 0;
    jj[u] = 0;
    pp[u] = 0;
    rr[u] = 0;
    if (t < J) {
      pp[u] = eslot[t];
      owned_range(pp[u], J, first, last, rr[u], nn[u]);
      if (nn[u]) jj[u] = order[t];
      c += nn[u];
    }
  }
  int excl;
  block_exclusive_scan(c, &excl);
  int64_t out = (int64_t)tiles[blockIdx.x] + excl;
#pragma unroll
  for (int u = 0; u < GP_ORDER_PER_THREAD; ++u) {
    for (int r = 0; r < nn[u]; ++r) {
      int64_t k = pp[u] + (rr[u] + r) * J;
      int64_t i = out++;
      if (i < 0 || i >= n_out) {  // only if Pi_e were not a bijection
        atomicOr(err, GP_EF_RANGE);
        continue;
      }
      put_query(i, gp_draw_query4(epts[base + u], k, epoch, k0, k1), jj[u], k, q, src, pos);
    }
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
            (ntiles >= 8 * (int64_t)ctx->num_sms
                 ? k_order_count<4><<<(unsigned)((ntiles + 3) / 4), GP_ORDER_THREADS, 0, ctx->stream>>>(
                       b->emit_slot, J, first, last, b->order_tiles, ntiles)
                 : k_order_count<1><<<(unsigned)ntiles, GP_ORDER_THREADS, 0, ctx->stream>>>(
                       b->emit_slot, J, first, last, b->order_tiles, ntiles)));
  GP_KERNEL(ctx, "k_order_tiles", k_order_tiles<<<1, GP_ORDER_THREADS, 0, ctx->stream>>>(b->order_tiles, ntiles));
  GP_KERNEL(ctx, "k_order_emit",
            k_order_emit<<<(unsigned)ntiles, GP_ORDER_THREADS, 0, ctx->stream>>>(
                b->emit_order, b->emit_slot, b->emit_pts, J, first, last, b->order_tiles, epoch, k0, k1, q_dev,
                src_dev, pos_dev, b->dev_ints + GP_DI_ERROR));
  return GP_OK;
}
