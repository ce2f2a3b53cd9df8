// Query sampling (Sec. 3): every epoch visits the points in a fresh random
// order and draws one Gaussian query around each visited point, q = s_j +
// sigma_j * z.  The visiting order Pi_e is a 4-round Feistel bijection of
// [0, J) (cycle walking), keyed by (seed, epoch); z comes from Philox4x32-10
// at counter (k, epoch, 0, 0) through Box-Muller.  Both are counter based, so
// any pool position is generated on its own, in any order.
#include "gp_internal.cuh"

namespace {

constexpr int WALK_LIMIT = 4096;  // cycle walks end in < 4 rounds on average

__global__ void k_perm(int64_t J, int half, uint32_t epoch, uint32_t k0, uint32_t k1, int32_t* __restrict__ perm,
                       int32_t* __restrict__ err) {
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
}

__global__ void k_sample(const float* __restrict__ pts, const float* __restrict__ sigma,
                         const int32_t* __restrict__ perm, int64_t J, int64_t first, int64_t count, uint32_t epoch,
                         uint32_t k0, uint32_t k1, float* __restrict__ q, int32_t* __restrict__ src) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  int64_t k = first + i;
  int32_t j = perm[k % J];
  float3 z = gp_box_muller3(gp_philox((uint32_t)k, epoch, 0u, 0u, k0, k1));
  float sg = sigma[j];
  q[3 * i + 0] = pts[3 * (int64_t)j + 0] + sg * z.x;
  q[3 * i + 1] = pts[3 * (int64_t)j + 1] + sg * z.y;
  q[3 * i + 2] = pts[3 * (int64_t)j + 2] + sg * z.z;
  if (src) src[i] = j;
}

}  // namespace

gp_status gp_build_permutation(gp_band* b, uint64_t seed, uint32_t epoch) {
  if (b->perm_valid && b->perm_seed == seed && b->perm_epoch == epoch) return GP_OK;
  gp_ctx* ctx = b->ctx;
  int half = gp_feistel_bits(b->J) / 2;
  GP_KERNEL(ctx, "k_perm", k_perm<<<gp_blocks(b->J, 256), 256, 0, ctx->stream>>>(b->J, half, epoch, (uint32_t)seed, (uint32_t)(seed >> 32),
                                                        b->perm, b->dev_ints + GP_DI_ERROR));
  b->perm_valid = true;
  b->perm_seed = seed;
  b->perm_epoch = epoch;
  return GP_OK;
}

extern "C" gp_status gp_sample(gp_band* b, uint64_t seed, uint32_t epoch, int64_t Q, int64_t first, int64_t count,
                               float* q_dev, int32_t* src_dev) {
  if (!b) return GP_ERR_ARG;
  gp_ctx* ctx = b->ctx;
  if (Q < 0 || Q >= (int64_t(1) << 31) || first < 0 || count < 0 || first + count > Q)
    return gp_fail(ctx, GP_ERR_ARG, "gp_sample: need 0 <= first, first + count <= Q < 2^31");
  if (count == 0) return GP_OK;
  if (!q_dev) return gp_fail(ctx, GP_ERR_ARG, "gp_sample: null output");
  if (!b->sigma) return gp_fail(ctx, GP_ERR_STATE, "gp_sample: band built with knn_k = 0 (no sigma)");
  gp_status st = gp_build_permutation(b, seed, epoch);
  if (st) return st;
  GP_KERNEL(ctx, "k_sample", k_sample<<<gp_blocks(count, 256), 256, 0, ctx->stream>>>(
                                 b->pts, b->sigma, b->perm, b->J, first, count, epoch, (uint32_t)seed,
                                 (uint32_t)(seed >> 32), q_dev, src_dev));
  return GP_OK;
}
