// gp_multi: many clouds of uneven size fitted together, one launch per stage
// for all of them.
//
// Each cloud keeps its own band (grid, bricks, values, Adam moments, point
// cell list, sigma).  Every stage of a fitting step - the epoch's order Pi_e,
// the batch's queries, nearest points, the L_TV sweep, the fused query forward
// + backward, Adam - is one persistent launch (a few blocks per SM) over a
// flattened work list of tiles.  A tile belongs to one cloud (a run of its
// records, of its points, or one of its bricks), so a block always knows the
// band it works on and clouds of any size mix in one launch.
//
// The step counter t lives on the device.  Every kernel derives its cloud's
// epoch, batch, learning rate and bias corrections from it and the last kernel
// advances it, so a step takes the same host arguments every time and can be
// captured once in a CUDA graph and replayed.
//
// Per cloud k at step t: nb_k = ceil(Q_k / B_k) batches per epoch, epoch
// e = t / nb_k, batch b = t mod nb_k = pool positions [b B_k, min((b+1) B_k,
// Q_k)) of Pi_e (Sec. 3 sampling, as gp_sample); the random streams of cloud k
// are keyed by seed + k.  Record slots past a short last batch hold NaN
// queries, which no stage counts.  Loss slots are written per cloud (n x 8
// floats, the gp_step layout).
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "gp_internal.cuh"
#include "gp_nn_device.cuh"
#include "gp_step_device.cuh"

namespace {

constexpr int PT_TILE = GP_ORDER_THREADS;  // points per point tile (one per thread)
constexpr int WALK_LIMIT = 4096;

struct MShape {
  Grid G;  // step view of the band
  NNGrid nn;
  float* D;
  float* m;
  float* v;
  float* grad;  // this cloud's slice of the gradient buffer
  unsigned long long* acc;  // its slice of the fixed-point query sums (deterministic multis), else null
  const float* pts;
  const float* sigma;
  const float* normals;
  const int32_t* order;  // points in Morton order of their cells
  const float4* epts;    // their (x, y, z, sigma)
  int32_t* perm;         // this cloud's slice of the multi's Pi_e
  int32_t* inv;          // and of Pi_e^-1
  int32_t* eslot;        // and of Pi_e^-1(order[u]), the pool slot of the u-th emitted point
  const int32_t* coord;
  const int32_t* nbr;  // 27 neighbour slots per brick
  const int32_t* active;
  int64_t J, Q, B, nb_epoch, V_tv;
  int64_t rec_off;  // first record slot of this cloud
  int64_t tile0;    // index of its first point tile
};

struct MTile {
  int32_t shape;
  int32_t first;  // record / point offset within the cloud, or brick index
};

struct MBatch {
  int64_t epoch, first, count;
};

__device__ __forceinline__ MBatch batch_at(const MShape& S, int64_t t) {
  MBatch b;
  b.epoch = t / S.nb_epoch;
  b.first = (t % S.nb_epoch) * S.B;
  b.count = min(S.B, S.Q - b.first);
  return b;
}

__device__ __forceinline__ void seed_key(uint64_t seed, int k, uint32_t& k0, uint32_t& k1) {
  const uint64_t s = seed + (uint64_t)k;
  k0 = (uint32_t)s;
  k1 = (uint32_t)(s >> 32);
}

__device__ __forceinline__ void put_nan_query(int64_t slot, float* __restrict__ q, int32_t* __restrict__ src) {
  const float nan = __int_as_float(0x7fc00000);
  q[3 * slot] = nan;
  q[3 * slot + 1] = nan;
  q[3 * slot + 2] = nan;
  src[slot] = -1;
}

__device__ __forceinline__ void put_query(int64_t slot, float3 v, int32_t j, float* __restrict__ q,
                                          int32_t* __restrict__ src) {
  q[3 * slot] = v.x;
  q[3 * slot + 1] = v.y;
  q[3 * slot + 2] = v.z;
  src[slot] = j;
}

// Pi_e and its inverse, for the clouds whose stored order is not that of the
// current epoch (k_m_finish records the epoch once the step is done).
__global__ void __launch_bounds__(PT_TILE) k_m_perm(const MShape* __restrict__ shapes,
                                                    const MTile* __restrict__ tiles, int64_t ntiles,
                                                    const int64_t* __restrict__ t_dev,
                                                    const int64_t* __restrict__ perm_epoch, uint64_t seed,
                                                    int32_t* __restrict__ err) {
  const int64_t t = *t_dev;
  for (int64_t ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
    const MTile tl = tiles[ti];
    const MShape& S = shapes[tl.shape];
    if (perm_epoch[tl.shape] == t / S.nb_epoch) continue;
    const int64_t p = (int64_t)tl.first + threadIdx.x;
    if (p >= S.J) continue;
    uint32_t k0, k1;
    seed_key(seed, tl.shape, k0, k1);
    const int half = gp_feistel_bits(S.J) / 2;
    const uint32_t epoch = (uint32_t)(t / S.nb_epoch);
    uint32_t x = (uint32_t)p;
    int it = 0;
    do {
      x = gp_feistel(x, half, epoch, k0, k1);
    } while ((int64_t)x >= S.J && ++it < WALK_LIMIT);
    if ((int64_t)x >= S.J) {
      atomicOr(err, GP_EF_RANGE);
      x = (uint32_t)(x % (uint64_t)S.J);
    }
    S.perm[p] = (int32_t)x;
    S.inv[x] = (int32_t)p;
  }
}

// Pi_e^-1 in emission order, for the clouds whose order was just rebuilt.
__global__ void __launch_bounds__(PT_TILE) k_m_emit_slots(const MShape* __restrict__ shapes,
                                                          const MTile* __restrict__ tiles, int64_t ntiles,
                                                          const int64_t* __restrict__ t_dev,
                                                          const int64_t* __restrict__ perm_epoch) {
  const int64_t t = *t_dev;
  for (int64_t ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
    const MTile tl = tiles[ti];
    const MShape& S = shapes[tl.shape];
    if (perm_epoch[tl.shape] == t / S.nb_epoch) continue;
    const int64_t u = (int64_t)tl.first + threadIdx.x;
    if (u < S.J) S.eslot[u] = S.inv[S.order[u]];
  }
}

// Position order: record slot i of cloud k holds pool position first + i.
__global__ void k_m_sample(const MShape* __restrict__ shapes, const MTile* __restrict__ tiles, int64_t ntiles,
                           int tq, const int64_t* __restrict__ t_dev, uint64_t seed, float* __restrict__ q,
                           int32_t* __restrict__ src) {
  const int64_t t = *t_dev;
  for (int64_t ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
    const MTile tl = tiles[ti];
    const MShape& S = shapes[tl.shape];
    const MBatch bt = batch_at(S, t);
    uint32_t k0, k1;
    seed_key(seed, tl.shape, k0, k1);
    const int64_t end = min((int64_t)tl.first + tq, S.B);
    for (int64_t i = (int64_t)tl.first + threadIdx.x; i < end; i += blockDim.x) {
      const int64_t slot = S.rec_off + i;
      if (i < bt.count) {
        const int64_t k = bt.first + i;
        const int32_t j = S.perm[k % S.J];
        put_query(slot, gp_draw_query(S.pts, S.sigma, j, k, (uint32_t)bt.epoch, k0, k1), j, q, src);
      } else {
        put_nan_query(slot, q, src);
      }
    }
  }
}

// Spatial order, pass 1: queries of the batch owned by each point tile (the
// cloud's points in Morton order; point j owns positions Pi_e^-1(j) + r J).
__global__ void __launch_bounds__(PT_TILE) k_m_order_count(const MShape* __restrict__ shapes,
                                                           const MTile* __restrict__ tiles, int64_t ntiles,
                                                           const int64_t* __restrict__ t_dev,
                                                           int32_t* __restrict__ counts) {
  const int64_t t = *t_dev;
  for (int64_t ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
    const MTile tl = tiles[ti];
    const MShape& S = shapes[tl.shape];
    const MBatch bt = batch_at(S, t);
    const int64_t u = (int64_t)tl.first + threadIdx.x;
    int c = 0;
    if (u < S.J) {
      int64_t r0;
      owned_range(S.eslot[u], S.J, bt.first, bt.first + bt.count, r0, c);
    }
    int excl;
    const int total = block_exclusive_scan(c, &excl);
    if (threadIdx.x == 0) counts[ti] = total;
  }
}

// Pass 2: exclusive scan of the tile counts over all clouds (one block).
__global__ void __launch_bounds__(GP_ORDER_THREADS) k_m_order_scan(int32_t* __restrict__ counts, int64_t ntiles) {
  gp_block_scan_inplace(counts, ntiles);
}

// Pass 3: every point writes its queries at its offset within the cloud's
// batch; the first tile of a cloud also pads a short batch with NaN queries.
__global__ void __launch_bounds__(PT_TILE) k_m_order_emit(const MShape* __restrict__ shapes,
                                                          const MTile* __restrict__ tiles, int64_t ntiles,
                                                          const int64_t* __restrict__ t_dev, uint64_t seed,
                                                          const int32_t* __restrict__ counts, float* __restrict__ q,
                                                          int32_t* __restrict__ src, int32_t* __restrict__ err) {
  const int64_t t = *t_dev;
  for (int64_t ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
    const MTile tl = tiles[ti];
    const MShape& S = shapes[tl.shape];
    const MBatch bt = batch_at(S, t);
    uint32_t k0, k1;
    seed_key(seed, tl.shape, k0, k1);
    const int64_t u = (int64_t)tl.first + threadIdx.x;
    int n = 0, j = 0;
    int64_t r0 = 0, p = 0;
    if (u < S.J) {
      p = S.eslot[u];
      owned_range(p, S.J, bt.first, bt.first + bt.count, r0, n);
      if (n) j = S.order[u];
    }
    int excl;
    block_exclusive_scan(n, &excl);
    int64_t out = (int64_t)counts[ti] - counts[S.tile0] + excl;
    for (int r = 0; r < n; ++r) {
      const int64_t k = p + (r0 + r) * S.J;
      const int64_t i = out++;
      if (i < 0 || i >= bt.count) {  // only if Pi_e were not a bijection
        atomicOr(err, GP_EF_RANGE);
        continue;
      }
      put_query(S.rec_off + i, gp_draw_query4(S.epts[u], k, (uint32_t)bt.epoch, k0, k1), j, q, src);
    }
    if (ti == S.tile0)
      for (int64_t i = bt.count + threadIdx.x; i < S.B; i += blockDim.x) put_nan_query(S.rec_off + i, q, src);
  }
}

// Nearest point of every query (seeded by its source point and the foot of q
// on the source's tangent plane), the step records, and the per-cloud count of
// valid records.
__global__ void __launch_bounds__(512) k_m_nn(const MShape* __restrict__ shapes, const MTile* __restrict__ tiles,
                                              int64_t ntiles, int tq, const float* __restrict__ q,
                                              const int32_t* __restrict__ src, float* __restrict__ rec,
                                              int32_t* __restrict__ nvalid) {
  for (int64_t ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
    const MTile tl = tiles[ti];
    const MShape& S = shapes[tl.shape];
    const int64_t end = min((int64_t)tl.first + tq, S.B);
    for (int64_t i0 = tl.first; i0 < end; i0 += blockDim.x) {
      const int64_t i = i0 + threadIdx.x;
      bool valid = false;
      if (i < end) {
        const int64_t slot = S.rec_off + i;
        float qq[3] = {q[3 * slot], q[3 * slot + 1], q[3 * slot + 2]};
        int best = -1;
        if (nn_query_ok(qq)) {
          int c[3] = {nn_cell(qq[0], S.nn), nn_cell(qq[1], S.nn), nn_cell(qq[2], S.nn)};
          NNState st{INFINITY, INFINITY, INFINITY, 0x7fffffff};
          const int32_t* hint = src + S.rec_off;
          nn_seed(st, qq, hint, i, S.J, S.pts);
          if (st.b1 < INFINITY) nn_seed_foot(st, qq, hint, i, S.J, S.pts, S.normals, S.nn);
          best = nn_thread_search(qq, c, S.nn, nn_margin(qq), st);
        }
        float s3[3];
        if (best >= 0) {
          s3[0] = S.pts[3 * (int64_t)best];
          s3[1] = S.pts[3 * (int64_t)best + 1];
          s3[2] = S.pts[3 * (int64_t)best + 2];
          Cells C;
          valid = classify(S.G, qq, s3, C);
        } else {
          s3[0] = s3[1] = s3[2] = __int_as_float(0x7fc00000);
        }
        rec[6 * slot + 0] = qq[0];
        rec[6 * slot + 1] = qq[1];
        rec[6 * slot + 2] = qq[2];
        rec[6 * slot + 3] = s3[0];
        rec[6 * slot + 4] = s3[1];
        rec[6 * slot + 5] = s3[2];
      }
      const int n = __syncthreads_count(valid);
      if (threadIdx.x == 0 && n) atomicAdd(nvalid + tl.shape, n);
    }
  }
}

// Sum over the block (any multiple of 32 threads up to 1024); the result is
// valid in thread 0.  Called by every thread of the block.
__device__ __forceinline__ float block_sum(float v, float* red) {
  v = gp_warp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float s = 0.f;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  return s;
}

// Loss sums of the deterministic mode: a block's float sum as an integer in
// units of 2^-24 (integer additions do not depend on their order).
__device__ __forceinline__ long long loss_fixed(float x) { return __double2ll_rn((double)x * 16777216.0); }

struct MultiTvSrc {
  const MShape* shapes;
  const MTile* tiles;
  __device__ __forceinline__ TvBrick brick(int64_t ti) const {
    const MTile tl = tiles[ti];
    const MShape& S = shapes[tl.shape];
    const int32_t* c = S.coord + 3 * (int64_t)tl.first;
    return TvBrick{S.G.D, S.G.masks, S.nbr + 27 * (int64_t)tl.first, S.G.R, __ldg(c) * 8, __ldg(c + 1) * 8,
                   __ldg(c + 2) * 8};
  }
};

// L_TV sweep: one brick per tile (TV_SWEEP_THREADS threads, pipelined across
// the block's tiles); the gradient is overwritten at every slot of every
// brick; the TV sums go to each cloud's slot 3, one atomic per run of tiles of
// the same cloud.
// DET: the query pass ran first into the fixed-point sums (its contributions
// already scaled by 1/B_v of the cloud), which are folded in here and
// cleared; the TV sums go to the integer loss sums.
template <bool DET>
__global__ void __launch_bounds__(TV_SWEEP_THREADS, TV_BLOCKS_PER_SM) k_m_tv(const MShape* __restrict__ shapes,
                                                           const MTile* __restrict__ tiles, int64_t ntiles,
                                                           float alpha, double* __restrict__ sums,
                                                           long long* __restrict__ isums) {
  __shared__ TvShared sh;
  __shared__ float red[32];
  int cur = -1;
  float acc = 0.f;
  auto flush = [&]() {
    const float bs = block_sum(acc, red);
    if (threadIdx.x == 0 && bs != 0.f) {
      if (DET)
        atomicAdd((unsigned long long*)(isums + 4 * cur + 3), (unsigned long long)loss_fixed(bs));
      else
        atomicAdd(sums + 4 * cur + 3, (double)bs);
    }
    acc = 0.f;
  };
  // DET: this thread's two vertices of each brick (those tv_gather hands
  // it) have their fixed-point sums loaded at the top of the brick's
  // iteration, under its halo copies; only trainable vertices can hold any.
  const int tt = threadIdx.x;
  const int lv0 = (tt & 7) + 16 * ((tt >> 3) & 3) + 64 * (tt >> 5);
  long long phi[2] = {0, 0}, plo[2] = {0, 0};
  bool ptr[2] = {false, false};
  auto out = [&](int64_t ti, int l0, float g0, int l1, float g1, float ts) {
        const MTile tl = tiles[ti];
        const MShape& S = shapes[tl.shape];
        if (tl.shape != cur) {
          if (cur >= 0) flush();
          cur = tl.shape;
        }
        acc += ts;
        const float tv_scale = S.V_tv > 0 ? alpha / (float)S.V_tv : 0.f;
        float* gp = S.grad + (int64_t)tl.first * 512;
        if (DET) {
          unsigned long long* ap = S.acc + 2 * (int64_t)tl.first * 512;
          const int ls[2] = {l0, l1};
          const float gs[2] = {g0, g1};
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            float g = tv_scale * gs[k];
            if (ptr[k]) {
              ap[2 * ls[k]] = 0ull;
              ap[2 * ls[k] + 1] = 0ull;
              const float qv = __fmaf_rn(__ll2float_rn(phi[k]), 9.5367431640625e-07f,
                                         __ll2float_rn(plo[k]) * 8.673617379884035e-19f);
              g = __fadd_rn(qv, g);
            }
            gp[ls[k]] = g;
          }
        } else {
          gp[l0] = tv_scale * g0;
          gp[l1] = tv_scale * g1;
        }
      };
  auto pre = [&](int64_t ti) {
        const MTile tl = tiles[ti];
        const MShape& S = shapes[tl.shape];
        const unsigned long long* ap = S.acc + 2 * (int64_t)tl.first * 512;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const int l = lv0 + 8 * k;
          const uint32_t word = __ldg(S.G.masks + (int64_t)tl.first * 48 + 16 + (l >> 5));
          ptr[k] = (word >> (l & 31)) & 1u;
          if (ptr[k]) {
            phi[k] = (long long)ap[2 * l];
            plo[k] = (long long)ap[2 * l + 1];
          }
        }
      };
  if constexpr (DET)
    tv_sweep(MultiTvSrc{shapes, tiles}, blockIdx.x, gridDim.x, ntiles, sh, out, pre);
  else
    tv_sweep(MultiTvSrc{shapes, tiles}, blockIdx.x, gridDim.x, ntiles, sh, out);
  if (cur >= 0) flush();
}

// Fused forward + hand-written backward of every valid record (the gp_step
// record code), loss sums per cloud.  At most 256 threads, so that the record
// code keeps its registers (at 512 it would spill).
template <bool DET>
__global__ void __launch_bounds__(256) k_m_query(const MShape* __restrict__ shapes, const MTile* __restrict__ tiles,
                                                 int64_t ntiles, int tq, const float* __restrict__ rec,
                                                 const int32_t* __restrict__ nvalid, float beta, float gamma,
                                                 double* __restrict__ sums, long long* __restrict__ isums,
                                                 int32_t* __restrict__ err) {
  __shared__ float red[32];
  // Loss sums stay in registers over a block's run of tiles of one cloud and
  // are reduced over the block when the cloud changes and at the end.
  int cur = -1;
  float sp = 0.f, sg = 0.f, ss = 0.f;
  auto flush = [&]() {
    const float a = block_sum(sp, red);
    const float b = block_sum(sg, red);
    const float c = block_sum(ss, red);
    if (threadIdx.x == 0) {
      if (DET) {
        unsigned long long* is = (unsigned long long*)(isums + 4 * cur);
        if (a != 0.f) atomicAdd(is + 0, (unsigned long long)loss_fixed(a));
        if (b != 0.f) atomicAdd(is + 1, (unsigned long long)loss_fixed(b));
        if (c != 0.f) atomicAdd(is + 2, (unsigned long long)loss_fixed(c));
      } else {
        if (a != 0.f) atomicAdd(sums + 4 * cur + 0, (double)a);
        if (b != 0.f) atomicAdd(sums + 4 * cur + 1, (double)b);
        if (c != 0.f) atomicAdd(sums + 4 * cur + 2, (double)c);
      }
    }
    sp = sg = ss = 0.f;
  };
  for (int64_t ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
    const MTile tl = tiles[ti];
    const MShape& S = shapes[tl.shape];
    if (tl.shape != cur) {
      if (cur >= 0) flush();
      cur = tl.shape;
    }
    const int bv = nvalid[tl.shape];
    const float w = bv > 0 ? 1.0f / (float)bv : 0.f;  // also for the fixed-point sums (taken pre-scaled)
    const int64_t end = min((int64_t)tl.first + tq, S.B);
    for (int64_t i = (int64_t)tl.first + threadIdx.x; i < end; i += blockDim.x) {
      float qq[3], s3[3];
      load_rec(rec, S.rec_off + i, qq, s3);
      query_record<DET, true>(S.G, qq, s3, w, beta, gamma, S.grad, S.acc, err, sp, sg, ss);
    }
  }
  if (cur >= 0) flush();
}

// Adam on every active brick of every cloud, as step t + 1, learning rate
// lr * decay^floor(t / every) (every = 0: constant); one thread per 4
// consecutive vertices (128 per active-brick tile).
__global__ void __launch_bounds__(256) k_m_adam(const MShape* __restrict__ shapes, const MTile* __restrict__ tiles,
                                                int64_t ntiles, const int64_t* __restrict__ t_dev, float lr,
                                                float decay, int64_t every, float b1, float b2, float eps) {
  const int64_t t = *t_dev;
  const float ibc1 = (float)(1.0 / (1.0 - pow((double)b1, (double)(t + 1))));
  const float ibc2 = (float)(1.0 / (1.0 - pow((double)b2, (double)(t + 1))));
  const float lr_t = every > 0 ? (float)((double)lr * pow((double)decay, (double)(t / every))) : lr;
  const int64_t n = ntiles * 128;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const MTile tl = tiles[i >> 7];
    const MShape& S = shapes[tl.shape];
    adam_quad(__ldg(S.active + tl.first), (int)(i & 127), S.G.masks, S.grad, S.D, S.m, S.v, lr_t, b1, b2, eps,
              ibc1, ibc2);
  }
}

// Loss slots of every cloud from its sums; clears the sums and counts for the
// next step, records the epoch of the stored orders and advances t.
__global__ void k_m_finish(const MShape* __restrict__ shapes, int n, int32_t* __restrict__ nvalid,
                           double* __restrict__ sums, long long* __restrict__ isums, int64_t* __restrict__ t_dev,
                           int64_t* __restrict__ perm_epoch, float alpha, float beta, float gamma,
                           float* __restrict__ loss) {
  const int64_t t = *t_dev;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    perm_epoch[k] = t / shapes[k].nb_epoch;
    const int bv = nvalid[k];
    if (isums) {  // deterministic: the integer sums in units of 2^-24
      for (int c = 0; c < 4; ++c) {
        sums[4 * k + c] = (double)isums[4 * k + c] * (1.0 / 16777216.0);
        isums[4 * k + c] = 0;
      }
    }
    const double* sk = sums + 4 * k;
    const double lp = bv > 0 ? sk[0] / bv : 0.0, lg = bv > 0 ? sk[1] / bv : 0.0, ls = bv > 0 ? sk[2] / bv : 0.0;
    const int64_t V_tv = shapes[k].V_tv;
    const double lt = V_tv > 0 ? sk[3] / (double)V_tv : 0.0;
    float* L = loss + 8 * k;
    L[GP_LOSS_TOTAL] = (float)(lp + alpha * lt + beta * ls + gamma * lg);
    L[GP_LOSS_PULL] = (float)lp;
    L[GP_LOSS_GRAD] = (float)lg;
    L[GP_LOSS_SURF] = (float)ls;
    L[GP_LOSS_TV] = (float)lt;
    L[GP_LOSS_BV] = (float)bv;
    L[GP_LOSS_T] = (float)V_tv;
    L[7] = 0.f;
    nvalid[k] = 0;
    for (int c = 0; c < 4; ++c) sums[4 * k + c] = 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) *t_dev += 1;
}

enum { ST_NN, ST_TV, ST_QUERY, ST_TUNED };

}  // namespace

struct gp_multi {
  gp_ctx* ctx = nullptr;
  int n = 0;
  uint64_t seed = 0;
  uint32_t flags = 0;
  std::vector<gp_band*> bands;
  std::vector<int64_t> B, rec_off, grad_off;
  int64_t total_B = 0, V_total = 0, J_total = 0;
  int tq = 256;                    // records per tile = block size of the record kernels
  int bpsm[ST_TUNED] = {4, TV_BLOCKS_PER_SM, 4};  // persistent blocks per SM of the tuned stages
  MShape* shapes = nullptr;
  MTile *rec_tiles = nullptr, *pt_tiles = nullptr, *brick_tiles = nullptr, *active_tiles = nullptr;
  int64_t n_rec_tiles = 0, n_pt_tiles = 0, n_brick_tiles = 0, n_active_tiles = 0;
  float *q = nullptr, *rec = nullptr, *grad = nullptr;
  int32_t *src = nullptr, *perm = nullptr, *inv = nullptr, *eslot = nullptr, *counts = nullptr, *nvalid = nullptr,
          *err = nullptr;
  double* sums = nullptr;
  unsigned long long* acc = nullptr;  // deterministic: two-word fixed-point query sums over all clouds
  long long* isums = nullptr;         // deterministic: integer loss sums (4 per cloud)
  int64_t* t = nullptr;
  int64_t* perm_epoch = nullptr;  // per cloud: epoch of the stored Pi_e (-1: none)
};

namespace {

void multi_free(gp_multi* m) {
  if (!m) return;
  for (void* p : {(void*)m->shapes, (void*)m->rec_tiles, (void*)m->pt_tiles, (void*)m->brick_tiles,
                  (void*)m->active_tiles, (void*)m->q, (void*)m->rec, (void*)m->grad, (void*)m->src,
                  (void*)m->perm, (void*)m->inv, (void*)m->eslot, (void*)m->counts, (void*)m->nvalid, (void*)m->err,
                  (void*)m->sums, (void*)m->acc, (void*)m->isums, (void*)m->t, (void*)m->perm_epoch})
    gp_free(p);
  delete m;
}

gp_status upload_tiles(gp_ctx* ctx, const std::vector<MTile>& h, MTile** d, int64_t* n) {
  gp_free(*d);
  *d = nullptr;
  *n = (int64_t)h.size();
  gp_status st = gp_alloc(ctx, d, h.size(), "multi tiles");
  if (st) return st;
  if (!h.empty())
    GP_CUDA(ctx, cudaMemcpyAsync(*d, h.data(), h.size() * sizeof(MTile), cudaMemcpyHostToDevice, ctx->stream));
  GP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));  // h is a temporary
  return GP_OK;
}

gp_status build_rec_tiles(gp_multi* m, int tq) {
  std::vector<MTile> h;
  for (int k = 0; k < m->n; ++k)
    for (int64_t i = 0; i < m->B[(size_t)k]; i += tq) h.push_back({k, (int32_t)i});
  m->tq = tq;
  return upload_tiles(m->ctx, h, &m->rec_tiles, &m->n_rec_tiles);
}

unsigned persistent_grid(const gp_multi* m, int bpsm, int64_t ntiles) {
  int64_t g = (int64_t)m->ctx->num_sms * bpsm;
  if (g > ntiles) g = ntiles;
  return (unsigned)(g < 1 ? 1 : g);
}

// The record stages and the TV sweep, separately (the autotuner times them).
gp_status launch_nn(gp_multi* m) {
  gp_ctx* ctx = m->ctx;
  GP_KERNEL(ctx, "k_m_nn",
            k_m_nn<<<persistent_grid(m, m->bpsm[ST_NN], m->n_rec_tiles), m->tq, 0, ctx->stream>>>(
                m->shapes, m->rec_tiles, m->n_rec_tiles, m->tq, m->q, m->src, m->rec, m->nvalid));
  return GP_OK;
}

gp_status launch_tv(gp_multi* m, const gp_loss_w* w) {
  gp_ctx* ctx = m->ctx;
  const unsigned grid = persistent_grid(m, m->bpsm[ST_TV], m->n_brick_tiles);
  if (m->acc)
    GP_KERNEL(ctx, "k_m_tv",
              k_m_tv<true><<<grid, TV_SWEEP_THREADS, 0, ctx->stream>>>(m->shapes, m->brick_tiles, m->n_brick_tiles,
                                                                       w->alpha, m->sums, m->isums));
  else
    GP_KERNEL(ctx, "k_m_tv",
              k_m_tv<false><<<grid, TV_SWEEP_THREADS, 0, ctx->stream>>>(m->shapes, m->brick_tiles, m->n_brick_tiles,
                                                                        w->alpha, m->sums, m->isums));
  return GP_OK;
}

gp_status launch_query(gp_multi* m, const gp_loss_w* w) {
  gp_ctx* ctx = m->ctx;
  const unsigned grid = persistent_grid(m, m->bpsm[ST_QUERY], m->n_rec_tiles);
  const int threads = std::min(m->tq, 256);
  if (m->acc)
    GP_KERNEL(ctx, "k_m_query",
              k_m_query<true><<<grid, threads, 0, ctx->stream>>>(m->shapes, m->rec_tiles, m->n_rec_tiles, m->tq,
                                                                 m->rec, m->nvalid, w->beta, w->gamma, m->sums,
                                                                 m->isums, m->err));
  else
    GP_KERNEL(ctx, "k_m_query",
              k_m_query<false><<<grid, threads, 0, ctx->stream>>>(m->shapes, m->rec_tiles, m->n_rec_tiles, m->tq,
                                                                  m->rec, m->nvalid, w->beta, w->gamma, m->sums,
                                                                  m->isums, m->err));
  return GP_OK;
}

// Pi_e (for clouds starting an epoch) and the batch's queries.
gp_status launch_sampling(gp_multi* m) {
  gp_ctx* ctx = m->ctx;
  cudaStream_t s = ctx->stream;
  const unsigned gp = persistent_grid(m, 4, m->n_pt_tiles);
  GP_KERNEL(ctx, "k_m_perm",
            k_m_perm<<<gp, PT_TILE, 0, s>>>(m->shapes, m->pt_tiles, m->n_pt_tiles, m->t, m->perm_epoch, m->seed,
                                            m->err));
  if (!(m->flags & GP_SAMPLE_SPATIAL)) {  // position order: no emission slots needed
    GP_KERNEL(ctx, "k_m_sample",
              k_m_sample<<<persistent_grid(m, 4, m->n_rec_tiles), 256, 0, s>>>(
                  m->shapes, m->rec_tiles, m->n_rec_tiles, m->tq, m->t, m->seed, m->q, m->src));
    return GP_OK;
  }
  GP_KERNEL(ctx, "k_m_emit_slots",
            k_m_emit_slots<<<gp, PT_TILE, 0, s>>>(m->shapes, m->pt_tiles, m->n_pt_tiles, m->t, m->perm_epoch));
  GP_KERNEL(ctx, "k_m_order_count",
            k_m_order_count<<<gp, PT_TILE, 0, s>>>(m->shapes, m->pt_tiles, m->n_pt_tiles, m->t, m->counts));
  GP_KERNEL(ctx, "k_m_order_scan", k_m_order_scan<<<1, GP_ORDER_THREADS, 0, s>>>(m->counts, m->n_pt_tiles));
  GP_KERNEL(ctx, "k_m_order_emit",
            k_m_order_emit<<<gp, PT_TILE, 0, s>>>(m->shapes, m->pt_tiles, m->n_pt_tiles, m->t, m->seed, m->counts,
                                                 m->q, m->src, m->err));
  return GP_OK;
}

gp_status launch_adam_finish(gp_multi* m, const gp_loss_w* w, const gp_adam* hp, float decay, int64_t every,
                             float* loss_dev) {
  gp_ctx* ctx = m->ctx;
  cudaStream_t s = ctx->stream;
  if (m->n_active_tiles > 0)
    GP_KERNEL(ctx, "k_m_adam",
              k_m_adam<<<persistent_grid(m, 8, m->n_active_tiles * 128 / 256 + 1), 256, 0, s>>>(
                  m->shapes, m->active_tiles, m->n_active_tiles, m->t, hp->lr, decay, every, hp->beta1, hp->beta2,
                  hp->eps));
  GP_KERNEL(ctx, "k_m_finish",
            k_m_finish<<<1, 256, 0, s>>>(m->shapes, m->n, m->nvalid, m->sums, m->isums, m->t, m->perm_epoch,
                                         w->alpha, w->beta, w->gamma, loss_dev));
  return GP_OK;
}

gp_status clear_step_state(gp_multi* m) {
  cudaStream_t s = m->ctx->stream;
  GP_CUDA(m->ctx, cudaMemsetAsync(m->nvalid, 0, m->n * sizeof(int32_t), s));
  GP_CUDA(m->ctx, cudaMemsetAsync(m->sums, 0, 4 * m->n * sizeof(double), s));
  if (m->isums) GP_CUDA(m->ctx, cudaMemsetAsync(m->isums, 0, 4 * m->n * sizeof(long long), s));
  if (m->acc) GP_CUDA(m->ctx, cudaMemsetAsync(m->acc, 0, 2 * m->V_total * sizeof(unsigned long long), s));
  return GP_OK;
}

}  // namespace

extern "C" gp_status gp_multi_create(gp_ctx* ctx, gp_band* const* bands, int32_t n, const int64_t* Q,
                                     const int64_t* B, uint64_t seed, uint32_t flags, gp_multi** out) {
  if (!ctx) return GP_ERR_ARG;
  if (!out) return gp_fail(ctx, GP_ERR_ARG, "gp_multi_create: null output");
  *out = nullptr;
  if (!bands || !Q || !B || n < 1) return gp_fail(ctx, GP_ERR_ARG, "gp_multi_create: null or empty input");
  if (flags & ~(uint32_t)(GP_SAMPLE_SPATIAL | GP_MULTI_DETERMINISTIC))
    return gp_fail(ctx, GP_ERR_ARG, "gp_multi_create: unknown flags");
  gp_multi* m = new (std::nothrow) gp_multi();
  if (!m) return gp_fail(ctx, GP_ERR_OOM, "gp_multi_create: host allocation");
  m->ctx = ctx;
  m->n = n;
  m->seed = seed;
  m->flags = flags;
  std::vector<MTile> pt, br, ac;
  for (int k = 0; k < n; ++k) {
    gp_band* b = bands[k];
    if (!b || b->ctx != ctx || !b->sigma || !b->emit_order || !b->emit_pts) {
      multi_free(m);
      return gp_fail(ctx, GP_ERR_ARG, "gp_multi_create: every band must come from this context, with sigma");
    }
    if (b->flags & GP_BAND_DETERMINISTIC) {
      multi_free(m);
      return gp_fail(ctx, GP_ERR_ARG, "gp_multi_create: deterministic bands step through gp_step only");
    }
    if (Q[k] < 1 || Q[k] >= (int64_t(1) << 31) || B[k] < 1 || B[k] > Q[k]) {
      multi_free(m);
      return gp_fail(ctx, GP_ERR_ARG, "gp_multi_create: need 1 <= B_k <= Q_k < 2^31");
    }
    for (int i = 0; i < k; ++i)
      if (bands[i] == b) {
        multi_free(m);
        return gp_fail(ctx, GP_ERR_ARG, "gp_multi_create: a band appears twice");
      }
    m->bands.push_back(b);
    m->B.push_back(B[k]);
    m->rec_off.push_back(m->total_B);
    m->grad_off.push_back(m->V_total);
    m->total_B += B[k];
    m->V_total += b->V_stored();
    for (int64_t p = 0; p < b->J; p += PT_TILE) pt.push_back({k, (int32_t)p});
    for (int64_t s = 0; s < b->n_bricks; ++s) br.push_back({k, (int32_t)s});
    for (int64_t a = 0; a < b->n_active; ++a) ac.push_back({k, (int32_t)a});
    m->J_total += b->J;
  }
  if (m->total_B >= (int64_t(1) << 31)) {
    multi_free(m);
    return gp_fail(ctx, GP_ERR_ARG, "gp_multi_create: sum of the batch sizes must stay below 2^31");
  }
  gp_status st = GP_OK;
  if (!st) st = gp_alloc(ctx, &m->grad, m->V_total, "multi gradient");
  if (!st && (flags & GP_MULTI_DETERMINISTIC)) st = gp_alloc(ctx, &m->acc, 2 * m->V_total, "multi fixed-point sums");
  if (!st && (flags & GP_MULTI_DETERMINISTIC)) st = gp_alloc(ctx, &m->isums, 4 * (size_t)n, "multi integer sums");
  if (!st) st = gp_alloc(ctx, &m->perm, m->J_total, "multi permutation");
  if (!st) st = gp_alloc(ctx, &m->inv, m->J_total, "multi inverse permutation");
  if (!st) st = gp_alloc(ctx, &m->eslot, m->J_total, "multi emission slots");
  if (!st) st = gp_alloc(ctx, &m->shapes, (size_t)n, "multi shapes");
  if (!st) st = gp_alloc(ctx, &m->q, 3 * m->total_B, "multi queries");
  if (!st) st = gp_alloc(ctx, &m->src, m->total_B, "multi sources");
  if (!st) st = gp_alloc(ctx, &m->rec, 6 * m->total_B, "multi records");
  if (!st) st = gp_alloc(ctx, &m->counts, pt.size(), "multi order counts");
  if (!st) st = gp_alloc(ctx, &m->nvalid, (size_t)n, "multi counts");
  if (!st) st = gp_alloc(ctx, &m->sums, 4 * (size_t)n, "multi sums");
  if (!st) st = gp_alloc(ctx, &m->t, 1, "multi step");
  if (!st) st = gp_alloc(ctx, &m->err, 1, "multi error flag");
  if (!st) st = gp_alloc(ctx, &m->perm_epoch, (size_t)n, "multi order epochs");
  if (st) {
    multi_free(m);
    return st;
  }
  std::vector<MShape> hs((size_t)n);
  int64_t joff = 0, tile0 = 0;
  for (int k = 0; k < n; ++k) {
    gp_band* b = m->bands[(size_t)k];
    MShape& S = hs[(size_t)k];
    S.G.table = b->brick_table;
    S.G.masks = b->masks;
    S.G.D = b->D;
    S.G.nb = b->nb;
    S.G.R = b->R;
    S.G.half_r = 0.5f * (float)b->R;
    S.nn = make_grid(b);
    S.D = b->D;
    S.m = b->m;
    S.v = b->v;
    S.grad = m->grad + m->grad_off[(size_t)k];
    S.acc = m->acc ? m->acc + 2 * m->grad_off[(size_t)k] : nullptr;
    S.pts = b->pts;
    S.sigma = b->sigma;
    S.normals = b->normals;
    S.order = b->emit_order;
    S.epts = b->emit_pts;
    S.perm = m->perm + joff;
    S.inv = m->inv + joff;
    S.eslot = m->eslot + joff;
    S.coord = b->brick_coord;
    S.nbr = b->brick_nbr;
    S.active = b->active;
    S.J = b->J;
    S.Q = Q[k];
    S.B = B[k];
    S.nb_epoch = (S.Q + S.B - 1) / S.B;
    S.V_tv = b->V_tv;
    S.rec_off = m->rec_off[(size_t)k];
    S.tile0 = tile0;
    joff += b->J;
    tile0 += (b->J + PT_TILE - 1) / PT_TILE;
  }
  cudaStream_t s = ctx->stream;
  cudaError_t e = cudaMemcpyAsync(m->shapes, hs.data(), n * sizeof(MShape), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->t, 0, sizeof(int64_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->err, 0, sizeof(int32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->perm_epoch, 0xff, n * sizeof(int64_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->grad, 0, m->V_total * sizeof(float), s);
  if (e != cudaSuccess) st = gp_cuda_fail(ctx, e, "gp_multi_create: upload");
  if (!st) st = clear_step_state(m);
  if (!st) st = upload_tiles(ctx, pt, &m->pt_tiles, &m->n_pt_tiles);  // synchronises (hs is freed after)
  if (!st) st = upload_tiles(ctx, br, &m->brick_tiles, &m->n_brick_tiles);
  if (!st) st = upload_tiles(ctx, ac, &m->active_tiles, &m->n_active_tiles);
  if (!st) st = build_rec_tiles(m, 256);
  if (st) {
    cudaStreamSynchronize(s);
    multi_free(m);
    return st;
  }
  *out = m;
  return GP_OK;
}

extern "C" void gp_multi_destroy(gp_multi* m) {
  if (!m) return;
  cudaStreamSynchronize(m->ctx->stream);
  multi_free(m);
}

extern "C" gp_status gp_multi_step(gp_multi* m, const gp_loss_w* w, const gp_adam* hp, float lr_decay,
                                   int64_t lr_every, float* loss_dev) {
  if (!m) return GP_ERR_ARG;
  if (!w || !hp || !loss_dev) return gp_fail(m->ctx, GP_ERR_ARG, "gp_multi_step: null pointer");
  if (lr_every < 0) return gp_fail(m->ctx, GP_ERR_ARG, "gp_multi_step: lr_every must be >= 0");
  gp_status st = launch_sampling(m);
  if (!st) st = launch_nn(m);
  if (m->acc) {  // deterministic: the query sums first, folded in by the sweep
    if (!st) st = launch_query(m, w);
    if (!st) st = launch_tv(m, w);
  } else {
    if (!st) st = launch_tv(m, w);
    if (!st) st = launch_query(m, w);
  }
  if (!st) st = launch_adam_finish(m, w, hp, lr_decay, lr_every, loss_dev);
  return st;
}

extern "C" gp_status gp_multi_autotune(gp_multi* m, const gp_loss_w* w) {
  if (!m) return GP_ERR_ARG;
  gp_ctx* ctx = m->ctx;
  if (!w) return gp_fail(ctx, GP_ERR_ARG, "gp_multi_autotune: null pointer");
  cudaStream_t s = ctx->stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  GP_CUDA(ctx, cudaEventCreate(&e0));
  gp_status st = GP_OK;
  cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) st = gp_cuda_fail(ctx, ce, "cudaEventCreate");
  // Best of three launches of one stage, in ms.
  auto time_stage = [&](int stage, float* ms) -> gp_status {
    float best = INFINITY;
    for (int rep = 0; rep < 3; ++rep) {
      GP_CUDA(ctx, cudaEventRecord(e0, s));
      gp_status r = stage == ST_NN ? launch_nn(m) : stage == ST_TV ? launch_tv(m, w) : launch_query(m, w);
      if (r) return r;
      GP_CUDA(ctx, cudaEventRecord(e1, s));
      GP_CUDA(ctx, cudaEventSynchronize(e1));
      float t = 0.f;
      GP_CUDA(ctx, cudaEventElapsedTime(&t, e0, e1));
      best = std::min(best, t);
    }
    *ms = best;
    return GP_OK;
  };
  // The current step's queries, as input of the record stages.
  if (!st) st = launch_sampling(m);
  // Records per tile (also the block size of the record kernels), timed on
  // the nearest-point stage, the heaviest.
  int best_tq = m->tq;
  float best_ms = INFINITY;
  for (int tq : {128, 256, 512}) {
    if (st) break;
    st = build_rec_tiles(m, tq);
    if (!st && !(m->flags & GP_SAMPLE_SPATIAL)) st = launch_sampling(m);  // sample tiles follow tq
    float ms = INFINITY;
    if (!st) st = time_stage(ST_NN, &ms);
    if (!st && ms < best_ms) {
      best_ms = ms;
      best_tq = tq;
    }
  }
  if (!st) st = build_rec_tiles(m, best_tq);
  if (!st && !(m->flags & GP_SAMPLE_SPATIAL)) st = launch_sampling(m);
  for (int stage : {ST_NN, ST_TV, ST_QUERY}) {
    int best_b = m->bpsm[stage];
    float bm = INFINITY;
    const int tv_c[3] = {TV_BLOCKS_PER_SM, 2 * TV_BLOCKS_PER_SM, 3 * TV_BLOCKS_PER_SM};
    const int gen_c[5] = {1, 2, 4, 8, 16};
    const int* cand = stage == ST_TV ? tv_c : gen_c;
    const int ncand = stage == ST_TV ? 3 : 5;
    for (int ci = 0; ci < ncand; ++ci) {
      const int c = cand[ci];
      if (st) break;
      m->bpsm[stage] = c;
      float ms = INFINITY;
      st = time_stage(stage, &ms);
      if (!st && ms < bm) {
        bm = ms;
        best_b = c;
      }
    }
    m->bpsm[stage] = best_b;
  }
  cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) return st;
  // The timed launches left counts and sums behind; the gradient is rewritten
  // by every step's TV sweep before it is read.
  st = clear_step_state(m);
  if (st) return st;
  GP_CUDA(ctx, cudaStreamSynchronize(s));
  return GP_OK;
}

extern "C" gp_status gp_multi_get_info(gp_multi* m, gp_multi_info* out) {
  if (!m) return GP_ERR_ARG;
  if (!out) return gp_fail(m->ctx, GP_ERR_ARG, "gp_multi_get_info: null output");
  out->n = m->n;
  out->flags = m->flags;
  out->records_per_tile = m->tq;
  out->blocks_per_sm_nn = m->bpsm[ST_NN];
  out->blocks_per_sm_tv = m->bpsm[ST_TV];
  out->blocks_per_sm_query = m->bpsm[ST_QUERY];
  out->total_B = m->total_B;
  out->V_total = m->V_total;
  int64_t t = 0;
  int32_t e = 0;
  GP_CUDA(m->ctx, cudaMemcpyAsync(&t, m->t, sizeof(int64_t), cudaMemcpyDeviceToHost, m->ctx->stream));
  GP_CUDA(m->ctx, cudaMemcpyAsync(&e, m->err, sizeof(int32_t), cudaMemcpyDeviceToHost, m->ctx->stream));
  GP_CUDA(m->ctx, cudaStreamSynchronize(m->ctx->stream));
  out->step = t;
  out->error_bits = e;
  return GP_OK;
}

extern "C" gp_status gp_multi_set_step(gp_multi* m, int64_t step) {
  if (!m) return GP_ERR_ARG;
  if (step < 0) return gp_fail(m->ctx, GP_ERR_ARG, "gp_multi_set_step: step must be >= 0");
  GP_CUDA(m->ctx, cudaMemcpyAsync(m->t, &step, sizeof(int64_t), cudaMemcpyHostToDevice, m->ctx->stream));
  GP_CUDA(m->ctx, cudaStreamSynchronize(m->ctx->stream));
  return GP_OK;
}

extern "C" gp_status gp_multi_buffers(gp_multi* m, int32_t k, float** rec_dev, int32_t** src_dev, float** grad_dev) {
  if (!m) return GP_ERR_ARG;
  if (k < 0 || k >= m->n) return gp_fail(m->ctx, GP_ERR_ARG, "gp_multi_buffers: cloud index out of range");
  if (rec_dev) *rec_dev = m->rec + 6 * m->rec_off[(size_t)k];
  if (src_dev) *src_dev = m->src + m->rec_off[(size_t)k];
  if (grad_dev) *grad_dev = m->grad + m->grad_off[(size_t)k];
  return GP_OK;
}
