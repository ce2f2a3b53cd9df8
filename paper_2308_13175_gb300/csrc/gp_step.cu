// gp_step: the loss of Eq. 8 and its gradient dL/dD in one forward +
// hand-written backward pass, and gp_update: Adam on the trainable vertices.
//
// Per valid query (q, s = NN(q)):
//   f, g = grad f at q from the 8 corners of cell(q) (Eq. 3, in the cell's
//          local coordinate t: trilinear lerps, g = dt f * R/2),
//   n = g / max(|g|, 1e-12),  p = q - f n  (Sec. 3),  r = (q - s) - f n,
//   l_pull = |r|  (Eq. 4),
//   f_s, g_s at s from the 8 corners of cell(s),  n_s = g_s / max(|g_s|, 1e-12),
//   l_grad = 1 - n . n_s  (Eq. 7),  l_surf = |f_s|  (Eq. 6).
// Backward (w = 1/B_v):  u = r / |r|;  dL/df = -w u.n;
//   dL/dn = -w f u - w gamma n_s;  dL/dg = (I - n n^T) dL/dn / |g|;
//   dL/dn_s = -w gamma n;  dL/dg_s = (I - n_s n_s^T) dL/dn_s / |g_s|;
//   dL/df_s = w beta sign(f_s);
// each corner c of a cell receives dL/df w_c(t) + sum_a dL/dt_a dw_c/dt_a.
// L_TV (Eq. 5): TV_i = sqrt(sum over in-grid axis neighbours (d_i - d_n)^2)
// over the TV set T, averaged; its gradient is gathered per vertex,
//   dTV/dd_i = [i in T] sum_n (d_i - d_n)/TV_i + sum_{n in T} (d_i - d_n)/TV_n.
#include <algorithm>
#include <cmath>

#include "gp_internal.cuh"
#include "gp_step_device.cuh"
#include "gp_query_win.cuh"
#include "gp_tv2.cuh"

namespace {

constexpr int Q_THREADS = 256;
constexpr int Q_BLOCKS_PER_SM = 3;  // resident k_query blocks per SM at its register cap
constexpr int TV_THREADS = TV_SWEEP_THREADS;
// Loss slots from the per-block partial sums, in a fixed order (run by one
// whole block).
struct FinalArgs {
  int32_t* done;       // blocks of the last kernel that have finished
  int q_blocks, tv_blocks;
  const int32_t* bv;
  int64_t n_tv;
  float alpha, beta, gamma;
  int tv_on;
  float* loss;
};

__device__ void finalize_loss(const double* __restrict__ partials, const FinalArgs& fa) {
  __shared__ double red[4][32];
  double sums[4] = {0, 0, 0, 0};
  for (int b = threadIdx.x; b < fa.q_blocks; b += blockDim.x) {
    sums[0] += __ldcg(partials + (int64_t)b * 8 + 0);
    sums[1] += __ldcg(partials + (int64_t)b * 8 + 1);
    sums[2] += __ldcg(partials + (int64_t)b * 8 + 2);
  }
  for (int b = threadIdx.x; b < fa.tv_blocks; b += blockDim.x) sums[3] += __ldcg(partials + (int64_t)b * 8 + 3);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    double v = gp_warp_sum_d(sums[c]);
    if ((threadIdx.x & 31) == 0) red[c][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[4] = {0, 0, 0, 0};
    for (int c = 0; c < 4; ++c)
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t[c] += red[c][w];
    int b = *fa.bv;
    double lp = b > 0 ? t[0] / b : 0.0, lg = b > 0 ? t[1] / b : 0.0, ls = b > 0 ? t[2] / b : 0.0;
    double lt = (fa.tv_on && fa.n_tv > 0) ? t[3] / (double)fa.n_tv : 0.0;
    float* loss = fa.loss;
    loss[GP_LOSS_TOTAL] = (float)(lp + fa.alpha * lt + fa.beta * ls + fa.gamma * lg);
    loss[GP_LOSS_PULL] = (float)lp;
    loss[GP_LOSS_GRAD] = (float)lg;
    loss[GP_LOSS_SURF] = (float)ls;
    loss[GP_LOSS_TV] = (float)lt;
    loss[GP_LOSS_BV] = (float)b;
    loss[GP_LOSS_T] = (float)fa.n_tv;
    loss[7] = 0.f;
  }
}

// The last block of the step's last kernel to finish (threadfence reduction)
// writes the loss slots and re-arms the counter for the next call.
__device__ void finish_if_last(const double* __restrict__ partials, const FinalArgs& fa) {
  __shared__ int am_last;
  __syncthreads();  // thread 0 has written this block's partials
  if (threadIdx.x == 0) {
    __threadfence();
    am_last = (atomicAdd(fa.done, 1) == (int)gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  finalize_loss(partials, fa);
  if (threadIdx.x == 0) *fa.done = 0;
}

__global__ void k_count_valid(Grid G, const float* __restrict__ rec, int64_t B, int32_t* __restrict__ nvalid) {
  int cnt = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < B; i += (int64_t)gridDim.x * blockDim.x) {
    float q[3], s[3];
    load_rec(rec, i, q, s);
    Cells C;
    cnt += classify(G, q, s, C) ? 1 : 0;
  }
  int w = gp_warp_sum_i(cnt);
  if ((threadIdx.x & 31) == 0 && w) atomicAdd(nvalid, w);
}

// Block reduction of three float sums into partials[block*8 + 0..2] (fp64).
__device__ __forceinline__ void block_store3(double* __restrict__ partials, float a, float b, float c) {
  __shared__ float red[3][Q_THREADS / 32];
  a = gp_warp_sum(a);
  b = gp_warp_sum(b);
  c = gp_warp_sum(c);
  int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[0][w] = a;
    red[1][w] = b;
    red[2][w] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0, s1 = 0, s2 = 0;
    for (int k = 0; k < Q_THREADS / 32; ++k) {
      s0 += red[0][k];
      s1 += red[1][k];
      s2 += red[2][k];
    }
    double* p = partials + (int64_t)blockIdx.x * 8;
    p[0] = s0;
    p[1] = s1;
    p[2] = s2;
  }
}

template <bool DET, bool GRAD, bool LAST>
__global__ void __launch_bounds__(Q_THREADS, Q_BLOCKS_PER_SM) k_query(Grid G, const float* __restrict__ rec, int64_t B,
                                                     const int32_t* __restrict__ bv, float beta, float gamma,
                                                     float* __restrict__ grad, unsigned long long* __restrict__ acc,
                                                     double* __restrict__ partials, int32_t* __restrict__ err,
                                                     FinalArgs fa) {
  const int64_t n = B;
  int bvv = *bv;
  float w = bvv > 0 ? 1.0f / (float)bvv : 0.f;
  float sp = 0.f, sg = 0.f, ss = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float q[3], s[3];
    load_rec(rec, i, q, s);
    query_record<DET, GRAD>(G, q, s, w, beta, gamma, grad, acc, err, sp, sg, ss);
  }
  block_store3(partials, sp, sg, ss);
  if (LAST) finish_if_last(partials, fa);
}

// The fused forward + backward with RPT records per thread and iteration:
// record i and i + stride (stride = the grid's threads) go through the
// phases together, so that the loads of one level of both records are in
// flight at once (the step is bound by the latency of these dependent
// gathers).  The 16 corner contributions of a record go to the gradient as
// vector reductions (GlobalSink; DET: the two-word fixed point).  MINB, the
// resident blocks per SM the kernel is compiled for, caps its registers.
template <bool DET, bool LAST, int RPT, int MINB>
__global__ void __launch_bounds__(Q_THREADS, MINB) k_query_ilp(Grid G, const float* __restrict__ rec, int64_t B,
                                                               const int32_t* __restrict__ bv, float beta,
                                                               float gamma, float* __restrict__ grad,
                                                               unsigned long long* __restrict__ acc,
                                                               double* __restrict__ partials,
                                                               int32_t* __restrict__ err, FinalArgs fa) {
  const int bvv = *bv;
  const float w = bvv > 0 ? 1.0f / (float)bvv : 0.f;  // also for the fixed-point sums (taken pre-scaled)
  float sp = 0.f, sg = 0.f, ss = 0.f;
  GlobalSink<DET> sink{G, grad, acc, err};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < B; i0 += RPT * stride) {
    RecState R[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const int64_t i = i0 + r * stride;
      float q[3] = {0.f, 0.f, 0.f}, s[3] = {0.f, 0.f, 0.f};
      if (i < B) load_rec(rec, i, q, s);
      rec_phase_a(G, q, s, i < B, R[r]);
    }
#pragma unroll
    for (int r = 0; r < RPT; ++r) rec_phase_b(G, R[r]);
#pragma unroll
    for (int r = 0; r < RPT; ++r) rec_phase_c<true>(G, R[r], w, beta, gamma, sink, err, sp, sg, ss);
  }
  block_store3(partials, sp, sg, ss);
  if (LAST) finish_if_last(partials, fa);
}

template <bool DET, bool LAST, int RPT, int MINB>
cudaError_t launch_query_ilp(gp_ctx* ctx, int64_t B, cudaStream_t s, Grid G, const float* rec, const int32_t* bv,
                             float beta, float gamma, float* grad, unsigned long long* acc, double* partials,
                             int32_t* err, FinalArgs& fa) {
  const unsigned grid = gp_blocks(B, Q_THREADS * RPT,
                                  std::min<int64_t>((int64_t)ctx->num_sms * MINB, GP_MAX_PARTIAL_BLOCKS));
  fa.q_blocks = (int)grid;
  k_query_ilp<DET, LAST, RPT, MINB><<<grid, Q_THREADS, 0, s>>>(G, rec, B, bv, beta, gamma, grad, acc, partials, err,
                                                               fa);
  return cudaGetLastError();
}

// The windowed form (gp_query_win.cuh): tiles of 256 RPT records, a
// persistent grid of MINB blocks per SM (MINB also caps the registers), each
// tile's window set up by warp 0 during the previous tile and, when staged,
// its bricks copied while the previous tile's window is written out.  Atomic
// mode only.
template <bool STAGE, bool LAST, int RPT, int MINB>
__global__ void __launch_bounds__(WQ_THREADS, MINB)
    k_query_win(Grid G, const int32_t* __restrict__ nbrs, const float* __restrict__ rec, int64_t B,
                const int32_t* __restrict__ bv, float beta, float gamma, float* __restrict__ grad,
                double* __restrict__ partials, int32_t* __restrict__ err, FinalArgs fa) {
  constexpr int TILE = WQ_THREADS * RPT;
  extern __shared__ __align__(128) unsigned char wq_smem[];
  float* acc = reinterpret_cast<float*>(wq_smem);
  float* val = acc + WIN_V;
  uint32_t* pull = reinterpret_cast<uint32_t*>(val + WIN_V);
  __shared__ int sh_slot[2][WIN_BRICKS];
  __shared__ int sh_lo[2][3];
  __shared__ uint32_t sh_present[2];
  __shared__ int sh_abort;
  __shared__ __align__(8) unsigned long long sh_bar;

  for (int i = threadIdx.x; i < WIN_V / 4; i += WQ_THREADS)
    reinterpret_cast<float4*>(acc)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  const int64_t ntiles = (B + TILE - 1) / TILE;
  int64_t tile = blockIdx.x;
  if (threadIdx.x < 32) win_setup(G, nbrs, rec, B, TILE, tile, ntiles, sh_slot[0], sh_lo[0], &sh_present[0]);
  if (threadIdx.x == 0) {
    sh_abort = 0;
    if (STAGE) mbar_init(&sh_bar, 1);
  }
  __syncthreads();
  if (STAGE && threadIdx.x == 0 && tile < ntiles && sh_present[0])
    win_issue(G, sh_slot[0], sh_present[0], val, pull, &sh_bar);
  uint32_t parity = 0;  // of the barrier phase the next staged tile completes
  const int bvv = *bv;
  const float w = bvv > 0 ? 1.0f / (float)bvv : 0.f;
  float sp = 0.f, sg = 0.f, ss = 0.f;
  for (int it = 0; tile < ntiles; ++it, tile += gridDim.x) {
    const int p = it & 1;
    Win W;
    W.lo[0] = sh_lo[p][0];
    W.lo[1] = sh_lo[p][1];
    W.lo[2] = sh_lo[p][2];
    W.present = sh_present[p];
    const int64_t next = tile + gridDim.x;
    if (threadIdx.x < 32)
      win_setup(G, nbrs, rec, B, TILE, next, ntiles, sh_slot[p ^ 1], sh_lo[p ^ 1], &sh_present[p ^ 1]);
    RecState R[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const int64_t i = tile * TILE + r * WQ_THREADS + threadIdx.x;
      float q[3] = {0.f, 0.f, 0.f}, s[3] = {0.f, 0.f, 0.f};
      if (i < B) load_rec(rec, i, q, s);
      win_phase_a<STAGE>(G, W, sh_slot[p], q, s, i < B, R[r]);
    }
    if (STAGE && W.present) {
      if (!mbar_wait(&sh_bar, parity)) {
        atomicOr(err, GP_EF_TIMEOUT);
        sh_abort = 1;
      }
      parity ^= 1u;
    }
#pragma unroll
    for (int r = 0; r < RPT; ++r) win_phase_b<STAGE>(G, W, sh_slot[p], val, pull, R[r]);
    WindowSink sink{G, grad, acc, W, err};
#pragma unroll
    for (int r = 0; r < RPT; ++r) rec_phase_c<true>(G, R[r], w, beta, gamma, sink, err, sp, sg, ss);
    __syncthreads();
    const bool abort = sh_abort != 0;
    if (STAGE && threadIdx.x == 0 && !abort && next < ntiles && sh_present[p ^ 1])
      win_issue(G, sh_slot[p ^ 1], sh_present[p ^ 1], val, pull, &sh_bar);
    win_flush(acc, sh_slot[p], grad);
    __syncthreads();
    if (abort) {
      // The copies of the phase that ran out may still be in flight: wait
      // for them (bounded) before the block leaves.
      if (STAGE && threadIdx.x == 0) mbar_wait(&sh_bar, parity ^ 1u);
      break;
    }
  }
  block_store3(partials, sp, sg, ss);
  if (LAST) finish_if_last(partials, fa);
}

template <bool STAGE, bool LAST, int RPT, int MINB>
cudaError_t launch_query_win(gp_ctx* ctx, const int32_t* nbrs, int64_t B, cudaStream_t s, Grid G, const float* rec,
                             const int32_t* bv, float beta, float gamma, float* grad, double* partials, int32_t* err,
                             FinalArgs& fa) {
  const size_t smem = STAGE ? WQ_SMEM_STAGED : WQ_SMEM_ACC;
  cudaError_t e = cudaFuncSetAttribute(k_query_win<STAGE, LAST, RPT, MINB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = gp_blocks(B, WQ_THREADS * RPT,
                                  std::min<int64_t>((int64_t)ctx->num_sms * MINB, GP_MAX_PARTIAL_BLOCKS));
  fa.q_blocks = (int)grid;
  k_query_win<STAGE, LAST, RPT, MINB><<<grid, WQ_THREADS, smem, s>>>(G, nbrs, rec, B, bv, beta, gamma, grad,
                                                                      partials, err, fa);
  return cudaGetLastError();
}

// The windowed forms at the band's launch shape: (RPT, MINB) as for the
// direct form; the staged form holds 110 KB of shared memory per block, so
// it runs 2 blocks per SM whatever MINB is.
template <bool LAST>
cudaError_t launch_query_window_tuned(const gp_band* b, int64_t B, cudaStream_t s, Grid G, const float* rec,
                                      const int32_t* bv, float beta, float gamma, float* grad, double* partials,
                                      int32_t* err, FinalArgs& fa) {
  gp_ctx* ctx = b->ctx;
  const int32_t* nb = b->brick_nbr;
#define GP_QW(ST_, R_, M_) \
  launch_query_win<ST_, LAST, R_, M_>(ctx, nb, B, s, G, rec, bv, beta, gamma, grad, partials, err, fa)
  if (b->q_form == GP_QUERY_WINDOW_STAGED) return b->q_rpt == 2 ? GP_QW(true, 2, 2) : GP_QW(true, 1, 2);
  if (b->q_rpt == 2) {
    if (b->q_bps == 3) return GP_QW(false, 2, 3);
    if (b->q_bps == 4) return GP_QW(false, 2, 4);
    return GP_QW(false, 2, 2);
  }
  if (b->q_bps == 3) return GP_QW(false, 1, 3);
  if (b->q_bps == 4) return GP_QW(false, 1, 4);
  return GP_QW(false, 1, 2);
#undef GP_QW
}

// The tuned launch shape: RPT in {1, 2} records per thread, MINB in {2, 3, 4}.
template <bool DET, bool LAST>
cudaError_t launch_query_tuned(const gp_band* b, int64_t B, cudaStream_t s, Grid G, const float* rec,
                               const int32_t* bv, float beta, float gamma, float* grad, double* partials,
                               int32_t* err, FinalArgs& fa) {
  gp_ctx* ctx = b->ctx;
  unsigned long long* acc = b->acc;
  if (!DET && b->q_form != GP_QUERY_DIRECT)
    return launch_query_window_tuned<LAST>(b, B, s, G, rec, bv, beta, gamma, grad, partials, err, fa);
  if (b->q_rpt == 2) {
    if (b->q_bps == 2)
      return launch_query_ilp<DET, LAST, 2, 2>(ctx, B, s, G, rec, bv, beta, gamma, grad, acc, partials, err, fa);
    if (b->q_bps == 4)
      return launch_query_ilp<DET, LAST, 2, 4>(ctx, B, s, G, rec, bv, beta, gamma, grad, acc, partials, err, fa);
    return launch_query_ilp<DET, LAST, 2, 3>(ctx, B, s, G, rec, bv, beta, gamma, grad, acc, partials, err, fa);
  }
  if (b->q_bps == 2)
    return launch_query_ilp<DET, LAST, 1, 2>(ctx, B, s, G, rec, bv, beta, gamma, grad, acc, partials, err, fa);
  if (b->q_bps == 4)
    return launch_query_ilp<DET, LAST, 1, 4>(ctx, B, s, G, rec, bv, beta, gamma, grad, acc, partials, err, fa);
  return launch_query_ilp<DET, LAST, 1, 3>(ctx, B, s, G, rec, bv, beta, gamma, grad, acc, partials, err, fa);
}

// The L_TV sweep over the band's bricks (tv_sweep: one brick at a time per
// block of TV_THREADS, one persistent wave of blocks, the next brick's halo
// copied while the current one is computed).  Writes the gradient of every
// stored slot: alpha/|T| * dTV/dd_i (+ the fixed-point query sums in
// deterministic mode, which are cleared for the next step).  Each TV_i enters
// the loss sum once, from the brick that stores i.
struct BandTvSrc {
  Grid G;
  const int32_t* coord;
  const int32_t* nbrs;
  __device__ __forceinline__ TvBrick brick(int64_t s) const {
    return TvBrick{G.D, G.masks, nbrs + 27 * s, G.R, __ldg(coord + 3 * s) * 8, __ldg(coord + 3 * s + 1) * 8,
                   __ldg(coord + 3 * s + 2) * 8};
  }
};

template <bool DET, bool GRAD, bool TV, bool LAST>
__global__ void __launch_bounds__(TV_THREADS, TV_BLOCKS_PER_SM) k_tv(Grid G, const int32_t* __restrict__ coord,
                                                   const int32_t* __restrict__ nbrs, int64_t n_bricks,
                                                   float tv_scale, float* __restrict__ grad,
                                                   unsigned long long* __restrict__ acc,
                                                   double* __restrict__ partials, int32_t* __restrict__ err,
                                                   FinalArgs fa) {
  __shared__ TvShared sh;
  float tsum = 0.f;
  const int l = threadIdx.x;
  auto emit = [&](int64_t addr, float gv) {
    if (!GRAD) return;
    if (DET) {
      long long hi = (long long)acc[2 * addr], lo = (long long)acc[2 * addr + 1];
      acc[2 * addr] = 0ull;
      acc[2 * addr + 1] = 0ull;
      // hi 2^-20 + lo 2^-60 in float32 (the scales are exact powers of two):
      // the same operations on the same integers, so still bit-reproducible.
      // The query pass added its contributions already scaled by 1/B_v.
      const float qv = __fmaf_rn(__ll2float_rn(hi), 9.5367431640625e-07f, __ll2float_rn(lo) * 8.673617379884035e-19f);
      gv = __fadd_rn(qv, gv);
    }
    grad[addr] = gv;
  };
  if (TV) {
    tv_sweep(BandTvSrc{G, coord, nbrs}, blockIdx.x, gridDim.x, n_bricks, sh,
             [&](int64_t slot, int l0, float g0, int l1, float g1, float ts) {
               tsum += ts;
               emit(slot * 512 + l0, tv_scale * g0);
               emit(slot * 512 + l1, tv_scale * g1);
             });
  } else {
    for (int64_t slot = blockIdx.x; slot < n_bricks; slot += gridDim.x) {
      emit(slot * 512 + l, 0.f);
      emit(slot * 512 + l + 256, 0.f);
    }
  }
  // block reduction of the TV sum into partials[block*8 + 3]
  __shared__ float red[TV_THREADS / 32];
  float w = gp_warp_sum(tsum);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = w;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0;
    for (int k = 0; k < TV_THREADS / 32; ++k) sum += red[k];
    partials[(int64_t)blockIdx.x * 8 + 3] = sum;
  }
  if (LAST) finish_if_last(partials, fa);
  (void)err;
}

// The two-pass L_TV of gp_step (gp_tv2.cuh).  Each block walks bricks
// blockIdx.x, + gridDim.x, ...: the next brick's copies are issued into the
// other of two stage buffers (cp.async) before the current one is computed,
// and the brick after that has its neighbour slots read meanwhile.
//
// Pass 1: 1/TV_i of every T vertex into inv (0 at every other slot), the
// block's sum of TV_i into partials[block*8 + 3].  The 6 squared differences
// are summed in the order of the single-sweep form (-x, +x, -y, +y, -z, +z),
// so inv is the same.
constexpr int TV2_INV_BLOCKS_PER_SM = 16;
constexpr int TV2_GRAD_BLOCKS_PER_SM = 12;
__global__ void __launch_bounds__(TV2_THREADS, TV2_INV_BLOCKS_PER_SM)
    k_tv_inv(Grid G, const int32_t* __restrict__ coord, const int32_t* __restrict__ nbrs, int64_t n_bricks,
             float* __restrict__ inv, double* __restrict__ partials) {
  __shared__ Tv2Stage s[2];
  __shared__ __align__(16) uint32_t Tw[2][16];
  const int t = threadIdx.x, x = t & 7, y = t >> 3;
  float tsum = 0.f;
  const int64_t first = blockIdx.x, stride = gridDim.x;
  auto issue = [&](int p, const Tv2Brick& k) {
    tv2_issue(s[p], G.D, k);
    if (t < 4) cp_async_cg16(&Tw[p][4 * t], G.masks + k.slot * 48 + 4 * t, 16);
  };
  Tv2Brick cur, nxt;
  if (first < n_bricks) {
    cur = tv2_brick(coord, nbrs, first);
    issue(0, cur);
  }
  cp_async_commit();
  if (first + stride < n_bricks) nxt = tv2_brick(coord, nbrs, first + stride);
  int p = 0;
  for (int64_t b = first; b < n_bricks; b += stride) {
    if (b + stride < n_bricks) issue(p ^ 1, nxt);
    cp_async_commit();
    Tv2Brick after;
    if (b + 2 * stride < n_bricks) after = tv2_brick(coord, nbrs, b + 2 * stride);
    cp_async_wait1();  // this thread's copies of brick b have landed
    __syncthreads();   // ... and everyone's
    const Tv2Stage& S = s[p];
#pragma unroll 2
    for (int z = 0; z < 8; ++z) {
      const int l = (z * 8 + y) * 8 + x;
      float iv = 0.f;
      if ((Tw[p][z * 2 + (y >> 2)] >> ((y & 3) * 8 + x)) & 1u) {
        float n[6];
        bool ok[6];
        tv2_nbrs(S, x, y, z, n);
        tv2_ingrid(cur.ox + x, cur.oy + y, cur.oz + z, G.R, ok);
        const float d = S.c[l];
        float s2 = 0.f;
#pragma unroll
        for (int j = 0; j < 6; ++j) {
          const float e = d - n[j];
          if (ok[j]) s2 = fmaf(e, e, s2);
        }
        iv = s2 > 0.f ? rsqrtf(s2) : 0.f;
        tsum += s2 * iv;
      }
      inv[b * 512 + l] = iv;
    }
    __syncthreads();  // buffer p is free for the copies of brick b + 2 stride
    cur = nxt;
    nxt = after;
    p ^= 1;
  }
  cp_async_wait0();
  __shared__ float red[TV2_THREADS / 32];
  const float w = gp_warp_sum(tsum);
  if ((t & 31) == 0) red[t >> 5] = w;
  __syncthreads();
  if (t == 0) {
    double sum = 0;
    for (int k = 0; k < TV2_THREADS / 32; ++k) sum += red[k];
    partials[(int64_t)blockIdx.x * 8 + 3] = sum;
  }
}

// Pass 2: the gradient of every stored slot, alpha/|T| dTV/dd (0 outside the
// grid), plus, DET, the fixed-point query sums (folded and cleared), in the
// single-sweep form's order of terms.  LAST: this kernel writes the loss slots.
template <bool DET, bool LAST>
__global__ void __launch_bounds__(TV2_THREADS, TV2_GRAD_BLOCKS_PER_SM)
    k_tv_grad(Grid G, const int32_t* __restrict__ coord, const int32_t* __restrict__ nbrs, int64_t n_bricks,
              const float* __restrict__ inv, float tv_scale, float* __restrict__ grad,
              unsigned long long* __restrict__ acc, double* __restrict__ partials, FinalArgs fa) {
  __shared__ Tv2Stage sd[2], si[2];
  const int t = threadIdx.x, x = t & 7, y = t >> 3;
  const int64_t first = blockIdx.x, stride = gridDim.x;
  auto issue = [&](int p, const Tv2Brick& k) {
    tv2_issue(sd[p], G.D, k);
    tv2_issue(si[p], inv, k);
  };
  Tv2Brick cur, nxt;
  if (first < n_bricks) {
    cur = tv2_brick(coord, nbrs, first);
    issue(0, cur);
  }
  cp_async_commit();
  if (first + stride < n_bricks) nxt = tv2_brick(coord, nbrs, first + stride);
  int p = 0;
  for (int64_t b = first; b < n_bricks; b += stride) {
    if (b + stride < n_bricks) issue(p ^ 1, nxt);
    cp_async_commit();
    Tv2Brick after;
    if (b + 2 * stride < n_bricks) after = tv2_brick(coord, nbrs, b + 2 * stride);
    cp_async_wait1();
    __syncthreads();
    const Tv2Stage& SD = sd[p];
    const Tv2Stage& SI = si[p];
#pragma unroll 2
    for (int z = 0; z < 8; ++z) {
      const int l = (z * 8 + y) * 8 + x;
      const int X = cur.ox + x, Y = cur.oy + y, Z = cur.oz + z;
      float nd[6], ni[6];
      bool ok[6];
      tv2_nbrs(SD, x, y, z, nd);
      tv2_nbrs(SI, x, y, z, ni);
      tv2_ingrid(X, Y, Z, G.R, ok);
      const float d = SD.c[l], own = SI.c[l];
      float g = 0.f;
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        // own != 0 only for T vertices, whose in-grid neighbours are all
        // stored; ni[j] != 0 only for neighbours in T.
        if (ok[j]) g = fmaf(d - nd[j], own + ni[j], g);
      }
      float gv = (X <= G.R && Y <= G.R && Z <= G.R) ? tv_scale * g : 0.f;
      const int64_t addr = b * 512 + l;
      if (DET) {
        const long long hi = (long long)acc[2 * addr], lo = (long long)acc[2 * addr + 1];
        acc[2 * addr] = 0ull;
        acc[2 * addr + 1] = 0ull;
        const float qv =
            __fmaf_rn(__ll2float_rn(hi), 9.5367431640625e-07f, __ll2float_rn(lo) * 8.673617379884035e-19f);
        gv = __fadd_rn(qv, gv);
      }
      grad[addr] = gv;
    }
    __syncthreads();
    cur = nxt;
    nxt = after;
    p ^= 1;
  }
  cp_async_wait0();
  if (LAST) finish_if_last(partials, fa);
}

// Adam's hyper-parameters for one step, with the bias corrections.
struct AdamArgs {
  float lr, b1, b2, eps, ibc1, ibc2;  // ibc = 1 / (1 - beta^t)
};

// L_TV and Adam in one sweep over the bricks (gp_step_update), after the
// query pass has added its contributions into qgrad (or, DET, into the
// fixed-point sums).  For every stored vertex of the brick: the gradient is
// alpha/|T| dTV/dd + the query part (which is read and reset to zero); a
// trainable vertex gets Adam's update, written to Dnext with its moments; any
// other vertex is copied to Dnext unchanged.  Reading the stencil from D and
// writing Dnext keeps every brick's neighbours at the step's values; the
// caller swaps the two buffers afterwards.  Each TV_i enters the loss once.
template <bool DET, bool TV>
__global__ void __launch_bounds__(TV_THREADS, TV_BLOCKS_PER_SM) k_tv_adam(
    Grid G, const int32_t* __restrict__ coord, const int32_t* __restrict__ nbrs, int64_t n_bricks, float tv_scale,
    float* __restrict__ qgrad, unsigned long long* __restrict__ acc, float* __restrict__ Dnext, float* __restrict__ m, float* __restrict__ v, AdamArgs ad,
    double* __restrict__ partials, int32_t* __restrict__ err, FinalArgs fa) {
  __shared__ TvShared sh;
  float tsum = 0.f;
  // This thread's two vertices of every brick (those tv_gather hands it), and
  // their Adam operands, loaded at the top of the brick's iteration.
  const int tt = threadIdx.x;
  const int lv[2] = {(tt & 7) + 16 * ((tt >> 3) & 3) + 64 * (tt >> 5), (tt & 7) + 16 * ((tt >> 3) & 3) + 64 * (tt >> 5) + 8};
  float pd[2], pm[2], pv[2], pq[2];
  uint32_t pw[2];
  auto load = [&](int64_t slot, int k, int l) {
    const int64_t addr = slot * 512 + l;
    pd[k] = __ldg(G.D + addr);
    pw[k] = __ldg(G.masks + slot * 48 + 16 + (l >> 5));
    if ((pw[k] >> (l & 31)) & 1u) {
      pm[k] = m[addr];
      pv[k] = v[addr];
      if (DET) {
        const long long hi = (long long)acc[2 * addr], lo = (long long)acc[2 * addr + 1];
        const float qv =
            __fmaf_rn(__ll2float_rn(hi), 9.5367431640625e-07f, __ll2float_rn(lo) * 8.673617379884035e-19f);
        pq[k] = qv;  // already scaled by 1/B_v by the query pass
      } else {
        pq[k] = qgrad[addr];
      }
    }
  };
  auto update = [&](int64_t slot, int k, int l, float g_tv) {
    const int64_t addr = slot * 512 + l;
    if (!((pw[k] >> (l & 31)) & 1u)) {
      Dnext[addr] = pd[k];
      return;
    }
    float g;
    if (DET) {
      acc[2 * addr] = 0ull;
      acc[2 * addr + 1] = 0ull;
      g = __fadd_rn(pq[k], tv_scale * g_tv);
    } else {
      qgrad[addr] = 0.f;
      g = tv_scale * g_tv + pq[k];
    }
    float mm = pm[k], vv = pv[k];
    const float dn = adam_elem(g, mm, vv, pd[k], ad.lr, ad.b1, ad.b2, ad.eps, ad.ibc1, ad.ibc2);
    m[addr] = mm;
    v[addr] = vv;
    Dnext[addr] = dn;
  };
  if (TV) {
    tv_sweep(
        BandTvSrc{G, coord, nbrs}, blockIdx.x, gridDim.x, n_bricks, sh,
        [&](int64_t slot, int l0, float g0, int l1, float g1, float ts) {
          tsum += ts;
          update(slot, 0, l0, g0);
          update(slot, 1, l1, g1);
        },
        [&](int64_t slot) {
          load(slot, 0, lv[0]);
          load(slot, 1, lv[1]);
        });
  } else {
    for (int64_t slot = blockIdx.x; slot < n_bricks; slot += gridDim.x) {
      load(slot, 0, threadIdx.x);
      load(slot, 1, threadIdx.x + 256);
      update(slot, 0, threadIdx.x, 0.f);
      update(slot, 1, threadIdx.x + 256, 0.f);
    }
  }
  __shared__ float red[TV_THREADS / 32];
  const float wsum = gp_warp_sum(tsum);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = wsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0;
    for (int k = 0; k < TV_THREADS / 32; ++k) sum += red[k];
    partials[(int64_t)blockIdx.x * 8 + 3] = sum;
  }
  finish_if_last(partials, fa);
  (void)err;
}

// One thread per 4 consecutive vertices of an active brick (128 per brick).
__global__ void __launch_bounds__(256) k_adam(const int32_t* __restrict__ active, int64_t n_active,
                                              const uint32_t* __restrict__ masks, const float* __restrict__ grad,
                                              float* __restrict__ D, float* __restrict__ m, float* __restrict__ v,
                                              float lr, float b1, float b2, float eps, float ibc1, float ibc2) {
  const int64_t n = n_active * 128;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    adam_quad(__ldg(active + (i >> 7)), (int)(i & 127), masks, grad, D, m, v, lr, b1, b2, eps, ibc1, ibc2);
}

// One resident wave of k_query: each thread takes several records and the
// block's loss reduction runs once per thread instead of once per record.
unsigned q_grid(const gp_ctx* ctx, int64_t B) {
  int64_t cap = (int64_t)ctx->num_sms * Q_BLOCKS_PER_SM;
  if (cap > GP_MAX_PARTIAL_BLOCKS) cap = GP_MAX_PARTIAL_BLOCKS;
  return gp_blocks(B, Q_THREADS, cap);
}

unsigned tv2_grid(const gp_ctx* ctx, int64_t n_bricks, int per_sm) {
  int64_t cap = (int64_t)ctx->num_sms * per_sm;
  if (cap > GP_MAX_PARTIAL_BLOCKS) cap = GP_MAX_PARTIAL_BLOCKS;
  return gp_blocks(n_bricks, 1, cap);
}

unsigned tv_grid(const gp_ctx* ctx, int64_t n_bricks) {
  int64_t cap = (int64_t)ctx->num_sms * TV_BLOCKS_PER_SM;  // persistent: one wave
  if (cap > GP_MAX_PARTIAL_BLOCKS) cap = GP_MAX_PARTIAL_BLOCKS;
  return gp_blocks(n_bricks, 1, cap);
}

}  // namespace

extern "C" gp_status gp_step(gp_band* b, const float* rec_dev, int64_t B, const int32_t* nvalid_dev,
                             const float* d_dev, const gp_loss_w* w, float* grad_dev, float* loss_dev,
                             uint32_t flags) {
  if (!b) return GP_ERR_ARG;
  gp_ctx* ctx = b->ctx;
  if (B < 0 || B >= (int64_t(1) << 31)) return gp_fail(ctx, GP_ERR_ARG, "gp_step: B must be in [0, 2^31)");
  if (!loss_dev || !w || (B > 0 && !rec_dev)) return gp_fail(ctx, GP_ERR_ARG, "gp_step: null pointer");
  const bool grad_on = !(flags & GP_STEP_LOSS_ONLY);
  const bool det = (flags & GP_STEP_DETERMINISTIC) != 0;
  const bool tv_on = !(flags & GP_STEP_NO_TV);
  if (grad_on && !grad_dev) return gp_fail(ctx, GP_ERR_ARG, "gp_step: null gradient output");
  if (((uintptr_t)rec_dev & 7u) != 0) return gp_fail(ctx, GP_ERR_ARG, "gp_step: records must be 8-byte aligned");
  if (((uintptr_t)grad_dev & 15u) != 0)
    return gp_fail(ctx, GP_ERR_ARG, "gp_step: the gradient must be 16-byte aligned");
  if (((uintptr_t)d_dev & 15u) != 0) return gp_fail(ctx, GP_ERR_ARG, "gp_step: the values must be 16-byte aligned");
  if (det && grad_on && !b->acc)
    return gp_fail(ctx, GP_ERR_STATE, "gp_step: deterministic mode needs a band built with GP_BAND_DETERMINISTIC");
  cudaStream_t s = ctx->stream;
  Grid G;
  G.table = b->brick_table;
  G.masks = b->masks;
  G.D = d_dev ? d_dev : b->D;
  G.nb = b->nb;
  G.R = b->R;
  G.half_r = 0.5f * (float)b->R;
  int32_t* err = b->dev_ints + GP_DI_ERROR;
  // B_v: given by the caller (e.g. counted by gp_nn) or counted here.
  const int32_t* bv = nvalid_dev;
  if (!bv) {
    int32_t* cnt = b->dev_ints + GP_DI_NVALID;
    GP_CUDA(ctx, cudaMemsetAsync(cnt, 0, sizeof(int32_t), s));
    if (B > 0) {
      GP_KERNEL(ctx, "k_count_valid", k_count_valid<<<q_grid(ctx, B), Q_THREADS, 0, s>>>(G, rec_dev, B, cnt));
    }
    bv = cnt;
  }
  const unsigned qb = q_grid(ctx, B);
  const unsigned tb = b->n_bricks ? tv_grid(ctx, b->n_bricks) : 1;
  const float tv_scale = (tv_on && b->V_tv > 0) ? w->alpha / (float)b->V_tv : 0.f;
  FinalArgs fa;
  fa.done = b->dev_ints + GP_DI_DONE;
  fa.q_blocks = (int)qb;
  fa.tv_blocks = (int)tb;
  fa.bv = bv;
  fa.n_tv = b->V_tv;
  fa.alpha = w->alpha;
  fa.beta = w->beta;
  fa.gamma = w->gamma;
  fa.tv_on = tv_on ? 1 : 0;
  fa.loss = loss_dev;
  // The TV sweep writes (overwrites) the gradient and the query pass adds to
  // it; in deterministic mode the query pass fills the fixed-point sums first
  // and the sweep folds them in.  Whichever runs second writes the loss.
  const bool tv_last = det && grad_on;
  const unsigned tb2 = b->n_bricks ? tv2_grid(ctx, b->n_bricks, TV2_INV_BLOCKS_PER_SM) : 1;
  const unsigned tg2 = b->n_bricks ? tv2_grid(ctx, b->n_bricks, TV2_GRAD_BLOCKS_PER_SM) : 1;
  if (tv_on) fa.tv_blocks = (int)tb2;
  auto launch_tv = [&]() -> gp_status {
    if (b->n_bricks == 0) {
      GP_CUDA(ctx, cudaMemsetAsync(b->partials + 3, 0, sizeof(double), s));
      return GP_OK;
    }
    if (tv_on) {
      // Two passes: 1/TV of the T vertices, then the gradient of every slot.
      GP_KERNEL(ctx, "k_tv_inv",
                k_tv_inv<<<tb2, TV2_THREADS, 0, s>>>(G, b->brick_coord, b->brick_nbr, b->n_bricks, b->tv_inv,
                                                      b->partials));
      if (!grad_on) return GP_OK;
#define GP_TV2(D_, L_)                                                                                          \
  k_tv_grad<D_, L_><<<tg2, TV2_THREADS, 0, s>>>(G, b->brick_coord, b->brick_nbr, b->n_bricks, b->tv_inv, tv_scale, \
                                                grad_dev, b->acc, b->partials, fa)
      if (tv_last)
        GP_KERNEL(ctx, "k_tv_grad", GP_TV2(true, true));
      else
        GP_KERNEL(ctx, "k_tv_grad", GP_TV2(false, false));
#undef GP_TV2
      return GP_OK;
    }
#define GP_TV(D_, G_, T_, L_)                                                                                  \
  k_tv<D_, G_, T_, L_><<<tb, TV_THREADS, 0, s>>>(G, b->brick_coord, b->brick_nbr, b->n_bricks, tv_scale, grad_dev, \
                                                 b->acc, b->partials, err, fa)
    gp_prof_pre(ctx);
    if (tv_last) {
      if (tv_on) GP_TV(true, true, true, true); else GP_TV(true, true, false, true);
    } else if (grad_on) {
      if (tv_on) GP_TV(false, true, true, false); else GP_TV(false, true, false, false);
    } else {
      if (tv_on) GP_TV(false, false, true, false); else GP_TV(false, false, false, false);
    }
#undef GP_TV
    gp_prof_post(ctx, "k_tv");
    GP_LAUNCH_CHECK(ctx, "k_tv");
    return GP_OK;
  };
  auto launch_q = [&]() -> gp_status {
    gp_prof_pre(ctx);
    cudaError_t e = cudaSuccess;
    if (det && grad_on) {
      e = launch_query_tuned<true, false>(b, B, s, G, rec_dev, bv, w->beta, w->gamma, grad_dev, b->partials, err,
                                          fa);
    } else if (grad_on) {
      e = launch_query_tuned<false, true>(b, B, s, G, rec_dev, bv, w->beta, w->gamma, grad_dev, b->partials, err,
                                          fa);
    } else {
      k_query<false, false, true><<<qb, Q_THREADS, 0, s>>>(G, rec_dev, B, bv, w->beta, w->gamma, grad_dev, b->acc,
                                                           b->partials, err, fa);
    }
    gp_prof_post(ctx, "k_query");
    if (e != cudaSuccess) return gp_cuda_fail(ctx, e, "k_query");
    GP_LAUNCH_CHECK(ctx, "k_query");
    return GP_OK;
  };
  gp_status st;
  if (tv_last) {
    if ((st = launch_q())) return st;
    if (b->n_bricks == 0) return gp_fail(ctx, GP_ERR_STATE, "gp_step: empty band");
    if ((st = launch_tv())) return st;
  } else {
    if ((st = launch_tv())) return st;
    if ((st = launch_q())) return st;
  }
  return GP_OK;
}

extern "C" gp_status gp_update(gp_band* b, const float* grad_dev, const gp_adam* hp, int64_t step) {
  if (!b) return GP_ERR_ARG;
  gp_ctx* ctx = b->ctx;
  if (!grad_dev || !hp) return gp_fail(ctx, GP_ERR_ARG, "gp_update: null pointer");
  if (step < 1) return gp_fail(ctx, GP_ERR_ARG, "gp_update: step must be >= 1");
  if (b->n_active == 0) return GP_OK;
  double bc1 = 1.0 - std::pow((double)hp->beta1, (double)step);
  double bc2 = 1.0 - std::pow((double)hp->beta2, (double)step);
  int64_t cap = (int64_t)ctx->num_sms * 8;
  GP_KERNEL(ctx, "k_adam", k_adam<<<gp_blocks(b->n_active * 128, 256, cap), 256, 0, ctx->stream>>>(b->active, b->n_active, b->masks, grad_dev, b->D,
                                                                  b->m, b->v, hp->lr, hp->beta1, hp->beta2, hp->eps,
                                                                  (float)(1.0 / bc1), (float)(1.0 / bc2)));
  return GP_OK;
}

// Times the fused step kernel's launch shapes on the given records and keeps
// the fastest in the band: records in flight per thread (1 or 2) and the
// resident blocks per SM it is compiled for (2, 3 or 4, i.e. a cap of 128, 80
// or 64 registers per thread).  The band's
// values are read, nothing of the band is written; a scratch gradient and
// loss are allocated and freed.
extern "C" gp_status gp_band_autotune(gp_band* b, const float* rec_dev, int64_t B, const int32_t* nvalid_dev,
                                      const gp_loss_w* w, int32_t* rpt_out, int32_t* bps_out) {
  if (!b) return GP_ERR_ARG;
  gp_ctx* ctx = b->ctx;
  if (B <= 0 || B >= (int64_t(1) << 31) || !rec_dev || !w)
    return gp_fail(ctx, GP_ERR_ARG, "gp_band_autotune: need 0 < B < 2^31 records and weights");
  if (((uintptr_t)rec_dev & 7u) != 0) return gp_fail(ctx, GP_ERR_ARG, "gp_band_autotune: records must be 8-byte aligned");
  cudaStream_t s = ctx->stream;
  float* grad = nullptr;
  float* loss = nullptr;
  gp_status st = gp_alloc(ctx, &grad, b->V_stored(), "autotune gradient");
  if (st) return st;
  if ((st = gp_alloc(ctx, &loss, 8, "autotune loss"))) {
    cudaFree(grad);
    return st;
  }
  Grid G;
  G.table = b->brick_table;
  G.masks = b->masks;
  G.D = b->D;
  G.nb = b->nb;
  G.R = b->R;
  G.half_r = 0.5f * (float)b->R;
  int32_t* err = b->dev_ints + GP_DI_ERROR;
  const int32_t* bv = nvalid_dev;
  cudaError_t e = cudaSuccess;
  if (!bv) {
    int32_t* cnt = b->dev_ints + GP_DI_NVALID;
    e = cudaMemsetAsync(cnt, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) {
      k_count_valid<<<q_grid(ctx, B), Q_THREADS, 0, s>>>(G, rec_dev, B, cnt);
      e = cudaGetLastError();
    }
    bv = cnt;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  int best_rpt = b->q_rpt, best_bps = b->q_bps;
  float best = INFINITY;
  const int rpts[2] = {1, 2}, bpss[3] = {2, 3, 4};
  const int save_rpt = b->q_rpt, save_bps = b->q_bps, save_form = b->q_form;
  b->q_form = GP_QUERY_DIRECT;
  for (int ri = 0; ri < 2 && e == cudaSuccess; ++ri) {
    for (int bi = 0; bi < 3 && e == cudaSuccess; ++bi) {
      b->q_rpt = rpts[ri];
      b->q_bps = bpss[bi];
      FinalArgs fa;
      fa.done = b->dev_ints + GP_DI_DONE;
      fa.q_blocks = 0;
      fa.tv_blocks = 0;
      fa.bv = bv;
      fa.n_tv = b->V_tv;
      fa.alpha = w->alpha;
      fa.beta = w->beta;
      fa.gamma = w->gamma;
      fa.tv_on = 0;
      fa.loss = loss;
      auto launch = [&]() -> cudaError_t {
        return launch_query_tuned<false, true>(b, B, s, G, rec_dev, bv, w->beta, w->gamma, grad, b->partials, err,
                                               fa);
      };
      e = launch();  // warm-up
      if (e == cudaSuccess) e = cudaEventRecord(e0, s);
      for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = launch();
      if (e == cudaSuccess) e = cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e == cudaSuccess && ms < best) {
        best = ms;
        best_rpt = rpts[ri];
        best_bps = bpss[bi];
      }
    }
  }
  // The windowed forms at the same shapes (the staged one at 2 blocks per
  // SM only), timed the same way.
  int best_form = GP_QUERY_DIRECT;
  const int wcand[8][3] = {{GP_QUERY_WINDOW, 1, 2}, {GP_QUERY_WINDOW, 1, 3}, {GP_QUERY_WINDOW, 1, 4},
                           {GP_QUERY_WINDOW, 2, 2}, {GP_QUERY_WINDOW, 2, 3}, {GP_QUERY_WINDOW, 2, 4},
                           {GP_QUERY_WINDOW_STAGED, 1, 2}, {GP_QUERY_WINDOW_STAGED, 2, 2}};
  for (int fi = 0; fi < 8 && e == cudaSuccess; ++fi) {
    b->q_form = wcand[fi][0];
    b->q_rpt = wcand[fi][1];
    b->q_bps = wcand[fi][2];
    FinalArgs fa;
    fa.done = b->dev_ints + GP_DI_DONE;
    fa.q_blocks = 0;
    fa.tv_blocks = 0;
    fa.bv = bv;
    fa.n_tv = b->V_tv;
    fa.alpha = w->alpha;
    fa.beta = w->beta;
    fa.gamma = w->gamma;
    fa.tv_on = 0;
    fa.loss = loss;
    auto launch = [&]() -> cudaError_t {
      return launch_query_tuned<false, true>(b, B, s, G, rec_dev, bv, w->beta, w->gamma, grad, b->partials, err, fa);
    };
    e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && ms < best) {
      best = ms;
      best_form = wcand[fi][0];
      best_rpt = wcand[fi][1];
      best_bps = wcand[fi][2];
    }
  }
  b->q_form = save_form;
  b->q_rpt = save_rpt;
  b->q_bps = save_bps;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  cudaFree(grad);
  cudaFree(loss);
  if (e != cudaSuccess) return gp_cuda_fail(ctx, e, "gp_band_autotune");
  b->q_rpt = best_rpt;
  b->q_bps = best_bps;
  b->q_form = best_form;
  if (rpt_out) *rpt_out = best_rpt;
  if (bps_out) *bps_out = best_bps;
  return GP_OK;
}

extern "C" gp_status gp_band_set_query_tiles(gp_band* b, int32_t rpt, int32_t bps) {
  if (!b) return GP_ERR_ARG;
  if (!(rpt == 1 || rpt == 2) || bps < 2 || bps > 4)
    return gp_fail(b->ctx, GP_ERR_ARG, "gp_band_set_query_tiles: rpt must be 1 or 2 and bps 2, 3 or 4");
  b->q_rpt = rpt;
  b->q_bps = bps;
  return GP_OK;
}

extern "C" gp_status gp_band_set_query_form(gp_band* b, int32_t form) {
  if (!b) return GP_ERR_ARG;
  if (form != GP_QUERY_DIRECT && form != GP_QUERY_WINDOW && form != GP_QUERY_WINDOW_STAGED)
    return gp_fail(b->ctx, GP_ERR_ARG, "gp_band_set_query_form: form must be a GP_QUERY_* value");
  b->q_form = form;
  return GP_OK;
}

extern "C" gp_status gp_band_query_shape(const gp_band* b, int32_t* rpt_out, int32_t* bps_out, int32_t* form_out) {
  if (!b) return GP_ERR_ARG;
  if (rpt_out) *rpt_out = b->q_rpt;
  if (bps_out) *bps_out = b->q_bps;
  if (form_out) *form_out = b->q_form;
  return GP_OK;
}

extern "C" gp_status gp_step_update(gp_band* b, const float* rec_dev, int64_t B, const int32_t* nvalid_dev,
                                    const gp_loss_w* w, const gp_adam* hp, int64_t step, float* loss_dev,
                                    uint32_t flags) {
  if (!b) return GP_ERR_ARG;
  gp_ctx* ctx = b->ctx;
  if (B < 0 || B >= (int64_t(1) << 31)) return gp_fail(ctx, GP_ERR_ARG, "gp_step_update: B must be in [0, 2^31)");
  if (!loss_dev || !w || !hp || (B > 0 && !rec_dev)) return gp_fail(ctx, GP_ERR_ARG, "gp_step_update: null pointer");
  if (step < 1) return gp_fail(ctx, GP_ERR_ARG, "gp_step_update: step must be >= 1");
  if (flags & ~(GP_STEP_DETERMINISTIC | GP_STEP_NO_TV))
    return gp_fail(ctx, GP_ERR_ARG, "gp_step_update: flags may only be GP_STEP_DETERMINISTIC and GP_STEP_NO_TV");
  const bool det = (flags & GP_STEP_DETERMINISTIC) != 0;
  const bool tv_on = !(flags & GP_STEP_NO_TV);
  if (((uintptr_t)rec_dev & 7u) != 0) return gp_fail(ctx, GP_ERR_ARG, "gp_step_update: records must be 8-byte aligned");
  if (det && !b->acc)
    return gp_fail(ctx, GP_ERR_STATE,
                   "gp_step_update: deterministic mode needs a band built with GP_BAND_DETERMINISTIC");
  if (b->n_bricks == 0) return gp_fail(ctx, GP_ERR_STATE, "gp_step_update: empty band");
  cudaStream_t s = ctx->stream;
  Grid G;
  G.table = b->brick_table;
  G.masks = b->masks;
  G.D = b->D;
  G.nb = b->nb;
  G.R = b->R;
  G.half_r = 0.5f * (float)b->R;
  int32_t* err = b->dev_ints + GP_DI_ERROR;
  const int32_t* bv = nvalid_dev;
  if (!bv) {
    int32_t* cnt = b->dev_ints + GP_DI_NVALID;
    GP_CUDA(ctx, cudaMemsetAsync(cnt, 0, sizeof(int32_t), s));
    if (B > 0) {
      GP_KERNEL(ctx, "k_count_valid", k_count_valid<<<q_grid(ctx, B), Q_THREADS, 0, s>>>(G, rec_dev, B, cnt));
    }
    bv = cnt;
  }
  const unsigned tb = tv_grid(ctx, b->n_bricks);
  FinalArgs fa;
  fa.done = b->dev_ints + GP_DI_DONE;
  fa.q_blocks = 0;
  fa.tv_blocks = (int)tb;
  fa.bv = bv;
  fa.n_tv = b->V_tv;
  fa.alpha = w->alpha;
  fa.beta = w->beta;
  fa.gamma = w->gamma;
  fa.tv_on = tv_on ? 1 : 0;
  fa.loss = loss_dev;
  // The query pass: its contributions into the band's zeroed query gradient
  // (or the fixed-point sums); its block sums are finished by the sweep.
  gp_prof_pre(ctx);
  cudaError_t e = det ? launch_query_tuned<true, false>(b, B, s, G, rec_dev, bv, w->beta, w->gamma, b->qgrad,
                                                        b->partials, err, fa)
                      : launch_query_tuned<false, false>(b, B, s, G, rec_dev, bv, w->beta, w->gamma, b->qgrad,
                                                         b->partials, err, fa);
  gp_prof_post(ctx, "k_query");
  if (e != cudaSuccess) return gp_cuda_fail(ctx, e, "k_query");
  GP_LAUNCH_CHECK(ctx, "k_query");
  AdamArgs ad;
  ad.lr = hp->lr;
  ad.b1 = hp->beta1;
  ad.b2 = hp->beta2;
  ad.eps = hp->eps;
  ad.ibc1 = (float)(1.0 / (1.0 - std::pow((double)hp->beta1, (double)step)));
  ad.ibc2 = (float)(1.0 / (1.0 - std::pow((double)hp->beta2, (double)step)));
  const float tv_scale = (tv_on && b->V_tv > 0) ? w->alpha / (float)b->V_tv : 0.f;
  gp_prof_pre(ctx);
#define GP_TVA(D_, T_)                                                                                             \
  k_tv_adam<D_, T_><<<tb, TV_THREADS, 0, s>>>(G, b->brick_coord, b->brick_nbr, b->n_bricks, tv_scale, b->qgrad,  \
                                              b->acc, b->D_alt, b->m, b->v, ad, b->partials, err, fa)
  if (det) {
    if (tv_on) GP_TVA(true, true); else GP_TVA(true, false);
  } else {
    if (tv_on) GP_TVA(false, true); else GP_TVA(false, false);
  }
#undef GP_TVA
  gp_prof_post(ctx, "k_tv_adam");
  GP_LAUNCH_CHECK(ctx, "k_tv_adam");
  std::swap(b->D, b->D_alt);
  return GP_OK;
}
