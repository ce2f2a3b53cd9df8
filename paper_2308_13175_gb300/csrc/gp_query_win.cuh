// The windowed form of the fused forward + backward pass (Eq. 3-8 per
// record, as in gp_step_device.cuh), for batches in spatial order.
//
// A block takes tiles of 256 x RPT consecutive records.  Records in spatial
// order (the sampler's GP_SAMPLE_SPATIAL batches: by source point, the points
// in Morton order of their cells) lie close together, and so do the corners
// their gradients go to.  Each tile gets a window: the 3 x 3 x 3 bricks
// around the brick of its middle record's NN(q) (the anchor), their slots
// taken from the anchor's row of the band's 27-neighbour table.
//   * Corner gradients of every cell whose 8 corners lie in stored window
//     bricks are added into a shared-memory copy of the window (55 KB) and
//     written to the gradient once per tile, one 16-byte vector reduction per
//     non-zero group of four slots: a block-level segmented reduction in
//     place of one global reduction per cell edge.  Cells outside the window
//     take the direct vector reductions.
//   * STAGE: the window bricks' values and pull-band masks are staged in
//     shared memory by bulk copies (cp.async.bulk, completion counted on an
//     mbarrier), issued for the next tile while the current tile's window is
//     written out; in-window cells then read no global memory.  Without
//     STAGE they are gathered from global memory, their brick slots read
//     from the window's slot list instead of the brick table.
// The results are those of the direct form up to the order of the float
// additions.
#pragma once

#include "gp_step_device.cuh"

constexpr int WQ_THREADS = 256;
constexpr int WIN_BRICKS = 27;                 // 3 x 3 x 3 bricks
constexpr int WIN_V = WIN_BRICKS * 512;        // 13,824 slots
// Dynamic shared memory: the gradient window, then (STAGE) the staged values
// and the pull-mask words of the window bricks.
constexpr size_t WQ_SMEM_ACC = sizeof(float) * WIN_V;
constexpr size_t WQ_SMEM_STAGED = WQ_SMEM_ACC + sizeof(float) * WIN_V + sizeof(uint32_t) * WIN_BRICKS * 16;
// A bounded wait for the staged copies: after this many cycles (about a
// second) the kernel raises GP_EF_TIMEOUT instead of waiting on.
constexpr long long WQ_WAIT_CYCLES = 2000000000ll;

// One tile's window as every thread holds it.
struct Win {
  int lo[3];         // vertex coordinates of the window's lowest corner ((anchor brick - 1) * 8)
  uint32_t present;  // bit k: window brick k (x fastest) is stored
};

// Window brick (0..26) of the lowest corner of cell c when all 8 corners lie
// in stored bricks of the window, else -1.  Integer arithmetic only: a host
// build of it and win_corner is checked on the CPU against the definition.
__host__ __device__ __forceinline__ int win_cell(const Win& W, const int c[3]) {
  const int rx = c[0] - W.lo[0], ry = c[1] - W.lo[1], rz = c[2] - W.lo[2];
  if ((unsigned)rx > 22u || (unsigned)ry > 22u || (unsigned)rz > 22u) return -1;
  const int b0 = (rx >> 3) + 3 * (ry >> 3) + 9 * (rz >> 3);
  // The bricks of the 8 corners: b0 plus, along each axis whose cell edge
  // crosses a brick face, the next brick.
  uint32_t need = 1u << b0;
  need |= need << (((rx + 1) >> 3) - (rx >> 3));
  need |= need << (3 * (((ry + 1) >> 3) - (ry >> 3)));
  need |= need << (9 * (((rz + 1) >> 3) - (rz >> 3)));
  return (need & ~W.present) ? -1 : b0;
}

// Window brick and in-brick slot of corner (dx, dy, dz) of an in-window cell c.
__host__ __device__ __forceinline__ int win_corner(const Win& W, const int c[3], int dx, int dy, int dz,
                                                   int& local) {
  const int x = c[0] + dx, y = c[1] + dy, z = c[2] + dz;
  local = gp_local(x, y, z);
  return ((x - W.lo[0]) >> 3) + 3 * ((y - W.lo[1]) >> 3) + 9 * ((z - W.lo[2]) >> 3);
}

// The 8 corner values of an in-window cell; window brick k's 512 values at
// brick(k) (shared memory when staged, the band's slot otherwise).
template <bool SMEM, class BrickPtr>
__device__ __forceinline__ void win_corners(const Win& W, const int c[3], int b0, BrickPtr brick, float d[8]) {
  auto ld = [](const float* p) { return SMEM ? *p : __ldg(p); };
  if ((c[0] & 7) != 7 && (c[1] & 7) != 7 && (c[2] & 7) != 7) {
    const float* base = brick(b0) + gp_local(c[0], c[1], c[2]);
    const int xm = c[0] & 3;
    if ((xm & 1) == 0) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float2* p = reinterpret_cast<const float2*>(base + (e & 1) * 8 + (e >> 1) * 64);
        const float2 v = SMEM ? *p : __ldg(p);
        d[2 * e] = v.x;
        d[2 * e + 1] = v.y;
      }
    } else if (xm == 1) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float4* p = reinterpret_cast<const float4*>(base - 1 + (e & 1) * 8 + (e >> 1) * 64);
        const float4 v = SMEM ? *p : __ldg(p);
        d[2 * e] = v.y;
        d[2 * e + 1] = v.z;
      }
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) d[k] = ld(base + (k & 1) + ((k >> 1) & 1) * 8 + (k >> 2) * 64);
    }
    return;
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    int local;
    const int wb = win_corner(W, c, k & 1, (k >> 1) & 1, k >> 2, local);
    d[k] = ld(brick(wb) + local);
  }
}

// Where a record's corner contributions go in the windowed form: cells in
// the window into the shared-memory sums, the others straight to the gradient.
struct WindowSink {
  const Grid& G;
  float* __restrict__ grad;
  float* acc;  // shared: WIN_V sums
  const Win& W;
  int32_t* __restrict__ err;
  __device__ __forceinline__ void cell(const int c[3], int slot, const float t[3], float A, const float Gt[3]) {
    const int b0 = win_cell(W, c);
    if (b0 < 0) {
      scatter8<false>(G, grad, nullptr, err, c, slot, t, A, Gt);
      return;
    }
    float v[8];
    corner_values(t, A, Gt, v);
    if ((c[0] & 7) != 7 && (c[1] & 7) != 7 && (c[2] & 7) != 7) {
      float* base = acc + b0 * 512 + gp_local(c[0], c[1], c[2]);
#pragma unroll
      for (int k = 0; k < 8; ++k) atomicAdd(base + (k & 1) + ((k >> 1) & 1) * 8 + (k >> 2) * 64, v[k]);
      return;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      int local;
      const int wb = win_corner(W, c, k & 1, (k >> 1) & 1, k >> 2, local);
      atomicAdd(acc + wb * 512 + local, v[k]);
    }
  }
};

// Phase a of a record in the windowed form: the cells, and the brick slots
// of cells outside the window (from the brick table).  In-window cells get
// their slot from the window's list (unused when staged).
template <bool STAGE>
__device__ __forceinline__ void win_phase_a(const Grid& G, const Win& W, const int* wslot, const float q[3],
                                            const float s[3], bool active, RecState& R) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    R.q[a] = q[a];
    R.s[a] = s[a];
  }
  R.ok = active && classify_cells(G, q, s, R.C);
  if (!R.ok) return;
  const int bq = win_cell(W, R.C.cq), bs = win_cell(W, R.C.cs);
  R.C.slot_q = bq >= 0 ? (STAGE ? 0 : wslot[bq]) : gp_brick_slot(G.table, G.nb, R.C.cq[0], R.C.cq[1], R.C.cq[2]);
  R.C.slot_s = bs >= 0 ? (STAGE ? 0 : wslot[bs]) : gp_brick_slot(G.table, G.nb, R.C.cs[0], R.C.cs[1], R.C.cs[2]);
}

// Phase b: the pull-mask words and the 16 corner values, from the staged
// window (STAGE), the window's slots, or the band.
template <bool STAGE>
__device__ __forceinline__ void win_phase_b(const Grid& G, const Win& W, const int* wslot, const float* val,
                                            const uint32_t* pull, RecState& R) {
  if (!R.ok) return;
  if (R.C.slot_q < 0 || R.C.slot_s < 0) {
    R.ok = false;
    return;
  }
  R.lq = gp_local(R.C.cq[0], R.C.cq[1], R.C.cq[2]);
  R.ls = gp_local(R.C.cs[0], R.C.cs[1], R.C.cs[2]);
  R.corners = true;
  const int bq = win_cell(W, R.C.cq), bs = win_cell(W, R.C.cs);
  auto staged = [val](int k) { return val + k * 512; };
  auto banded = [&G, wslot](int k) { return G.D + (int64_t)wslot[k] * 512; };
  if (bq >= 0 && STAGE) {
    R.wq = pull[bq * 16 + (R.lq >> 5)];
    win_corners<true>(W, R.C.cq, bq, staged, R.dq);
  } else if (bq >= 0) {
    R.wq = __ldg(G.masks + (int64_t)R.C.slot_q * 48 + 32 + (R.lq >> 5));
    win_corners<false>(W, R.C.cq, bq, banded, R.dq);
  } else {
    R.wq = __ldg(G.masks + (int64_t)R.C.slot_q * 48 + 32 + (R.lq >> 5));
    load_corners(G, R.C.cq, R.C.slot_q, R.dq, R.corners);
  }
  if (bs >= 0 && STAGE) {
    R.ws = pull[bs * 16 + (R.ls >> 5)];
    win_corners<true>(W, R.C.cs, bs, staged, R.ds);
  } else if (bs >= 0) {
    R.ws = __ldg(G.masks + (int64_t)R.C.slot_s * 48 + 32 + (R.ls >> 5));
    win_corners<false>(W, R.C.cs, bs, banded, R.ds);
  } else {
    R.ws = __ldg(G.masks + (int64_t)R.C.slot_s * 48 + 32 + (R.ls >> 5));
    load_corners(G, R.C.cs, R.C.slot_s, R.ds, R.corners);
  }
}

// The window of tile `tile` (warp 0, all lanes): anchor = the brick of the
// clamped cell of the middle record's s; slot[k] = the anchor's 27-neighbour
// row; present = the stored ones.  An absent anchor (a non-finite s, or a
// brick the band does not store) or a tile past the end gives an empty
// window, and every cell of the tile then takes the direct path.
__device__ __forceinline__ void win_setup(const Grid& G, const int32_t* __restrict__ nbrs,
                                          const float* __restrict__ rec, int64_t B, int tile_n, int64_t tile,
                                          int64_t ntiles, int* slot, int* lo, uint32_t* present) {
  const int lane = threadIdx.x & 31;
  int sl = -1;
  int c[3] = {0, 0, 0};
  if (tile < ntiles) {
    const int64_t t0 = tile * tile_n;
    const int64_t n = B - t0 < tile_n ? B - t0 : tile_n;
    float q[3], s[3];
    load_rec(rec, t0 + n / 2, q, s);
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const gp_cell1 h = gp_cell_exact(s[a], G.half_r);
      if (h.c == -(1 << 30)) ok = false;
      c[a] = min(max(h.c, 0), G.R - 1);
    }
    if (ok) sl = gp_brick_slot(G.table, G.nb, c[0], c[1], c[2]);
  }
  int mine = -1;
  if (sl >= 0 && lane < WIN_BRICKS) mine = __ldg(nbrs + (int64_t)WIN_BRICKS * sl + lane);
  const uint32_t pres = __ballot_sync(0xffffffffu, mine >= 0);
  if (lane < WIN_BRICKS) slot[lane] = mine;
  if (lane == 0) {
#pragma unroll
    for (int a = 0; a < 3; ++a) lo[a] = ((c[a] >> 3) - 1) * 8;
    *present = pres;
  }
}

// --------------------------------------------- bulk copies and the mbarrier
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, uint32_t bytes) {
  asm volatile(
      "{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(smem_u32(bar)),
      "r"(bytes)
      : "memory");
}

// Waits until the barrier's phase of the given parity has completed, for at
// most WQ_WAIT_CYCLES; returns false when the wait ran out.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > WQ_WAIT_CYCLES) return false;
  }
}

// One bulk copy global -> shared of `bytes` (a multiple of 16; both
// addresses 16-byte aligned), its completion counted on bar.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Thread 0: the bulk copies of a window's stored bricks (2 KB of values and
// the 64-byte pull-mask row each) into the staging buffers.  Earlier generic
// reads of the buffers are ordered before the copies by the barrier the
// caller passed and the proxy fence here.
__device__ __forceinline__ void win_issue(const Grid& G, const int* slot, uint32_t present, float* val,
                                          uint32_t* pull, unsigned long long* bar) {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  mbar_arrive_expect_tx(bar, (uint32_t)__popc(present) * (2048u + 64u));
  for (int k = 0; k < WIN_BRICKS; ++k) {
    if (!((present >> k) & 1u)) continue;
    const int64_t sl = slot[k];
    bulk_g2s(val + k * 512, G.D + sl * 512, 2048u, bar);
    bulk_g2s(pull + k * 16, G.masks + sl * 48 + 32, 64u, bar);
  }
}

// Adds the tile's window sums to the gradient (one 16-byte reduction per
// non-zero group of four slots) and clears them.  Only stored window bricks
// receive contributions.
__device__ __forceinline__ void win_flush(float* acc, const int* slot, float* __restrict__ grad) {
  float4* a4 = reinterpret_cast<float4*>(acc);
  for (int g = threadIdx.x; g < WIN_V / 4; g += WQ_THREADS) {
    const float4 v = a4[g];
    if (v.x != 0.f || v.y != 0.f || v.z != 0.f || v.w != 0.f) {
      const int sl = slot[g >> 7];
      if (sl >= 0) red_add_v4(grad + (int64_t)sl * 512 + (g & 127) * 4, v.x, v.y, v.z, v.w);
      a4[g] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
}
