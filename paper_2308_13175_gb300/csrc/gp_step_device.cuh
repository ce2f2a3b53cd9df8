// Device functions of the step shared by the single-band kernels (gp_step.cu)
// and the many-band kernels (gp_multi.cu): Eq. 3 interpolation, the per-record
// forward + hand-written backward, one brick of the L_TV sweep, one Adam update.
// The formulas are stated in the header comment of gp_step.cu.
#pragma once

#include "gp_internal.cuh"

constexpr float NORM_FLOOR = 1e-12f;
// Deterministic sums: each contribution v is split into two integers,
// hi = round(v * 2^20) and lo = round((v - hi * 2^-20) * 2^60), accumulated
// with 64-bit integer atomics (exact, so the order of the additions does not
// matter).  The sum is hi * 2^-20 + lo * 2^-60: a resolution of 2^-60, no
// overflow below 2^42 per contribution and 2^23 contributions per vertex.
constexpr double FIX_HI = 1048576.0;                     // 2^20
constexpr double FIX_LO = 1152921504606846976.0;         // 2^60
constexpr double FIX_LIMIT = 4398046511104.0;            // 2^42

struct Eval {
  float f;
  float gt[3];  // df/dt (t = local coordinate in cell units)
};

__device__ __forceinline__ void load_corners(const Grid& G, const int c[3], int slot, float d[8], bool& ok) {
  if ((c[0] & 7) != 7 && (c[1] & 7) != 7 && (c[2] & 7) != 7) {
    const float* base = G.D + gp_vaddr(slot, c[0], c[1], c[2]);
#pragma unroll
    for (int k = 0; k < 8; ++k) d[k] = __ldg(base + (k & 1) + ((k >> 1) & 1) * 8 + (k >> 2) * 64);
    return;
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    int i = c[0] + (k & 1), j = c[1] + ((k >> 1) & 1), kk = c[2] + (k >> 2);
    int s = gp_brick_slot(G.table, G.nb, i, j, kk);
    if (s < 0) {
      ok = false;
      d[k] = 0.f;
    } else {
      d[k] = __ldg(G.D + gp_vaddr(s, i, j, kk));
    }
  }
}

// Trilinear interpolation of Eq. 3.  f is a lerp along x, then y, then z.
// Each gradient component is the bilinear blend, over the other two axes, of
// the four cell-edge differences along its own axis: a difference of two close
// grid values is exact (Sterbenz), so no component suffers the cancellation
// that differencing two interpolated values would bring.
__device__ __forceinline__ float lerp1(float t, float a, float b) { return fmaf(t, b - a, a); }

__device__ __forceinline__ Eval trilerp(const float d[8], const float t[3]) {
  Eval r;
  float e00 = lerp1(t[0], d[0], d[1]), e10 = lerp1(t[0], d[2], d[3]);
  float e01 = lerp1(t[0], d[4], d[5]), e11 = lerp1(t[0], d[6], d[7]);
  r.f = lerp1(t[2], lerp1(t[1], e00, e10), lerp1(t[1], e01, e11));
  // x edges at (y,z) = 00, 10, 01, 11
  float a00 = d[1] - d[0], a10 = d[3] - d[2], a01 = d[5] - d[4], a11 = d[7] - d[6];
  r.gt[0] = lerp1(t[2], lerp1(t[1], a00, a10), lerp1(t[1], a01, a11));
  // y edges at (x,z) = 00, 10, 01, 11
  float b00 = d[2] - d[0], b10 = d[3] - d[1], b01 = d[6] - d[4], b11 = d[7] - d[5];
  r.gt[1] = lerp1(t[2], lerp1(t[0], b00, b10), lerp1(t[0], b01, b11));
  // z edges at (x,y) = 00, 10, 01, 11
  float c00 = d[4] - d[0], c10 = d[5] - d[1], c01 = d[6] - d[2], c11 = d[7] - d[3];
  r.gt[2] = lerp1(t[1], lerp1(t[0], c00, c10), lerp1(t[0], c01, c11));
  return r;
}

// Scatter of one cell's 8 corner contributions.
template <bool DET>
__device__ __forceinline__ void scatter8(const Grid& G, float* __restrict__ grad, unsigned long long* __restrict__ acc,
                                         int32_t* __restrict__ err, const int c[3], int slot, const float t[3],
                                         float A, const float Gt[3]) {
  float wx[2] = {1.f - t[0], t[0]}, wy[2] = {1.f - t[1], t[1]}, wz[2] = {1.f - t[2], t[2]};
  bool fast = (c[0] & 7) != 7 && (c[1] & 7) != 7 && (c[2] & 7) != 7;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    int dx = k & 1, dy = (k >> 1) & 1, dz = k >> 2;
    float sx = dx ? 1.f : -1.f, sy = dy ? 1.f : -1.f, sz = dz ? 1.f : -1.f;
    float wyz = wy[dy] * wz[dz];
    float val = A * wx[dx] * wyz + Gt[0] * sx * wyz + Gt[1] * wx[dx] * sy * wz[dz] + Gt[2] * wx[dx] * wy[dy] * sz;
    int64_t addr;
    if (fast) {
      addr = gp_vaddr(slot, c[0], c[1], c[2]) + dx + dy * 8 + dz * 64;
    } else {
      int i = c[0] + dx, j = c[1] + dy, kk = c[2] + dz;
      int s = gp_brick_slot(G.table, G.nb, i, j, kk);
      if (s < 0) continue;
      addr = gp_vaddr(s, i, j, kk);
    }
    if (DET) {
      double x = (double)val;
      if (!(fabs(x) < FIX_LIMIT)) {
        atomicOr(err, GP_EF_NUMERIC);
        continue;
      }
      double hi = rint(x * FIX_HI);
      double lo = rint((x - hi / FIX_HI) * FIX_LO);
      atomicAdd(acc + 2 * addr, (unsigned long long)(long long)hi);
      atomicAdd(acc + 2 * addr + 1, (unsigned long long)(long long)lo);
    } else {
      atomicAdd(grad + addr, val);
    }
  }
}


// One step record: classify it, evaluate Eq. 3 at q and at s, add its loss
// terms to sp / sg / ss and (GRAD) scatter its gradient to the 8 + 8 corners,
// scaled by w (1/B_v; 1 for the fixed-point sums, scaled at the end).
template <bool DET, bool GRAD>
__device__ __forceinline__ bool query_record(const Grid& G, const float q[3], const float s[3], float w, float beta,
                                             float gamma, float* __restrict__ grad,
                                             unsigned long long* __restrict__ acc, int32_t* __restrict__ err,
                                             float& sp, float& sg, float& ss) {
  Cells C;
  if (!classify(G, q, s, C)) return false;
  bool ok = true;
  float dq[8], ds[8];
  load_corners(G, C.cq, C.slot_q, dq, ok);
  load_corners(G, C.cs, C.slot_s, ds, ok);
  if (!ok) {
    atomicOr(err, GP_EF_RANGE);
    return false;
  }
  Eval eq = trilerp(dq, C.tq);
  Eval es = trilerp(ds, C.ts);
  float g[3] = {eq.gt[0] * G.half_r, eq.gt[1] * G.half_r, eq.gt[2] * G.half_r};
  float gs[3] = {es.gt[0] * G.half_r, es.gt[1] * G.half_r, es.gt[2] * G.half_r};
  float gl = sqrtf(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
  float gls = sqrtf(gs[0] * gs[0] + gs[1] * gs[1] + gs[2] * gs[2]);
  float inv = 1.0f / fmaxf(gl, NORM_FLOOR), invs = 1.0f / fmaxf(gls, NORM_FLOOR);
  float nv[3] = {g[0] * inv, g[1] * inv, g[2] * inv};
  float ns[3] = {gs[0] * invs, gs[1] * invs, gs[2] * invs};
  float f = eq.f, fs = es.f;
  float r[3] = {(q[0] - s[0]) - f * nv[0], (q[1] - s[1]) - f * nv[1], (q[2] - s[2]) - f * nv[2]};
  float lp = sqrtf(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  float cosv = nv[0] * ns[0] + nv[1] * ns[1] + nv[2] * ns[2];
  sp += lp;
  sg += 1.0f - cosv;
  ss += fabsf(fs);
  if (!GRAD) return true;
  float ilp = lp > 0.f ? 1.0f / lp : 0.f;
  float u[3] = {r[0] * ilp, r[1] * ilp, r[2] * ilp};
  float un = u[0] * nv[0] + u[1] * nv[1] + u[2] * nv[2];
  float dfq = -w * un;
  float dn[3], dns[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    dn[a] = -w * f * u[a] - w * gamma * ns[a];
    dns[a] = -w * gamma * nv[a];
  }
  float ndn = nv[0] * dn[0] + nv[1] * dn[1] + nv[2] * dn[2];
  float nsdns = ns[0] * dns[0] + ns[1] * dns[1] + ns[2] * dns[2];
  bool big = gl > NORM_FLOOR, bigs = gls > NORM_FLOOR;
  float Gq[3], Gs[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float dg = big ? (dn[a] - nv[a] * ndn) * inv : dn[a] * inv;
    float dgs = bigs ? (dns[a] - ns[a] * nsdns) * invs : dns[a] * invs;
    Gq[a] = dg * G.half_r;  // dL/dt = dL/dg * dg/dt
    Gs[a] = dgs * G.half_r;
  }
  float dfs = fs > 0.f ? w * beta : (fs < 0.f ? -w * beta : 0.f);
  scatter8<DET>(G, grad, acc, err, C.cq, C.slot_q, C.tq, dfq, Gq);
  scatter8<DET>(G, grad, acc, err, C.cs, C.slot_s, C.ts, dfs, Gs);
  return true;
}
constexpr int HS = 12;            // staged edge: brick (8) + 2 on each side
constexpr int HN = HS * HS * HS;  // 1728
constexpr int IS = 10;            // TV edge: brick + 1 on each side
constexpr int IN = IS * IS * IS;  // 1000

__device__ __forceinline__ int hidx(int x, int y, int z) { return ((z + 2) * HS + (y + 2)) * HS + (x + 2); }
__device__ __forceinline__ int iidx(int x, int y, int z) { return ((z + 1) * IS + (y + 1)) * IS + (x + 1); }


// The L_TV sweep, one brick at a time per block of TV_SWEEP_THREADS threads
// (each owns vertex l and vertex l + 256 of the brick).  For each brick: stage
// the brick plus a two-vertex halo (12^3 values) and the T masks of its 27
// neighbour bricks in shared memory, compute 1/TV_n on the brick plus a
// one-vertex halo (10^3), then gather every vertex's
//   dTV/dd_i = [i in T] sum_n (d_i - d_n) / TV_i + sum_{n in T} (d_i - d_n) / TV_n
// over the stored in-grid axis neighbours n.  Each TV_i enters the sum once,
// from the brick that stores i.
//
// Pipeline: the halo of the next brick is copied by cp.async (zero-filled
// where absent) into the other of two buffers while the current brick is
// computed; the neighbour slots of the brick after that are fetched in two
// steps spread over the current brick's phases.  No halo value is held in
// registers, so several blocks fit on an SM.
constexpr int TV_SWEEP_THREADS = 256;

// Brick b as the sweep sees it: values, masks, its row of the 27-neighbour
// table (3x3x3, x fastest, -1 absent), grid size and origin vertex.
struct TvBrick {
  const float* D;
  const uint32_t* masks;
  const int32_t* nbr;
  int R, ox, oy, oz;
};

struct TvShared {
  float D[2][HN];          // staged values (0 where not stored)
  uint32_t T[2][27 * 16];  // T-mask words of the 27 neighbour bricks (0 where absent)
  uint8_t S[2][HN];        // 1: stored and inside [0, R]^3
  float inv[IN];           // 1/TV of T vertices of the inner region, else 0
  int slot[2][27];
  TvBrick bk[2];
};

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem, int src_bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Neighbour-brick index (0..26) of halo offset (hx, hy, hz), each in [-2, 9].
__device__ __forceinline__ int tv_region(int hx, int hy, int hz) {
  return ((hz >> 3) + 1) * 9 + ((hy >> 3) + 1) * 3 + ((hx >> 3) + 1);
}

// Issue the copies of brick bk[q]'s halo and neighbour T masks into buffer q
// and write its stored flags (plain stores).
__device__ __forceinline__ void tv_issue(TvShared& sh, int q) {
  const TvBrick bk = sh.bk[q];
  for (int h = threadIdx.x; h < HN; h += TV_SWEEP_THREADS) {
    const int hx = h % HS - 2, hy = (h / HS) % HS - 2, hz = h / (HS * HS) - 2;
    const int i = bk.ox + hx, j = bk.oy + hy, k = bk.oz + hz;
    const int sl = sh.slot[q][tv_region(hx, hy, hz)];
    const bool ok = sl >= 0 && i <= bk.R && j <= bk.R && k <= bk.R;  // negative i lies in an absent brick
    const float* src = ok ? bk.D + (int64_t)sl * 512 + gp_local(i, j, k) : bk.D;
    cp_async4(&sh.D[q][h], src, ok ? 4 : 0);
    sh.S[q][h] = ok ? 1 : 0;
  }
  for (int w = threadIdx.x; w < 27 * 16; w += TV_SWEEP_THREADS) {
    const int sl = sh.slot[q][w >> 4];
    const uint32_t* src = sl >= 0 ? bk.masks + (int64_t)sl * 48 + (w & 15) : bk.masks;
    cp_async4(&sh.T[q][w], src, sl >= 0 ? 4 : 0);
  }
}

// 1/TV over the inner region of buffer p; adds this thread's share of the
// brick's own TV_i to tsum.
__device__ __forceinline__ void tv_inverse(TvShared& sh, int p, float& tsum) {
  const float* D = sh.D[p];
  const uint8_t* S = sh.S[p];
  for (int h = threadIdx.x; h < IN; h += TV_SWEEP_THREADS) {
    const int x = h % IS - 1, y = (h / IS) % IS - 1, z = h / (IS * IS) - 1;
    const int c = hidx(x, y, z);
    float inv = 0.f;
    if (S[c]) {
      const int loc = ((z & 7) << 6) | ((y & 7) << 3) | (x & 7);
      const uint32_t tw = sh.T[p][tv_region(x, y, z) * 16 + (loc >> 5)];
      if ((tw >> (loc & 31)) & 1u) {
        const float dc = D[c];
        float acc2 = 0.f;
        const int nb6[6] = {c - 1, c + 1, c - HS, c + HS, c - HS * HS, c + HS * HS};
#pragma unroll
        for (int t = 0; t < 6; ++t) {
          if (S[nb6[t]]) {
            const float e = dc - D[nb6[t]];
            acc2 = fmaf(e, e, acc2);
          }
        }
        const float tv = sqrtf(acc2);
        if (x >= 0 && y >= 0 && z >= 0 && x < 8 && y < 8 && z < 8) tsum += tv;
        inv = tv > 0.f ? 1.0f / tv : 0.f;
      }
    }
    sh.inv[h] = inv;
  }
}

// dTV/dd of vertex l of the brick in buffer p (0 for padding).
__device__ __forceinline__ float tv_gather(const TvShared& sh, int p, int l) {
  const int lx = l & 7, ly = (l >> 3) & 7, lz = l >> 6;
  const int c = hidx(lx, ly, lz);
  const float* D = sh.D[p];
  const uint8_t* S = sh.S[p];
  if (!S[c]) return 0.f;
  const float di = D[c];
  const int ci = iidx(lx, ly, lz);
  const float own = sh.inv[ci];
  const int hn[6] = {c - 1, c + 1, c - HS, c + HS, c - HS * HS, c + HS * HS};
  const int in6[6] = {ci - 1, ci + 1, ci - IS, ci + IS, ci - IS * IS, ci + IS * IS};
  float gsum = 0.f;
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    if (!S[hn[t]]) continue;  // outside the grid or not stored
    const float e = di - D[hn[t]];
    gsum += e * own + e * sh.inv[in6[t]];
  }
  return gsum;
}

// The sweep over work items first, first + stride, ... < n of this block.
// src.brick(i) gives item i's TvBrick.  out(i, g0, g1, tsum) is called by
// every thread once per item, in order, with the unscaled dTV/dd of vertices
// l and l + 256 and the thread's share of the item's sum of TV_i; it may
// synchronise the block.
template <class Src, class Out>
__device__ __forceinline__ void tv_sweep(const Src& src, int64_t first, int64_t stride, int64_t n, TvShared& sh,
                                         Out&& out) {
  const int l = threadIdx.x;
  if (first >= n) return;
  if (l == 0) sh.bk[0] = src.brick(first);
  __syncthreads();
  if (l < 27) sh.slot[0][l] = __ldg(sh.bk[0].nbr + l);
  __syncthreads();
  tv_issue(sh, 0);
  cp_async_commit();
  if (first + stride < n) {
    if (l == 0) sh.bk[1] = src.brick(first + stride);
    __syncthreads();
    if (l < 27) sh.slot[1][l] = __ldg(sh.bk[1].nbr + l);
  }
  int p = 0;
  for (int64_t i = first; i < n; i += stride) {
    __syncthreads();  // the previous item is done with buffer p ^ 1 and inv; bk / slot[p ^ 1] written
    const int64_t next = i + stride, after = next + stride;
    if (next < n) tv_issue(sh, p ^ 1);
    cp_async_commit();
    TvBrick ab;
    if (l == 0 && after < n) ab = src.brick(after);
    cp_async_wait1();  // this thread's copies of item i have landed
    __syncthreads();   // ... and everyone's
    float tsum = 0.f;
    tv_inverse(sh, p, tsum);
    if (l == 0 && after < n) sh.bk[p] = ab;  // item i's own TvBrick was last read by tv_issue
    __syncthreads();  // inv ready, bk[p] published
    int rs = -1;
    if (l < 27 && after < n) rs = __ldg(sh.bk[p].nbr + l);
    const float g0 = tv_gather(sh, p, l), g1 = tv_gather(sh, p, l + 256);
    if (l < 27 && after < n) sh.slot[p][l] = rs;  // slot[p] was last read by tv_issue of item i
    out(i, g0, g1, tsum);
    p ^= 1;
  }
  cp_async_wait0();
}

// Adam (Kingma and Ba) on vertex `l` of brick `slot`, if it is trainable.
__device__ __forceinline__ void adam_vertex(int slot, int l, const uint32_t* __restrict__ masks,
                                            const float* __restrict__ grad, float* __restrict__ D,
                                            float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2,
                                            float eps, float bc1, float bc2) {
  if (!gp_mask_bit(masks, slot, 1, l)) return;
  int64_t addr = (int64_t)slot * 512 + l;
  float g = grad[addr];
  float mm = fmaf(b1, m[addr], (1.0f - b1) * g);
  float vv = fmaf(b2, v[addr], (1.0f - b2) * g * g);
  m[addr] = mm;
  v[addr] = vv;
  float mh = mm / bc1, vh = vv / bc2;
  D[addr] -= lr * mh / (sqrtf(vh) + eps);
}
