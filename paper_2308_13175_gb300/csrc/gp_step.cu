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
#include <cmath>

#include "gp_internal.cuh"

namespace {

constexpr int Q_THREADS = 256;
constexpr int TV_THREADS = 512;
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
__global__ void __launch_bounds__(Q_THREADS, 4) k_query(Grid G, const float* __restrict__ rec, int64_t B,
                                                     const int32_t* __restrict__ bv, float beta, float gamma,
                                                     float* __restrict__ grad, unsigned long long* __restrict__ acc,
                                                     double* __restrict__ partials, int32_t* __restrict__ err,
                                                     FinalArgs fa) {
  const int64_t n = B;
  int bvv = *bv;
  float w = bvv > 0 ? 1.0f / (float)bvv : 0.f;
  if (DET) w = 1.0f;  // fixed-point sums are scaled by 1/B_v at the end
  float sp = 0.f, sg = 0.f, ss = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float q[3], s[3];
    load_rec(rec, i, q, s);
    Cells C;
    if (!classify(G, q, s, C)) continue;
    bool ok = true;
    float dq[8], ds[8];
    load_corners(G, C.cq, C.slot_q, dq, ok);
    load_corners(G, C.cs, C.slot_s, ds, ok);
    if (!ok) {
      atomicOr(err, GP_EF_RANGE);
      continue;
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
    if (!GRAD) continue;
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
  }
  block_store3(partials, sp, sg, ss);
  if (LAST) finish_if_last(partials, fa);
}

// One block of 512 threads per brick (grid-stride over bricks).  The brick and
// a two-vertex halo (12^3 values, with stored / in-grid / T flags) are staged in
// shared memory; TV and 1/TV are computed for the brick plus a one-vertex halo
// (10^3), and each of the 512 vertices then gathers its gradient from shared
// memory.  Writes the gradient of every stored slot: alpha/|T| * dTV/dd_i (+ the
// fixed-point query sums in deterministic mode, which are cleared for the next
// step).  Each TV_i enters the loss sum once, from the brick that stores i.
constexpr int HS = 12;            // staged edge: brick (8) + 2 on each side
constexpr int HN = HS * HS * HS;  // 1728
constexpr int IS = 10;            // TV edge: brick + 1 on each side
constexpr int IN = IS * IS * IS;  // 1000

__device__ __forceinline__ int hidx(int x, int y, int z) { return ((z + 2) * HS + (y + 2)) * HS + (x + 2); }
__device__ __forceinline__ int iidx(int x, int y, int z) { return ((z + 1) * IS + (y + 1)) * IS + (x + 1); }

template <bool DET, bool GRAD, bool TV, bool LAST>
__global__ void __launch_bounds__(TV_THREADS) k_tv(Grid G, const int32_t* __restrict__ coord, int64_t n_bricks,
                                                   float tv_scale, float* __restrict__ grad,
                                                   unsigned long long* __restrict__ acc,
                                                   const int32_t* __restrict__ bv, double* __restrict__ partials,
                                                   int32_t* __restrict__ err, FinalArgs fa) {
  __shared__ float sD[HN];
  __shared__ uint8_t sF[HN];  // bit0: stored and inside [0,R]^3, bit1: in T
  __shared__ float sInv[IN];  // 1/TV of T vertices of the inner region, else 0
  __shared__ int sSlot[27];   // slots of the 3x3x3 bricks around the current one (-1: absent)
  __shared__ uint32_t sT[27 * 16];  // their T masks
  float tsum = 0.f;
  double qscale = 0.0;
  if (DET) {
    int b = *bv;
    qscale = b > 0 ? 1.0 / (double)b : 0.0;
  }
  const int l = threadIdx.x;
  const int lx = l & 7, ly = (l >> 3) & 7, lz = l >> 6;
  for (int64_t slot = blockIdx.x; slot < n_bricks; slot += gridDim.x) {
    const int ox = coord[3 * slot] * 8, oy = coord[3 * slot + 1] * 8, oz = coord[3 * slot + 2] * 8;
    const int64_t addr = slot * 512 + l;
    if (TV) {
      __syncthreads();  // previous brick done with the shared arrays
      // The 27 bricks around this one: slots and T masks, once per brick.
      if (l < 27) {
        int bx = (ox >> 3) + l % 3 - 1, by = (oy >> 3) + (l / 3) % 3 - 1, bz = (oz >> 3) + l / 9 - 1;
        sSlot[l] = gp_brick_slot(G.table, G.nb, bx * 8, by * 8, bz * 8);
      }
      __syncthreads();
      for (int w = l; w < 27 * 16; w += TV_THREADS) {
        int sl = sSlot[w >> 4];
        sT[w] = sl >= 0 ? __ldg(G.masks + (int64_t)sl * 48 + (w & 15)) : 0u;
      }
      __syncthreads();
      for (int h = l; h < HN; h += TV_THREADS) {
        int hx = h % HS - 2, hy = (h / HS) % HS - 2, hz = h / (HS * HS) - 2;
        int i = ox + hx, j = oy + hy, k = oz + hz;
        float v = 0.f;
        uint8_t f = 0;
        if (i >= 0 && j >= 0 && k >= 0 && i <= G.R && j <= G.R && k <= G.R) {
          int nbi = ((hz >> 3) + 1) * 9 + ((hy >> 3) + 1) * 3 + ((hx >> 3) + 1);  // hx in [-2, 9]
          int sl = sSlot[nbi];
          if (sl >= 0) {
            int loc = gp_local(i, j, k);
            v = __ldg(G.D + (int64_t)sl * 512 + loc);
            f = 1 | (((sT[nbi * 16 + (loc >> 5)] >> (loc & 31)) & 1u) ? 2 : 0);
          }
        }
        sD[h] = v;
        sF[h] = f;
      }
      __syncthreads();
      for (int h = l; h < IN; h += TV_THREADS) {
        int x = h % IS - 1, y = (h / IS) % IS - 1, z = h / (IS * IS) - 1;
        int c = hidx(x, y, z);
        float inv = 0.f;
        if ((sF[c] & 3) == 3) {
          float dc = sD[c], acc2 = 0.f;
          const int nb6[6] = {hidx(x - 1, y, z), hidx(x + 1, y, z), hidx(x, y - 1, z),
                              hidx(x, y + 1, z), hidx(x, y, z - 1), hidx(x, y, z + 1)};
#pragma unroll
          for (int t = 0; t < 6; ++t) {
            if (sF[nb6[t]] & 1) {
              float e = dc - sD[nb6[t]];
              acc2 = fmaf(e, e, acc2);
            }
          }
          float tv = sqrtf(acc2);
          if (x >= 0 && y >= 0 && z >= 0 && x < 8 && y < 8 && z < 8) tsum += tv;
          inv = tv > 0.f ? 1.0f / tv : 0.f;
        }
        sInv[h] = inv;
      }
      __syncthreads();
    }
    if (GRAD) {
      float gv = 0.f;
      if (TV) {
        int c = hidx(lx, ly, lz);
        if (sF[c] & 1) {
          float di = sD[c];
          float own = sInv[iidx(lx, ly, lz)];
          const int hn[6] = {hidx(lx - 1, ly, lz), hidx(lx + 1, ly, lz), hidx(lx, ly - 1, lz),
                             hidx(lx, ly + 1, lz), hidx(lx, ly, lz - 1), hidx(lx, ly, lz + 1)};
          const int in6[6] = {iidx(lx - 1, ly, lz), iidx(lx + 1, ly, lz), iidx(lx, ly - 1, lz),
                              iidx(lx, ly + 1, lz), iidx(lx, ly, lz - 1), iidx(lx, ly, lz + 1)};
          float gsum = 0.f;
#pragma unroll
          for (int t = 0; t < 6; ++t) {
            if (!(sF[hn[t]] & 1)) continue;  // outside the grid or not stored
            float e = di - sD[hn[t]];
            gsum += e * own + e * sInv[in6[t]];
          }
          gv = tv_scale * gsum;
        }
      }
      if (DET) {
        long long hi = (long long)acc[2 * addr], lo = (long long)acc[2 * addr + 1];
        acc[2 * addr] = 0ull;
        acc[2 * addr + 1] = 0ull;
        double q = ((double)hi / FIX_HI + (double)lo / FIX_LO) * qscale;
        gv = (float)((double)gv + q);
      }
      grad[addr] = gv;
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

__global__ void __launch_bounds__(512) k_adam(const int32_t* __restrict__ active, int64_t n_active,
                                              const uint32_t* __restrict__ masks, const float* __restrict__ grad,
                                              float* __restrict__ D, float* __restrict__ m, float* __restrict__ v,
                                              float lr, float b1, float b2, float eps, float bc1, float bc2) {
  const int l = threadIdx.x;
  for (int64_t a = blockIdx.x; a < n_active; a += gridDim.x) {
    int slot = active[a];
    if (!gp_mask_bit(masks, slot, 1, l)) continue;
    int64_t addr = (int64_t)slot * 512 + l;
    float g = grad[addr];
    float mm = fmaf(b1, m[addr], (1.0f - b1) * g);
    float vv = fmaf(b2, v[addr], (1.0f - b2) * g * g);
    m[addr] = mm;
    v[addr] = vv;
    float mh = mm / bc1, vh = vv / bc2;
    D[addr] -= lr * mh / (sqrtf(vh) + eps);
  }
}

unsigned q_grid(const gp_ctx* ctx, int64_t B) {
  return gp_blocks(B, Q_THREADS, GP_MAX_PARTIAL_BLOCKS);
}

unsigned tv_grid(const gp_ctx* ctx, int64_t n_bricks) {
  int64_t cap = (int64_t)ctx->num_sms * 4;
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
  auto launch_tv = [&]() -> gp_status {
    if (b->n_bricks == 0) {
      GP_CUDA(ctx, cudaMemsetAsync(b->partials + 3, 0, sizeof(double), s));
      return GP_OK;
    }
#define GP_TV(D_, G_, T_, L_)                                                                                  \
  k_tv<D_, G_, T_, L_><<<tb, TV_THREADS, 0, s>>>(G, b->brick_coord, b->n_bricks, tv_scale, grad_dev, b->acc, bv, \
                                                 b->partials, err, fa)
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
    if (det && grad_on)
      k_query<true, true, false><<<qb, Q_THREADS, 0, s>>>(G, rec_dev, B, bv, w->beta, w->gamma, grad_dev, b->acc,
                                                          b->partials, err, fa);
    else if (grad_on)
      k_query<false, true, true><<<qb, Q_THREADS, 0, s>>>(G, rec_dev, B, bv, w->beta, w->gamma, grad_dev, b->acc,
                                                          b->partials, err, fa);
    else
      k_query<false, false, true><<<qb, Q_THREADS, 0, s>>>(G, rec_dev, B, bv, w->beta, w->gamma, grad_dev, b->acc,
                                                           b->partials, err, fa);
    gp_prof_post(ctx, "k_query");
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
  int64_t cap = (int64_t)ctx->num_sms * 4;
  GP_KERNEL(ctx, "k_adam", k_adam<<<gp_blocks(b->n_active, 1, cap), 512, 0, ctx->stream>>>(b->active, b->n_active, b->masks, grad_dev, b->D,
                                                                  b->m, b->v, hp->lr, hp->beta1, hp->beta2, hp->eps,
                                                                  (float)bc1, (float)bc2));
  return GP_OK;
}
