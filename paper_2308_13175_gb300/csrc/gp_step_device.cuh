// Device functions of the step shared by the single-band kernels (gp_step.cu)
// and the many-band kernels (gp_multi.cu): Eq. 3 interpolation, the per-record
// forward + hand-written backward, one brick of the L_TV sweep, one Adam update.
// The formulas are stated in the header comment of gp_step.cu.
#pragma once

#include <string.h>

#include "gp_internal.cuh"

constexpr float NORM_FLOOR = 1e-12f;
// Deterministic sums: each contribution v is split into two integers, hi in
// units of 2^-20 and lo in units of 2^-60 (fix_split), accumulated with 64-bit
// integer atomics (exact, so the order of the additions does not matter).
// The sum is hi * 2^-20 + lo * 2^-60: a resolution of 2^-60; a contribution
// of magnitude 2^42 (FIX_LIMIT) or more, or a non-finite one, raises
// GP_EF_NUMERIC instead.
constexpr double FIX_HI = 1048576.0;                     // 2^20
constexpr double FIX_LO = 1152921504606846976.0;         // 2^60
constexpr double FIX_LIMIT = 4398046511104.0;            // 2^42

struct Eval {
  float f;
  float gt[3];  // df/dt (t = local coordinate in cell units)
};

// The 8 corner values of cell c (corner k = dx + 2 dy + 4 dz).  Inside a
// brick the two corners (x, x + 1) of each of the cell's four x edges are
// adjacent floats: one 8-byte load per edge at even x, one aligned 16-byte
// load from x - 1 at x = 1 mod 4, two 4-byte loads at x = 3 mod 4.  A cell
// whose corners span bricks looks each corner's brick up.
__device__ __forceinline__ void load_corners(const Grid& G, const int c[3], int slot, float d[8], bool& ok) {
  if ((c[0] & 7) != 7 && (c[1] & 7) != 7 && (c[2] & 7) != 7) {
    const float* base = G.D + gp_vaddr(slot, c[0], c[1], c[2]);
    const int xm = c[0] & 3;
    if ((xm & 1) == 0) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float2 v = __ldg(reinterpret_cast<const float2*>(base + (e & 1) * 8 + (e >> 1) * 64));
        d[2 * e] = v.x;
        d[2 * e + 1] = v.y;
      }
    } else if (xm == 1) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(base - 1 + (e & 1) * 8 + (e >> 1) * 64));
        d[2 * e] = v.y;
        d[2 * e + 1] = v.z;
      }
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) d[k] = __ldg(base + (k & 1) + ((k >> 1) & 1) * 8 + (k >> 2) * 64);
    }
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

// Two adjacent floats added as one 8-byte vector reduction (address 8-byte aligned).
__device__ __forceinline__ void red_add_v2(float* addr, float a, float b) {
  asm volatile("red.global.add.v2.f32 [%0], {%1, %2};\n" ::"l"(addr), "f"(a), "f"(b) : "memory");
}
// Four adjacent floats as one 16-byte vector reduction (address 16-byte aligned).
__device__ __forceinline__ void red_add_v4(float* addr, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};\n" ::"l"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
               : "memory");
}

// Deterministic sums: each contribution v is taken exactly (to 2^-60) into
// two integers, hi in units of 2^-20 and lo in units of 2^-60 with
// hi 2^40 + lo = v 2^60 rounded toward zero below 2^-60, by integer
// arithmetic on v's bits.  Integer sums do not depend on the order of the
// additions.  Returns false for a non-finite v or |v| >= 2^42 (FIX_LIMIT).
// Integer arithmetic only, so the host build (a CPU test of its boundaries)
// computes the same integers as the device.
__host__ __device__ __forceinline__ bool fix_split(float v, long long& hi, long long& lo) {
#ifdef __CUDA_ARCH__
  const uint32_t u = __float_as_uint(v);
#else
  uint32_t u;
  memcpy(&u, &v, sizeof(u));
#endif
  const int ex = (int)((u >> 23) & 0xffu);
  if (ex == 0xff) return false;
  long long m = (long long)(u & 0x7fffffu);
  int e;
  if (ex == 0) {
    e = -149;
  } else {
    m |= 0x800000ll;
    e = ex - 150;
  }
  hi = 0;
  lo = 0;
  if (m == 0) return true;
  const int sh = e + 60;  // v 2^60 = m 2^sh, m < 2^24
  // |v| >= 2^42 exactly when e >= 19 (m >= 2^23 for a normal v), i.e. sh >= 79;
  // below that hi = m 2^(sh - 40) < 2^62 fits its 64-bit word.
  if (sh >= 79) return false;
  if (sh >= 40) {
    hi = m << (sh - 40);
  } else if (sh >= 0) {
    const long long val = m << sh;  // < 2^63
    hi = val >> 40;
    lo = val & ((1ll << 40) - 1);
  } else if (sh > -64) {
    lo = m >> (-sh);
  }
  if (u >> 31) {
    hi = -hi;
    lo = -lo;
  }
  return true;
}

// Scatter of one cell's 8 corner contributions.
template <bool DET>
__device__ __forceinline__ void scatter8(const Grid& G, float* __restrict__ grad, unsigned long long* __restrict__ acc,
                                         int32_t* __restrict__ err, const int c[3], int slot, const float t[3],
                                         float A, const float Gt[3]) {
  float wx[2] = {1.f - t[0], t[0]}, wy[2] = {1.f - t[1], t[1]}, wz[2] = {1.f - t[2], t[2]};
  bool fast = (c[0] & 7) != 7 && (c[1] & 7) != 7 && (c[2] & 7) != 7;
  if (!DET && fast && (c[0] & 3) != 3) {
    // The corners (x, x + 1) of each of the 4 (y, z) edges are adjacent: one
    // vector reduction per edge - 8 bytes at even x, 16 bytes from x - 1 (the
    // outer two lanes adding zero) at x = 1 mod 4.
    float* base = grad + gp_vaddr(slot, c[0], c[1], c[2]);
    const bool odd = c[0] & 1;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int dy = e & 1, dz = e >> 1;
      const float sy = dy ? 1.f : -1.f, sz = dz ? 1.f : -1.f;
      const float wyz = wy[dy] * wz[dz];
      float v[2];
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        const float sx = dx ? 1.f : -1.f;
        v[dx] = A * wx[dx] * wyz + Gt[0] * sx * wyz + Gt[1] * wx[dx] * sy * wz[dz] + Gt[2] * wx[dx] * wy[dy] * sz;
      }
      if (odd)
        red_add_v4(base - 1 + dy * 8 + dz * 64, 0.f, v[0], v[1], 0.f);
      else
        red_add_v2(base + dy * 8 + dz * 64, v[0], v[1]);
    }
    return;
  }
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
      long long hi, lo;
      if (!fix_split(val, hi, lo)) {
        atomicOr(err, GP_EF_NUMERIC);
        continue;
      }
      if (hi) atomicAdd(acc + 2 * addr, (unsigned long long)hi);
      if (lo) atomicAdd(acc + 2 * addr + 1, (unsigned long long)lo);
    } else {
      atomicAdd(grad + addr, val);
    }
  }
}


// dL/dd_c of the cell's corner c = dx + 2 dy + 4 dz from dL/df = A and
// dL/dt = Gt at local coordinate t: A w_c(t) + sum_a Gt_a dw_c/dt_a.
__device__ __forceinline__ void corner_values(const float t[3], float A, const float Gt[3], float v[8]) {
  const float wx[2] = {1.f - t[0], t[0]}, wy[2] = {1.f - t[1], t[1]}, wz[2] = {1.f - t[2], t[2]};
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int dx = k & 1, dy = (k >> 1) & 1, dz = k >> 2;
    const float sx = dx ? 1.f : -1.f, sy = dy ? 1.f : -1.f, sz = dz ? 1.f : -1.f;
    const float wyz = wy[dy] * wz[dz];
    v[k] = A * wx[dx] * wyz + Gt[0] * sx * wyz + Gt[1] * wx[dx] * sy * wz[dz] + Gt[2] * wx[dx] * wy[dy] * sz;
  }
}

// Where a record's corner contributions go: straight to the gradient with
// global reductions (float atomics, or the two-word fixed point).
template <bool DET>
struct GlobalSink {
  const Grid& G;
  float* __restrict__ grad;
  unsigned long long* __restrict__ acc;
  int32_t* __restrict__ err;
  __device__ __forceinline__ void cell(const int c[3], int slot, const float t[3], float A, const float Gt[3]) {
    scatter8<DET>(G, grad, acc, err, c, slot, t, A, Gt);
  }
};

// One step record: classify it, evaluate Eq. 3 at q and at s, add its loss
// terms to sp / sg / ss and (GRAD) scatter its gradient to the 8 + 8 corners,
// scaled by w = 1/B_v (the fixed-point sums too: a contribution below 2^-20
// then has no high word, and most corners take one 64-bit atomic, not two).
//
// The validity test is the one of classify(), with its memory reads arranged
// for latency: both brick slots are read together, then both pull-mask words
// and all 16 corner values together (the corners of a record that turns out
// invalid are read for nothing).
// l_grad = 1 - n . n_s (Eq. 7) without the cancellation of 1 - cos near
// cos = 1: 1 - n.m = |n - m|^2 / 2 + (1 - |n|^2) / 2 + (1 - |m|^2) / 2, whose
// last two terms vanish for a unit vector (a gradient above the floor).  The
// difference n - m of two close unit vectors is computed almost exactly.
__device__ __forceinline__ float grad_term(const float n[3], const float m[3], bool n_unit, bool m_unit) {
  const float d0 = n[0] - m[0], d1 = n[1] - m[1], d2 = n[2] - m[2];
  float l = 0.5f * (d0 * d0 + d1 * d1 + d2 * d2);
  if (!n_unit) l += 0.5f * (1.0f - (n[0] * n[0] + n[1] * n[1] + n[2] * n[2]));
  if (!m_unit) l += 0.5f * (1.0f - (m[0] * m[0] + m[1] * m[1] + m[2] * m[2]));
  return l;
}

// The backward pass of one record from its forward quantities.  With
// u = r / |r| (0 at r = 0), for the pull term dL/df = -w u.n and
// dL/dn = -w f u - w gamma n_s, for the gradient term dL/dn_s = -w gamma n;
// through n = g / |g|, dL/dg = (I - n n^T) dL/dn / |g| (dL/dn / 1e-12 below the
// floor), and dL/dt = dL/dg R/2.  For a unit n the projections are taken from
// small differences instead of differences of large terms:
//   u.n = ((q - s).n - f) / |r|,  (I - n n^T) u = ((q - s) - ((q - s).n) n) / |r|,
//   (I - n n^T) n_s = (n_s - n) - ((n_s - n).n) n,
// which are the same quantities, but keep float32 accuracy when |f| >> |q - s|
// or n ~ n_s (the residual r = (q - s) - f n loses the small perpendicular
// part of q - s to the rounding of f n).
__device__ __forceinline__ void backward_terms(const float q[3], const float s[3], float f, const float nv[3],
                                               const float ns[3], float lp, float inv, float invs, bool big,
                                               bool bigs, float w, float gamma, float half_r, float Gq[3],
                                               float Gs[3], float& dfq) {
  const float ilp = lp > 0.f ? 1.0f / lp : 0.f;
  const float d[3] = {q[0] - s[0], q[1] - s[1], q[2] - s[2]};
  if (big) {
    const float dn = d[0] * nv[0] + d[1] * nv[1] + d[2] * nv[2];
    const float e[3] = {ns[0] - nv[0], ns[1] - nv[1], ns[2] - nv[2]};
    const float en = e[0] * nv[0] + e[1] * nv[1] + e[2] * nv[2];
    dfq = -w * (dn - f) * ilp;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float u_perp = (d[a] - dn * nv[a]) * ilp;
      const float ns_perp = e[a] - en * nv[a];
      Gq[a] = (-w * f * u_perp - w * gamma * ns_perp) * inv * half_r;
    }
  } else {
    const float r[3] = {d[0] - f * nv[0], d[1] - f * nv[1], d[2] - f * nv[2]};
    const float un = (r[0] * nv[0] + r[1] * nv[1] + r[2] * nv[2]) * ilp;
    dfq = -w * un;
#pragma unroll
    for (int a = 0; a < 3; ++a) Gq[a] = (-w * f * r[a] * ilp - w * gamma * ns[a]) * inv * half_r;
  }
  if (bigs) {
    const float e[3] = {nv[0] - ns[0], nv[1] - ns[1], nv[2] - ns[2]};
    const float en = e[0] * ns[0] + e[1] * ns[1] + e[2] * ns[2];
#pragma unroll
    for (int a = 0; a < 3; ++a) Gs[a] = -w * gamma * (e[a] - en * ns[a]) * invs * half_r;
  } else {
#pragma unroll
    for (int a = 0; a < 3; ++a) Gs[a] = -w * gamma * nv[a] * invs * half_r;
  }
}

// A record between the phases of its evaluation.  The three phases issue
// the record's dependent loads level by level - the brick slots (phase a),
// then the pull-mask words and the 16 corner values (phase b) - so that a
// thread working on several records issues all of one level's loads before it
// waits for any of them.
struct RecState {
  float q[3], s[3];
  Cells C;
  int lq, ls;
  uint32_t wq, ws;
  float dq[8], ds[8];
  bool ok;       // still a candidate for a valid record
  bool corners;  // every corner was found in the band
};

__device__ __forceinline__ void rec_phase_a(const Grid& G, const float q[3], const float s[3], bool active,
                                            RecState& R) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    R.q[a] = q[a];
    R.s[a] = s[a];
  }
  R.ok = active && classify_cells(G, q, s, R.C);
  if (!R.ok) return;
  R.C.slot_q = gp_brick_slot(G.table, G.nb, R.C.cq[0], R.C.cq[1], R.C.cq[2]);
  R.C.slot_s = gp_brick_slot(G.table, G.nb, R.C.cs[0], R.C.cs[1], R.C.cs[2]);
}

__device__ __forceinline__ void rec_phase_b(const Grid& G, RecState& R) {
  if (!R.ok) return;
  if (R.C.slot_q < 0 || R.C.slot_s < 0) {
    R.ok = false;
    return;
  }
  R.lq = gp_local(R.C.cq[0], R.C.cq[1], R.C.cq[2]);
  R.ls = gp_local(R.C.cs[0], R.C.cs[1], R.C.cs[2]);
  R.wq = __ldg(G.masks + (int64_t)R.C.slot_q * 48 + 32 + (R.lq >> 5));
  R.ws = __ldg(G.masks + (int64_t)R.C.slot_s * 48 + 32 + (R.ls >> 5));
  R.corners = true;
  load_corners(G, R.C.cq, R.C.slot_q, R.dq, R.corners);
  load_corners(G, R.C.cs, R.C.slot_s, R.ds, R.corners);
}

// Validity (cell(q) and cell(s) in the pull band, Sec. 3), the forward terms
// and, with GRAD, the backward pass into the sink.  Returns whether the
// record is valid.
template <bool GRAD, class Sink>
__device__ __forceinline__ bool rec_phase_c(const Grid& G, RecState& R, float w, float beta, float gamma,
                                            Sink& sink, int32_t* __restrict__ err, float& sp, float& sg,
                                            float& ss) {
  if (!R.ok) return false;
  if (!((R.wq >> (R.lq & 31)) & 1u) || !((R.ws >> (R.ls & 31)) & 1u)) return false;
  if (!R.corners) {
    atomicOr(err, GP_EF_RANGE);
    return false;
  }
  const float* q = R.q;
  const float* s = R.s;
  const Cells& C = R.C;
  Eval eq = trilerp(R.dq, C.tq);
  Eval es = trilerp(R.ds, C.ts);
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
  bool big = gl > NORM_FLOOR, bigs = gls > NORM_FLOOR;
  sp += lp;
  sg += grad_term(nv, ns, big, bigs);
  ss += fabsf(fs);
  if (!GRAD) return true;
  float Gq[3], Gs[3], dfq;
  backward_terms(q, s, f, nv, ns, lp, inv, invs, big, bigs, w, gamma, G.half_r, Gq, Gs, dfq);
  float dfs = fs > 0.f ? w * beta : (fs < 0.f ? -w * beta : 0.f);
  sink.cell(C.cq, C.slot_q, C.tq, dfq, Gq);
  sink.cell(C.cs, C.slot_s, C.ts, dfs, Gs);
  return true;
}

template <bool GRAD, class Sink>
__device__ __forceinline__ bool query_record_to(const Grid& G, const float q[3], const float s[3], float w,
                                                float beta, float gamma, Sink& sink, int32_t* __restrict__ err,
                                                float& sp, float& sg, float& ss) {
  RecState R;
  rec_phase_a(G, q, s, true, R);
  rec_phase_b(G, R);
  return rec_phase_c<GRAD>(G, R, w, beta, gamma, sink, err, sp, sg, ss);
}

// The record with its contributions reduced straight into the gradient.
template <bool DET, bool GRAD>
__device__ __forceinline__ bool query_record(const Grid& G, const float q[3], const float s[3], float w, float beta,
                                             float gamma, float* __restrict__ grad,
                                             unsigned long long* __restrict__ acc, int32_t* __restrict__ err,
                                             float& sp, float& sg, float& ss) {
  GlobalSink<DET> sink{G, grad, acc, err};
  return query_record_to<GRAD>(G, q, s, w, beta, gamma, sink, err, sp, sg, ss);
}

constexpr int HS = 12;            // staged edge: brick (8) + 2 on each side
constexpr int HN = HS * HS * HS;  // 1728
constexpr int IS = 10;            // TV edge: brick + 1 on each side
constexpr int IN = IS * IS * IS;  // 1000

__device__ __forceinline__ int hidx(int x, int y, int z) { return ((z + 2) * HS + (y + 2)) * HS + (x + 2); }
// The inner region's 1/TV array: rows of IS values padded to TV_IROW floats,
// so that the gather's warps (rows y, y + 2, y + 4, y + 6) meet no bank
// conflict.
constexpr int TV_IROW = 12;
constexpr int TV_IPLANE = IS * TV_IROW;
__device__ __forceinline__ int iidx(int x, int y, int z) { return ((z + 1) * IS + (y + 1)) * TV_IROW + (x + 1); }


// The L_TV sweep, one brick at a time per block of TV_SWEEP_THREADS threads
// (each owns two vertices of the brick).  For each brick: stage
// the brick plus a two-vertex halo (12^3 values) and the T masks of its 27
// neighbour bricks in shared memory, compute 1/TV_n on the brick plus a
// one-vertex halo (10^3), then gather every vertex's
//   dTV/dd_i = [i in T] sum_n (d_i - d_n) / TV_i + sum_{n in T} (d_i - d_n) / TV_n
// over the in-grid axis neighbours n.  Each TV_i enters the sum once, from the
// brick that stores i.
//
// The band stores every in-grid axis neighbour of a T vertex, so a value the
// sums use is always present: absent bricks are staged as zeros and only the
// grid boundary needs checks (bricks within two vertices of it take a checked
// path).  Staging copies rows: each halo row (fixed y, z) is four cp.async
// pieces (x = -2..-1 from the brick below in x, 0..3 and 4..7 from the centre
// column, 8..9 from the brick above), into rows padded to 16 floats.  The next
// brick's halo is copied into the other of two buffers while the current one
// is computed; the neighbour slots of the brick after that are fetched in two
// steps spread over the current brick's phases.
constexpr int TV_SWEEP_THREADS = 256;
constexpr int TV_BLOCKS_PER_SM = 5;  // resident blocks per SM at the register cap below (48 per thread)
constexpr int TV_ROW = 20;        // floats per staged row: x = -2..9 at columns 2..13 (20: fewer bank conflicts)
constexpr int TV_ROWS = HS * HS;  // 144 rows: y, z = -2..9

// Brick b as the sweep sees it: values, masks, its row of the 27-neighbour
// table (3x3x3, x fastest, -1 absent), grid size and origin vertex.
struct TvBrick {
  const float* D;
  const uint32_t* masks;
  const int32_t* nbr;
  int R, ox, oy, oz;
};

struct TvShared {
  __align__(16) float D[2][TV_ROWS * TV_ROW];   // staged values (0 in absent bricks)
  __align__(16) uint32_t T[2][27 * 16];         // T-mask words of the 27 neighbour bricks (0 if absent)
  float inv[IS * TV_IPLANE];                    // 1/TV of T vertices of the inner region, else 0
  int slot[2][27];
  TvBrick bk[2];
};

__device__ __forceinline__ int tv_hc(int x, int y, int z) { return ((z + 2) * HS + (y + 2)) * TV_ROW + (x + 4); }

__device__ __forceinline__ void cp_async_ca8(void* smem, const void* gmem, int src_bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_cg16(void* smem, const void* gmem, int src_bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// This thread's fixed share of every brick's work, decoded once: its row
// pieces to copy and its inner-region entries.
constexpr int TV_TASKS = (TV_ROWS * 4 + TV_SWEEP_THREADS - 1) / TV_SWEEP_THREADS;  // 3
constexpr int TV_INNER = (IN + TV_SWEEP_THREADS - 1) / TV_SWEEP_THREADS;          // 4
struct TvPlan {
  uint32_t task[TV_TASKS];   // region | local << 5 | destination << 14 | 16-byte piece << 26 | valid << 27
  uint32_t entry[TV_INNER];  // halo index | region << 12 | local << 17 | inner << 26 | valid << 27
};

__device__ __forceinline__ TvPlan tv_plan() {
  TvPlan pl;
#pragma unroll
  for (int k = 0; k < TV_TASKS; ++k) {
    const int r = threadIdx.x + k * TV_SWEEP_THREADS;
    pl.task[k] = 0;
    if (r >= TV_ROWS * 4) continue;
    const int row = r >> 2, seg = r & 3;
    const int hy = row % HS - 2, hz = row / HS - 2;
    const int dx = seg == 0 ? 0 : (seg == 3 ? 2 : 1);  // brick column: below / centre / above
    const int lx0 = seg == 0 ? 6 : (seg == 2 ? 4 : 0);
    const int col = seg == 0 ? 2 : (seg == 1 ? 4 : (seg == 2 ? 8 : 12));
    const uint32_t reg = ((hz >> 3) + 1) * 9 + ((hy >> 3) + 1) * 3 + dx;
    const uint32_t loc = ((hz & 7) << 6) | ((hy & 7) << 3) | lx0;
    const uint32_t dst = row * TV_ROW + col;
    const uint32_t big = (seg == 1 || seg == 2) ? 1u : 0u;
    pl.task[k] = reg | (loc << 5) | (dst << 14) | (big << 26) | (1u << 27);
  }
#pragma unroll
  for (int k = 0; k < TV_INNER; ++k) {
    const int h = threadIdx.x + k * TV_SWEEP_THREADS;
    pl.entry[k] = 0;
    if (h >= IN) continue;
    const int x = h % IS - 1, y = (h / IS) % IS - 1, z = h / (IS * IS) - 1;
    const uint32_t reg = ((z >> 3) + 1) * 9 + ((y >> 3) + 1) * 3 + ((x >> 3) + 1);
    const uint32_t loc = ((z & 7) << 6) | ((y & 7) << 3) | (x & 7);
    const uint32_t inner = (x >= 0 && y >= 0 && z >= 0 && x < 8 && y < 8 && z < 8) ? 1u : 0u;
    pl.entry[k] = (uint32_t)tv_hc(x, y, z) | (reg << 12) | (loc << 17) | (inner << 26) | (1u << 27);
  }
  return pl;
}

// Issue the copies of brick bk[q]'s halo rows and neighbour T masks into
// buffer q (zero-filled where the brick is absent).
__device__ __forceinline__ void tv_issue(TvShared& sh, int q, const TvPlan& pl) {
  const float* D = sh.bk[q].D;
#pragma unroll
  for (int k = 0; k < TV_TASKS; ++k) {
    const uint32_t t = pl.task[k];
    if (!(t >> 27)) continue;
    const int sl = sh.slot[q][t & 31];
    const float* src = sl >= 0 ? D + (size_t)sl * 512u + ((t >> 5) & 511) : D;
    float* dst = &sh.D[q][(t >> 14) & 4095];
    if ((t >> 26) & 1)
      cp_async_cg16(dst, src, sl >= 0 ? 16 : 0);
    else
      cp_async_ca8(dst, src, sl >= 0 ? 8 : 0);
  }
  if (threadIdx.x < 27 * 4) {
    const int w = threadIdx.x;
    const int sl = sh.slot[q][w >> 2];
    const uint32_t* masks = sh.bk[q].masks;
    const uint32_t* src = sl >= 0 ? masks + (size_t)sl * 48u + 4u * (w & 3) : masks;
    cp_async_cg16(&sh.T[q][4 * w], src, sl >= 0 ? 16 : 0);
  }
}

// Is every vertex of the halo inside [0, R]^3?
__device__ __forceinline__ bool tv_interior(const TvBrick& bk) {
  return bk.ox >= 2 && bk.oy >= 2 && bk.oz >= 2 && bk.ox + 9 <= bk.R && bk.oy + 9 <= bk.R && bk.oz + 9 <= bk.R;
}

// 1/TV over the inner region of buffer p; adds this thread's share of the
// brick's own TV_i to tsum.  CHECK: skip out-of-grid neighbours.
template <bool CHECK>
__device__ __forceinline__ void tv_inverse(TvShared& sh, int p, const TvBrick& bk, const TvPlan& pl, float& tsum) {
  const float* D = sh.D[p];
  const uint32_t* T = sh.T[p];
#pragma unroll
  for (int k = 0; k < TV_INNER; ++k) {
    const uint32_t e = pl.entry[k];
    if (!(e >> 27)) continue;
    const int h = threadIdx.x + k * TV_SWEEP_THREADS;
    const int c = e & 4095, reg = (e >> 12) & 31, loc = (e >> 17) & 511;
    float inv = 0.f;
    if ((T[reg * 16 + (loc >> 5)] >> (loc & 31)) & 1u) {
      const float dc = D[c];
      const int nb6[6] = {c - 1, c + 1, c - TV_ROW, c + TV_ROW, c - TV_ROW * HS, c + TV_ROW * HS};
      bool ok[6] = {true, true, true, true, true, true};
      if (CHECK) {
        const int x = h % IS - 1 + bk.ox, y = (h / IS) % IS - 1 + bk.oy, z = h / (IS * IS) - 1 + bk.oz;
        ok[0] = x > 0;
        ok[1] = x < bk.R;
        ok[2] = y > 0;
        ok[3] = y < bk.R;
        ok[4] = z > 0;
        ok[5] = z < bk.R;
      }
      float acc2 = 0.f;
#pragma unroll
      for (int t = 0; t < 6; ++t) {
        const float d = dc - D[nb6[t]];
        if (ok[t]) acc2 = fmaf(d, d, acc2);
      }
      inv = acc2 > 0.f ? rsqrtf(acc2) : 0.f;  // 1/TV_n
      if ((e >> 26) & 1) tsum += acc2 * inv;  // TV_n
    }
    sh.inv[(h / IS) * TV_IROW + h % IS] = inv;  // iidx of the entry
  }
}

// dTV/dd of this thread's two vertices of the brick in buffer p: (lx, ly, lz)
// and (lx, ly + 1, lz) with lx = t & 7, ly = 2 ((t >> 3) & 3), lz = t >> 5,
// vertex indices l0 = lx + 8 ly + 64 lz and l0 + 8.  A warp's four rows y are
// two apart, which keeps both the staged values (rows 40 floats apart) and
// the inverses (24 apart) free of bank conflicts.  0 outside the grid.
template <bool CHECK>
__device__ __forceinline__ void tv_gather(const TvShared& sh, int p, const TvBrick& bk, float& g0, float& g1,
                                          int& l0) {
  const int t = threadIdx.x;
  const int lx = t & 7, ly0 = 2 * ((t >> 3) & 3), lz = t >> 5;
  const float* D = sh.D[p];
  const float* I = sh.inv;
  l0 = lx + 8 * ly0 + 64 * lz;
  float out[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int ly = ly0 + k;
    bool ok[6] = {true, true, true, true, true, true};
    bool inside = true;
    if (CHECK) {
      const int x = bk.ox + lx, y = bk.oy + ly, z = bk.oz + lz;
      inside = x <= bk.R && y <= bk.R && z <= bk.R;
      ok[0] = x > 0;
      ok[1] = x < bk.R;
      ok[2] = y > 0;
      ok[3] = y < bk.R;
      ok[4] = z > 0;
      ok[5] = z < bk.R;
    }
    const int c = tv_hc(lx, ly, lz), ci = iidx(lx, ly, lz);
    const float di = D[c], own = I[ci];
    const int hn[6] = {c - 1, c + 1, c - TV_ROW, c + TV_ROW, c - TV_ROW * HS, c + TV_ROW * HS};
    const int in6[6] = {ci - 1, ci + 1, ci - TV_IROW, ci + TV_IROW, ci - TV_IPLANE, ci + TV_IPLANE};
    float gsum = 0.f;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      // own != 0 only for i in T, whose in-grid neighbours are all stored;
      // inv[n] != 0 only for n in T (inside the grid and stored).
      if (ok[j]) gsum = fmaf(di - D[hn[j]], own + I[in6[j]], gsum);
    }
    out[k] = inside ? gsum : 0.f;
  }
  g0 = out[0];
  g1 = out[1];
}

// The sweep over work items first, first + stride, ... < n of this block.
// src.brick(i) gives item i's TvBrick.  out(i, l0, g0, l1, g1, tsum) is called
// by every thread once per item, in order, with the unscaled dTV/dd of the
// thread's two vertices l0, l1 (tv_gather) and its share of the item's sum of
// TV_i; it may synchronise the block.
struct TvNoPre {
  __device__ __forceinline__ void operator()(int64_t) const {}
};

// pre(i) (optional) is called by every thread at the top of item i's
// iteration, while the item's halo copies are still in flight: a place to
// issue loads whose latency the stencil work then hides.
template <class Src, class Out, class Pre = TvNoPre>
__device__ __forceinline__ void tv_sweep(const Src& src, int64_t first, int64_t stride, int64_t n, TvShared& sh,
                                         Out&& out, Pre&& pre = Pre()) {
  const int l = threadIdx.x;
  if (first >= n) return;
  const TvPlan pl = tv_plan();
  if (l == 0) sh.bk[0] = src.brick(first);
  __syncthreads();
  if (l < 27) sh.slot[0][l] = __ldg(sh.bk[0].nbr + l);
  __syncthreads();
  tv_issue(sh, 0, pl);
  cp_async_commit();
  if (first + stride < n) {
    if (l == 0) sh.bk[1] = src.brick(first + stride);
    __syncthreads();
    if (l < 27) sh.slot[1][l] = __ldg(sh.bk[1].nbr + l);
  }
  int p = 0;
  for (int64_t i = first; i < n; i += stride) {
    pre(i);
    __syncthreads();  // the previous item is done with buffer p ^ 1 and inv; bk / slot[p ^ 1] written
    const int64_t next = i + stride, after = next + stride;
    if (next < n) tv_issue(sh, p ^ 1, pl);
    cp_async_commit();
    TvBrick ab;
    if (l < 27 && after < n) ab = src.brick(after);  // warp 0: one broadcast load per field
    const TvBrick bk = sh.bk[p];
    const bool check = !tv_interior(bk);
    cp_async_wait1();  // this thread's copies of item i have landed
    __syncthreads();   // ... and everyone's
    float tsum = 0.f;
    if (check)
      tv_inverse<true>(sh, p, bk, pl, tsum);
    else
      tv_inverse<false>(sh, p, bk, pl, tsum);
    __syncthreads();  // inv ready; bk[p] and slot[p] are free
    if (l == 0 && after < n) sh.bk[p] = ab;
    int rs = -1;
    if (l < 27 && after < n) rs = __ldg(ab.nbr + l);
    float g0, g1;
    int l0;
    if (check)
      tv_gather<true>(sh, p, bk, g0, g1, l0);
    else
      tv_gather<false>(sh, p, bk, g0, g1, l0);
    if (l < 27 && after < n) sh.slot[p][l] = rs;
    out(i, l0, g0, l0 + 8, g1, tsum);
    p ^= 1;
  }
  cp_async_wait0();
}

// One Adam step (Kingma and Ba; Sec. 4 "Details") of one vertex, the bias
// corrections given as their reciprocals ibc = 1 / (1 - beta^t):
//   m <- b1 m + (1 - b1) g,  v <- b2 v + (1 - b2) g^2,
//   d <- d - lr (m ibc1) / (sqrt(v ibc2) + eps).
// The root is x rsqrt(x) and the division __fdividef: a few ulp each, far
// inside the step's tolerance, and neither has a slow path.
__device__ __forceinline__ float adam_elem(float g, float& m, float& v, float d, float lr, float b1, float b2,
                                           float eps, float ibc1, float ibc2) {
  const float mm = fmaf(b1, m, (1.0f - b1) * g);
  const float vv = fmaf(b2, v, (1.0f - b2) * g * g);
  m = mm;
  v = vv;
  const float mh = mm * ibc1, vh = vv * ibc2;
  const float root = (vh > 0.f && vh < INFINITY) ? vh * rsqrtf(vh) : vh;
  return d - __fdividef(lr * mh, root + eps);
}

// Adam on the trainable vertices among 4q .. 4q + 3 of brick `slot` (q in
// [0, 128)): one 16-byte load and store per array.  Vertices of the quad that
// are not trainable are written back unchanged.
__device__ __forceinline__ void adam_quad(int slot, int q, const uint32_t* __restrict__ masks,
                                          const float* __restrict__ grad, float* __restrict__ D,
                                          float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2,
                                          float eps, float ibc1, float ibc2) {
  const uint32_t bits = (__ldg(masks + (int64_t)slot * 48 + 16 + (q >> 3)) >> ((4 * q) & 31)) & 15u;
  if (!bits) return;
  const int64_t a = (int64_t)slot * 512 + 4 * q;
  const float4 g4 = __ldg(reinterpret_cast<const float4*>(grad + a));
  float4 m4 = *reinterpret_cast<const float4*>(m + a);
  float4 v4 = *reinterpret_cast<const float4*>(v + a);
  float4 d4 = *reinterpret_cast<const float4*>(D + a);
  const float* gp = reinterpret_cast<const float*>(&g4);
  float* mp = reinterpret_cast<float*>(&m4);
  float* vp = reinterpret_cast<float*>(&v4);
  float* dp = reinterpret_cast<float*>(&d4);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (!((bits >> k) & 1u)) continue;
    dp[k] = adam_elem(gp[k], mp[k], vp[k], dp[k], lr, b1, b2, eps, ibc1, ibc2);
  }
  *reinterpret_cast<float4*>(m + a) = m4;
  *reinterpret_cast<float4*>(v + a) = v4;
  *reinterpret_cast<float4*>(D + a) = d4;
}
