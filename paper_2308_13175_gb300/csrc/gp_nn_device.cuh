// Device side of the exact nearest-point search (shared by gp_nn.cu and
// gp_multi.cu): the uniform cell list, the float32 screen with its proven
// margins, the seeded ball walk, the ring search for unseeded queries and the
// float64 tie-break.  The exactness argument is in the header of gp_nn.cu.
#pragma once

#include <math.h>

#include "gp_internal.cuh"

constexpr float NN_EPS = 3.814697265625e-06f;  // 2^-18
constexpr float NN_TINY = 1e-30f;

struct NNGrid {
  const float4* __restrict__ pts;      // sorted by cell: x, y, z, original index bits
  const int32_t* __restrict__ start;   // G^3 + 1
  int G;
  float half_g;  // G / 2
  float cs;      // 2 / G
};

__device__ __forceinline__ int nn_cell(float x, const NNGrid& g) {
  float t = __fmul_rn(__fadd_rn(x, 1.0f), g.half_g);
  int c = (t < 0.f) ? -1 : (int)floorf(fminf(t, 1.0e6f));
  return min(max(c, 0), g.G - 1);
}

// Lower bound on the distance from q to any point outside the box of cells
// [c - r, c + r]; returns +inf when the box covers the whole grid.
__device__ __forceinline__ float nn_gap(const float q[3], const int c[3], int r, const NNGrid& g) {
  float gap = INFINITY;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (c[a] - r > 0) {
      float lo = -1.0f + (float)(c[a] - r) * g.cs;
      gap = fminf(gap, q[a] - lo);
    }
    if (c[a] + r < g.G - 1) {
      float hi = -1.0f + (float)(c[a] + r + 1) * g.cs;
      gap = fminf(gap, hi - q[a]);
    }
  }
  return gap;
}

// sqrt(x) for the x-range of a row, as x rsqrt(x): within a relative 3e-7
// of the correctly rounded root, which the range's factor 1.000001 and its
// additive margin (>= 2e-5) cover.  0 for x <= 0.
__device__ __forceinline__ float nn_row_sqrt(float x) { return x > 0.f ? x * rsqrtf(x) : 0.f; }

__device__ __forceinline__ float nn_margin(const float q[3]) {
  float m = fmaxf(fabsf(q[0]), fmaxf(fabsf(q[1]), fabsf(q[2])));
  return 1e-5f * (2.0f + m);
}

// Visit every cell of ring r (Chebyshev shell) as contiguous point ranges.
template <typename F>
__device__ __forceinline__ void nn_ring(const int c[3], int r, const NNGrid& g, F&& visit) {
  const int G = g.G;
  for (int dz = -r; dz <= r; ++dz) {
    int cz = c[2] + dz;
    if (cz < 0 || cz >= G) continue;
    for (int dy = -r; dy <= r; ++dy) {
      int cy = c[1] + dy;
      if (cy < 0 || cy >= G) continue;
      int64_t row = ((int64_t)cz * G + cy) * G;
      bool full = (dz == -r || dz == r || dy == -r || dy == r);
      if (full) {
        int x0 = max(c[0] - r, 0), x1 = min(c[0] + r, G - 1);
        visit(__ldg(g.start + row + x0), __ldg(g.start + row + x1 + 1));
      } else {
        int xa = c[0] - r, xb = c[0] + r;
        if (xa >= 0) visit(__ldg(g.start + row + xa), __ldg(g.start + row + xa + 1));
        if (xb < G) visit(__ldg(g.start + row + xb), __ldg(g.start + row + xb + 1));
      }
    }
  }
}

__device__ __forceinline__ double nn_d64(const float q[3], float4 p) {
  double dx = __dsub_rn((double)q[0], (double)p.x);
  double dy = __dsub_rn((double)q[1], (double)p.y);
  double dz = __dsub_rn((double)q[2], (double)p.z);
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// Lower bound on |p_a - q_a| for any point p in cell `ca` along one axis
// (edge cells extend to infinity outwards); the margin absorbs the rounding of
// the point-to-cell assignment and of the cell faces.
__device__ __forceinline__ float nn_axis_gap(float qa, int ca, const NNGrid& g, float margin) {
  float lo = -1.0f + (float)ca * g.cs, hi = lo + g.cs;
  float d = 0.f;
  if (ca > 0 && qa < lo) d = lo - qa;
  if (ca < g.G - 1 && qa > hi) d = qa - hi;
  return fmaxf(d - margin, 0.f);
}

// Exact nearest point: b1/j1 = best float32 distance and its index, b2 = the
// runner-up distance (any other point), thr = b1 (1 + 8 eps) + tiny = the
// pruning radius squared.  Only cells that may hold a point with squared
// distance <= thr are read: a row of cells (fixed y, z) is skipped when its y/z
// lower bound already exceeds thr, and its x-range is clipped to the cells
// that intersect the remaining radius.
struct NNState {
  float b1, b2, thr;
  int j1;
};

__device__ __forceinline__ void nn_update(NNState& st, float d, int j) {
  if (d > st.b2) return;   // neither the best nor the runner-up (b1 <= b2)
  if (j == st.j1) return;  // the seeded point, met again in the scan
  if (d < st.b1 || (d == st.b1 && j < st.j1)) {
    st.b2 = st.b1;
    st.b1 = d;
    st.j1 = j;
    st.thr = d * (1.0f + 8.0f * NN_EPS) + NN_TINY;
  } else if (d < st.b2) {
    st.b2 = d;
  }
}

// Lower bound on the y/z distance from q to any point in a row outside the
// square of rows [c - r, c + r]^2 (y, z); +inf when that square covers the grid.
__device__ __forceinline__ float nn_gap_yz(const float q[3], const int c[3], int r, const NNGrid& g) {
  float gap = INFINITY;
#pragma unroll
  for (int a = 1; a < 3; ++a) {
    if (c[a] - r > 0) gap = fminf(gap, q[a] - (-1.0f + (float)(c[a] - r) * g.cs));
    if (c[a] + r < g.G - 1) gap = fminf(gap, (-1.0f + (float)(c[a] + r + 1) * g.cs) - q[a]);
  }
  return gap;
}

// Visit the rows (fixed y, z) of square ring r around the query's row, each
// clipped to the cells whose points may lie within sqrt(thr) of q.  Rows whose
// y/z lower bound alone exceeds thr are skipped.  thr is read live, so rows
// visited later use the tighter radius.
template <typename F>
__device__ __forceinline__ void nn_row_ring(const float q[3], const int c[3], int r, const NNGrid& g, float margin,
                                            const float& thr, F&& visit) {
  const int G = g.G;
  for (int dz = -r; dz <= r; ++dz) {
    int cz = c[2] + dz;
    if (cz < 0 || cz >= G) continue;
    float lz = nn_axis_gap(q[2], cz, g, margin);
    float lz2 = lz * lz;
    bool zedge = (dz == -r || dz == r);
    int step = zedge ? 1 : 2 * r;
    for (int dy = -r; dy <= r; dy += (step > 0 ? step : 1)) {
      int cy = c[1] + dy;
      if (cy < 0 || cy >= G) continue;
      float ly = nn_axis_gap(q[1], cy, g, margin);
      float lyz2 = fmaf(ly, ly, lz2);
      if (lyz2 > thr) continue;
      int xa = 0, xb = G - 1;
      float rem = thr - lyz2;
      if (rem < 16.0f) {
        float rad = nn_row_sqrt(rem) * 1.000001f + margin;
        xa = nn_cell(q[0] - rad, g);
        xb = nn_cell(q[0] + rad, g);
      }
      int64_t row = ((int64_t)cz * G + cy) * G;
      visit(__ldg(g.start + row + xa), __ldg(g.start + row + xb + 1));
      if (r == 0) break;
    }
  }
}

// Scan rows ring by ring until no unscanned row can hold a point within the
// pruning radius; returns the last ring visited.
template <typename F>
__device__ __forceinline__ int nn_ball_scan(const float q[3], const int c[3], const NNGrid& g, float margin,
                                            const float& thr, const float& b1, F&& visit) {
  int r = 0;
  for (; r <= g.G; ++r) {
    if (r > 0) {
      float gap = nn_gap_yz(q, c, r - 1, g);
      if (gap == INFINITY) break;
      float gs = gap - margin;
      if (b1 < INFINITY && gs > 0.f && gs * gs > thr) break;
    }
    nn_row_ring(q, c, r, g, margin, thr, visit);
  }
  return r - 1;
}

// Count of the records gp_step will treat as valid (q inside the domain, the
// cells of q and of its nearest point in the pull band), one atomic per warp.
__device__ __forceinline__ void nn_count_valid(int32_t* nvalid, bool valid) {
  unsigned m = __activemask();
  unsigned vb = __ballot_sync(m, valid);
  if ((int)(threadIdx.x & 31) == __ffs(m) - 1 && vb) atomicAdd(nvalid, __popc(vb));
}

// NaN surface point for queries outside the domain of the search.
__device__ __forceinline__ void nn_invalid(int64_t i, const float q[3], int32_t* nn_out, float* rec) {
  if (nn_out) nn_out[i] = -1;
  if (rec) {
    for (int a = 0; a < 6; ++a) rec[6 * i + a] = a < 3 ? q[a] : __int_as_float(0x7fc00000);
  }
}

// Seed the search with a known point (the query's source point): its distance
// bounds the nearest one from above.
__device__ __forceinline__ void nn_seed(NNState& st, const float q[3], const int32_t* __restrict__ hint, int64_t i,
                                        int64_t J, const float* __restrict__ pts_orig) {
  if (!hint) return;
  int j = hint[i];
  if (j < 0 || j >= J) return;
  float dx = q[0] - pts_orig[3 * (int64_t)j], dy = q[1] - pts_orig[3 * (int64_t)j + 1];
  float dz = q[2] - pts_orig[3 * (int64_t)j + 2];
  float d = dx * dx + dy * dy + dz * dz;
  if (d < INFINITY) {
    st.b1 = d;
    st.j1 = j;
    st.thr = d * (1.0f + 8.0f * NN_EPS) + NN_TINY;
  }
}

// Seeded search (thr finite from the start): walk the slabs (fixed z) and, in
// each, the rows (fixed y) closest first, two at a time (one each side), each
// clipped to the cells within the radius as it stood when the pair was
// tested; a side stops at its first slab or row whose lower bound exceeds
// thr, since bounds only grow outwards and thr only shrinks.  Every point
// with squared distance <= the final thr lies in a row that was visited,
// within the x-range read.
template <typename F>
__device__ __forceinline__ void nn_ball_walk(const float q[3], const int c[3], const NNGrid& g, float margin,
                                             const float& thr, F&& visit) {
  const int G = g.G;
  bool z_done[2] = {false, false};
  for (int kz = 0; !(z_done[0] && z_done[1]); ++kz) {
#pragma unroll
    for (int sz = 0; sz < 2; ++sz) {
      if (z_done[sz] || (kz == 0 && sz == 1)) continue;
      const int cz = c[2] + (sz ? -kz : kz);
      if (cz < 0 || cz >= G) {
        z_done[sz] = true;
        continue;
      }
      const float lz = nn_axis_gap(q[2], cz, g, margin);
      const float lz2 = lz * lz;
      if (lz2 > thr) {
        z_done[sz] = true;
        continue;
      }
      bool y_done[2] = {false, false};
      for (int ky = 0; !(y_done[0] && y_done[1]); ++ky) {
        // Both rows of this distance (c_y + ky, c_y - ky) are tested and
        // their cell starts loaded before either is scanned, so that the two
        // rows' loads are in flight together.  The second row's test and
        // x-range then use the radius from before the first row's scan: a
        // superset of what the shrunken radius needs.
        int a[2] = {0, 0}, b[2] = {0, 0};
#pragma unroll
        for (int sy = 0; sy < 2; ++sy) {
          if (y_done[sy] || (ky == 0 && sy == 1)) continue;
          const int cy = c[1] + (sy ? -ky : ky);
          if (cy < 0 || cy >= G) {
            y_done[sy] = true;
            continue;
          }
          const float ly = nn_axis_gap(q[1], cy, g, margin);
          const float lyz2 = fmaf(ly, ly, lz2);
          if (lyz2 > thr) {
            y_done[sy] = true;
            continue;
          }
          const float rad = nn_row_sqrt(thr - lyz2) * 1.000001f + margin;
          const int xa = nn_cell(q[0] - rad, g), xb = nn_cell(q[0] + rad, g);
          const int64_t row = ((int64_t)cz * G + cy) * G;
          a[sy] = __ldg(g.start + row + xa);
          b[sy] = __ldg(g.start + row + xb + 1);
        }
#pragma unroll
        for (int sy = 0; sy < 2; ++sy)
          if (b[sy] > a[sy]) visit(a[sy], b[sy]);
      }
    }
  }
}

// Near tie (another point within the float32 margin of the best): rank every
// point within the margin by its float64 distance and index.  Rings 0..r_end
// (or, for r_end < 0, the ball walk) cover every row within the pruning radius.
__device__ __forceinline__ int nn_break_tie(const float q[3], const int c[3], const NNGrid& g, float margin,
                                            const NNState& st, int r_end, int* work = nullptr) {
  const float tie = st.b1 * (1.0f + 2.0f * NN_EPS) + NN_TINY;
  if (st.b2 > tie) return st.j1;
  double bd = INFINITY;
  int bj = 0x7fffffff;
  const float thr = st.thr;
  auto rank = [&](int a, int b) {
    if (work) *work += b > a ? b - a : 0;
    for (int p = a; p < b; ++p) {
      float4 P = g.pts[p];
      float dx = q[0] - P.x, dy = q[1] - P.y, dz = q[2] - P.z;
      float d = dx * dx + dy * dy + dz * dz;
      if (d > tie) continue;
      int j = __float_as_int(P.w);
      double dd = nn_d64(q, P);
      if (dd < bd || (dd == bd && j < bj)) {
        bd = dd;
        bj = j;
      }
    }
  };
  if (r_end < 0)
    nn_ball_walk(q, c, g, margin, thr, rank);
  else
    for (int r = 0; r <= r_end; ++r) nn_row_ring(q, c, r, g, margin, thr, rank);
  return bj != 0x7fffffff ? bj : st.j1;
}

// The whole search for one query by one thread, from whatever seed st holds.
// Returns the nearest point's index, or -1 if none compares below +inf.
// work (optional): incremented by the number of point distances evaluated.
__device__ __forceinline__ int nn_thread_search(const float q[3], const int c[3], const NNGrid& g, float margin,
                                                NNState& st, int* work = nullptr) {
  auto one = [&](float4 P) {
    float dx = q[0] - P.x, dy = q[1] - P.y, dz = q[2] - P.z;
    nn_update(st, dx * dx + dy * dy + dz * dz, __float_as_int(P.w));
  };
  // Points of a range, four loads in flight at a time (same visiting order).
  auto scan = [&](int a, int b) {
    if (work) *work += b > a ? b - a : 0;
    int p = a;
    for (; p + 4 <= b; p += 4) {
      float4 P0 = __ldg(g.pts + p), P1 = __ldg(g.pts + p + 1), P2 = __ldg(g.pts + p + 2), P3 = __ldg(g.pts + p + 3);
      one(P0);
      one(P1);
      one(P2);
      one(P3);
    }
    for (; p < b; ++p) one(__ldg(g.pts + p));
  };
  int r_end = -1;
  if (st.b1 < INFINITY)
    nn_ball_walk(q, c, g, margin, st.thr, scan);  // seeded: closest-first walk of the ball
  else
    r_end = nn_ball_scan(q, c, g, margin, st.thr, st.b1, scan);
  if (st.j1 == 0x7fffffff) return -1;
  return nn_break_tie(q, c, g, margin, st, r_end, work);
}

__device__ __forceinline__ void nn_finish(int64_t i, const float q[3], int best, const float* __restrict__ pts_orig,
                                          int32_t* __restrict__ nn_out, float* __restrict__ rec, const Grid& band,
                                          int32_t* __restrict__ nvalid) {
  if (best < 0) {
    nn_invalid(i, q, nn_out, rec);
    if (nvalid) nn_count_valid(nvalid, false);
    return;
  }
  float s3[3] = {pts_orig[3 * (int64_t)best], pts_orig[3 * (int64_t)best + 1], pts_orig[3 * (int64_t)best + 2]};
  if (nn_out) nn_out[i] = best;
  if (rec) {
    rec[6 * i + 0] = q[0];
    rec[6 * i + 1] = q[1];
    rec[6 * i + 2] = q[2];
    rec[6 * i + 3] = s3[0];
    rec[6 * i + 4] = s3[1];
    rec[6 * i + 5] = s3[2];
  }
  if (nvalid) {
    Cells C;
    nn_count_valid(nvalid, classify(band, q, s3, C));
  }
}

__device__ __forceinline__ bool nn_query_ok(const float q[3]) {
  return fabsf(q[0]) <= 1e18f && fabsf(q[1]) <= 1e18f && fabsf(q[2]) <= 1e18f;
}

// Extra seeds: the points of the cell holding the foot of q on the tangent
// plane of its source point, f = q - ((q - s) . n) n.  The nearest point tends
// to lie near f, much closer to q than s is, which shrinks the ball to walk.
__device__ __forceinline__ void nn_seed_foot(NNState& st, const float q[3], const int32_t* __restrict__ hint,
                                             int64_t i, int64_t J, const float* __restrict__ pts_orig,
                                             const float* __restrict__ normals, const NNGrid& g,
                                             int* work = nullptr) {
  if (!hint || !normals) return;
  const int j = hint[i];
  if (j < 0 || j >= J) return;
  const float n0 = normals[3 * (int64_t)j], n1 = normals[3 * (int64_t)j + 1], n2 = normals[3 * (int64_t)j + 2];
  const float s0 = pts_orig[3 * (int64_t)j], s1 = pts_orig[3 * (int64_t)j + 1], s2 = pts_orig[3 * (int64_t)j + 2];
  const float h = (q[0] - s0) * n0 + (q[1] - s1) * n1 + (q[2] - s2) * n2;
  const int cx = nn_cell(q[0] - h * n0, g), cy = nn_cell(q[1] - h * n1, g), cz = nn_cell(q[2] - h * n2, g);
  const int64_t cell = ((int64_t)cz * g.G + cy) * g.G + cx;
  const int a = __ldg(g.start + cell), b = __ldg(g.start + cell + 1);
  if (work) *work += b > a ? b - a : 0;
  for (int p = a; p < b; ++p) {
    float4 P = __ldg(g.pts + p);
    float dx = q[0] - P.x, dy = q[1] - P.y, dz = q[2] - P.z;
    nn_update(st, dx * dx + dy * dy + dz * dz, __float_as_int(P.w));
  }
}

inline NNGrid make_grid(const gp_band* b) {
  NNGrid g;
  g.pts = b->pts_sorted;
  g.start = b->cell_start;
  g.G = b->G;
  g.half_g = 0.5f * (float)b->G;
  g.cs = 2.0f / (float)b->G;
  return g;
}

