// Nearest surface point NN(q) (Eq. 4) and the per-point sampling sigma
// (distance to the k-th nearest other point), both by an exact search over a
// uniform cell list of the cloud.  The paper organises the points in a KD-tree
// (Sec. 3 "Discrete Grids"); a GPU walks a uniform grid far better than a
// pointer-chasing tree, and the search below is exact all the same.
//
// Exactness of gp_nn.  The answer is defined in float64:
//   D_j = ((qx-sx)^2 + (qy-sy)^2) + (qz-sz)^2 from the float32 inputs,
//   NN = argmin_j D_j, ties to the lowest j.
// The scan works in float32.  With E_j the exact squared distance, the float32
// value is within a relative 5u (u = 2^-24) of E_j (plus an absolute 1e-30
// covering underflow) and the float64 value within 3*2^-53.  Keeping the
// smallest float32 distance b1 (index j1) and the second smallest b2 over all
// scanned points: if b2 > b1 (1 + 2 eps) + 1e-30 with eps = 2^-18 >> 5u, every
// other point has E_k > E_j1 (1 + eps), hence a larger float64 value, so j1 is
// the float64 answer.  Otherwise (a near tie, e.g. duplicate points) the
// scanned cells are visited again and every point within that margin is ranked
// by its float64 value and index.  Rings of cells are scanned around the
// query's cell until the distance from q to the scanned box, less a rounding
// margin of 1e-5 (1 + |q|_inf), exceeds sqrt(b1 (1 + 8 eps)), so no unscanned
// point can enter the comparison.
#include <algorithm>
#include <cmath>
#include <vector>

#include "gp_internal.cuh"

namespace {

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

__global__ void k_point_cells(const float* __restrict__ pts, int64_t J, NNGrid g, int32_t* __restrict__ cid,
                              int32_t* __restrict__ counts) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= J) return;
  int cx = nn_cell(pts[3 * j], g), cy = nn_cell(pts[3 * j + 1], g), cz = nn_cell(pts[3 * j + 2], g);
  int32_t c = (int32_t)(((int64_t)cz * g.G + cy) * g.G + cx);
  cid[j] = c;
  atomicAdd(counts + c, 1);
}

__global__ void k_point_scatter(const float* __restrict__ pts, int64_t J, const int32_t* __restrict__ cid,
                                const int32_t* __restrict__ start, int32_t* __restrict__ cursor,
                                float4* __restrict__ sorted) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= J) return;
  int32_t c = cid[j];
  int32_t pos = start[c] + atomicAdd(cursor + c, 1);
  sorted[pos] = make_float4(pts[3 * j], pts[3 * j + 1], pts[3 * j + 2], __int_as_float((int)j));
}

// sigma_j: distance to the k-th nearest other point, by a bounded max-heap.
__global__ void __launch_bounds__(128) k_knn_sigma(NNGrid g, int64_t J, int k, float* __restrict__ sigma) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= J) return;
  float4 me = g.pts[t];
  int self = __float_as_int(me.w);
  float heap[64];
  int cnt = 0;
  if (k <= 0) {
    sigma[self] = 0.f;
    return;
  }
  float q[3] = {me.x, me.y, me.z};
  int c[3] = {nn_cell(q[0], g), nn_cell(q[1], g), nn_cell(q[2], g)};
  float margin = nn_margin(q);
  for (int r = 0; r <= g.G; ++r) {
    nn_ring(c, r, g, [&](int a, int b) {
      for (int p = a; p < b; ++p) {
        float4 P = g.pts[p];
        if (__float_as_int(P.w) == self) continue;
        float dx = q[0] - P.x, dy = q[1] - P.y, dz = q[2] - P.z;
        float d = dx * dx + dy * dy + dz * dz;
        if (cnt < k) {
          // sift up
          int i = cnt++;
          while (i > 0) {
            int par = (i - 1) >> 1;
            if (heap[par] >= d) break;
            heap[i] = heap[par];
            i = par;
          }
          heap[i] = d;
        } else if (d < heap[0]) {
          // replace root, sift down
          int i = 0;
          while (true) {
            int l = 2 * i + 1;
            if (l >= k) break;
            int m = (l + 1 < k && heap[l + 1] > heap[l]) ? l + 1 : l;
            if (heap[m] <= d) break;
            heap[i] = heap[m];
            i = m;
          }
          heap[i] = d;
        }
      }
    });
    if (cnt == k) {
      float gap = nn_gap(q, c, r, g);
      if (gap == INFINITY) break;
      float gs = gap - margin;
      if (gs > 0.f && gs * gs > heap[0] * (1.0f + 8.0f * NN_EPS) + NN_TINY) break;
    } else if (nn_gap(q, c, r, g) == INFINITY) {
      break;
    }
  }
  sigma[self] = cnt > 0 ? sqrtf(heap[0]) : 0.f;
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
        float rad = sqrtf(rem) * 1.000001f + margin;
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
// each, the rows (fixed y) closest first, alternating sides, each clipped to
// the cells within the current radius; a side stops at its first slab or row
// whose lower bound exceeds thr, since bounds only grow outwards and thr only
// shrinks.  Every point with squared distance <= the final thr lies in a row
// that was visited, within the x-range read.
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
          const float rad = sqrtf(thr - lyz2) * 1.000001f + margin;
          const int xa = nn_cell(q[0] - rad, g), xb = nn_cell(q[0] + rad, g);
          const int64_t row = ((int64_t)cz * G + cy) * G;
          visit(__ldg(g.start + row + xa), __ldg(g.start + row + xb + 1));
        }
      }
    }
  }
}

// Near tie (another point within the float32 margin of the best): rank every
// point within the margin by its float64 distance and index.  Rings 0..r_end
// (or, for r_end < 0, the ball walk) cover every row within the pruning radius.
__device__ __forceinline__ int nn_break_tie(const float q[3], const int c[3], const NNGrid& g, float margin,
                                            const NNState& st, int r_end) {
  const float tie = st.b1 * (1.0f + 2.0f * NN_EPS) + NN_TINY;
  if (st.b2 > tie) return st.j1;
  double bd = INFINITY;
  int bj = 0x7fffffff;
  const float thr = st.thr;
  auto rank = [&](int a, int b) {
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
__device__ __forceinline__ int nn_thread_search(const float q[3], const int c[3], const NNGrid& g, float margin,
                                                NNState& st) {
  auto one = [&](float4 P) {
    float dx = q[0] - P.x, dy = q[1] - P.y, dz = q[2] - P.z;
    nn_update(st, dx * dx + dy * dy + dz * dz, __float_as_int(P.w));
  };
  // Points of a range, four loads in flight at a time (same visiting order).
  auto scan = [&](int a, int b) {
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
  return nn_break_tie(q, c, g, margin, st, r_end);
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

// One thread per query.  Queries with a NaN, infinite or huge coordinate (whose
// squared distances would overflow float32) get -1 and a NaN surface point.
// Smallest-eigenvalue eigenvector of a symmetric 3x3 matrix (Smith, "Eigenvalues
// of a symmetric 3x3 matrix", CACM 1961: the characteristic cubic solved by
// trigonometry), then a null vector of A - l I from the largest cross product
// of its rows.  Returns false when the matrix is (nearly) isotropic.
__device__ bool smallest_eigvec(const double A[6], double v[3]) {
  // A = [a00 a01 a02; . a11 a12; . . a22] packed as a00, a01, a02, a11, a12, a22
  const double a00 = A[0], a01 = A[1], a02 = A[2], a11 = A[3], a12 = A[4], a22 = A[5];
  const double p1 = a01 * a01 + a02 * a02 + a12 * a12;
  const double qm = (a00 + a11 + a22) / 3.0;
  const double p2 = (a00 - qm) * (a00 - qm) + (a11 - qm) * (a11 - qm) + (a22 - qm) * (a22 - qm) + 2.0 * p1;
  if (!(p2 > 1e-300)) return false;
  const double p = sqrt(p2 / 6.0);
  const double b00 = (a00 - qm) / p, b11 = (a11 - qm) / p, b22 = (a22 - qm) / p;
  const double b01 = a01 / p, b02 = a02 / p, b12 = a12 / p;
  double r = 0.5 * (b00 * (b11 * b22 - b12 * b12) - b01 * (b01 * b22 - b12 * b02) + b02 * (b01 * b12 - b11 * b02));
  r = fmin(1.0, fmax(-1.0, r));
  const double phi = acos(r) / 3.0;
  const double lmin = qm + 2.0 * p * cos(phi + 2.0943951023931954923);  // + 2 pi / 3
  const double r0[3] = {a00 - lmin, a01, a02}, r1[3] = {a01, a11 - lmin, a12}, r2[3] = {a02, a12, a22 - lmin};
  double c[3][3] = {{r0[1] * r1[2] - r0[2] * r1[1], r0[2] * r1[0] - r0[0] * r1[2], r0[0] * r1[1] - r0[1] * r1[0]},
                    {r0[1] * r2[2] - r0[2] * r2[1], r0[2] * r2[0] - r0[0] * r2[2], r0[0] * r2[1] - r0[1] * r2[0]},
                    {r1[1] * r2[2] - r1[2] * r2[1], r1[2] * r2[0] - r1[0] * r2[2], r1[0] * r2[1] - r1[1] * r2[0]}};
  int best = 0;
  double bn = -1.0;
  for (int k = 0; k < 3; ++k) {
    double nk = c[k][0] * c[k][0] + c[k][1] * c[k][1] + c[k][2] * c[k][2];
    if (nk > bn) {
      bn = nk;
      best = k;
    }
  }
  if (!(bn > 1e-300)) return false;
  const double inv = 1.0 / sqrt(bn);
  v[0] = c[best][0] * inv;
  v[1] = c[best][1] * inv;
  v[2] = c[best][2] * inv;
  return true;
}

// Normal of each point: direction of least spread of the points within
// sigma_j (its k-nearest-neighbour ball), by PCA.  Used only to seed gp_nn.
__global__ void __launch_bounds__(128) k_normals(NNGrid g, int64_t J, const float* __restrict__ sigma,
                                                 float* __restrict__ normals) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= J) return;
  const float4 me = g.pts[t];
  const int self = __float_as_int(me.w);
  const float q[3] = {me.x, me.y, me.z};
  const int c[3] = {nn_cell(q[0], g), nn_cell(q[1], g), nn_cell(q[2], g)};
  const float rad = sigma[self];
  const float r2 = rad * rad * 1.000001f;
  const float margin = nn_margin(q);
  double m[3] = {0, 0, 0}, S[6] = {0, 0, 0, 0, 0, 0};
  int cnt = 0;
  for (int r = 0; r <= g.G; ++r) {
    nn_ring(c, r, g, [&](int a, int b) {
      for (int p = a; p < b; ++p) {
        float4 P = g.pts[p];
        float dx = P.x - q[0], dy = P.y - q[1], dz = P.z - q[2];
        if (dx * dx + dy * dy + dz * dz > r2) continue;
        m[0] += dx;
        m[1] += dy;
        m[2] += dz;
        S[0] += (double)dx * dx;
        S[1] += (double)dx * dy;
        S[2] += (double)dx * dz;
        S[3] += (double)dy * dy;
        S[4] += (double)dy * dz;
        S[5] += (double)dz * dz;
        ++cnt;
      }
    });
    float gap = nn_gap(q, c, r, g);
    if (gap == INFINITY || gap - margin > rad) break;
  }
  float nv[3] = {0.f, 0.f, 0.f};
  if (cnt >= 3) {
    for (int a = 0; a < 3; ++a) m[a] /= cnt;
    double C[6] = {S[0] / cnt - m[0] * m[0], S[1] / cnt - m[0] * m[1], S[2] / cnt - m[0] * m[2],
                   S[3] / cnt - m[1] * m[1], S[4] / cnt - m[1] * m[2], S[5] / cnt - m[2] * m[2]};
    double v[3];
    if (smallest_eigvec(C, v)) {
      nv[0] = (float)v[0];
      nv[1] = (float)v[1];
      nv[2] = (float)v[2];
    }
  }
  normals[3 * (int64_t)self + 0] = nv[0];
  normals[3 * (int64_t)self + 1] = nv[1];
  normals[3 * (int64_t)self + 2] = nv[2];
}

// Extra seeds: the points of the cell holding the foot of q on the tangent
// plane of its source point, f = q - ((q - s) . n) n.  The nearest point tends
// to lie near f, much closer to q than s is, which shrinks the ball to walk.
__device__ __forceinline__ void nn_seed_foot(NNState& st, const float q[3], const int32_t* __restrict__ hint,
                                             int64_t i, int64_t J, const float* __restrict__ pts_orig,
                                             const float* __restrict__ normals, const NNGrid& g) {
  if (!hint || !normals) return;
  const int j = hint[i];
  if (j < 0 || j >= J) return;
  const float n0 = normals[3 * (int64_t)j], n1 = normals[3 * (int64_t)j + 1], n2 = normals[3 * (int64_t)j + 2];
  const float s0 = pts_orig[3 * (int64_t)j], s1 = pts_orig[3 * (int64_t)j + 1], s2 = pts_orig[3 * (int64_t)j + 2];
  const float h = (q[0] - s0) * n0 + (q[1] - s1) * n1 + (q[2] - s2) * n2;
  const int cx = nn_cell(q[0] - h * n0, g), cy = nn_cell(q[1] - h * n1, g), cz = nn_cell(q[2] - h * n2, g);
  const int64_t cell = ((int64_t)cz * g.G + cy) * g.G + cx;
  const int a = __ldg(g.start + cell), b = __ldg(g.start + cell + 1);
  for (int p = a; p < b; ++p) {
    float4 P = __ldg(g.pts + p);
    float dx = q[0] - P.x, dy = q[1] - P.y, dz = q[2] - P.z;
    nn_update(st, dx * dx + dy * dy + dz * dz, __float_as_int(P.w));
  }
}

__global__ void __launch_bounds__(256) k_nn(NNGrid g, const float* __restrict__ qin, int64_t n,
                                            const int32_t* __restrict__ hint, int64_t J,
                                            const float* __restrict__ pts_orig, int32_t* __restrict__ nn_out,
                                            float* __restrict__ rec, Grid band, int32_t* __restrict__ nvalid,
                                            const float* __restrict__ normals) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = i < n;
  float q[3] = {0.f, 0.f, 0.f};
  if (active) {
    q[0] = qin[3 * i];
    q[1] = qin[3 * i + 1];
    q[2] = qin[3 * i + 2];
  }
  const bool ok = active && nn_query_ok(q);
  int c[3] = {0, 0, 0};
  float margin = 0.f;
  NNState st{INFINITY, INFINITY, INFINITY, 0x7fffffff};
  if (ok) {
    c[0] = nn_cell(q[0], g);
    c[1] = nn_cell(q[1], g);
    c[2] = nn_cell(q[2], g);
    margin = nn_margin(q);
    nn_seed(st, q, hint, i, J, pts_orig);
    if (st.b1 < INFINITY) nn_seed_foot(st, q, hint, i, J, pts_orig, normals, g);
  }
  int best = -1;
  if (ok) best = nn_thread_search(q, c, g, margin, st);
  if (active) nn_finish(i, q, best, pts_orig, nn_out, rec, band, nvalid);
}

NNGrid make_grid(const gp_band* b) {
  NNGrid g;
  g.pts = b->pts_sorted;
  g.start = b->cell_start;
  g.G = b->G;
  g.half_g = 0.5f * (float)b->G;
  g.cs = 2.0f / (float)b->G;
  return g;
}

}  // namespace

// Emission order of the spatial batches: point indices sorted by the Morton
// code of their cell-list cell (ties by index), so that consecutive points, and
// the queries drawn around them, stay close in all three directions.  Set-up
// only: the sort runs once per cloud on the host.
static uint64_t spread3(uint64_t x) {
  x &= 0x1fffff;
  x = (x | x << 32) & 0x1f00000000ffffull;
  x = (x | x << 16) & 0x1f0000ff0000ffull;
  x = (x | x << 8) & 0x100f00f00f00f00full;
  x = (x | x << 4) & 0x10c30c30c30c30c3ull;
  x = (x | x << 2) & 0x1249249249249249ull;
  return x;
}

static gp_status build_emit_order(gp_band* b) {
  gp_ctx* ctx = b->ctx;
  const int64_t J = b->J;
  std::vector<float> pts((size_t)(3 * J));
  GP_CUDA(ctx, cudaMemcpyAsync(pts.data(), b->pts, 3 * J * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
  GP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  const float half_g = 0.5f * (float)b->G;
  std::vector<uint64_t> key((size_t)J);
  for (int64_t j = 0; j < J; ++j) {
    uint64_t c[3];
    for (int a = 0; a < 3; ++a) {
      float t = (pts[3 * j + a] + 1.0f) * half_g;
      int ci = (t < 0.f) ? 0 : (int)std::floor(std::fmin(t, 1.0e6f));
      c[a] = (uint64_t)std::min(std::max(ci, 0), b->G - 1);
    }
    uint64_t m = spread3(c[0]) | (spread3(c[1]) << 1) | (spread3(c[2]) << 2);
    key[(size_t)j] = (m << 31) | (uint64_t)j;  // Morton code (<= 30 bits), then index
  }
  std::sort(key.begin(), key.end());
  std::vector<int32_t> order((size_t)J);
  for (int64_t t = 0; t < J; ++t) order[(size_t)t] = (int32_t)(key[(size_t)t] & 0x7fffffffull);
  gp_status st = gp_alloc(ctx, &b->emit_order, J, "emission order");
  if (st) return st;
  GP_CUDA(ctx, cudaMemcpyAsync(b->emit_order, order.data(), J * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
  GP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return GP_OK;
}

// Point copy, cell list and sigma (called by gp_build_band).
gp_status gp_build_points(gp_band* b, const float* pts_dev) {
  gp_ctx* ctx = b->ctx;
  cudaStream_t s = ctx->stream;
  const int64_t J = b->J;
  if (b->G <= 0) {
    int G = (int)std::sqrt((double)J / 3.0);
    b->G = std::min(std::max(G, 4), 512);
  }
  const int G = b->G;
  const int64_t ncell = (int64_t)G * G * G;
  gp_status st;
  if ((st = gp_alloc(ctx, &b->pts, 3 * J, "points"))) return st;
  GP_CUDA(ctx, cudaMemcpyAsync(b->pts, pts_dev, 3 * J * sizeof(float), cudaMemcpyDeviceToDevice, s));
  if ((st = gp_alloc(ctx, &b->pts_sorted, J, "sorted points"))) return st;
  if ((st = gp_alloc(ctx, &b->cell_start, ncell + 1, "cell starts"))) return st;
  int32_t *cid = nullptr, *cursor = nullptr;
  if ((st = gp_alloc(ctx, &cid, J, "point cells"))) return st;
  if ((st = gp_alloc(ctx, &cursor, ncell, "cell cursor"))) {
    cudaFree(cid);
    return st;
  }
  NNGrid g = make_grid(b);
  cudaError_t e = cudaMemsetAsync(b->cell_start, 0, (ncell + 1) * sizeof(int32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(cursor, 0, ncell * sizeof(int32_t), s);
  if (e == cudaSuccess) {
    k_point_cells<<<gp_blocks(J, 256), 256, 0, s>>>(b->pts, J, g, cid, b->cell_start);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    int64_t total = 0;
    st = gp_exclusive_scan_i32(ctx, b->cell_start, ncell + 1, &total);
    if (!st) {
      k_point_scatter<<<gp_blocks(J, 256), 256, 0, s>>>(b->pts, J, cid, b->cell_start, cursor, b->pts_sorted);
      e = cudaGetLastError();
    }
  }
  cudaStreamSynchronize(s);
  cudaFree(cid);
  cudaFree(cursor);
  if (st) return st;
  if (e != cudaSuccess) return gp_cuda_fail(ctx, e, "point cell list");
  if (b->knn_k > 0) {
    if ((st = gp_alloc(ctx, &b->sigma, J, "sigma"))) return st;
    if ((st = gp_alloc(ctx, &b->perm, J, "permutation"))) return st;
    if ((st = gp_alloc(ctx, &b->inv_perm, J, "inverse permutation"))) return st;
    if ((st = gp_alloc(ctx, &b->order_tiles, (J + GP_ORDER_TILE - 1) / GP_ORDER_TILE + 1, "order tiles"))) return st;
    if ((st = build_emit_order(b))) return st;
    int k = (int)std::min<int64_t>(b->knn_k, J - 1);
    GP_KERNEL(ctx, "k_knn_sigma", k_knn_sigma<<<gp_blocks(J, 128), 128, 0, s>>>(g, J, k, b->sigma));
    if ((st = gp_alloc(ctx, &b->normals, 3 * J, "normals"))) return st;
    GP_KERNEL(ctx, "k_normals", k_normals<<<gp_blocks(J, 128), 128, 0, s>>>(g, J, b->sigma, b->normals));
  }
  return GP_OK;
}

extern "C" gp_status gp_band_sigma(const gp_band* b, float* sigma_dev) {
  if (!b) return GP_ERR_ARG;
  if (!sigma_dev) return gp_fail(b->ctx, GP_ERR_ARG, "gp_band_sigma: null output");
  if (!b->sigma) return gp_fail(b->ctx, GP_ERR_STATE, "gp_band_sigma: band built with knn_k = 0");
  GP_CUDA(b->ctx, cudaMemcpyAsync(sigma_dev, b->sigma, b->J * sizeof(float), cudaMemcpyDeviceToDevice,
                                  b->ctx->stream));
  return GP_OK;
}

extern "C" gp_status gp_nn(gp_band* b, const float* q_dev, int64_t n, const int32_t* hint_dev, int32_t* nn_dev,
                           float* rec_dev, int32_t* nvalid_dev) {
  if (!b) return GP_ERR_ARG;
  gp_ctx* ctx = b->ctx;
  if (n < 0 || n >= (int64_t(1) << 31)) return gp_fail(ctx, GP_ERR_ARG, "gp_nn: n must be in [0, 2^31)");
  if (nvalid_dev) GP_CUDA(ctx, cudaMemsetAsync(nvalid_dev, 0, sizeof(int32_t), ctx->stream));
  if (n == 0) return GP_OK;
  if (!q_dev || (!nn_dev && !rec_dev)) return gp_fail(ctx, GP_ERR_ARG, "gp_nn: null pointer");
  NNGrid g = make_grid(b);
  Grid band;
  band.table = b->brick_table;
  band.masks = b->masks;
  band.D = b->D;
  band.nb = b->nb;
  band.R = b->R;
  band.half_r = 0.5f * (float)b->R;
  GP_KERNEL(ctx, "k_nn", k_nn<<<gp_blocks(n, 256), 256, 0, ctx->stream>>>(g, q_dev, n, hint_dev, b->J, b->pts,
                                                                           nn_dev, rec_dev, band, nvalid_dev,
                                                                           b->normals));
  return GP_OK;
}
