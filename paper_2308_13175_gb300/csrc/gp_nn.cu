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
#include "gp_nn_device.cuh"

namespace {

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

__device__ __forceinline__ void nn_add_work(unsigned long long* total, int v) {
  unsigned long long w = (unsigned long long)v;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
  if ((threadIdx.x & 31) == 0 && w) atomicAdd(total, w);
}

// One thread per query.  Queries with a NaN, infinite or huge coordinate (whose
// squared distances would overflow float32) get -1 and a NaN surface point.
#ifndef GP_NN_BLOCK
#define GP_NN_BLOCK 256
#endif
#ifdef GP_NN_MIN_BLOCKS
#define GP_NN_BOUNDS __launch_bounds__(GP_NN_BLOCK, GP_NN_MIN_BLOCKS)
#else
#define GP_NN_BOUNDS __launch_bounds__(GP_NN_BLOCK)
#endif
// COUNT: also add the number of point distances evaluated (seeds, walk and
// tie-break) to *work_total, for measurement; the search is the same.
template <bool COUNT>
__global__ void GP_NN_BOUNDS k_nn(NNGrid g, const float* __restrict__ qin, int64_t n,
                                            const int32_t* __restrict__ hint, int64_t J,
                                            const float* __restrict__ pts_orig, int32_t* __restrict__ nn_out,
                                            float* __restrict__ rec, Grid band, int32_t* __restrict__ nvalid,
                                            const float* __restrict__ normals,
                                            unsigned long long* __restrict__ work_total) {
  int work_v = 0;
  int* work = COUNT ? &work_v : nullptr;
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
    if (COUNT && st.b1 < INFINITY) ++work_v;
    if (st.b1 < INFINITY) nn_seed_foot(st, q, hint, i, J, pts_orig, normals, g, work);
  }
  int best = -1;
  if (ok) best = nn_thread_search(q, c, g, margin, st, work);
  if (active) nn_finish(i, q, best, pts_orig, nn_out, rec, band, nvalid);
  if (COUNT) nn_add_work(work_total, work_v);
}

// The same search for large seeded batches.  Each thread first seeds its own query; the block then sorts its queries (in
// segments of NN_SPAN), stably, by the seeded radius (a counting sort on thr in
// quarters of the squared cell size: the walk visits about thr / cs^2 rows),
// and every thread searches the query of its rank, so that the lanes of a warp
// have walks of similar length while queries of equal key keep their spatial
// order.  Which thread searches a query does not change its result.
// Measured on GB300: 18% faster than k_nn on the 4,194,304-query superquadric
// batch and 10% on the 2,097,152-query scene batch, 6-10% slower on the
// 262,144-query single-object batch, hence NN_SORTED_MIN_QUERIES.  Blocks of
// 128 (sorted together) beat 256 by 4% on the scene: a block's slot is held
// until its slowest warp ends, and smaller blocks leave shorter tails; 64
// or a 64-query sort span lose more than that.
constexpr int NN_THREADS = 128;
constexpr int NN_SPAN = 128;  // queries sorted together (a multiple of 32 dividing NN_THREADS)
constexpr int NN_SEGS = NN_THREADS / NN_SPAN;
constexpr int NN_SPAN_WARPS = NN_SPAN / 32;
constexpr int NN_BUCKETS = 16;
constexpr int64_t NN_SORTED_MIN_QUERIES = int64_t(1) << 20;
static_assert(NN_SPAN % 32 == 0 && NN_THREADS % NN_SPAN == 0, "sort span");

template <bool COUNT>
__global__ void __launch_bounds__(NN_THREADS) k_nn_sorted(NNGrid g, const float* __restrict__ qin, int64_t n,
                                                   const int32_t* __restrict__ hint, int64_t J,
                                                   const float* __restrict__ pts_orig, int32_t* __restrict__ nn_out,
                                                   float* __restrict__ rec, Grid band, int32_t* __restrict__ nvalid,
                                                   const float* __restrict__ normals,
                                                   unsigned long long* __restrict__ work_total) {
  int work_v = 0;
  int* work = COUNT ? &work_v : nullptr;
  __shared__ int s_off[NN_SEGS][NN_BUCKETS][NN_SPAN_WARPS];  // count, then first rank in the segment
  __shared__ float4 s_q[NN_THREADS];   // q, and the query's offset in the block (int bits; -1 - offset if invalid)
  __shared__ float4 s_st[NN_THREADS];  // b1, b2, thr, j1 (int bits)
  const int t = threadIdx.x, lane = t & 31, seg = t / NN_SPAN, wseg = (t % NN_SPAN) >> 5;
  const int64_t base = (int64_t)blockIdx.x * NN_THREADS;
  int64_t i = base + t;
  const bool active = i < n;
  float q[3] = {0.f, 0.f, 0.f};
  if (active) {
    q[0] = qin[3 * i];
    q[1] = qin[3 * i + 1];
    q[2] = qin[3 * i + 2];
  }
  bool ok = active && nn_query_ok(q);
  NNState st{INFINITY, INFINITY, INFINITY, 0x7fffffff};
  int key = 0;
  if (ok) {
    nn_seed(st, q, hint, i, J, pts_orig);
    if (COUNT && st.b1 < INFINITY) ++work_v;
    if (st.b1 < INFINITY) {
      nn_seed_foot(st, q, hint, i, J, pts_orig, normals, g, work);
      key = (int)fminf(4.0f * st.thr / (g.cs * g.cs), (float)(NN_BUCKETS - 2));
    } else {
      key = NN_BUCKETS - 1;  // unseeded: the ring search
    }
  }
  // Stable counting sort within each segment of NN_SPAN queries:
  // rank = (smaller key) + (same key, lower warp) + (same key, lower lane).
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  const int in_warp = __popc(peers & ((1u << lane) - 1u));
  for (int k = t; k < NN_SEGS * NN_BUCKETS * NN_SPAN_WARPS; k += NN_THREADS) (&s_off[0][0][0])[k] = 0;
  __syncthreads();
  if (in_warp == 0) s_off[seg][key][wseg] = __popc(peers);
  __syncthreads();
  if (t < NN_SEGS) {
    int run = 0;
    for (int b = 0; b < NN_BUCKETS; ++b)
      for (int w = 0; w < NN_SPAN_WARPS; ++w) {
        const int c = s_off[t][b][w];
        s_off[t][b][w] = run;
        run += c;
      }
  }
  __syncthreads();
  const int rank = seg * NN_SPAN + s_off[seg][key][wseg] + in_warp;
  s_q[rank] = make_float4(q[0], q[1], q[2], __int_as_float(ok ? t : -1 - t));
  s_st[rank] = make_float4(st.b1, st.b2, st.thr, __int_as_float(st.j1));
  __syncthreads();
  const float4 mq = s_q[t], ms = s_st[t];
  const int off = __float_as_int(mq.w);
  ok = off >= 0;
  i = base + (ok ? off : -1 - off);
  q[0] = mq.x;
  q[1] = mq.y;
  q[2] = mq.z;
  st = NNState{ms.x, ms.y, ms.z, __float_as_int(ms.w)};
  int best = -1;
  if (ok) {
    const int c[3] = {nn_cell(q[0], g), nn_cell(q[1], g), nn_cell(q[2], g)};
    best = nn_thread_search(q, c, g, nn_margin(q), st, work);
  }
  if (i < n) nn_finish(i, q, best, pts_orig, nn_out, rec, band, nvalid);
  if (COUNT) nn_add_work(work_total, work_v);
}

// Points and sigma in emission order, for the sampler's coalesced reads.
__global__ void k_emit_pts(const int32_t* __restrict__ order, const float* __restrict__ pts,
                           const float* __restrict__ sigma, int64_t J, float4* __restrict__ out) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= J) return;
  const int64_t j = order[u];
  out[u] = make_float4(pts[3 * j], pts[3 * j + 1], pts[3 * j + 2], sigma[j]);
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

constexpr double NN_POINTS_PER_CELL = 6.5;

// Point copy, cell list and sigma (called by gp_build_band).
gp_status gp_build_points(gp_band* b, const float* pts_dev) {
  gp_ctx* ctx = b->ctx;
  cudaStream_t s = ctx->stream;
  const int64_t J = b->J;
  if (b->G <= 0) {
    // About 6.5 points per occupied cell of the search grid, the measured
    // optimum (4.9 to 8 points per cell were within 1-3% on the benchmark
    // clouds).  The cloud is a surface, so the cells it occupies at grid G are
    // about n_occ (G / R)^2, n_occ being its occupied cells at the band's R.
    // That estimate fails for a cloud too sparse to cover its surface at R
    // (n_occ near J); there sqrt(J / 3) cells per axis, the bound that served
    // such clouds before, is the smaller one and is taken.
    const double occ = (double)std::max<int64_t>(b->n_occ, 1);
    const double g_area = (double)b->R * std::sqrt((double)J / (NN_POINTS_PER_CELL * occ));
    const double g_count = std::sqrt((double)J / 3.0);
    const int G = (int)std::min(g_area, g_count);
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
    if ((st = gp_alloc(ctx, &b->emit_slot, J, "emission slots"))) return st;
    int k = (int)std::min<int64_t>(b->knn_k, J - 1);
    GP_KERNEL(ctx, "k_knn_sigma", k_knn_sigma<<<gp_blocks(J, 128), 128, 0, s>>>(g, J, k, b->sigma));
    if ((st = gp_alloc(ctx, &b->normals, 3 * J, "normals"))) return st;
    GP_KERNEL(ctx, "k_normals", k_normals<<<gp_blocks(J, 128), 128, 0, s>>>(g, J, b->sigma, b->normals));
    if ((st = gp_alloc(ctx, &b->emit_pts, J, "emission points"))) return st;
    GP_KERNEL(ctx, "k_emit_pts", k_emit_pts<<<gp_blocks(J, 256), 256, 0, s>>>(b->emit_order, b->pts, b->sigma, J,
                                                                            b->emit_pts));
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

// The launch of gp_nn; work_total (device, NULL = not counted) receives the
// number of point distances evaluated.
static gp_status nn_launch(gp_band* b, const float* q_dev, int64_t n, const int32_t* hint_dev, int32_t* nn_dev,
                           float* rec_dev, int32_t* nvalid_dev, unsigned long long* work_total) {
  gp_ctx* ctx = b->ctx;
  NNGrid g = make_grid(b);
  Grid band;
  band.table = b->brick_table;
  band.masks = b->masks;
  band.D = b->D;
  band.nb = b->nb;
  band.R = b->R;
  band.half_r = 0.5f * (float)b->R;
  if (hint_dev && n >= NN_SORTED_MIN_QUERIES) {
    if (work_total)
      GP_KERNEL(ctx, "k_nn_sorted_count",
                k_nn_sorted<true><<<gp_blocks(n, NN_THREADS), NN_THREADS, 0, ctx->stream>>>(
                    g, q_dev, n, hint_dev, b->J, b->pts, nn_dev, rec_dev, band, nvalid_dev, b->normals, work_total));
    else
      GP_KERNEL(ctx, "k_nn_sorted",
                k_nn_sorted<false><<<gp_blocks(n, NN_THREADS), NN_THREADS, 0, ctx->stream>>>(
                    g, q_dev, n, hint_dev, b->J, b->pts, nn_dev, rec_dev, band, nvalid_dev, b->normals, nullptr));
    return GP_OK;
  }
  if (work_total)
    GP_KERNEL(ctx, "k_nn_count",
              k_nn<true><<<gp_blocks(n, GP_NN_BLOCK), GP_NN_BLOCK, 0, ctx->stream>>>(
                  g, q_dev, n, hint_dev, b->J, b->pts, nn_dev, rec_dev, band, nvalid_dev, b->normals, work_total));
  else
    GP_KERNEL(ctx, "k_nn",
              k_nn<false><<<gp_blocks(n, GP_NN_BLOCK), GP_NN_BLOCK, 0, ctx->stream>>>(
                  g, q_dev, n, hint_dev, b->J, b->pts, nn_dev, rec_dev, band, nvalid_dev, b->normals, nullptr));
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
  return nn_launch(b, q_dev, n, hint_dev, nn_dev, rec_dev, nvalid_dev, nullptr);
}

extern "C" gp_status gp_nn_work(gp_band* b, const float* q_dev, int64_t n, const int32_t* hint_dev,
                                int32_t* nn_dev, int64_t* work_host) {
  if (!b) return GP_ERR_ARG;
  gp_ctx* ctx = b->ctx;
  if (n < 0 || n >= (int64_t(1) << 31)) return gp_fail(ctx, GP_ERR_ARG, "gp_nn_work: n must be in [0, 2^31)");
  if (!work_host || !nn_dev || (n > 0 && !q_dev)) return gp_fail(ctx, GP_ERR_ARG, "gp_nn_work: null pointer");
  *work_host = 0;
  if (n == 0) return GP_OK;
  unsigned long long* dev = nullptr;
  gp_status st = gp_alloc(ctx, &dev, 1, "gp_nn_work counter");
  if (st) return st;
  cudaError_t e = cudaMemsetAsync(dev, 0, sizeof(unsigned long long), ctx->stream);
  if (e == cudaSuccess) {
    st = nn_launch(b, q_dev, n, hint_dev, nn_dev, nullptr, nullptr, dev);
    unsigned long long h = 0;
    if (!st) e = cudaMemcpyAsync(&h, dev, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream);
    if (!st && e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    *work_host = (int64_t)h;
  }
  cudaFree(dev);
  if (st) return st;
  if (e != cudaSuccess) return gp_cuda_fail(ctx, e, "gp_nn_work");
  return GP_OK;
}
