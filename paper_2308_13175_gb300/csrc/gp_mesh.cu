// gp_mesh_extract: the surface of the fitted field as a triangle soup,
// marching cubes (Lorensen and Cline, SIGGRAPH 1987) over the cells the fit
// optimised.  Sec. 3 "Overview" meshes the zero level set of the learned field
// with marching cubes; Sec. 3 (after Eq. 8) skips the cells that were not
// optimised; Sec. 4 "Details" meshes at the grid's own resolution.
//
// Cell rule: a cell is meshed iff its 8 corners are all trainable.  Corner c
// (c = dx + 2 dy + 4 dz) is negative iff d < iso.  Topology: on every face of
// the cell, walked counter-clockwise as seen from outside, each maximal run of
// negative corners gives one segment from the cut edge where the walk enters
// the run to the cut edge where it leaves it.  A face's segments depend on its
// four corners only, so neighbouring cells agree and the soup closes up; the
// segments of a cell chain into cycles, each fanned from its lowest edge id
// (cycles in order of that id), which orients every triangle's normal
// (v1 - v0) x (v2 - v0) from the negative to the positive side.  Edge ids:
// 4 * axis + p + 2 q, (p, q) the lower corner's coordinates on the other two
// axes, lower-numbered axis first.  The crossing on an edge from corner lo to
// corner hi lies at t = (iso - d_lo) / (d_hi - d_lo), at the world point
// -1 + h * lo + h * t along the edge's axis.
//
// Launch plan: a meshed cell's lowest corner is trainable, so its brick is
// active; the active bricks are meshed either by one 512-thread block each (one
// cell per thread) or, on large bands, by one warp each (8 per block, 16
// consecutive cells per lane, no block barrier).  Either stages the brick's
// 9^3 corner values and trainable bits in shared memory through the
// 27-neighbour brick table.
// Pass 1 counts triangles per brick, a device scan turns the counts into
// offsets, pass 2 writes the triangles: bricks in active-list order, cells in
// x-fastest order within a brick, each cell's triangles in table order.
#include <cmath>
#include <mutex>

#include "gp_internal.cuh"

namespace {

constexpr int MC_MAX_TRI = 5;       // most triangles any of the 256 cases yields
constexpr int MB_THREADS = 512;     // small bands: one thread per cell of a brick
constexpr int MC_WARPS = 8;         // large bands: bricks per block, one warp each
constexpr int MC_BLOCK = 32 * MC_WARPS;
constexpr int MC_CELLS = 16;        // consecutive cells per lane (512 / 32)
// Bricks per SM from which a warp per brick pays: below it one block per
// brick keeps more threads busy (single object, 7 bricks per SM: 12 / 24 us
// against 18 / 71 us); above it the warp form keeps more bricks in flight
// (dense 257^3, 236 per SM: 88 / 150 us against 184 / 239 us).
constexpr int MC_WARP_MIN_BRICKS_PER_SM = 32;

static_assert(MB_THREADS == GP_ORDER_THREADS, "block_exclusive_scan is sized for GP_ORDER_THREADS");
constexpr int MC_S = 9;             // staged corners per axis (8 + the +1 apron)
constexpr int MC_STAGED = MC_S * MC_S * MC_S;


struct McTable {
  uint8_t ntri[256];
  uint8_t edge[256][3 * MC_MAX_TRI];
};

__constant__ McTable c_mc;

// ------------------------------------------------------ case table (host)
// Corner of a face walk: face (axis a, side s), step (pu, pw) on the two
// other axes u = a+1, w = a+2 (mod 3), so that e_u x e_w = e_a.
int walk_corner(int a, int s, int pu, int pw) {
  const int u = (a + 1) % 3, w = (a + 2) % 3;
  return (s << a) | (pu << u) | (pw << w);
}

// Id of the edge joining two corners that differ in exactly one bit.
int edge_of(int c1, int c2) {
  const int diff = c1 ^ c2;
  const int a = diff == 1 ? 0 : (diff == 2 ? 1 : 2);
  const int lo = c1 & c2;
  const int x = lo & 1, y = (lo >> 1) & 1, z = (lo >> 2) & 1;
  if (a == 0) return 0 + y + 2 * z;
  if (a == 1) return 4 + x + 2 * z;
  return 8 + x + 2 * y;
}

bool build_case(int cas, uint8_t* ntri, uint8_t* edges) {
  int next[12];
  for (int e = 0; e < 12; ++e) next[e] = -1;
  // Counter-clockwise walks about the outward normal: (0,0) (1,0) (1,1) (0,1)
  // in (u, w) on the + side of an axis, the reverse turn on the - side.
  static const int plus_u[4] = {0, 1, 1, 0}, plus_w[4] = {0, 0, 1, 1};
  for (int a = 0; a < 3; ++a) {
    for (int s = 0; s < 2; ++s) {
      int ring[4];
      for (int k = 0; k < 4; ++k) {
        const int kk = s ? k : (4 - k) % 4;  // reversed order, same start
        ring[k] = walk_corner(a, s, plus_u[kk], plus_w[kk]);
      }
      bool neg[4];
      int first_pos = -1;
      for (int k = 0; k < 4; ++k) {
        neg[k] = (cas >> ring[k]) & 1;
        if (!neg[k] && first_pos < 0) first_pos = k;
      }
      if (first_pos < 0) continue;  // the whole face is negative
      int enter = -1;
      for (int k = 1; k <= 4; ++k) {
        const int p0 = (first_pos + k - 1) & 3, p1 = (first_pos + k) & 3;
        if (!neg[p0] && neg[p1]) enter = edge_of(ring[p0], ring[p1]);
        if (neg[p0] && !neg[p1]) {
          const int leave = edge_of(ring[p0], ring[p1]);
          if (enter < 0 || next[enter] >= 0) return false;
          next[enter] = leave;
          enter = -1;
        }
      }
    }
  }
  int n = 0;
  bool used[12] = {};
  for (int e0 = 0; e0 < 12; ++e0) {
    if (next[e0] < 0 || used[e0]) continue;
    int cyc[12], len = 0;
    int e = e0;
    do {
      if (len >= 12 || used[e] || next[e] < 0) return false;
      used[e] = true;
      cyc[len++] = e;
      e = next[e];
    } while (e != e0);
    for (int k = 1; k + 1 < len; ++k) {
      if (n >= MC_MAX_TRI) return false;
      edges[3 * n + 0] = (uint8_t)cyc[0];
      edges[3 * n + 1] = (uint8_t)cyc[k];
      edges[3 * n + 2] = (uint8_t)cyc[k + 1];
      ++n;
    }
  }
  *ntri = (uint8_t)n;
  return true;
}

const McTable* mc_table() {
  static McTable table;
  static bool ok = false;
  static std::once_flag once;
  std::call_once(once, [] {
    ok = true;
    for (int c = 0; c < 256; ++c) ok = ok && build_case(c, &table.ntri[c], table.edge[c]);
  });
  return ok ? &table : nullptr;
}

// --------------------------------------------------------------- kernels
struct MeshArgs {
  const int32_t* active;
  const int32_t* brick_coord;
  const int32_t* brick_nbr;
  const uint32_t* masks;
  const float* D;
  int R;
  float iso;
  float h;
};

struct MeshShared {
  float d[MC_STAGED];
  uint8_t tr[MC_STAGED];
};

// Stage the corners (x, y, z) in [0, 8]^3 of the brick: the brick's own 8^3
// and the +x / +y / +z apron from its neighbours; absent bricks read as not
// trainable.
__device__ __forceinline__ void mesh_stage(const MeshArgs& a, int slot, MeshShared& sh) {
  for (int s = threadIdx.x; s < MC_STAGED; s += MB_THREADS) {
    const int x = s % MC_S, y = (s / MC_S) % MC_S, z = s / (MC_S * MC_S);
    const int dx = x >> 3, dy = y >> 3, dz = z >> 3;
    const int src = (dx | dy | dz) ? __ldg(a.brick_nbr + (int64_t)slot * 27 + (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1))
                                   : slot;
    float d = 0.f;
    uint8_t t = 0;
    if (src >= 0) {
      const int l = (((z & 7) << 3) | (y & 7)) << 3 | (x & 7);
      d = __ldg(a.D + (int64_t)src * 512 + l);
      t = gp_mask_bit(a.masks, src, 1, l) ? 1 : 0;
    }
    sh.d[s] = d;
    sh.tr[s] = t;
  }
}

// Case of this thread's cell (one thread per cell), or -1 when it is not meshed.
__device__ __forceinline__ int mesh_case_thread(const MeshArgs& a, const MeshShared& sh, int bx, int by, int bz) {
  const int x = threadIdx.x & 7, y = (threadIdx.x >> 3) & 7, z = threadIdx.x >> 6;
  if (bx * 8 + x >= a.R || by * 8 + y >= a.R || bz * 8 + z >= a.R) return -1;
  int cas = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int s = (z + (c >> 2)) * (MC_S * MC_S) + (y + ((c >> 1) & 1)) * MC_S + (x + (c & 1));
    if (!sh.tr[s]) return -1;
    cas |= (sh.d[s] < a.iso ? 1 : 0) << c;
  }
  return cas;
}

// Small bands: one 512-thread block per active brick, one cell per thread.
__global__ void __launch_bounds__(MB_THREADS) k_mesh_count(MeshArgs a, int32_t* __restrict__ counts) {
  __shared__ MeshShared sh;
  __shared__ int wsum[MB_THREADS / 32];
  const int slot = __ldg(a.active + blockIdx.x);
  mesh_stage(a, slot, sh);
  __syncthreads();
  const int cas = mesh_case_thread(a, sh, __ldg(a.brick_coord + 3 * slot), __ldg(a.brick_coord + 3 * slot + 1),
                            __ldg(a.brick_coord + 3 * slot + 2));
  int n = cas >= 0 ? c_mc.ntri[cas] : 0;
  n = gp_warp_sum_i(n);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = n;
  __syncthreads();
  if (threadIdx.x < 32) {
    int v = threadIdx.x < MB_THREADS / 32 ? wsum[threadIdx.x] : 0;
    v = gp_warp_sum_i(v);
    if (threadIdx.x == 0) counts[blockIdx.x] = v;
  }
}

__global__ void __launch_bounds__(MB_THREADS) k_mesh_emit(MeshArgs a, const int32_t* __restrict__ offsets,
                                                          float* __restrict__ tri, int64_t* __restrict__ tri_cell) {
  __shared__ MeshShared sh;
  const int slot = __ldg(a.active + blockIdx.x);
  const int bx = __ldg(a.brick_coord + 3 * slot), by = __ldg(a.brick_coord + 3 * slot + 1),
            bz = __ldg(a.brick_coord + 3 * slot + 2);
  mesh_stage(a, slot, sh);
  __syncthreads();
  const int cas = mesh_case_thread(a, sh, bx, by, bz);
  const int n = cas >= 0 ? c_mc.ntri[cas] : 0;
  int local;
  block_exclusive_scan(n, &local);
  if (n == 0) return;
  const int x = threadIdx.x & 7, y = (threadIdx.x >> 3) & 7, z = threadIdx.x >> 6;
  const int gi = bx * 8 + x, gj = by * 8 + y, gk = bz * 8 + z;
  const int64_t first = (int64_t)__ldg(offsets + blockIdx.x) + local;
  const int64_t key = gi + (int64_t)a.R * (gj + (int64_t)a.R * gk);
  for (int k = 0; k < n; ++k) {
    float* out = tri + (first + k) * 9;
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      const int e = c_mc.edge[cas][3 * k + v];
      const int axis = e >> 2, r = e & 3;
      // lower corner of the edge: the edge's own axis at 0, (p, q) on the others
      const int lo = axis == 0 ? ((r & 1) << 1) | ((r >> 1) << 2)
                               : (axis == 1 ? (r & 1) | ((r >> 1) << 2) : (r & 1) | ((r >> 1) << 1));
      const int hi = lo | (1 << axis);
      const int slo = (z + (lo >> 2)) * (MC_S * MC_S) + (y + ((lo >> 1) & 1)) * MC_S + (x + (lo & 1));
      const int shi = (z + (hi >> 2)) * (MC_S * MC_S) + (y + ((hi >> 1) & 1)) * MC_S + (x + (hi & 1));
      const float dlo = sh.d[slo], dhi = sh.d[shi];
      const float t = __fdiv_rn(__fsub_rn(a.iso, dlo), __fsub_rn(dhi, dlo));
      // -1 + h * (integer corner) is exact in float32 for R <= 2048
      float px = __fadd_rn(-1.0f, __fmul_rn(a.h, (float)(gi + (lo & 1))));
      float py = __fadd_rn(-1.0f, __fmul_rn(a.h, (float)(gj + ((lo >> 1) & 1))));
      float pz = __fadd_rn(-1.0f, __fmul_rn(a.h, (float)(gk + (lo >> 2))));
      const float step = __fmul_rn(a.h, t);
      if (axis == 0) px = __fadd_rn(px, step);
      else if (axis == 1) py = __fadd_rn(py, step);
      else pz = __fadd_rn(pz, step);
      out[3 * v + 0] = px;
      out[3 * v + 1] = py;
      out[3 * v + 2] = pz;
    }
    if (tri_cell) tri_cell[first + k] = key;
  }
}

struct MeshStage {
  float d[MC_STAGED];
  uint8_t tr[MC_STAGED];
};

// Stage, by one warp, the corners (x, y, z) in [0, 8]^3 of a brick: its own
// 8^3 and the +x / +y / +z apron.  The 8 bricks involved (the brick and its
// +x, +y, +z, ... neighbours) are looked up once by lanes 0-7 and shuffled,
// so every lane's 23 value loads are independent of one another.  Absent
// bricks read as not trainable.
__device__ __forceinline__ void mesh_stage_warp(const MeshArgs& a, int slot, MeshStage& sh, int lane) {
  int nbr = -1;
  if (lane < 8) {
    const int dx = lane & 1, dy = (lane >> 1) & 1, dz = lane >> 2;
    nbr = lane == 0 ? slot : __ldg(a.brick_nbr + (int64_t)slot * 27 + (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1));
  }
#pragma unroll 4
  for (int it = 0; it < (MC_STAGED + 31) / 32; ++it) {
    const int s = lane + 32 * it;
    const int sc = s < MC_STAGED ? s : MC_STAGED - 1;
    const int x = sc % MC_S, y = (sc / MC_S) % MC_S, z = sc / (MC_S * MC_S);
    const int src = __shfl_sync(0xffffffffu, nbr, (x >> 3) | ((y >> 3) << 1) | ((z >> 3) << 2));
    if (s < MC_STAGED) {
      float d = 0.f;
      uint8_t t = 0;
      if (src >= 0) {
        const int l = (((z & 7) << 3) | (y & 7)) << 3 | (x & 7);
        d = __ldg(a.D + (int64_t)src * 512 + l);
        t = gp_mask_bit(a.masks, src, 1, l) ? 1 : 0;
      }
      sh.d[s] = d;
      sh.tr[s] = t;
    }
  }
  __syncwarp();
}

// Case of cell c (x-fastest index in the brick), or -1 when it is not meshed.
__device__ __forceinline__ int mesh_case(const MeshArgs& a, const MeshStage& sh, int c, int bx, int by, int bz) {
  const int x = c & 7, y = (c >> 3) & 7, z = c >> 6;
  if (bx * 8 + x >= a.R || by * 8 + y >= a.R || bz * 8 + z >= a.R) return -1;
  int cas = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int s = (z + (k >> 2)) * (MC_S * MC_S) + (y + ((k >> 1) & 1)) * MC_S + (x + (k & 1));
    if (!sh.tr[s]) return -1;
    cas |= (sh.d[s] < a.iso ? 1 : 0) << k;
  }
  return cas;
}

// Large bands: one warp per active brick, MC_WARPS bricks per block; lane L
// owns the MC_CELLS consecutive cells [MC_CELLS L, MC_CELLS (L + 1)).
__global__ void __launch_bounds__(MC_BLOCK) k_mesh_count_w(MeshArgs a, int64_t n_active, int32_t* __restrict__ counts) {
  __shared__ MeshStage st[MC_WARPS];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t b = (int64_t)blockIdx.x * MC_WARPS + w;
  if (b >= n_active) return;  // the whole warp; no block barrier follows
  const int slot = __ldg(a.active + b);
  const int bx = __ldg(a.brick_coord + 3 * slot), by = __ldg(a.brick_coord + 3 * slot + 1),
            bz = __ldg(a.brick_coord + 3 * slot + 2);
  MeshStage& sh = st[w];
  mesh_stage_warp(a, slot, sh, lane);
  // Only the total matters here, so the cells go round-robin over the lanes
  // (cell lane + 32 k): a warp's staged reads then spread over the banks.
  int n = 0;
#pragma unroll
  for (int k = 0; k < MC_CELLS; ++k) {
    const int cas = mesh_case(a, sh, lane + 32 * k, bx, by, bz);
    if (cas >= 0) n += c_mc.ntri[cas];
  }
  n = gp_warp_sum_i(n);
  if (lane == 0) counts[b] = n;
}

__global__ void __launch_bounds__(MC_BLOCK) k_mesh_emit_w(MeshArgs a, int64_t n_active,
                                                        const int32_t* __restrict__ offsets, float* __restrict__ tri,
                                                        int64_t* __restrict__ tri_cell) {
  __shared__ MeshStage st[MC_WARPS];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t b = (int64_t)blockIdx.x * MC_WARPS + w;
  if (b >= n_active) return;
  const int slot = __ldg(a.active + b);
  const int bx = __ldg(a.brick_coord + 3 * slot), by = __ldg(a.brick_coord + 3 * slot + 1),
            bz = __ldg(a.brick_coord + 3 * slot + 2);
  MeshStage& sh = st[w];
  mesh_stage_warp(a, slot, sh, lane);
  int n = 0;
#pragma unroll
  for (int k = 0; k < MC_CELLS; ++k) {
    const int cas = mesh_case(a, sh, lane * MC_CELLS + k, bx, by, bz);
    if (cas >= 0) n += c_mc.ntri[cas];
  }
  // exclusive scan of the lanes' counts keeps the x-fastest cell order
  int incl = n;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (n == 0) return;
  int64_t next = (int64_t)__ldg(offsets + b) + (incl - n);
#pragma unroll 1
  for (int k = 0; k < MC_CELLS; ++k) {
    const int c = lane * MC_CELLS + k;
    const int cc = mesh_case(a, sh, c, bx, by, bz);  // recomputed: no per-lane case array
    if (cc < 0) continue;
    const int x = c & 7, y = (c >> 3) & 7, z = c >> 6;
    const int gi = bx * 8 + x, gj = by * 8 + y, gk = bz * 8 + z;
    const int64_t key = gi + (int64_t)a.R * (gj + (int64_t)a.R * gk);
    const int nt = c_mc.ntri[cc];
    for (int j = 0; j < nt; ++j) {
      float* out = tri + (next + j) * 9;
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        const int e = c_mc.edge[cc][3 * j + v];
        const int axis = e >> 2, r = e & 3;
        // lower corner of the edge: the edge's own axis at 0, (p, q) on the others
        const int lo = axis == 0 ? ((r & 1) << 1) | ((r >> 1) << 2)
                                 : (axis == 1 ? (r & 1) | ((r >> 1) << 2) : (r & 1) | ((r >> 1) << 1));
        const int hi = lo | (1 << axis);
        const int slo = (z + (lo >> 2)) * (MC_S * MC_S) + (y + ((lo >> 1) & 1)) * MC_S + (x + (lo & 1));
        const int shi = (z + (hi >> 2)) * (MC_S * MC_S) + (y + ((hi >> 1) & 1)) * MC_S + (x + (hi & 1));
        const float dlo = sh.d[slo], dhi = sh.d[shi];
        const float t = __fdiv_rn(__fsub_rn(a.iso, dlo), __fsub_rn(dhi, dlo));
        // -1 + h * (integer corner) is exact in float32 for R <= 2048
        float px = __fadd_rn(-1.0f, __fmul_rn(a.h, (float)(gi + (lo & 1))));
        float py = __fadd_rn(-1.0f, __fmul_rn(a.h, (float)(gj + ((lo >> 1) & 1))));
        float pz = __fadd_rn(-1.0f, __fmul_rn(a.h, (float)(gk + (lo >> 2))));
        const float step = __fmul_rn(a.h, t);
        if (axis == 0) px = __fadd_rn(px, step);
        else if (axis == 1) py = __fadd_rn(py, step);
        else pz = __fadd_rn(pz, step);
        out[3 * v + 0] = px;
        out[3 * v + 1] = py;
        out[3 * v + 2] = pz;
      }
      if (tri_cell) tri_cell[next + j] = key;
    }
    next += nt;
  }
}

}  // namespace

extern "C" gp_status gp_mesh_case_table(uint8_t* ntri, uint8_t* edges) {
  if (!ntri || !edges) return GP_ERR_ARG;
  const McTable* table = mc_table();
  if (!table) return GP_ERR_STATE;
  for (int c = 0; c < 256; ++c) {
    ntri[c] = table->ntri[c];
    for (int k = 0; k < 3 * MC_MAX_TRI; ++k) edges[c * 3 * MC_MAX_TRI + k] = k < 3 * table->ntri[c] ? table->edge[c][k] : 255;
  }
  return GP_OK;
}

extern "C" gp_status gp_mesh_extract(gp_band* b, float iso, float* tri_dev, int64_t* cell_dev, int64_t cap,
                                     int64_t* n_tri) {
  if (!b) return GP_ERR_ARG;
  gp_ctx* ctx = b->ctx;
  if (!n_tri) return gp_fail(ctx, GP_ERR_ARG, "gp_mesh_extract: n_tri is null");
  *n_tri = 0;
  if (!std::isfinite(iso)) return gp_fail(ctx, GP_ERR_ARG, "gp_mesh_extract: iso must be finite");
  if (cap < 0) return gp_fail(ctx, GP_ERR_ARG, "gp_mesh_extract: cap must be >= 0");
  if (cap > 0 && !tri_dev) return gp_fail(ctx, GP_ERR_ARG, "gp_mesh_extract: tri_dev is null");
  if (b->n_active == 0) return GP_OK;
  const McTable* table = mc_table();
  if (!table) return gp_fail(ctx, GP_ERR_STATE, "gp_mesh_extract: case table failed its own checks");
  GP_CUDA(ctx, cudaMemcpyToSymbolAsync(c_mc, table, sizeof(McTable), 0, cudaMemcpyHostToDevice, ctx->stream));

  MeshArgs a;
  a.active = b->active;
  a.brick_coord = b->brick_coord;
  a.brick_nbr = b->brick_nbr;
  a.masks = b->masks;
  a.D = b->D;
  a.R = b->R;
  a.iso = iso;
  a.h = 2.0f / (float)b->R;

  const int64_t nb = b->n_active;
  if (nb > 0x7fffffff) return gp_fail(ctx, GP_ERR_ARG, "gp_mesh_extract: too many active bricks");
  int32_t* counts = nullptr;
  gp_status st = gp_alloc(ctx, &counts, (size_t)nb, "mesh counts");
  if (st) return st;
  int64_t total = 0;
  do {
    gp_prof_pre(ctx);
    const bool warp_form = nb >= (int64_t)MC_WARP_MIN_BRICKS_PER_SM * ctx->num_sms;
    const unsigned grid = (unsigned)((nb + MC_WARPS - 1) / MC_WARPS);
    if (warp_form) {
      k_mesh_count_w<<<grid, MC_BLOCK, 0, ctx->stream>>>(a, nb, counts);
      gp_prof_post(ctx, "k_mesh_count_w");
    } else {
      k_mesh_count<<<(unsigned)nb, MB_THREADS, 0, ctx->stream>>>(a, counts);
      gp_prof_post(ctx, "k_mesh_count");
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { st = gp_cuda_fail(ctx, e, "k_mesh_count"); break; }
    // Each brick holds at most 512 * 5 triangles, so the int32 offsets are
    // exact while the total stays below 2^31.
    if ((st = gp_exclusive_scan_i32(ctx, counts, nb, &total))) break;
    if (total > 0x7fffffffLL) { st = gp_fail(ctx, GP_ERR_ARG, "gp_mesh_extract: more than 2^31 - 1 triangles"); break; }
    *n_tri = total;
    if (total == 0 || total > cap) break;
    gp_prof_pre(ctx);
    if (warp_form) {
      k_mesh_emit_w<<<grid, MC_BLOCK, 0, ctx->stream>>>(a, nb, counts, tri_dev, cell_dev);
      gp_prof_post(ctx, "k_mesh_emit_w");
    } else {
      k_mesh_emit<<<(unsigned)nb, MB_THREADS, 0, ctx->stream>>>(a, counts, tri_dev, cell_dev);
      gp_prof_post(ctx, "k_mesh_emit");
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) { st = gp_cuda_fail(ctx, e, "k_mesh_emit"); break; }
    // counts is freed below: wait until the emit pass has read it.
    e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) st = gp_cuda_fail(ctx, e, "gp_mesh_extract");
  } while (false);
  gp_free(counts);
  return st;
}
