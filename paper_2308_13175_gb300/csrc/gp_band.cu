// gp_build_band: the uniform grid's near-surface band (Sec. 3 "Discrete
// Grids", the M1 pull bandwidth and the M2 TV bandwidth) stored as 8^3-vertex
// bricks, plus the band queries (info, init, export, values).
#include <algorithm>
#include <vector>

#include "gp_internal.cuh"

gp_status gp_build_points(gp_band* band, const float* pts_dev);  // gp_nn.cu

namespace {

// Cell map bits.
constexpr uint8_t C_OCC = 1, C_M1 = 2, C_M2 = 4, C_MX = 8;
// Vertex map bits (match the export flags).
constexpr uint8_t V_T = 1, V_TRAIN = 2, V_PULL = 8;

__global__ void k_mark_occupied(const float* __restrict__ pts, int64_t J, int R, uint8_t* __restrict__ cells) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= J) return;
  float half_r = 0.5f * (float)R;
  int c[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    gp_cell1 g = gp_cell_exact(pts[3 * j + a], half_r);
    c[a] = min(max(g.c, 0), R - 1);
  }
  cells[((int64_t)c[2] * R + c[1]) * R + c[0]] = C_OCC;
}

// One axis of the separable Chebyshev dilation.  Pass 0 dilates the occupied
// bit into the three band bits; later passes dilate each band bit by its own
// radius.  Bit C_OCC is carried through.
__global__ void k_dilate_axis(const uint8_t* __restrict__ in, uint8_t* __restrict__ out, int R, int axis,
                              int M1, int M2, int MX, int first) {
  int64_t n = (int64_t)R * R * R;
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  int x = (int)(idx % R), y = (int)((idx / R) % R), z = (int)(idx / ((int64_t)R * R));
  int pos = axis == 0 ? x : (axis == 1 ? y : z);
  int64_t stride = axis == 0 ? 1 : (axis == 1 ? R : (int64_t)R * R);
  int mm = max(M1, max(M2, MX));
  uint8_t acc = in[idx] & C_OCC;
  for (int d = -mm; d <= mm; ++d) {
    int p = pos + d;
    if (p < 0 || p >= R) continue;
    uint8_t v = in[idx + d * stride];
    int ad = d < 0 ? -d : d;
    uint8_t s1 = first ? (v & C_OCC) : (v & C_M1);
    uint8_t s2 = first ? (v & C_OCC) : (v & C_M2);
    uint8_t s3 = first ? (v & C_OCC) : (v & C_MX);
    if (s1 && ad <= M1) acc |= C_M1;
    if (s2 && ad <= M2) acc |= C_M2;
    if (s3 && ad <= MX) acc |= C_MX;
  }
  out[idx] = acc;
}

__global__ void k_set_all_bits(uint8_t* __restrict__ cells, int64_t n, uint8_t bits) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < n) cells[idx] |= bits;
}

__global__ void k_count_cells(const uint8_t* __restrict__ cells, int64_t n, unsigned long long* counts) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint8_t v = idx < n ? cells[idx] : 0;
  int occ = __syncthreads_count(v & C_OCC);
  int pull = __syncthreads_count(v & C_M1);
  if (threadIdx.x == 0) {
    if (occ) atomicAdd(counts + 0, (unsigned long long)occ);
    if (pull) atomicAdd(counts + 1, (unsigned long long)pull);
  }
}

// Vertex flags: T = corner of an M2 cell, trainable = corner of an MX cell,
// pull = lowest corner of an M1 cell.
__global__ void k_vertex_flags(const uint8_t* __restrict__ cells, uint8_t* __restrict__ verts, int R) {
  int n1 = R + 1;
  int64_t nv = (int64_t)n1 * n1 * n1;
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nv) return;
  int i = (int)(idx % n1), j = (int)((idx / n1) % n1), k = (int)(idx / ((int64_t)n1 * n1));
  uint8_t any = 0;
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        int ci = i - dx, cj = j - dy, ck = k - dz;
        if (ci < 0 || cj < 0 || ck < 0 || ci >= R || cj >= R || ck >= R) continue;
        any |= cells[((int64_t)ck * R + cj) * R + ci];
      }
  uint8_t f = 0;
  if (any & C_M2) f |= V_T;
  if (any & C_MX) f |= V_TRAIN;
  if (i < R && j < R && k < R && (cells[((int64_t)k * R + j) * R + i] & C_M1)) f |= V_PULL;
  verts[idx] = f;
}

// Required vertices (T, trainable and the axis neighbours of T) mark their brick.
__global__ void k_required(uint8_t* __restrict__ verts, int R, int nb, uint8_t* __restrict__ need) {
  int n1 = R + 1;
  int64_t nv = (int64_t)n1 * n1 * n1;
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nv) return;
  int i = (int)(idx % n1), j = (int)((idx / n1) % n1), k = (int)(idx / ((int64_t)n1 * n1));
  uint8_t f = verts[idx];
  bool req = (f & (V_T | V_TRAIN)) != 0;
  if (!req) {
    const int di[6] = {-1, 1, 0, 0, 0, 0}, dj[6] = {0, 0, -1, 1, 0, 0}, dk[6] = {0, 0, 0, 0, -1, 1};
    for (int t = 0; t < 6 && !req; ++t) {
      int a = i + di[t], b = j + dj[t], c = k + dk[t];
      if (a < 0 || b < 0 || c < 0 || a > R || b > R || c > R) continue;
      if (verts[((int64_t)c * n1 + b) * n1 + a] & V_T) req = true;
    }
  }
  if (req) need[((int64_t)(k >> 3) * nb + (j >> 3)) * nb + (i >> 3)] = 1;
}

__device__ __forceinline__ uint32_t compact3(uint32_t x) {  // every third bit -> contiguous
  x &= 0x09249249u;
  x = (x ^ (x >> 2)) & 0x030C30C3u;
  x = (x ^ (x >> 4)) & 0x0300F00Fu;
  x = (x ^ (x >> 8)) & 0x030000FFu;
  x = (x ^ (x >> 16)) & 0x000003FFu;
  return x;
}

// Morton-ordered flags of the needed bricks.
__global__ void k_morton_flags(const uint8_t* __restrict__ need, int nb, int64_t nm, int32_t* __restrict__ flags) {
  int64_t mi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (mi >= nm) return;
  uint32_t bx = compact3((uint32_t)mi), by = compact3((uint32_t)(mi >> 1)), bz = compact3((uint32_t)(mi >> 2));
  int32_t f = 0;
  if (bx < (uint32_t)nb && by < (uint32_t)nb && bz < (uint32_t)nb)
    f = need[((int64_t)bz * nb + by) * nb + bx];
  flags[mi] = f;
}

__global__ void k_assign_slots(const uint8_t* __restrict__ need, const int32_t* __restrict__ offs, int nb,
                               int64_t nm, int32_t* __restrict__ table, int32_t* __restrict__ coord) {
  int64_t mi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (mi >= nm) return;
  uint32_t bx = compact3((uint32_t)mi), by = compact3((uint32_t)(mi >> 1)), bz = compact3((uint32_t)(mi >> 2));
  if (bx >= (uint32_t)nb || by >= (uint32_t)nb || bz >= (uint32_t)nb) return;
  int64_t b = ((int64_t)bz * nb + by) * nb + bx;
  if (!need[b]) return;
  int32_t slot = offs[mi];
  table[b] = slot;
  coord[3 * slot + 0] = bx;
  coord[3 * slot + 1] = by;
  coord[3 * slot + 2] = bz;
}

// Slots of the 27 bricks around each brick (itself included), x fastest.
__global__ void k_brick_nbr(const int32_t* __restrict__ table, const int32_t* __restrict__ coord, int nb,
                            int64_t n_bricks, int32_t* __restrict__ nbr) {
  int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n_bricks * 27) return;
  int64_t slot = a / 27;
  int t = (int)(a - slot * 27);
  int bx = coord[3 * slot] + t % 3 - 1, by = coord[3 * slot + 1] + (t / 3) % 3 - 1, bz = coord[3 * slot + 2] + t / 9 - 1;
  int32_t v = -1;
  if ((unsigned)bx < (unsigned)nb && (unsigned)by < (unsigned)nb && (unsigned)bz < (unsigned)nb)
    v = table[((int64_t)bz * nb + by) * nb + bx];
  nbr[a] = v;
}

// One block of 512 threads per brick: masks by warp ballots, counts, active flag.
__global__ void k_brick_masks(const uint8_t* __restrict__ verts, int R, const int32_t* __restrict__ coord,
                              uint32_t* __restrict__ masks, int32_t* __restrict__ active_flag,
                              unsigned long long* counts) {
  int slot = blockIdx.x;
  int l = threadIdx.x;
  int i = coord[3 * slot] * 8 + (l & 7);
  int j = coord[3 * slot + 1] * 8 + ((l >> 3) & 7);
  int k = coord[3 * slot + 2] * 8 + (l >> 6);
  int n1 = R + 1;
  uint8_t f = 0;
  if (i <= R && j <= R && k <= R) f = verts[((int64_t)k * n1 + j) * n1 + i];
  uint32_t bt = __ballot_sync(0xffffffffu, f & V_T);
  uint32_t br = __ballot_sync(0xffffffffu, f & V_TRAIN);
  uint32_t bp = __ballot_sync(0xffffffffu, f & V_PULL);
  int w = l >> 5;
  if ((l & 31) == 0) {
    uint32_t* mk = masks + (int64_t)slot * 48;
    mk[w] = bt;
    mk[16 + w] = br;
    mk[32 + w] = bp;
    if (bt) atomicAdd(counts + 2, (unsigned long long)__popc(bt));
    if (br) atomicAdd(counts + 3, (unsigned long long)__popc(br));
  }
  int any = __syncthreads_or(f & V_TRAIN);
  if (l == 0) active_flag[slot] = any ? 1 : 0;
}

__global__ void k_compact_active(const int32_t* __restrict__ flags, const int32_t* __restrict__ offs, int64_t n,
                                 int32_t* __restrict__ out) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n && flags[s]) out[offs[s]] = (int32_t)s;
}

__global__ void k_init_sphere(float* __restrict__ D, const int32_t* __restrict__ coord, int64_t nslots, int R,
                              float cx, float cy, float cz, float radius, float noise, uint32_t k0, uint32_t k1) {
  int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nslots) return;
  int slot = (int)(a >> 9), l = (int)(a & 511);
  int i = coord[3 * slot] * 8 + (l & 7);
  int j = coord[3 * slot + 1] * 8 + ((l >> 3) & 7);
  int k = coord[3 * slot + 2] * 8 + (l >> 6);
  if (i > R || j > R || k > R) {
    D[a] = 0.f;
    return;
  }
  float h = 2.0f / (float)R;
  float x = -1.0f + h * (float)i - cx, y = -1.0f + h * (float)j - cy, z = -1.0f + h * (float)k - cz;
  float d = sqrtf(x * x + y * y + z * z) - radius;
  if (noise != 0.f) {
    uint64_t key = (uint64_t)i + (uint64_t)(R + 1) * ((uint64_t)j + (uint64_t)(R + 1) * (uint64_t)k);
    float3 zz = gp_box_muller3(gp_philox((uint32_t)key, (uint32_t)(key >> 32), 0u, 2u, k0, k1));
    d += noise * zz.x;
  }
  D[a] = d;
}

__global__ void k_export(const int32_t* __restrict__ coord, const uint32_t* __restrict__ masks, const float* __restrict__ D,
                         int64_t nslots, int R, int32_t* __restrict__ ijk, float* __restrict__ dout,
                         uint8_t* __restrict__ flags) {
  int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nslots) return;
  int slot = (int)(a >> 9), l = (int)(a & 511);
  int i = coord[3 * slot] * 8 + (l & 7);
  int j = coord[3 * slot + 1] * 8 + ((l >> 3) & 7);
  int k = coord[3 * slot + 2] * 8 + (l >> 6);
  if (ijk) {
    ijk[3 * a] = i;
    ijk[3 * a + 1] = j;
    ijk[3 * a + 2] = k;
  }
  if (dout) dout[a] = D[a];
  if (flags) {
    uint8_t f = 0;
    if (gp_mask_bit(masks, slot, 0, l)) f |= 1;
    if (gp_mask_bit(masks, slot, 1, l)) f |= 2;
    if (i <= R && j <= R && k <= R) f |= 4;
    if (gp_mask_bit(masks, slot, 2, l)) f |= 8;
    flags[a] = f;
  }
}

void band_free(gp_band* b) {
  if (!b) return;
  gp_free(b->brick_table);
  gp_free(b->brick_coord);
  gp_free(b->brick_nbr);
  gp_free(b->masks);
  gp_free(b->active);
  gp_free(b->D);
  gp_free(b->m);
  gp_free(b->v);
  gp_free(b->acc);
  gp_free(b->D_alt);
  gp_free(b->qgrad);
  gp_free(b->tv_inv);
  gp_free(b->pts);
  gp_free(b->pts_sorted);
  gp_free(b->cell_start);
  gp_free(b->sigma);
  gp_free(b->normals);
  gp_free(b->perm);
  gp_free(b->inv_perm);
  gp_free(b->order_tiles);
  gp_free(b->emit_order);
  gp_free(b->emit_slot);
  gp_free(b->emit_pts);
  gp_free(b->partials);
  gp_free(b->dev_ints);
  delete b;
}

struct TempBufs {
  std::vector<void*> ptrs;
  ~TempBufs() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <typename T>
  gp_status alloc(gp_ctx* ctx, T** p, size_t n, const char* what) {
    gp_status st = gp_alloc(ctx, p, n, what);
    if (!st) ptrs.push_back(*p);
    return st;
  }
};

gp_status build_band_sets(gp_band* b, const float* pts_dev) {
  gp_ctx* ctx = b->ctx;
  cudaStream_t s = ctx->stream;
  const int R = b->R;
  const int64_t ncell = (int64_t)R * R * R;
  const int64_t nvert = (int64_t)(R + 1) * (R + 1) * (R + 1);
  const int nb = b->nb;
  const int64_t nbr = (int64_t)nb * nb * nb;
  TempBufs tmp;
  uint8_t *cA = nullptr, *cB = nullptr, *verts = nullptr, *need = nullptr;
  unsigned long long* counts = nullptr;
  gp_status st;
  if ((st = tmp.alloc(ctx, &cA, ncell, "cell map"))) return st;
  if ((st = tmp.alloc(ctx, &cB, ncell, "cell map"))) return st;
  if ((st = tmp.alloc(ctx, &counts, 8, "band counts"))) return st;
  GP_CUDA(ctx, cudaMemsetAsync(cA, 0, ncell, s));
  GP_CUDA(ctx, cudaMemsetAsync(counts, 0, 8 * sizeof(unsigned long long), s));
  GP_KERNEL(ctx, "k_mark_occupied", k_mark_occupied<<<gp_blocks(b->J, 256), 256, 0, s>>>(pts_dev, b->J, R, cA));

  // Negative widths mean "every cell": dilate by 0 and set the bit afterwards.
  int m1 = b->M1 < 0 ? 0 : std::min(b->M1, R);
  int m2 = b->M2 < 0 ? 0 : std::min(b->M2, R);
  bool all1 = b->M1 < 0, all2 = b->M2 < 0;
  bool allx = all1 || all2;
  int mx = allx ? 0 : std::max(m1, m2);
  uint8_t* in = cA;
  uint8_t* out = cB;
  for (int axis = 0; axis < 3; ++axis) {
    GP_KERNEL(ctx, "k_dilate_axis", k_dilate_axis<<<gp_blocks(ncell, 256), 256, 0, s>>>(in, out, R, axis, m1, m2, mx, axis == 0));
    std::swap(in, out);
  }
  uint8_t all_bits = (all1 ? C_M1 : 0) | (all2 ? C_M2 : 0) | (allx ? C_MX : 0);
  if (all_bits) {
    GP_KERNEL(ctx, "k_set_all_bits", k_set_all_bits<<<gp_blocks(ncell, 256), 256, 0, s>>>(in, ncell, all_bits));
  }
  GP_KERNEL(ctx, "k_count_cells", k_count_cells<<<gp_blocks(ncell, 256), 256, 0, s>>>(in, ncell, counts));

  if ((st = tmp.alloc(ctx, &verts, nvert, "vertex map"))) return st;
  GP_KERNEL(ctx, "k_vertex_flags", k_vertex_flags<<<gp_blocks(nvert, 256), 256, 0, s>>>(in, verts, R));
  if ((st = tmp.alloc(ctx, &need, nbr, "brick flags"))) return st;
  GP_CUDA(ctx, cudaMemsetAsync(need, 0, nbr, s));
  GP_KERNEL(ctx, "k_required", k_required<<<gp_blocks(nvert, 256), 256, 0, s>>>(verts, R, nb, need));

  // Slots in Morton order of the brick coordinates.
  int nbm = 1;
  while (nbm < nb) nbm <<= 1;
  const int64_t nm = (int64_t)nbm * nbm * nbm;
  int32_t* mflags = nullptr;
  if ((st = tmp.alloc(ctx, &mflags, nm, "morton flags"))) return st;
  GP_KERNEL(ctx, "k_morton_flags", k_morton_flags<<<gp_blocks(nm, 256), 256, 0, s>>>(need, nb, nm, mflags));
  int64_t n_bricks = 0;
  if ((st = gp_exclusive_scan_i32(ctx, mflags, nm, &n_bricks))) return st;
  b->n_bricks = n_bricks;
  if ((st = gp_alloc(ctx, &b->brick_table, nbr, "brick table"))) return st;
  GP_CUDA(ctx, cudaMemsetAsync(b->brick_table, 0xFF, nbr * sizeof(int32_t), s));
  if ((st = gp_alloc(ctx, &b->brick_coord, 3 * n_bricks, "brick coords"))) return st;
  GP_KERNEL(ctx, "k_assign_slots", k_assign_slots<<<gp_blocks(nm, 256), 256, 0, s>>>(need, mflags, nb, nm, b->brick_table, b->brick_coord));
  if ((st = gp_alloc(ctx, &b->brick_nbr, 27 * n_bricks, "brick neighbours"))) return st;
  if (n_bricks > 0)
    GP_KERNEL(ctx, "k_brick_nbr", k_brick_nbr<<<gp_blocks(27 * n_bricks, 256), 256, 0, s>>>(b->brick_table, b->brick_coord, nb, n_bricks, b->brick_nbr));

  if ((st = gp_alloc(ctx, &b->masks, 48 * n_bricks, "brick masks"))) return st;
  int32_t *aflag = nullptr, *aoffs = nullptr;
  if ((st = tmp.alloc(ctx, &aflag, n_bricks, "active flags"))) return st;
  if ((st = tmp.alloc(ctx, &aoffs, n_bricks, "active offsets"))) return st;
  if (n_bricks > 0) {
    GP_KERNEL(ctx, "k_brick_masks", k_brick_masks<<<(unsigned)n_bricks, 512, 0, s>>>(verts, R, b->brick_coord, b->masks, aflag, counts));
    GP_CUDA(ctx, cudaMemcpyAsync(aoffs, aflag, n_bricks * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  }
  int64_t n_active = 0;
  if ((st = gp_exclusive_scan_i32(ctx, aoffs, n_bricks, &n_active))) return st;
  b->n_active = n_active;
  if ((st = gp_alloc(ctx, &b->active, n_active, "active list"))) return st;
  if (n_bricks > 0) {
    GP_KERNEL(ctx, "k_compact_active", k_compact_active<<<gp_blocks(n_bricks, 256), 256, 0, s>>>(aflag, aoffs, n_bricks, b->active));
  }
  unsigned long long hc[8];
  GP_CUDA(ctx, cudaMemcpyAsync(hc, counts, sizeof(hc), cudaMemcpyDeviceToHost, s));
  GP_CUDA(ctx, cudaStreamSynchronize(s));
  b->n_occ = (int64_t)hc[0];
  b->n_pull = (int64_t)hc[1];
  b->V_tv = (int64_t)hc[2];
  b->V_trainable = (int64_t)hc[3];
  return GP_OK;
}

}  // namespace

extern "C" gp_status gp_build_band(gp_ctx* ctx, const float* pts_dev, int64_t J, const gp_grid_desc* desc,
                                   gp_band** out) {
  if (!ctx) return GP_ERR_ARG;
  if (!out || !pts_dev || !desc) return gp_fail(ctx, GP_ERR_ARG, "gp_build_band: null argument");
  *out = nullptr;
  int R = desc->R;
  if (R < 8 || R > 2048 || (R & (R - 1)))
    return gp_fail(ctx, GP_ERR_ARG, "gp_build_band: R must be a power of two in [8, 2048]");
  if (J < 1 || J >= (int64_t(1) << 31)) return gp_fail(ctx, GP_ERR_ARG, "gp_build_band: J must be in [1, 2^31)");
  if (desc->knn_k < 0 || desc->knn_k > 64) return gp_fail(ctx, GP_ERR_ARG, "gp_build_band: knn_k must be in [0, 64]");
  if (desc->nn_grid < 0 || desc->nn_grid > 1024)
    return gp_fail(ctx, GP_ERR_ARG, "gp_build_band: nn_grid must be in [0, 1024]");
  GP_CUDA(ctx, cudaSetDevice(ctx->device));
  gp_band* b = new (std::nothrow) gp_band();
  if (!b) return gp_fail(ctx, GP_ERR_OOM, "gp_build_band: host allocation");
  b->ctx = ctx;
  b->R = R;
  b->M1 = desc->M1;
  b->M2 = desc->M2;
  b->nb = R / 8 + 1;
  b->knn_k = desc->knn_k;
  b->flags = desc->flags;
  b->J = J;
  b->G = desc->nn_grid;
  gp_status st = build_band_sets(b, pts_dev);
  int64_t V = b->V_stored();
  if (!st) st = gp_alloc(ctx, &b->D, V, "values");
  if (!st) st = gp_alloc(ctx, &b->m, V, "adam m");
  if (!st) st = gp_alloc(ctx, &b->v, V, "adam v");
  if (!st && (b->flags & GP_BAND_DETERMINISTIC)) st = gp_alloc(ctx, &b->acc, 2 * V, "fixed-point accumulator");
  if (!st) st = gp_alloc(ctx, &b->D_alt, V, "second value buffer");
  if (!st) st = gp_alloc(ctx, &b->qgrad, V, "query gradient");
  if (!st) st = gp_alloc(ctx, &b->tv_inv, V, "1/TV of the two-pass L_TV");
  if (!st) st = gp_alloc(ctx, &b->partials, (size_t)GP_MAX_PARTIAL_BLOCKS * 8, "partials");
  if (!st) st = gp_alloc(ctx, &b->dev_ints, GP_DI_COUNT, "device ints");
  if (!st) {
    cudaStream_t s = ctx->stream;
    cudaError_t e = cudaMemsetAsync(b->D, 0, V * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->m, 0, V * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->v, 0, V * sizeof(float), s);
    if (e == cudaSuccess && b->acc) e = cudaMemsetAsync(b->acc, 0, 2 * V * sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->D_alt, 0, V * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->qgrad, 0, V * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->dev_ints, 0, GP_DI_COUNT * sizeof(int32_t), s);
    if (e != cudaSuccess) st = gp_cuda_fail(ctx, e, "gp_build_band: memset");
  }
  if (!st) st = gp_build_points(b, pts_dev);
  if (!st) {
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) st = gp_cuda_fail(ctx, e, "gp_build_band: synchronise");
  }
  if (st) {
    band_free(b);
    return st;
  }
  ctx->live_bands += 1;
  *out = b;
  return GP_OK;
}

extern "C" void gp_band_destroy(gp_band* band) {
  if (!band) return;
  gp_ctx* ctx = band->ctx;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  cudaGetLastError();
  band_free(band);
  ctx->live_bands -= 1;
  if (ctx->live_bands == 0 && ctx->destroy_pending) gp_ctx_release(ctx);
}

extern "C" gp_status gp_band_get_info(const gp_band* b, gp_band_info* out) {
  if (!b || !out) return GP_ERR_ARG;
  out->R = b->R;
  out->nb = b->nb;
  out->n_bricks = b->n_bricks;
  out->n_active_bricks = b->n_active;
  out->V_stored = b->V_stored();
  out->V_trainable = b->V_trainable;
  out->V_tv = b->V_tv;
  out->n_pull_cells = b->n_pull;
  out->n_occupied_cells = b->n_occ;
  out->J = b->J;
  out->nn_grid = b->G;
  out->knn_k = b->knn_k;
  return GP_OK;
}

extern "C" gp_status gp_band_init_sphere(gp_band* b, float cx, float cy, float cz, float radius, float noise_std,
                                         uint64_t seed) {
  if (!b) return GP_ERR_ARG;
  gp_ctx* ctx = b->ctx;
  int64_t V = b->V_stored();
  if (V == 0) return GP_OK;
  GP_KERNEL(ctx, "k_init_sphere", k_init_sphere<<<gp_blocks(V, 256), 256, 0, ctx->stream>>>(b->D, b->brick_coord, V, b->R, cx, cy, cz, radius,
                                                            noise_std, (uint32_t)seed, (uint32_t)(seed >> 32)));
  return GP_OK;
}

extern "C" gp_status gp_band_set_values(gp_band* b, const float* d_dev) {
  if (!b) return GP_ERR_ARG;
  if (!d_dev) return gp_fail(b->ctx, GP_ERR_ARG, "gp_band_set_values: null values");
  GP_CUDA(b->ctx, cudaMemcpyAsync(b->D, d_dev, b->V_stored() * sizeof(float), cudaMemcpyDeviceToDevice,
                                  b->ctx->stream));
  return GP_OK;
}

extern "C" gp_status gp_band_export(const gp_band* b, int32_t* ijk_dev, float* d_dev, uint8_t* flags_dev) {
  if (!b) return GP_ERR_ARG;
  gp_ctx* ctx = b->ctx;
  int64_t V = b->V_stored();
  if (V == 0 || (!ijk_dev && !d_dev && !flags_dev)) return GP_OK;
  GP_KERNEL(ctx, "k_export", k_export<<<gp_blocks(V, 256), 256, 0, ctx->stream>>>(b->brick_coord, b->masks, b->D, V, b->R, ijk_dev, d_dev,
                                                       flags_dev));
  return GP_OK;
}

extern "C" gp_status gp_band_values(gp_band* b, float** d_dev, float** m_dev, float** v_dev) {
  if (!b) return GP_ERR_ARG;
  if (d_dev) *d_dev = b->D;
  if (m_dev) *m_dev = b->m;
  if (v_dev) *v_dev = b->v;
  return GP_OK;
}

extern "C" gp_status gp_band_reset_adam(gp_band* b) {
  if (!b) return GP_ERR_ARG;
  int64_t V = b->V_stored();
  GP_CUDA(b->ctx, cudaMemsetAsync(b->m, 0, V * sizeof(float), b->ctx->stream));
  GP_CUDA(b->ctx, cudaMemsetAsync(b->v, 0, V * sizeof(float), b->ctx->stream));
  return GP_OK;
}

extern "C" gp_status gp_band_check(gp_band* b) {
  if (!b) return GP_ERR_ARG;
  gp_ctx* ctx = b->ctx;
  int32_t flag = 0;
  GP_CUDA(ctx, cudaMemcpyAsync(&flag, b->dev_ints + GP_DI_ERROR, 4, cudaMemcpyDeviceToHost, ctx->stream));
  GP_CUDA(ctx, cudaMemsetAsync(b->dev_ints + GP_DI_ERROR, 0, 4, ctx->stream));
  GP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (flag & GP_EF_TIMEOUT) return gp_fail(ctx, GP_ERR_TIMEOUT, "a bounded device wait gave up");
  if (flag & (GP_EF_NUMERIC | GP_EF_RANGE))
    return gp_fail(ctx, GP_ERR_NUMERIC, "a device numeric or range check fired");
  return GP_OK;
}
