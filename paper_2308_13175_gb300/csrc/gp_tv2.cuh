// L_TV (Eq. 5) and its gradient in two passes over the bricks, for gp_step:
//   pass 1: inv_i = 1 / TV_i for i in T (0 elsewhere, and where TV_i = 0),
//           TV_i = sqrt(sum over in-grid axis neighbours n of (d_i - d_n)^2),
//           written to a per-slot array; the block sums of TV_i;
//   pass 2: dTV/dd_j = sum over in-grid axis neighbours n of
//           (d_j - d_n) (inv_j + inv_n), which is the gathered form
//           [j in T] sum_n (d_j - d_n)/TV_j + sum_{n in T} (d_j - d_n)/TV_n.
// Each pass needs a brick's values (and, in pass 2, its inverses) and the
// face of each of its 6 axis-neighbour bricks that touches it: a radius-1
// stencil, with no halo ring to recompute (the single-sweep form stages a
// 12^3 halo from 27 bricks and computes 1/TV on the 10^3 inner region).
// One block of 64 threads per brick at a time, thread (x, y) walking its
// column z = 0..7.
#pragma once

#include "gp_step_device.cuh"

constexpr int TV2_THREADS = 64;
// Face order: -x, +x, -y, +y, -z, +z; their rows of the 27-neighbour table
// ((dx + 1) + 3 (dy + 1) + 9 (dz + 1)).
__device__ __forceinline__ int tv2_face_nbr(int f) {
  return f == 0 ? 12 : f == 1 ? 14 : f == 2 ? 10 : f == 3 ? 16 : f == 4 ? 4 : 22;
}
// In-brick slot of the face value thread t holds for face f: the layer of
// the neighbour brick that touches this one (x = 7 of the -x brick, ...).
// Face arrays are indexed (z, y) for the x faces, (z, x) for the y faces,
// (y, x) for the z faces, 8 x 8 each: index t = 8 * first + second.
__device__ __forceinline__ int tv2_face_local(int f, int t) {
  const int a = t >> 3, b = t & 7;
  switch (f) {
    case 0: return (a * 8 + b) * 8 + 7;  // (z, y) of the -x brick at x = 7
    case 1: return (a * 8 + b) * 8 + 0;
    case 2: return (a * 8 + 7) * 8 + b;  // (z, x) of the -y brick at y = 7
    case 3: return (a * 8 + 0) * 8 + b;
    case 4: return (7 * 8 + a) * 8 + b;  // (y, x) of the -z brick at z = 7
    default: return (0 * 8 + a) * 8 + b;
  }
}

// A staged brick: its 512 values and the 6 faces (0 where a neighbour brick
// is absent: only frozen vertices, outside T, can sit next to one).
struct __align__(16) Tv2Stage {
  float c[512];
  float f[6][64];
};

// The slots a brick's copies read: its own and its 6 face neighbours' (-1
// absent), and its origin vertex.
struct Tv2Brick {
  int64_t slot;
  int nb[6];
  int ox, oy, oz;
};
__device__ __forceinline__ Tv2Brick tv2_brick(const int32_t* __restrict__ coord, const int32_t* __restrict__ nbrs,
                                             int64_t b) {
  Tv2Brick k;
  k.slot = b;
#pragma unroll
  for (int f = 0; f < 6; ++f) k.nb[f] = __ldg(nbrs + 27 * b + tv2_face_nbr(f));
  k.ox = __ldg(coord + 3 * b) * 8;
  k.oy = __ldg(coord + 3 * b + 1) * 8;
  k.oz = __ldg(coord + 3 * b + 2) * 8;
  return k;
}

__device__ __forceinline__ void tv2_cp4(void* smem, const void* gmem, int src_bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gmem), "r"(src_bytes) : "memory");
}

// This thread's asynchronous copies of brick k of array src into s (64
// threads): two 16-byte pieces of the centre; one 16-byte piece of a z face
// (threads 0-31) or of a y face (threads 32-63); one value of each x face.
// An absent neighbour's pieces are zero-filled (no bytes read).
__device__ __forceinline__ void tv2_issue(Tv2Stage& s, const float* __restrict__ src, const Tv2Brick& k) {
  const int t = threadIdx.x;
  const float* c = src + k.slot * 512;
  cp_async_cg16(&s.c[4 * t], c + 4 * t, 16);
  cp_async_cg16(&s.c[4 * (t + 64)], c + 4 * (t + 64), 16);
  {
    // z faces (t < 32): plane z = 7 of the -z brick, z = 0 of the +z brick,
    // face index 8 y + x; y faces: row y = 7 (0) at each z, index 8 z + x.
    const int f = t < 16 ? 4 : t < 32 ? 5 : t < 48 ? 2 : 3;
    const int piece = t & 15;  // 16 pieces of 4 floats per face
    const int ns = f == 2 ? k.nb[2] : f == 3 ? k.nb[3] : f == 4 ? k.nb[4] : k.nb[5];  // no indexed registers
    int local;
    if (f >= 4)
      local = (f == 4 ? 7 * 64 : 0) + 4 * piece;
    else
      local = (piece >> 1) * 64 + (f == 2 ? 56 : 0) + 4 * (piece & 1);
    const float* g = ns >= 0 ? src + (int64_t)ns * 512 + local : src;
    cp_async_cg16(&s.f[f][4 * piece], g, ns >= 0 ? 16 : 0);
  }
#pragma unroll
  for (int f = 0; f < 2; ++f) {
    const int ns = k.nb[f];
    const float* g = ns >= 0 ? src + (int64_t)ns * 512 + tv2_face_local(f, t) : src;
    tv2_cp4(&s.f[f][t], g, ns >= 0 ? 4 : 0);
  }
}

// The 6 axis neighbours of (x, y, z) in the staged brick (-x, +x, -y, +y, -z, +z).
__device__ __forceinline__ void tv2_nbrs(const Tv2Stage& s, int x, int y, int z, float n[6]) {
  const int l = (z * 8 + y) * 8 + x;
  n[0] = x > 0 ? s.c[l - 1] : s.f[0][z * 8 + y];
  n[1] = x < 7 ? s.c[l + 1] : s.f[1][z * 8 + y];
  n[2] = y > 0 ? s.c[l - 8] : s.f[2][z * 8 + x];
  n[3] = y < 7 ? s.c[l + 8] : s.f[3][z * 8 + x];
  n[4] = z > 0 ? s.c[l - 64] : s.f[4][y * 8 + x];
  n[5] = z < 7 ? s.c[l + 64] : s.f[5][y * 8 + x];
}

// Which of the 6 neighbours of vertex (X, Y, Z) lie inside [0, R]^3.
__device__ __forceinline__ void tv2_ingrid(int X, int Y, int Z, int R, bool ok[6]) {
  ok[0] = X > 0;
  ok[1] = X < R;
  ok[2] = Y > 0;
  ok[3] = Y < R;
  ok[4] = Z > 0;
  ok[5] = Z < R;
}
