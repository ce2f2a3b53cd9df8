// Reconstruction metrics against a reference surface: the measures Sec. 4
// "Datasets and Metrics" reports (Chamfer L1 and L2, Hausdorff, normal
// consistency, F-score), for two oriented point sets.
//
// gp_mesh_quadrature turns a triangle soup into weighted oriented points: every
// triangle is split at m equal steps along its edges into m^2 congruent
// triangles, and each contributes its centroid, the triangle's unit normal and
// area / m^2 (the one-point rule on each piece, so a weighted mean over the
// points is a quadrature of the mean over the surface).
//
// gp_eval_nearest takes one direction: for every query point its exact nearest
// point in a band's cloud (gp_nn), the distance d = sqrt(((dx^2 + dy^2) + dz^2))
// in float64 from the float32 coordinates (no contraction), and the weighted
// sums of d, d^2, |n_q . n_nn| and [d < tau_k], and the largest d.  Two calls
// (mesh -> reference, reference -> mesh) give CD_L1, CD_L2, HD, NC and F.
#include <cmath>
#include <cstring>

#include "gp_internal.cuh"

namespace {

constexpr int EV_THREADS = 256;
constexpr int EV_MAX_TAU = 16;
constexpr int EV_SUMS = 4 + EV_MAX_TAU;  // w, w d, w d^2, w |cos|, w [d < tau_k]

struct EvTaus {
  double t[EV_MAX_TAU];
};

__global__ void __launch_bounds__(EV_THREADS) k_mesh_quad(const float* __restrict__ tri, int64_t T, int m,
                                                          float* __restrict__ pts, float* __restrict__ nrm,
                                                          float* __restrict__ w) {
  const int64_t per = (int64_t)m * m;
  const int64_t total = T * per;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = g / per;
    int k = (int)(g - i * per);
    // k-th piece in the order: for i = 0..m-1, j = 0..m-1-i: upright (i, j),
    // then inverted (i, j) when i + j < m - 1.
    int pi = 0, pj = 0;
    bool inverted = false;
    for (int a = 0; a < m; ++a) {
      const int row = 2 * (m - a) - 1;  // pieces with first index a
      if (k < row) {
        pi = a;
        pj = k / 2;
        inverted = (k & 1) != 0;
        break;
      }
      k -= row;
    }
    const float* t = tri + 9 * i;
    const float x0 = t[0], y0 = t[1], z0 = t[2];
    const float e1x = __fsub_rn(t[3], x0), e1y = __fsub_rn(t[4], y0), e1z = __fsub_rn(t[5], z0);
    const float e2x = __fsub_rn(t[6], x0), e2y = __fsub_rn(t[7], y0), e2z = __fsub_rn(t[8], z0);
    const float inv = 1.0f / (3.0f * (float)m);
    const float a = (float)(3 * pi + (inverted ? 2 : 1)) * inv;
    const float b = (float)(3 * pj + (inverted ? 2 : 1)) * inv;
    pts[3 * g + 0] = x0 + a * e1x + b * e2x;
    pts[3 * g + 1] = y0 + a * e1y + b * e2y;
    pts[3 * g + 2] = z0 + a * e1z + b * e2z;
    const float cx = e1y * e2z - e1z * e2y, cy = e1z * e2x - e1x * e2z, cz = e1x * e2y - e1y * e2x;
    const float len = sqrtf(cx * cx + cy * cy + cz * cz);
    const float s = len > 0.f ? 1.0f / len : 0.f;
    nrm[3 * g + 0] = cx * s;
    nrm[3 * g + 1] = cy * s;
    nrm[3 * g + 2] = cz * s;
    w[g] = 0.5f * len / (float)per;
  }
}

__global__ void __launch_bounds__(EV_THREADS) k_eval_terms(const float* __restrict__ q, const float* __restrict__ q_nrm,
                                                           const float* __restrict__ q_w, int64_t n,
                                                           const int32_t* __restrict__ nn,
                                                           const float* __restrict__ pts,
                                                           const float* __restrict__ t_nrm, EvTaus taus, int ntau,
                                                           double* __restrict__ sums,
                                                           unsigned long long* __restrict__ max_bits) {
  __shared__ double red[EV_THREADS / 32][EV_SUMS];
  __shared__ unsigned long long red_max[EV_THREADS / 32];
  double acc[EV_SUMS];
#pragma unroll
  for (int k = 0; k < EV_SUMS; ++k) acc[k] = 0.0;
  double dmax = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int j = nn[i];
    const double w = q_w ? (double)q_w[i] : 1.0;
    if (j < 0 || !(w > 0.0)) continue;
    const double dx = __dsub_rn((double)q[3 * i + 0], (double)pts[3 * (int64_t)j + 0]);
    const double dy = __dsub_rn((double)q[3 * i + 1], (double)pts[3 * (int64_t)j + 1]);
    const double dz = __dsub_rn((double)q[3 * i + 2], (double)pts[3 * (int64_t)j + 2]);
    const double d = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
    acc[0] += w;
    acc[1] += w * d;
    acc[2] += w * (d * d);
    if (q_nrm && t_nrm) {
      const double c = (double)q_nrm[3 * i] * (double)t_nrm[3 * (int64_t)j] +
                       (double)q_nrm[3 * i + 1] * (double)t_nrm[3 * (int64_t)j + 1] +
                       (double)q_nrm[3 * i + 2] * (double)t_nrm[3 * (int64_t)j + 2];
      acc[3] += w * fabs(c);
    }
#pragma unroll
    for (int k = 0; k < EV_MAX_TAU; ++k)
      if (k < ntau && d < taus.t[k]) acc[4 + k] += w;
    dmax = fmax(dmax, d);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < EV_SUMS; ++k) {
    double v = acc[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[wid][k] = v;
  }
  for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_down_sync(0xffffffffu, dmax, o));
  if (lane == 0) red_max[wid] = (unsigned long long)__double_as_longlong(dmax);
  __syncthreads();
  if (threadIdx.x < EV_SUMS) {
    double v = 0.0;
    for (int w = 0; w < EV_THREADS / 32; ++w) v += red[w][threadIdx.x];
    if (v != 0.0) atomicAdd(sums + threadIdx.x, v);
  }
  if (threadIdx.x == 0) {
    unsigned long long m = 0;
    for (int w = 0; w < EV_THREADS / 32; ++w) m = red_max[w] > m ? red_max[w] : m;
    // non-negative doubles order like their bit patterns
    atomicMax(max_bits, m);
  }
}

}  // namespace

extern "C" gp_status gp_mesh_quadrature(gp_ctx* ctx, const float* tri_dev, int64_t T, int32_t m, float* pts_dev,
                                        float* nrm_dev, float* w_dev) {
  if (!ctx) return GP_ERR_ARG;
  if (T < 0 || m < 1 || m > 64) return gp_fail(ctx, GP_ERR_ARG, "gp_mesh_quadrature: need T >= 0 and m in [1, 64]");
  if (T == 0) return GP_OK;
  if (!tri_dev || !pts_dev || !nrm_dev || !w_dev) return gp_fail(ctx, GP_ERR_ARG, "gp_mesh_quadrature: null pointer");
  if (T > (int64_t(1) << 40) / ((int64_t)m * m)) return gp_fail(ctx, GP_ERR_ARG, "gp_mesh_quadrature: too many points");
  GP_KERNEL(ctx, "k_mesh_quad",
            k_mesh_quad<<<gp_blocks(T * m * m, EV_THREADS, (int64_t)ctx->num_sms * 16), EV_THREADS, 0, ctx->stream>>>(
                tri_dev, T, m, pts_dev, nrm_dev, w_dev));
  return GP_OK;
}

extern "C" gp_status gp_eval_nearest(gp_band* b, const float* q_dev, const float* q_nrm_dev, const float* q_w_dev,
                                     int64_t n, const float* target_nrm_dev, const double* tau_host, int32_t ntau,
                                     double* out_host) {
  if (!b) return GP_ERR_ARG;
  gp_ctx* ctx = b->ctx;
  if (!out_host) return gp_fail(ctx, GP_ERR_ARG, "gp_eval_nearest: out is null");
  if (ntau < 0 || ntau > EV_MAX_TAU || (ntau > 0 && !tau_host))
    return gp_fail(ctx, GP_ERR_ARG, "gp_eval_nearest: ntau must be in [0, 16] with a tau array");
  if (n < 0 || n >= (int64_t(1) << 31)) return gp_fail(ctx, GP_ERR_ARG, "gp_eval_nearest: n must be in [0, 2^31)");
  const bool with_nc = q_nrm_dev && target_nrm_dev;
  for (int k = 0; k < 5 + ntau; ++k) out_host[k] = 0.0;
  if (n == 0) {
    for (int k = 1; k < 5 + ntau; ++k) out_host[k] = NAN;
    out_host[3] = 0.0;
    return GP_OK;
  }
  if (!q_dev) return gp_fail(ctx, GP_ERR_ARG, "gp_eval_nearest: q is null");
  EvTaus taus{};
  for (int k = 0; k < ntau; ++k) taus.t[k] = tau_host[k];

  int32_t* nn = nullptr;
  double* acc = nullptr;  // EV_SUMS sums, then the max as bits
  gp_status st = gp_alloc(ctx, &nn, (size_t)n, "eval nn");
  if (st) return st;
  if ((st = gp_alloc(ctx, &acc, EV_SUMS + 1, "eval sums"))) {
    gp_free(nn);
    return st;
  }
  double host[EV_SUMS + 1];
  do {
    cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(double) * (EV_SUMS + 1), ctx->stream);
    if (e != cudaSuccess) { st = gp_cuda_fail(ctx, e, "gp_eval_nearest memset"); break; }
    if ((st = gp_nn(b, q_dev, n, nullptr, nn, nullptr, nullptr))) break;
    gp_prof_pre(ctx);
    k_eval_terms<<<gp_blocks(n, EV_THREADS, (int64_t)ctx->num_sms * 8), EV_THREADS, 0, ctx->stream>>>(
        q_dev, with_nc ? q_nrm_dev : nullptr, q_w_dev, n, nn, b->pts, with_nc ? target_nrm_dev : nullptr, taus, ntau,
        acc, reinterpret_cast<unsigned long long*>(acc + EV_SUMS));
    gp_prof_post(ctx, "k_eval_terms");
    e = cudaGetLastError();
    if (e != cudaSuccess) { st = gp_cuda_fail(ctx, e, "k_eval_terms"); break; }
    e = cudaMemcpyAsync(host, acc, sizeof(host), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) { st = gp_cuda_fail(ctx, e, "gp_eval_nearest"); break; }
  } while (false);
  gp_free(nn);
  gp_free(acc);
  if (st) return st;
  const double W = host[0];
  out_host[0] = W;
  out_host[1] = W > 0 ? host[1] / W : NAN;
  out_host[2] = W > 0 ? host[2] / W : NAN;
  double dmax;
  std::memcpy(&dmax, &host[EV_SUMS], sizeof(double));
  out_host[3] = dmax;
  out_host[4] = (W > 0 && with_nc) ? host[3] / W : NAN;
  for (int k = 0; k < ntau; ++k) out_host[5 + k] = W > 0 ? host[4 + k] / W : NAN;
  return GP_OK;
}
