/*
 * gridpull.h - C ABI of the GB300 GridPull step library (libgridpull.so).
 *
 * GridPull (Chen, Liu, Han, ICCV 2023) fits a discrete signed distance field
 * D = {d_i} held on the vertices of a uniform grid to a point cloud S by
 * minimising, over D, the loss of Eq. 8 on sampled queries q (Sec. 3).  This
 * library runs one optimisation step of that fit on one GPU:
 *
 *   gp_build_band  uniform grid + near-surface brick table (Sec. 3 "Discrete
 *                  Grids", the M1 / M2 bandwidths) and the per-point sampling
 *                  sigma;
 *   gp_sample      Gaussian queries around randomly visited points (Sec. 3);
 *   gp_nn          NN(q), the nearest surface point of each query (Eq. 4);
 *   gp_step        the loss of Eq. 8 (Eq. 3-7 inside) and its gradient dL/dD,
 *                  forward and hand-written backward in one pass;
 *   gp_update      Adam on the trainable vertices (Sec. 4 "Details").
 *
 * Conventions shared by every call:
 *   - Geometry.  The domain is [-1,1]^3 split into R^3 cells (R a power of two),
 *     h = 2/R, vertex (i,j,k) at (-1,-1,-1) + h*(i,j,k), i,j,k in [0,R].  The
 *     cell of a point x is floor((x+1)/h) per axis, taken exactly on the
 *     float32 input; surface points are clamped to [0,R-1]; a query outside the
 *     domain, or whose cell or whose NN's cell is outside the pull band, is
 *     masked (weight 0, not counted in B_v).
 *   - Storage.  Grid values live in bricks of 8x8x8 vertices.  Brick b covers
 *     vertices [8*bx, 8*bx+7] x ...; the value of vertex (i,j,k) is at slot
 *     index  s*512 + ((k&7)*8 + (j&7))*8 + (i&7)  where s is the brick's slot.
 *     "V_stored" = 512 * n_bricks; slots whose coordinate exceeds R are padding.
 *   - Memory.  Pointers named *_dev are device pointers on the context's device
 *     owned by the caller; the library never frees them and never keeps them
 *     after the call returns.  The library owns the band (brick table, D, Adam
 *     moments, point cell list, scratch) and frees it in gp_band_destroy.
 *   - Streams.  Every call is asynchronous on the context's stream, except
 *     gp_build_band and the gp_band_* queries that return host values, which
 *     synchronise that stream.  gp_sample, gp_nn, gp_step and gp_update never
 *     allocate memory.
 *   - Errors.  Every call returns a gp_status; on failure gp_last_error(ctx)
 *     holds a one-line message.  No C++ exception crosses this interface.
 *     Invalid arguments are reported before anything is launched.
 */
#ifndef GRIDPULL_H
#define GRIDPULL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gp_status {
  GP_OK = 0,
  GP_ERR_ARG = 1,     /* invalid argument: null pointer, bad size or descriptor  */
  GP_ERR_OOM = 2,     /* a device allocation failed                              */
  GP_ERR_CUDA = 3,    /* a CUDA runtime call or a kernel launch failed           */
  GP_ERR_TIMEOUT = 4, /* a bounded device-side wait gave up                      */
  GP_ERR_STATE = 5,   /* the call is not valid in the object's current state     */
  GP_ERR_NUMERIC = 6  /* a device-side numeric or range check fired              */
} gp_status;

typedef struct gp_ctx gp_ctx;
typedef struct gp_band gp_band;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device` whose calls run on `stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out receives the
 * context; destroy it with gp_destroy after every band made from it. */
gp_status gp_create(gp_ctx** out, int device, void* stream);

/* Change the stream later calls run on (e.g. torch's current stream). */
gp_status gp_set_stream(gp_ctx* ctx, void* stream);

/* Free the context (NULL is ignored).  If bands made from it are still alive,
 * the context is released when the last of them is destroyed, so the two may
 * be destroyed in either order. */
void gp_destroy(gp_ctx* ctx);

/* Message of the last failing call on this context ("" if none).  The string
 * is owned by the context and valid until its next call. */
const char* gp_last_error(const gp_ctx* ctx);

/* Library version string, e.g. "gridpull-gb300 0.1". */
const char* gp_version(void);

/* ---------------------------------------------------------------- tracing */

/* Start (enable != 0) or stop recording a pair of CUDA events around every
 * kernel this context launches, on its stream.  Off by default; recording adds
 * two event records per launch and no synchronisation. */
gp_status gp_profile(gp_ctx* ctx, int enable);

/* Aggregate the recorded launches by kernel name and clear the record
 * (synchronises the stream).  Up to max_kernels entries are written: names as
 * 32-byte NUL-terminated strings (names + 32*k), total_ms[k] the summed event
 * durations, launches[k] the launch count; *n_kernels receives the number of
 * distinct kernels seen (may exceed max_kernels). */
gp_status gp_profile_read(gp_ctx* ctx, char* names, double* total_ms, int64_t* launches, int32_t max_kernels,
                          int32_t* n_kernels);

/* Kernels launched through this context since its creation (always counted;
 * -1 for a NULL context). */
int64_t gp_launch_count(const gp_ctx* ctx);

/* ------------------------------------------------------------------- band */

/* Band flags (gp_grid_desc.flags). */
#define GP_BAND_DETERMINISTIC 1u /* also allocate the fixed-point gradient
                                    accumulator used by GP_STEP_DETERMINISTIC  */

typedef struct gp_grid_desc {
  int32_t R;       /* cells per axis: a power of two in [8, 2048]                */
  int32_t M1;      /* pull bandwidth (Sec. 3): Chebyshev dilation, in cells, of
                      the cells holding points; < 0 = every cell                 */
  int32_t M2;      /* TV bandwidth (Sec. 3 "Continuous Distance Fields"): L_TV is
                      imposed on the corners of the M2 dilation; < 0 = all      */
  int32_t knn_k;   /* sigma_j = distance from s_j to its knn_k-th nearest other
                      point (0 = do not compute; gp_sample then fails)           */
  int32_t nn_grid; /* cells per axis of the point cell list used by gp_nn
                      (0 = chosen for about 6.5 points per occupied cell, at
                      most sqrt(J/3) and 512)                                    */
  uint32_t flags;  /* GP_BAND_* flags                                            */
} gp_grid_desc;

typedef struct gp_band_info {
  int32_t R;                 /* cells per axis                                  */
  int32_t nb;                /* bricks per axis of the virtual brick grid       */
  int64_t n_bricks;          /* stored bricks                                   */
  int64_t n_active_bricks;   /* bricks holding at least one trainable vertex    */
  int64_t V_stored;          /* 512 * n_bricks value slots                      */
  int64_t V_trainable;       /* corners of the max(M1,M2) band                  */
  int64_t V_tv;              /* |T|: corners of the M2 band                     */
  int64_t n_pull_cells;      /* cells of the M1 band                            */
  int64_t n_occupied_cells;  /* cells holding at least one point                */
  int64_t J;                 /* points in the cloud                             */
  int32_t nn_grid;           /* cells per axis of the point cell list           */
  int32_t knn_k;             /* k used for sigma (0 if not computed)            */
} gp_band_info;

/* Build the band for the cloud `pts_dev` (J x 3 float32, xyz interleaved, in
 * [-1,1]^3; points outside are clamped to the boundary cells).  Computes the
 * occupied cells, the M1 pull band, the TV vertex set, the trainable set,
 * allocates the bricks that hold them plus the one-vertex apron L_TV reads, and
 * initialises every stored value to 0 and the Adam state to zero.  Also builds
 * the point cell list for gp_nn and sigma_j (knn_k > 0).  Synchronises the
 * stream.  Errors: GP_ERR_ARG (R not a power of two in range, J < 1 or
 * J >= 2^31, null pointer), GP_ERR_OOM, GP_ERR_CUDA. */
gp_status gp_build_band(gp_ctx* ctx, const float* pts_dev, int64_t J,
                        const gp_grid_desc* desc, gp_band** out);

/* Free the band and everything it owns (NULL is ignored). */
void gp_band_destroy(gp_band* band);

/* Sizes of the band (host struct).  Does not synchronise. */
gp_status gp_band_get_info(const gp_band* band, gp_band_info* out);

/* Geometric initialisation (Sec. 3): every stored value (trainable or not) is
 * set to |v - c| - radius + noise_std * z, z ~ N(0,1) the first Box-Muller
 * normal of Philox4x32-10 at counter (key_lo, key_hi, 0, 2) and key (seed_lo,
 * seed_hi), key = i + (R+1)*(j + (R+1)*k).  Padding slots are set to 0. */
gp_status gp_band_init_sphere(gp_band* band, float cx, float cy, float cz, float radius,
                              float noise_std, uint64_t seed);

/* Overwrite all V_stored values from `d_dev` (V_stored floats, storage order). */
gp_status gp_band_set_values(gp_band* band, const float* d_dev);

/* Export the stored vertices in storage order.  Any output may be NULL.
 * ijk_dev: V_stored x 3 int32 vertex coordinates (padding slots have a
 * coordinate > R); d_dev: V_stored current values; flags_dev: V_stored bytes,
 * bit0 = in the TV set T, bit1 = trainable, bit2 = inside [0,R]^3,
 * bit3 = lowest corner of a pull-band cell. */
gp_status gp_band_export(const gp_band* band, int32_t* ijk_dev, float* d_dev, uint8_t* flags_dev);

/* Zero-copy device pointers of the band's values and Adam moments (each
 * V_stored floats, storage order).  Any output may be NULL.  The pointers stay
 * valid until gp_band_destroy; the values pointer is the current one of the
 * band's two value buffers, which gp_step_update swaps. */
gp_status gp_band_values(gp_band* band, float** d_dev, float** m_dev, float** v_dev);

/* Copy sigma_j (J floats, original point order) to `sigma_dev`. */
gp_status gp_band_sigma(const gp_band* band, float* sigma_dev);

/* Zero the Adam moments (the step counter is the caller's). */
gp_status gp_band_reset_adam(gp_band* band);

/* Read and clear the band's device-side error flag (synchronises the stream).
 * Returns GP_OK, GP_ERR_NUMERIC (a fixed-point accumulator overflowed or a
 * non-finite value reached a deterministic sum) or GP_ERR_TIMEOUT. */
gp_status gp_band_check(gp_band* band);

/* --------------------------------------------------------------- sampling */

#define GP_SAMPLE_SPATIAL 1u /* emit the batch grouped by source point, points in
                                Morton order of their cells                   */

/* Queries of the epoch-`epoch` pool of Q queries, pool positions
 * [first, first + count), written to q_dev (count x 3 float32).  Sec. 3: each
 * epoch visits the points in a fresh random order and draws a Gaussian query
 * around each visited point.  Position k visits point j = Pi_e(k mod J), where
 * Pi_e is a 4-round Feistel bijection of [0, J) keyed by (seed, epoch), and
 * q = s_j + sigma_j * z with z ~ N(0, I) from Philox4x32-10 at counter
 * (k, epoch, 0, 0), key (seed_lo, seed_hi), via Box-Muller.  Without flags the
 * i-th output is position first + i; with GP_SAMPLE_SPATIAL the same set of
 * queries is emitted grouped by source point, points in Morton order of their
 * cell-list cells (replicas of a point in increasing k): neighbouring outputs are close
 * in space.  Optional outputs (NULL to skip, count int32 each): src_dev = j
 * (a valid gp_nn hint), pos_dev = k.  Requires knn_k > 0 at build.  Errors:
 * GP_ERR_ARG (Q > 2^31-1, first + count > Q, null q_dev with count > 0),
 * GP_ERR_STATE (no sigma). */
gp_status gp_sample(gp_band* band, uint64_t seed, uint32_t epoch, int64_t Q, int64_t first, int64_t count,
                    uint32_t flags, float* q_dev, int32_t* src_dev, int32_t* pos_dev);

/* ---------------------------------------------------------- nearest point */

/* NN(q) of Eq. 4 for n queries q_dev (n x 3 float32): nn_dev[i] receives the
 * index (original order) of the cloud point minimising
 * ((qx-sx)^2 + (qy-sy)^2) + (qz-sz)^2 evaluated in float64 from the float32
 * coordinates, ties to the lowest index.  If rec_dev is not NULL it receives
 * the step record (qx,qy,qz,sx,sy,sz) per query (n x 6 float32).  nn_dev may
 * be NULL when rec_dev is given.  Exact: a float32 screen with a proven error
 * margin keeps every candidate that could be the float64 minimum.  A query
 * with a NaN, infinite or larger-than-1e18 coordinate (whose squared
 * distances would overflow float32) gets index -1 and NaN for s.  hint_dev
 * (NULL, or n int32 point indices, e.g. gp_sample's src_dev) seeds each search
 * with a known point: it only speeds the search up, the result is the same
 * for any hint; out-of-range hints are ignored.  If nvalid_dev is not NULL
 * (one int32) it receives the number of records gp_step will count as valid
 * (q inside the domain, cell(q) and cell(NN(q)) in the pull band): pass it to
 * gp_step to skip its own count. */
gp_status gp_nn(gp_band* band, const float* q_dev, int64_t n, const int32_t* hint_dev, int32_t* nn_dev,
                float* rec_dev, int32_t* nvalid_dev);

/* The same search as gp_nn (same kernel and launch shape, same results in
 * nn_dev), counting the point distances it evaluates: the seeds, every point
 * of every cell range the walk reads and the float64 tie-break's re-reads.
 * *work_host receives the count.  For measurement: the search's work in
 * candidate evaluations.  Synchronises the stream; allocates and frees one
 * 8-byte counter.  Errors: as gp_nn, plus GP_ERR_ARG for a null work_host or
 * nn_dev, GP_ERR_OOM. */
gp_status gp_nn_work(gp_band* band, const float* q_dev, int64_t n, const int32_t* hint_dev, int32_t* nn_dev,
                     int64_t* work_host);

/* ------------------------------------------------------------------- step */

typedef struct gp_loss_w {
  float alpha;  /* weight of L_TV      (Eq. 8; paper: 1, or 2 for noisy input) */
  float beta;   /* weight of L_Surface (Eq. 8; paper: 1)                        */
  float gamma;  /* weight of L_grad    (Eq. 8; paper: 0.005)                    */
} gp_loss_w;

#define GP_STEP_DETERMINISTIC 1u /* fixed-point gradient sums: bitwise equal
                                    results run to run (band needs
                                    GP_BAND_DETERMINISTIC)                      */
#define GP_STEP_NO_TV 2u         /* leave out the L_TV term and its gradient   */
#define GP_STEP_LOSS_ONLY 4u     /* compute the loss only; grad_dev untouched  */

/* Loss slots written to loss_dev (8 floats). */
#define GP_LOSS_TOTAL 0 /* L = L_Pull + alpha L_TV + beta L_Surface + gamma L_grad */
#define GP_LOSS_PULL 1  /* mean over valid queries of |p - NN(q)|  (Eq. 4)         */
#define GP_LOSS_GRAD 2  /* mean of 1 - cos(grad f(q), grad f(NN(q))) (Eq. 7)       */
#define GP_LOSS_SURF 3  /* mean of |f(NN(q))|                         (Eq. 6)       */
#define GP_LOSS_TV 4    /* mean over T of sqrt(sum of 6 squared differences) (Eq. 5) */
#define GP_LOSS_BV 5    /* B_v, the number of valid queries (as float)             */
#define GP_LOSS_T 6     /* |T| (as float)                                          */

/* One forward + hand-written backward pass of Eq. 8 over B step records
 * rec_dev (B x 6 float32: q then NN(q), e.g. from gp_nn; 8-byte aligned).  Query terms are
 * averaged over the B_v valid queries, L_TV over T.  Writes the loss slots to
 * loss_dev (8 floats) and, unless GP_STEP_LOSS_ONLY, overwrites grad_dev
 * (V_stored floats, storage order) with dL/dD at every stored slot (0 at
 * padding).  All B records are read; invalid ones are masked.  If nvalid_dev is
 * not NULL it holds B_v, the number of valid records among them (as gp_nn
 * counts it); otherwise gp_step counts them first.  If d_dev is not NULL the values are
 * read from it (V_stored floats) instead of the band's own.  Errors:
 * GP_ERR_ARG (B < 0, null rec/loss, B >= 2^31, rec_dev not 8-byte aligned,
 * grad_dev not 16-byte aligned: its corner pairs are added as vector reductions;
 * d_dev not 16-byte aligned: corners are read as vectors and bricks copied in bulk),
 * GP_ERR_STATE (deterministic
 * flag on a band built without GP_BAND_DETERMINISTIC). */
gp_status gp_step(gp_band* band, const float* rec_dev, int64_t B, const int32_t* nvalid_dev,
                  const float* d_dev, const gp_loss_w* w, float* grad_dev, float* loss_dev,
                  uint32_t flags);

/* Forms of the atomic-mode query pass (gp_step, gp_step_update; the
 * deterministic sums always take the direct form).  All give the same
 * results up to the order of the float additions.
 *   GP_QUERY_DIRECT: every record's 16 corner contributions go to the
 *     gradient as global vector reductions (8 or 16 bytes per cell edge).
 *   GP_QUERY_WINDOW: tiles of 512 consecutive records; each tile's window is
 *     the 3 x 3 x 3 bricks around the brick of its middle record's NN(q).
 *     Cells inside the window add their corner gradients into a shared-memory
 *     copy of the window, written to the gradient once per tile (one 16-byte
 *     reduction per non-zero group of four slots); the other cells take the
 *     direct path.  Pays off on batches in spatial order (gp_sample with
 *     GP_SAMPLE_SPATIAL), whose consecutive records share corners.
 *   GP_QUERY_WINDOW_STAGED: as GP_QUERY_WINDOW, and the window bricks' values
 *     and pull-band masks are staged in shared memory by bulk copies
 *     (cp.async.bulk), so that in-window cells read no global memory.
 * The gradient the corners of a cell receive is the derivative of Eq. 3-7
 * at its record, as in the direct form. */
#define GP_QUERY_DIRECT 0
#define GP_QUERY_WINDOW 1
#define GP_QUERY_WINDOW_STAGED 2

/* Chooses the launch shape of gp_step's fused forward + backward kernel: the
 * records each thread keeps in flight (*rpt_out = 1 or 2; with 2, both
 * records' gathers of one level are issued before either is waited for) and
 * the resident blocks per SM it is compiled for (*bps_out = 2, 3 or 4, i.e. a
 * cap of 128, 80 or 64 registers per thread), by timing each candidate with
 * CUDA events on the B records rec_dev (a representative batch, e.g. from
 * gp_nn; nvalid_dev as for gp_step, NULL = counted here).  The choice is kept
 * in the band and used by later gp_step calls; the windowed forms
 * (GP_QUERY_WINDOW, GP_QUERY_WINDOW_STAGED) are timed too, and the form of the
 * fastest candidate is kept (gp_band_query_shape reads it).  Reads the band's values,
 * writes nothing of the band but the choice; allocates and frees a scratch
 * gradient; synchronises.  rpt_out, bps_out may be NULL.  Errors: GP_ERR_ARG
 * (B outside (0, 2^31), null records or weights, misaligned records),
 * GP_ERR_OOM, GP_ERR_CUDA. */
gp_status gp_band_autotune(gp_band* band, const float* rec_dev, int64_t B, const int32_t* nvalid_dev,
                           const gp_loss_w* w, int32_t* rpt_out, int32_t* bps_out);

/* Sets that launch shape directly: rpt records per thread (1 or 2) and bps
 * blocks per SM (2, 3 or 4).  The windowed forms take the same shape (tiles
 * of 256 rpt records); the staged one runs 2 blocks per SM whatever bps is.
 * Errors: GP_ERR_ARG. */
gp_status gp_band_set_query_tiles(gp_band* band, int32_t rpt, int32_t bps);

/* Sets the form of the atomic-mode query pass (GP_QUERY_*).  gp_band_autotune
 * also times the two windowed forms (after the direct shapes) and keeps the
 * fastest of all.  Errors: GP_ERR_ARG. */
gp_status gp_band_set_query_form(gp_band* band, int32_t form);

/* The band's current query-pass choice: records per thread, blocks per SM
 * (direct form) and the form (GP_QUERY_*).  Any pointer may be NULL. */
gp_status gp_band_query_shape(const gp_band* band, int32_t* rpt_out, int32_t* bps_out, int32_t* form_out);

/* ----------------------------------------------------------------- update */

typedef struct gp_adam {
  float lr;     /* learning rate (world units per step)                 */
  float beta1;  /* 0.9   */
  float beta2;  /* 0.999 */
  float eps;    /* 1e-8  */
} gp_adam;

/* Adam (Kingma and Ba) at step `step` >= 1 on every trainable vertex:
 * m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 * d -= lr * (m / (1-b1^step)) / (sqrt(v / (1-b2^step)) + eps),
 * with g = grad_dev (V_stored floats, storage order).  Vertices outside the
 * trainable set are left untouched (Sec. 3: only variables in the bandwidth are
 * optimised).  Errors: GP_ERR_ARG (step < 1, null pointers). */
gp_status gp_update(gp_band* band, const float* grad_dev, const gp_adam* hp, int64_t step);

/* One fitting step on the band's own values: the loss and gradient of gp_step
 * followed by gp_update's Adam at step `step` (>= 1), in two kernels and
 * without a gradient array: the query pass adds its corner contributions into
 * the band's internal query gradient (kept all zero between calls), then one
 * sweep over the bricks computes each vertex's L_TV gradient, adds and resets
 * the query part and applies Adam to the trainable vertices (Sec. 3: only the
 * band is optimised).  The new values are written to the band's second value
 * buffer while the stencil reads the current one; the two are swapped when
 * the call returns, so the pointer gp_band_values gives changes with every
 * call (fetch it again) and a band stepped this way must not belong to a
 * gp_multi.  The values, moments and loss slots equal those of gp_step (same
 * records, weights and flags) then gp_update with the same hyper-parameters,
 * bit for bit with GP_STEP_DETERMINISTIC, to float rounding otherwise.
 * flags: GP_STEP_DETERMINISTIC and/or GP_STEP_NO_TV.  Never allocates; the
 * swap is a host-side pointer exchange, so a CUDA graph must capture two
 * consecutive calls.  Errors: GP_ERR_ARG (as gp_step, step < 1, null hp, other
 * flags), GP_ERR_STATE (deterministic flag without GP_BAND_DETERMINISTIC,
 * empty band). */
gp_status gp_step_update(gp_band* band, const float* rec_dev, int64_t B, const int32_t* nvalid_dev,
                         const gp_loss_w* w, const gp_adam* hp, int64_t step, float* loss_dev, uint32_t flags);

/* ------------------------------------------------------------------ mesh */

/* The surface of the fitted field at level `iso` as a triangle soup: marching
 * cubes (Sec. 3 "Overview") over the cells whose 8 corners are all trainable
 * (cells the fit did not optimise are skipped, Sec. 3 after Eq. 8), at the
 * grid's resolution (Sec. 4 "Details").
 *
 * Corner c = dx + 2 dy + 4 dz of a cell is negative iff d < iso.  On each face
 * of the cell, walked counter-clockwise as seen from outside, every maximal run
 * of negative corners gives one segment from the cut edge where the walk
 * enters the run to the one where it leaves it; the segments chain into cycles,
 * each fanned from its lowest edge id (edge id 4 axis + p + 2 q, (p, q) the
 * lower corner's coordinates on the other two axes, lower axis first).  Every
 * triangle's normal (v1 - v0) x (v2 - v0) points to the positive side.  A
 * crossing lies at t = (iso - d_lo) / (d_hi - d_lo) from the edge's lower
 * corner.  Two cells sharing a face produce the same crossings on it, bit for
 * bit, so the soup welds into a closed mesh wherever all cells are meshed.
 *
 * tri_dev: cap x 9 float32 (three xyz vertices per triangle); cell_dev: cap
 * int64 keys i + R (j + R k) of each triangle's cell, or NULL.  Triangles come
 * in a fixed order (active bricks in storage order, cells x-fastest within a
 * brick, a cell's triangles in fan order).  *n_tri (host) receives the total;
 * the buffers are written only if it is <= cap, so a call with cap = 0 sizes
 * them.  Synchronises the stream; allocates and frees a small count array.
 * Errors: GP_ERR_ARG (null n_tri, iso not finite, cap < 0, cap > 0 with a null
 * tri_dev, more than 2^31 - 1 triangles), GP_ERR_OOM, GP_ERR_CUDA. */
gp_status gp_mesh_extract(gp_band* band, float iso, float* tri_dev, int64_t* cell_dev, int64_t cap,
                          int64_t* n_tri);

/* The 256-case table gp_mesh_extract uses, built on the host from the face
 * rule above (no GPU needed): ntri[c] triangles for the cell whose negative
 * corners are the set bits of c, and edges[15 c + 3 k + v] the edge id of
 * vertex v of triangle k (255 past the last triangle).  At most 5 triangles.
 * Errors: GP_ERR_ARG (null pointer), GP_ERR_STATE (the table failed its own
 * consistency checks). */
gp_status gp_mesh_case_table(uint8_t* ntri, uint8_t* edges);

/* --------------------------------------------------------------- metrics */

/* Weighted oriented points of a triangle soup for the metrics of Sec. 4
 * "Datasets and Metrics": every triangle of tri_dev (T x 9 float32) is split at
 * m equal steps along its edges into m^2 congruent triangles, and each gives
 * its centroid, the triangle's unit normal and area / m^2 (zero normal and
 * weight for a degenerate triangle).  Point k of triangle i is row i m^2 + k;
 * pieces are ordered by (i, j) of their lowest lattice corner, i outer, the
 * upright piece (corners (i,j), (i+1,j), (i,j+1)) before the inverted one
 * (corners (i+1,j), (i,j+1), (i+1,j+1)); the centroid is
 * v0 + a (v1 - v0) + b (v2 - v0) with (a, b) = ((3i+1)/(3m), (3j+1)/(3m))
 * upright and ((3i+2)/(3m), (3j+2)/(3m)) inverted.  Outputs: pts_dev and
 * nrm_dev T m^2 x 3 float32, w_dev T m^2 float32.  Asynchronous.  Errors:
 * GP_ERR_ARG (T < 0, m outside [1, 64], null pointers with T > 0). */
gp_status gp_mesh_quadrature(gp_ctx* ctx, const float* tri_dev, int64_t T, int32_t m, float* pts_dev,
                             float* nrm_dev, float* w_dev);

/* One direction of the metrics: for each of the n query points q_dev (n x 3
 * float32) its exact nearest point in the band's cloud (as gp_nn), at distance
 * d = sqrt((dx^2 + dy^2) + dz^2) in float64 from the float32 coordinates.
 * q_w_dev: n float32 weights (NULL = 1); points of weight <= 0 are skipped.
 * q_nrm_dev and target_nrm_dev (n x 3 and J x 3 float32 unit normals, the
 * latter in the cloud's original order) give the normal term; NULL skips it.
 * out_host (5 + ntau doubles): [0] the weight sum W, [1] sum w d / W,
 * [2] sum w d^2 / W, [3] the largest d, [4] sum w |n_q . n_NN(q)| / W (NaN
 * without normals), [5 + k] sum w [d < tau_k] / W.  With the two directions
 * (A into a band over B, B into a band over A):
 * CD_L1 = ([1]_AB + [1]_BA) / 2, CD_L2 = ([2]_AB + [2]_BA) / 2,
 * HD = max([3]_AB, [3]_BA), NC = ([4]_AB + [4]_BA) / 2, F(tau_k) = 2 P R /
 * (P + R) with P = [5+k]_AB, R = [5+k]_BA.  Means are NaN when W = 0.
 * Synchronises the stream; allocates and frees n int32 of scratch.  Errors:
 * GP_ERR_ARG (n outside [0, 2^31), ntau outside [0, 16] or without taus,
 * null out_host or q_dev), GP_ERR_OOM, GP_ERR_CUDA. */
gp_status gp_eval_nearest(gp_band* band, const float* q_dev, const float* q_nrm_dev, const float* q_w_dev,
                          int64_t n, const float* target_nrm_dev, const double* tau_host, int32_t ntau,
                          double* out_host);

/* ------------------------------------------------------------- many clouds */

/* Several clouds of uneven size fitted together: the whole step of Sec. 3
 * (sampling, NN, Eq. 3-8 forward and backward, L_TV, Adam) for every cloud in
 * one launch per stage, each a persistent kernel over a work list that mixes
 * the clouds' tiles.  Each cloud keeps its own band (its values and Adam
 * moments are the band's own D, m, v, which gp_band_values and gp_band_export
 * read); the multi owns the records, the per-cloud orders Pi_e, the gradient
 * buffer and a step counter t kept on the device.
 *
 * Cloud k at step t takes batch t mod nb_k of epoch t / nb_k, nb_k =
 * ceil(Q_k / B_k): pool positions [b B_k, min((b+1) B_k, Q_k)), the queries
 * gp_sample draws with key seed + k; with GP_SAMPLE_SPATIAL they are emitted in
 * the spatial order (the same set).  Adam runs as step t + 1 with learning
 * rate lr * lr_decay^floor(t / lr_every) (lr_every = 0: constant lr). */
typedef struct gp_multi gp_multi;

typedef struct gp_multi_info {
  int32_t n;                    /* clouds                                      */
  uint32_t flags;               /* creation flags                              */
  int32_t records_per_tile;     /* also the block size of the record kernels   */
  int32_t blocks_per_sm_nn;     /* persistent blocks per SM, NN stage          */
  int32_t blocks_per_sm_tv;     /* ... L_TV sweep                              */
  int32_t blocks_per_sm_query;  /* ... fused query forward + backward          */
  int32_t error_bits;           /* kernel error flags raised so far (0 = none) */
  int32_t reserved;
  int64_t total_B;              /* sum of the batch sizes (record slots)       */
  int64_t V_total;              /* sum of the bands' V_stored (gradient size)  */
  int64_t step;                 /* t, the next step to run                     */
} gp_multi_info;

#define GP_MULTI_DETERMINISTIC 2u /* gp_multi_create: bitwise repeatable steps -
                                     the query sums in two-word integer fixed
                                     point (folded in by the L_TV sweep, which
                                     then runs after the query pass) and the
                                     loss sums in integers of 2^-24           */

/* Bands: n distinct bands of ctx, built with knn_k > 0 and without
 * GP_BAND_DETERMINISTIC; they must outlive the multi.  Q[k], B[k]: pool size
 * and batch size of cloud k, 1 <= B[k] <= Q[k] < 2^31, sum of B[k] < 2^31.
 * flags: GP_SAMPLE_SPATIAL and/or GP_MULTI_DETERMINISTIC (which allocates 16
 * more bytes per stored vertex).  Allocates the multi's buffers (the
 * dominant ones: 36 bytes per record slot, 4 bytes per stored vertex, 8 bytes
 * per point) and synchronises.  t starts at 0.  Errors: GP_ERR_ARG,
 * GP_ERR_OOM, GP_ERR_CUDA. */
gp_status gp_multi_create(gp_ctx* ctx, gp_band* const* bands, int32_t n, const int64_t* Q, const int64_t* B,
                          uint64_t seed, uint32_t flags, gp_multi** out);

/* Step t of every cloud, then t += 1 on the device.  Stream-ordered on the
 * context's stream; allocates nothing and does not synchronise, so a call can
 * be captured into a CUDA graph and replayed: the weights, hyper-parameters
 * and loss_dev of the captured call then stay fixed while t advances.  Writes
 * 8 loss slots per cloud to loss_dev (n x 8 floats, the gp_step layout).
 * Errors: GP_ERR_ARG (null pointers, lr_every < 0), GP_ERR_CUDA. */
gp_status gp_multi_step(gp_multi* m, const gp_loss_w* w, const gp_adam* hp, float lr_decay, int64_t lr_every,
                        float* loss_dev);

/* Chooses the records per tile (128, 256 or 512) and the persistent blocks
 * per SM of the NN, L_TV and query stages by timing each candidate with CUDA
 * events on the current step's data.  Leaves D, m, v and t as they were;
 * synchronises.  Call it before capturing a graph of gp_multi_step. */
gp_status gp_multi_autotune(gp_multi* m, const gp_loss_w* w);

/* Configuration, step counter and error flags (synchronises). */
gp_status gp_multi_get_info(gp_multi* m, gp_multi_info* out);

/* Sets t (to resume a fit; synchronises).  Errors: GP_ERR_ARG (step < 0). */
gp_status gp_multi_set_step(gp_multi* m, int64_t step);

/* Device views of cloud k's slices of the multi's buffers, as the last step
 * left them: its B_k records (B_k x 6 floats; slots past a short batch hold
 * NaN queries), their source points (B_k ints, -1 for those slots) and its
 * gradient (V_stored floats).  Any pointer may be NULL.  Valid until
 * gp_multi_destroy; gp_multi_autotune rewrites them. */
gp_status gp_multi_buffers(gp_multi* m, int32_t k, float** rec_dev, int32_t** src_dev, float** grad_dev);

/* Waits for the context's stream and frees the multi (not the bands). */
void gp_multi_destroy(gp_multi* m);

/* ------------------------------------------------------- no allocation */

/* An allocation-free form of the query part of gp_step (L_Pull + beta
 * L_Surface + gamma L_grad, averaged over the valid records, and its
 * gradient) on a dense grid the caller owns.  It is for callers that cannot
 * allocate device memory: a plugin whose host framework owns every device
 * allocation, a real-time loop that may not block on the allocator, or code
 * that plans all of its memory up front.  Such callers cannot build a band,
 * since gp_build_band allocates.  The paper has no counterpart to this entry
 * point; its results equal those of gp_step with GP_STEP_NO_TV on a band built
 * with M1 = M2 = -1 (every cell in the pull band).
 *
 * d_dev: (R+1)^3 float32 grid values, vertex (i,j,k) at i + (R+1)(j + (R+1)k).
 * rec_dev: B step records (qx,qy,qz,sx,sy,sz); a record is valid when q lies in
 * the domain and s is finite.  grad_dev: (R+1)^3 floats, overwritten with the
 * gradient (NULL = loss only).  loss_dev: 8 floats, the gp_step slots (L_TV and
 * |T| are 0).  R is a power of two in [8, 1024]; B <= 1,048,576.
 *
 * Nothing is allocated: the call's scratch (one row of partial sums per 256
 * records, two counters) is a fixed array of about 128 KiB compiled into the
 * library, which every GPU that loads the library holds until the process
 * exits.  The call makes the context's device current while it runs and puts
 * the caller's current device back before it returns.  The first call on a
 * device looks up that array's device address and keeps it: make that first
 * call before any stream capture.  Every call shares the array and clears the
 * counters it needs; calls whose work overlaps on the GPU (other streams or
 * host threads) race on it and give wrong results.
 * Errors: GP_ERR_ARG (R or B out of range, null pointers), GP_ERR_CUDA. */
gp_status gp_step_dense_noalloc(gp_ctx* ctx, int32_t R, const float* d_dev, const float* rec_dev, int64_t B,
                                const gp_loss_w* w, float* grad_dev, float* loss_dev);

#ifdef __cplusplus
}
#endif

#endif /* GRIDPULL_H */
