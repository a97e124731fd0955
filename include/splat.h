/*
 * splat.h -- C ABI of the GB300 (sm_103a) hybrid 3D-4D Gaussian rasterizer.
 *
 * The library renders a mixed set of static 3D Gaussians and dynamic 4D
 * Gaussians ("Hybrid 3D-4D Gaussian Splatting for Fast Dynamic Scene
 * Representation", Sec. 4.3 and Alg. 1 "GPU Rasterization of 3D&4D
 * Gaussians") and differentiates the result with respect to every Gaussian
 * parameter.  One call of each stage handles a batch of V views (cameras and
 * timestamps, resolutions may differ).  Stages, in order:
 *
 *   splat_slice_project     Alg. 1 CullGaussian, ProjGaussian4D, ProjGaussian3D
 *   splat_bin_sort          Alg. 1 CreateTiles, DuplicateWithKeys, SortByKeys,
 *                           IdentifyTileRanges
 *   splat_composite_fwd     Alg. 1 BlendInOrder (Eq. 3)
 *   splat_composite_bwd     reverse mode of all of the above
 *   splat_convert_4d_to_3d  Sec. 4.1 static/dynamic identification and
 *                           Sec. 4.2 conversion (Eq. 9)
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every pointer inside the structs below is DEVICE memory owned by the
 *    caller, unless a comment says "host".  The library never allocates; its
 *    scratch memory is a caller-supplied workspace of splat_workspace_size()
 *    bytes (256-byte aligned).  Pointers are borrowed for the call only.
 *  - Calls are asynchronous on the caller's CUDA stream (`stream`, a
 *    cudaStream_t; NULL = legacy default stream) and may be captured into a
 *    CUDA graph: no entry point synchronises or reads device memory on the
 *    host.
 *  - The return value reports argument errors found on the host
 *    (SPLAT_ERR_INVALID_ARG) and launch failures (SPLAT_ERR_CUDA).  Errors
 *    found on the device are written to `status`, a device int32[4]:
 *      status[0]  first error code (0 = OK), never overwritten once set
 *      status[1]  stage that set it (SPLAT_STAGE_*)
 *      status[2]  low 32 bits of an auxiliary value (CAPACITY: required count)
 *      status[3]  high 32 bits of it
 *    splat_slice_project clears status at its start; later stages skip their
 *    work while status[0] != 0.  Kernels never trap: bounded waits that run
 *    out set SPLAT_ERR_TIMEOUT and return.
 *  - Gaussian parameters are raw, before activation: log-scales, opacity
 *    logits, quaternions that need not be normalised, quaternion order
 *    (w,x,y,z) for 3D and (a,b,c,d) / (p,q,r,s) for the 4D left / right
 *    quaternions of Eq. 4.  4D coordinates are (x,y,z,t).  All fields of one
 *    set share one storage dtype (SPLAT_F32, SPLAT_BF16, SPLAT_F16); all
 *    arithmetic is FP32, gradients are always FP32.
 *  - Merged index: inside one view, Gaussian i in [0, N4) is the i-th 4D
 *    Gaussian and i in [N4, N4+N3) the (i-N4)-th 3D Gaussian (Alg. 1 fills M'
 *    with the 4D Gaussians first, then appends the 3D ones).  Projected rows
 *    are indexed r = v*N + i with N = N4 + N3.
 *  - Tiles are 16x16 pixels.  View v has TX = ceil(W/16) by TY = ceil(H/16)
 *    tiles; tiles of all views are numbered consecutively, view by view, row
 *    major inside a view.  Pixel (u, y) of a view is evaluated at the point
 *    (u, y) of the image plane, where a camera-space point (x, y, z) lands at
 *    (fx x/z + cx, fy y/z + cy).
 *  - Images of all views are stored back to back: view v starts at pixel
 *    offset P_v = sum_{w<v} W_w H_w; rgb is planar per view, [3][H][W]
 *    starting at float offset 3 P_v; final_T and last start at offset P_v.
 */
#ifndef SPLAT_H
#define SPLAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SPLAT_OK = 0,
    SPLAT_ERR_INVALID_ARG = 1, /* host-side argument check failed                */
    SPLAT_ERR_CAPACITY = 2,    /* a caller buffer is too small; see status[2..3] */
    SPLAT_ERR_TIMEOUT = 3,     /* a bounded device-side wait ran out             */
    SPLAT_ERR_NONFINITE = 4,   /* a projected quantity was NaN or infinite        */
    SPLAT_ERR_CUDA = 5         /* a CUDA runtime call or launch failed            */
} splat_status;

typedef enum { SPLAT_F32 = 0, SPLAT_BF16 = 1, SPLAT_F16 = 2 } splat_dtype;

enum {
    SPLAT_STAGE_SLICE_PROJECT = 1,
    SPLAT_STAGE_DEPTH_SORT = 2,
    SPLAT_STAGE_SCAN = 3,
    SPLAT_STAGE_DUPLICATE = 4,
    SPLAT_STAGE_TILE_SORT = 5,
    SPLAT_STAGE_COMPOSITE_FWD = 6,
    SPLAT_STAGE_COMPOSITE_BWD = 7,
    SPLAT_STAGE_ADJOINT = 8,
    SPLAT_STAGE_CONVERT = 9,
    SPLAT_STAGE_DENSIFY = 10
};

#define SPLAT_MAX_VIEWS 16
#define SPLAT_TILE 16
#define SPLAT_SH_COEFFS 16           /* degree 3, 3 channels each              */
#define SPLAT_MAX_INSTANCES (1 << 30) /* upper bound of splat_bins.capacity    */

/* Parameter arrays: FP32 arrays of 4-wide fields (quat, the 4D fields) and the
 * SH arrays 16-byte aligned; with BF16 / FP16 storage the 4-wide fields 8-byte
 * and the SH arrays 16-byte aligned (entry points return SPLAT_ERR_INVALID_ARG
 * otherwise). */

/* Static 3D Gaussians (Eq. 1, Eq. 2). */
typedef struct {
    int64_t n;        /* N3                                                     */
    int64_t capacity; /* rows allocated in every field (>= n); convert appends  */
    int32_t dtype;    /* splat_dtype of every field                             */
    int32_t reserved;
    void *mean;       /* [capacity][3] world position                           */
    void *log_scale;  /* [capacity][3] s, scale = exp(s)                        */
    void *quat;       /* [capacity][4] (w,x,y,z)                                */
    void *opacity;    /* [capacity]    logit, opacity = sigmoid(o)              */
    void *sh;         /* [capacity][16][3] SH coefficients, degree 3            */
} splat_g3;

/* Dynamic 4D Gaussians (Eq. 4 - Eq. 6).  The colour is degree-3 SH, or with
 * sh_time = T > 0 the time-dependent model of 4D spherindrical harmonics that
 * Sec. 3.2 defers to 4DGS for: colour(d, t) = max(0, 0.5 + sum_{n=0..T}
 * cos(2 pi n t) sum_k c_nk Y_k(d)), t in units of the sequence length. */
typedef struct {
    int64_t n;        /* N4                                                     */
    int32_t dtype;
    int32_t sh_time;  /* T, 0 .. SPLAT_MAX_SH_TIME (0: plain SH)                */
    void *mean;       /* [n][4] (x,y,z,t)                                       */
    void *log_scale;  /* [n][4] (s_x,s_y,s_z,s_t)                               */
    void *ql;         /* [n][4] left quaternion (a,b,c,d)                       */
    void *qr;         /* [n][4] right quaternion (p,q,r,s)                      */
    void *opacity;    /* [n]                                                    */
    void *sh;         /* [n][T+1][16][3]: a coefficient block per time frequency */
} splat_g4;

#define SPLAT_MAX_SH_TIME 4

/* One camera and timestamp (host memory; the library copies it into kernel
 * parameters).  x_cam = R x_world + T, R row major. */
typedef struct {
    float R[9];
    float T[3];
    float fx, fy, cx, cy;
    int32_t W, H;     /* image size in pixels, each in [1, 16384]               */
    float t;          /* timestamp the 4D Gaussians are sliced at (Eq. 5/6)     */
    float z_near;     /* Gaussians with camera depth <= z_near are culled       */
    float bg[3];      /* background colour added with the final transmittance   */
    float reserved;
} splat_view;

/* Projected Gaussians (Alg. 1 M'), one row per (view, merged Gaussian). */
typedef struct {
    int64_t n;             /* N = N4 + N3 rows per view                         */
    int32_t views;         /* V                                                 */
    int32_t reserved;
    float *xy;             /* [V*N][2]  projected mean (px, py)                  */
    float *conic_opacity;  /* [V*N][4]  (a, b, c, alpha_max): inverse 2D covariance
                              [[a,b],[b,c]] and the peak opacity                 */
    float *rgb_depth;      /* [V*N][4]  (r, g, b, camera depth)                  */
    int32_t *rect;         /* [V*N][4]  tile rectangle x0,y0,x1,y1 (half open)   */
    int32_t *radius;       /* [V*N]     support radius in pixels, 0 = culled     */
    uint32_t *n_tiles;     /* [V*N]     tiles in the rectangle, 0 = culled        */
} splat_proj;

/* Per-tile sorted instance lists (Alg. 1 L, K and R). */
typedef struct {
    int64_t capacity;      /* entries allocated in keys / vals, <= 2^30          */
    uint32_t *keys;        /* [capacity] global tile index, ascending             */
    uint32_t *vals;        /* [capacity] projected row v*N + i                    */
    uint32_t *ranges;      /* [total_tiles][2] [start, end) of each tile in vals  */
    int64_t *n_instances;  /* [1] K, the number of (tile, Gaussian) instances;
                              on SPLAT_ERR_CAPACITY the count that was needed    */
    uint32_t *tile_order;  /* optional (may be NULL), [total_tiles]: written by
                              splat_bin_sort with the tiles in decreasing
                              order of list length (classes of eight per power
                              of two: the exponent and the next three bits;
                              order inside a class unspecified); the
                              compositing kernels take tiles in this order,
                              the longest first, so that the last wave of
                              warps is short.  Results do not depend on it.
                              NULL: raster order.                            */
    int64_t *n_needed;     /* optional (may be NULL), [1]: the capacity the call
                              needed, K or, on the binned path, the larger of K
                              and the super-tile list length (which shares the
                              capacity-sized buffers and, with the saturation
                              cut, is often the larger)                      */
} splat_bins;

/* Rendered images and the per-pixel state the backward pass replays. */
typedef struct {
    float *rgb;            /* [sum_v 3 W_v H_v] planar per view                  */
    float *final_T;        /* [sum_v W_v H_v] transmittance after the last blend */
    int32_t *last;         /* [sum_v W_v H_v] end of the pixel's walk: the
                              index in its tile list of the entry that would
                              bring T below 1e-4 (not blended), else the list
                              length; the backward walks entries [0, last)   */
} splat_image;

/* FP32 gradients, same shapes as splat_g3 / splat_g4 (first n rows). */
typedef struct {
    float *mean, *log_scale, *quat, *opacity, *sh;
} splat_grads3;

typedef struct {
    float *mean, *log_scale, *ql, *qr, *opacity, *sh;
} splat_grads4;

/* Workspace selectors for splat_workspace_size. */
enum {
    SPLAT_OP_BIN_SORT = 1,
    SPLAT_OP_COMPOSITE_BWD = 2,
    SPLAT_OP_CONVERT = 3,
    SPLAT_OP_ALL = 4,      /* one workspace good for every entry point           */
    SPLAT_OP_CONVERT_STATE = 5
};

/*
 * Optimizer state of one parameter set for a training step: FP32 master
 * values and Adam's first and second moments, one array per field, each
 * shaped like the field ([rows][width] floats, dense, 16-byte aligned).  Field
 * order is that of splat_g3 (mean, log_scale, quat, opacity, sh; entries 0-4,
 * entry 5 unused) or of splat_g4 (mean, log_scale, ql, qr, opacity, sh).  The
 * arrays of a 3D set have splat_g3.capacity rows.
 */
typedef struct {
    float *param[6];
    float *m[6];
    float *v[6];
} splat_adam_set;

/* Step sizes and Adam constants of one update (host memory). */
typedef struct {
    float lr3[5];       /* per 3D field; for sh, the degree-0 coefficients   */
    float lr4[6];       /* per 4D field; for sh, the degree-0 coefficients   */
    float lr_sh_rest;   /* SH coefficients of degree 1-3, both sets           */
    float beta1, beta2, eps;
    int32_t step;       /* t >= 1, for the bias corrections 1 - beta^t        */
} splat_adam_hyper;

/* splat_composite_bwd flags */
#define SPLAT_BWD_STOP_2D 1u      /* stop after the 2D gradients (dproj), skip the adjoint */
#define SPLAT_BWD_ADJOINT_ONLY 2u /* skip the compositing adjoint: chain the caller's dproj
                                     (not cleared) through the projection into dg3 / dg4 */

/*
 * Bytes of workspace an entry point needs.  N3, N4: Gaussian counts (for
 * CONVERT, N4 is the 4D count); V views of sizes W[v] x H[v] (host arrays);
 * capacity: splat_bins.capacity.  Returns 0 on invalid arguments.
 */
size_t splat_workspace_size(int op, int64_t N3, int64_t N4, int V, const int32_t *W, const int32_t *H,
                            int64_t capacity);

/* Total number of tiles of V views (host arrays W, H): the length of
 * splat_bins.ranges / 2. */
int64_t splat_total_tiles(int V, const int32_t *W, const int32_t *H);

/*
 * Alg. 1 CullGaussian + ProjGaussian4D + ProjGaussian3D, for every view.
 * 4D Gaussians are sliced at the view's t: conditional mean (Eq. 5) and
 * Schur-complement covariance (Eq. 6) of Sigma_4D = R S S^T R^T with R from
 * Eq. 4, and opacity scaled by exp(-(t-mu_t)^2 / (2 Sigma_tt)).  Every Gaussian
 * is culled when its camera depth is <= z_near or its peak opacity is below
 * 1/255, EWA-projected (Jacobian at the mean with x/z, y/z clamped to
 * +-1.3 W/(2 fx), +-1.3 H/(2 fy); 0.3 px^2 added to the 2D covariance
 * diagonal), given the radius ceil(3 sqrt(lambda_max)), the tile rectangle
 * [floor((px-r)/16), ceil((px+r)/16)) x [...] clipped to the image's tiles, and
 * the colour max(0, 0.5 + sum_k sh_k Y_k(d)) of the degree-3 real SH at the
 * unit direction d from the camera centre to the (sliced) mean.
 * g3 / g4 may be NULL or have n == 0.  out->n must be N4 + N3 and
 * out->views == V.  Clears status[] first.
 */
splat_status splat_slice_project(const splat_g3 *g3, const splat_g4 *g4, const splat_view *views, int V,
                                 splat_proj *out, int32_t *status, void *stream);

/*
 * Alg. 1 CreateTiles + DuplicateWithKeys + SortByKeys + IdentifyTileRanges.
 * Every visible row emits one instance per tile of its rectangle, keyed by
 * (global tile index, camera depth); the instances are sorted by that key,
 * stably, ties in emission order (row r ascending, tiles row major).  Because
 * the depth part of the key is the same for every instance of a row, the
 * depth digits of this LSD radix sort are sorted once per row before the
 * duplication, then the tile digits after it; the resulting order is the
 * same.  Writes bins->keys/vals (first K entries), bins->ranges (every tile,
 * [0,0) when empty) and *bins->n_instances = K.  K > capacity sets
 * SPLAT_ERR_CAPACITY with the required count in status[2..3] and n_instances;
 * on the binned path (see splat_set_tile_sort) the intermediate super-tile
 * list may overflow first, and the count reported is then a lower bound of K
 * (retrying with at least that capacity converges in a few calls).
 * bins->keys may be NULL when the binned partition is in use (see
 * splat_set_tile_sort); the tile of entry s is then implied by ranges.
 */
splat_status splat_bin_sort(const splat_proj *proj, const splat_view *views, int V, splat_bins *bins,
                            int32_t *status, void *workspace, size_t workspace_bytes, void *stream);

/*
 * Alg. 1 BlendInOrder, Eq. 3 front to back per pixel over its tile's list:
 * power = -(a dx^2 + c dy^2)/2 - b dx dy with (dx, dy) = mean - pixel; skip
 * when power > 0; alpha = min(0.99, alpha_max exp(power)); skip when
 * alpha < 1/255; stop (without blending) when T (1 - alpha) < 1e-4;
 * otherwise C += rgb alpha T, T *= 1 - alpha.  Finally C += T bg.
 */
splat_status splat_composite_fwd(const splat_proj *proj, const splat_bins *bins, const splat_view *views, int V,
                                 splat_image *img, int32_t *status, void *stream);

/*
 * splat_composite_fwd with the L1 loss of splat_l1_loss fused into it: as
 * each pixel's colour is written it is compared with target (device floats,
 * the layout of img->rgb): *loss = sum |rgb - target| (device float,
 * overwritten), dL_drgb = scale * sign(rgb - target) with sign(0) = 0.  The
 * image and the gradient are the same as from the two calls, the loss up to
 * the order of its float sum; the image is not read back.  When the status
 * word already holds an error, nothing is rendered and dL_drgb is not written.
 */
splat_status splat_composite_fwd_l1(const splat_proj *proj, const splat_bins *bins, const splat_view *views, int V,
                                    splat_image *img, const float *target, float scale, float *dL_drgb,
                                    float *loss, int32_t *status, void *stream);

/*
 * Reverse mode of the forward pipeline for a loss with pixel gradient
 * dL_drgb (same layout as img->rgb).  Replays each pixel back to front from
 * its stored final_T and last (T_i = T_{i+1} / (1 - alpha_i)); no per-splat
 * state is stored by the forward.  Writes the 2D gradients to dproj (caller
 * memory [V*N][12] f32, 16-byte aligned, or workspace when dproj is NULL): per row
 * (dpx, dpy, da, db, dc, dalpha_max, dr, dg, db, 0, 0, 0), then chains them
 * through the colour, EWA, slicing and covariance of every Gaussian and
 * OVERWRITES dg3 / dg4 with the gradient summed over the V views.  With
 * SPLAT_BWD_STOP_2D only dproj is written; with SPLAT_BWD_ADJOINT_ONLY the
 * given dproj (caller memory, required) is only chained through the
 * projection (img and dL_drgb are then unused).  g3, g4 must be the
 * parameters the forward used.
 */
splat_status splat_composite_bwd(const splat_proj *proj, const splat_bins *bins, const splat_view *views, int V,
                                 const splat_image *img, const float *dL_drgb, const splat_g3 *g3,
                                 const splat_g4 *g4, splat_grads3 *dg3, splat_grads4 *dg4, float *dproj,
                                 uint32_t flags, int32_t *status, void *workspace, size_t workspace_bytes,
                                 void *stream);

/*
 * Sec. 4.1 + Sec. 4.2: every 4D Gaussian with exp(s_t) > tau is static.  Its
 * (mu_x, q_3D, s_x, s_y, s_z, opacity, SH) is appended to g3 in increasing 4D
 * index order, where q_3D comes from the top-left 3x3 block of R_4D by Eq. 9
 * (the largest-diagonal branch of Shepperd's method when 1 + tr < 1e-2),
 * normalised with w >= 0; mu_t and s_t are dropped.  The remaining 4D
 * Gaussians are compacted in place, order kept.  *n_moved_dev receives the
 * number moved; g3->n and g4->n are NOT updated (the host reads n_moved and
 * updates them).  g3 and g4 must share one dtype.  If g3->n + moved exceeds
 * g3->capacity nothing is changed and status reports SPLAT_ERR_CAPACITY.
 * Does not clear status.
 */
splat_status splat_convert_4d_to_3d(splat_g4 *g4, splat_g3 *g3, float tau, int64_t *n_moved_dev, int32_t *status,
                                    void *workspace, size_t workspace_bytes, void *stream);

/*
 * Parameter update of a training step (Sec. 4.3 optimises the 3D and the 4D
 * set in every iteration): one Adam step (Kingma and Ba, 2015) over every
 * float of the first g3->n rows of each 3D field and g4->n rows of each 4D
 * field, in one launch:
 *   m = beta1 m + (1 - beta1) g,  v = beta2 v + (1 - beta2) g^2,
 *   p -= lr (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps),
 * with g from dg3 / dg4 (as splat_composite_bwd wrote them) and p, m, v in
 * s3 / s4; then the storage copies g3 / g4 (the arrays the rasterizer reads,
 * any dtype, round to nearest) receive the new p.  For FP32 storage a field
 * of g3 / g4 may be the master array itself.  g3->dtype == g4->dtype.  Skips
 * its work when status already holds an error.
 */
splat_status splat_adam_step(const splat_adam_hyper *h, splat_adam_set *s3, const splat_grads3 *dg3, splat_g3 *g3,
                             splat_adam_set *s4, const splat_grads4 *dg4, splat_g4 *g4, int32_t *status, void *stream);

/*
 * Storage copies of FP32 master values: the first src3->n rows of every field
 * of src3 (dtype F32) are rounded to nearest into dst3 (any dtype), likewise
 * src4 into dst4; dst->n is not read.  After splat_convert_4d_to_3d on the
 * master sets this refreshes the arrays the rasterizer reads.
 */
splat_status splat_cast_params(const splat_g3 *src3, splat_g3 *dst3, const splat_g4 *src4, splat_g4 *dst4,
                               void *stream);

/*
 * The optimizer-state side of splat_convert_4d_to_3d (Sec. 4.1-4.2 during
 * training).  Call it first, with the same g4 / g3 and tau: the decision
 * exp(s_t) > tau reads g4's log_scale, which the conversion then rewrites.
 * The moments s4->m / s4->v of the kept 4D Gaussians are compacted in place
 * like their parameters (order kept); the 3D moments s3->m / s3->v of rows
 * g3->n .. g3->n + moved - 1, where the converted Gaussians will land, are set
 * to zero (a converted Gaussian starts with fresh moments, as a Gaussian added
 * by densification does).  The param arrays are not touched.  Workspace:
 * splat_workspace_size(SPLAT_OP_CONVERT_STATE, 0, N4, ...).  Capacity overflow
 * changes nothing and sets SPLAT_ERR_CAPACITY, as the conversion does.
 */
splat_status splat_convert_adam_state(const splat_g4 *g4, const splat_g3 *g3, float tau, splat_adam_set *s4,
                                      splat_adam_set *s3, int32_t *status, void *workspace, size_t workspace_bytes,
                                      void *stream);

/*
 * Densification statistics (Sec. 4.3 densifies with the 3DGS rule, which
 * reads the positional gradient of the projected means): for every merged
 * Gaussian i (4D first) and every view v that sees it (proj->n_tiles[v N + i]
 * > 0), accum[i] += |(dpx W_v / 2, dpy H_v / 2)| -- the norm of dL/d(mean in
 * normalised device coordinates), from the dproj splat_composite_bwd wrote
 * (16-byte aligned) -- and count[i] += 1.  accum, count: [N] f32, device,
 * accumulated across calls (the caller zeroes them).
 */
splat_status splat_densify_stats(const splat_proj *proj, const splat_view *views, int V, const float *dproj,
                                 float *accum, float *count, void *stream);

/* Rules of splat_densify (host memory). */
typedef struct {
    float grad_threshold;  /* mean accum / count at which a Gaussian densifies (3DGS: 2e-4) */
    float dense_scale;     /* largest spatial scale exp(s) of a clone; larger ones split  */
    float min_opacity;     /* sigmoid(o) below this prunes the Gaussian (3DGS: 5e-3)      */
    float split_shrink;    /* log-scale decrease of the two children of a split (log 1.6) */
} splat_densify_rule;

/* One parameter set as splat_densify sees it. */
typedef struct {
    int64_t n;             /* rows in use                                               */
    int64_t capacity;      /* rows allocated in every array of state                    */
    splat_adam_set *state; /* FP32 master values and Adam moments (splat_adam_set)      */
    const float *accum;    /* [n] statistics of splat_densify_stats (this set's rows)   */
    const float *count;    /* [n]                                                       */
    const float *noise;    /* [n][2][3] (3D set) or [n][2][4] (4D set) N(0, 1) draws    */
    int32_t sh_time;       /* 4D set: the colour's time frequencies (splat_g4.sh_time); 3D: 0 */
    int32_t reserved;
} splat_densify_set;

/*
 * Adaptive densification and pruning of each set on its own (Sec. 4.3, the
 * clone / split / prune rules of 3DGS densification the paper adopts, without
 * opacity resets).  Per row: sigmoid(o) < min_opacity -> removed; else, when
 * accum / count >= grad_threshold (count 0 reads as 0), a Gaussian whose
 * largest spatial scale max(exp(s_x), exp(s_y), exp(s_z)) <= dense_scale is
 * cloned (an identical copy is added) and a larger one is split: it is
 * replaced by two Gaussians at mean + M z_h, h = 0, 1 (z from noise, M =
 * R diag(exp(s)) with R the 3x3 rotation of the quaternion for a 3D Gaussian
 * and the 4x4 R of Eq. 4 for a 4D one, which moves (x, y, z, t)), every
 * log-scale lowered by split_shrink, the other fields copied.  New layout of
 * each set: the kept rows in order, then the clones in order, then the
 * children two by two in order; new rows get zero moments.  n_out[0] /
 * n_out[1] (device int64) receive the new 3D / 4D row counts; set->n is not
 * updated.  A set whose new count exceeds its capacity sets SPLAT_ERR_CAPACITY
 * and neither set changes.  Workspace: splat_densify_workspace_size().
 */
splat_status splat_densify(const splat_densify_rule *rule, splat_densify_set *set3, splat_densify_set *set4,
                           int64_t *n_out, int32_t *status, void *workspace, size_t workspace_bytes, void *stream);

/* Bytes of workspace splat_densify needs for sets of n rows and the given capacities
 * (sh_time4: the 4D set's colour time frequencies). */
size_t splat_densify_workspace_size(int64_t n3, int64_t capacity3, int64_t n4, int64_t capacity4, int sh_time4);

/* Workspace of SPLAT_OP_CONVERT / SPLAT_OP_CONVERT_STATE for a 4D set of N4 rows
 * whose colour has sh_time time frequencies (splat_workspace_size assumes 0). */
size_t splat_workspace_size_4d(int op, int64_t N4, int sh_time);

/*
 * L1 photometric loss of a training step (Sec. 4.3 trains the rendered
 * images against the captured frames): *loss = sum_i |img_i - target_i|
 * (device float, overwritten), dL_dimg_i = scale * sign(img_i - target_i).
 * n floats, all three arrays 16-byte aligned (any layout, e.g. img->rgb).
 */
splat_status splat_l1_loss(const float *img, const float *target, int64_t n, float scale, float *dL_dimg,
                           float *loss, void *stream);

/*
 * splat_bin_sort for callers that cannot allocate device memory when they
 * sort -- e.g. a plugin whose host application has reserved the whole GPU
 * memory budget, or a frame loop that must not reach cudaMalloc / cudaFree
 * because those calls can synchronise the device.  The paper has no
 * counterpart to this entry point.  Same arguments and results as
 * splat_bin_sort minus the workspace: the scratch is a fixed array of
 * SPLAT_NOALLOC_SCRATCH_BYTES compiled into the library, which every GPU that
 * loads this part of the library keeps until the process exits.
 *  - Problems whose splat_bin_sort workspace would exceed that size are
 *    rejected on the host with SPLAT_ERR_CAPACITY, before any device work.
 *  - The first call on each device looks up the array's device address with
 *    the device current (cudaGetSymbolAddress); make that first call before
 *    any stream capture.  The address is kept for the life of the process: a
 *    cudaDeviceReset (or a reset of the primary context) unloads the array and
 *    voids this entry point on that device until the process restarts.
 *  - All calls share the array and its contents persist between calls (the
 *    sort clears what must start at zero); calls that overlap on the GPU --
 *    other streams, or other host threads without ordering -- race on it.
 * No allocation routine is called.
 */
#define SPLAT_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)
splat_status splat_bin_sort_noalloc(const splat_proj *proj, const splat_view *views, int V, splat_bins *bins,
                                    int32_t *status, void *stream);

/*
 * Per-call tuning (host memory), for callers that run several rasterizers
 * with different settings in one process, or from several threads: the
 * *_opts entry points below take it as their second-to-last argument and
 * otherwise behave exactly as the entry point of the same name without the
 * suffix.  Each field at its "library default" value (0, -1 or NULL as noted)
 * takes the library-wide setting of the matching splat_set_* call, so a
 * zero-initialised struct with tile_sort = tile_cull = spin_limit = -1 (or a
 * NULL pointer) changes nothing.  Out-of-range values are rejected with
 * SPLAT_ERR_INVALID_ARG (splat_workspace_size_opts returns 0).  The struct is
 * read during the call only.
 */
typedef struct {
    int32_t pixels_per_lane_fwd;  /* 2, 4 or 8; 0: library default (splat_set_pixels_per_lane) */
    int32_t pixels_per_lane_bwd;  /* 2, 4 or 8; 0: library default                           */
    int32_t tile_sort;            /* 0 automatic, 1 radix, 2 binned; -1: splat_set_tile_sort */
    int32_t tile_cull;            /* 0 off, 1 on; -1: splat_set_tile_cull                    */
    int64_t spin_limit;           /* >= 0; -1: splat_set_spin_limit                          */
    unsigned long long *stats;    /* device uint64[8] (see splat_set_stats); NULL: library default */
} splat_options;

/* splat_workspace_size for a call made with the given options (the sort's
 * workspace depends on the tile sort mode). */
size_t splat_workspace_size_opts(int op, int64_t N3, int64_t N4, int V, const int32_t *W, const int32_t *H,
                                 int64_t capacity, const splat_options *opt);

/* splat_bin_sort with per-call options (tile_sort, tile_cull, spin_limit). */
splat_status splat_bin_sort_opts(const splat_proj *proj, const splat_view *views, int V, splat_bins *bins,
                                 int32_t *status, void *workspace, size_t workspace_bytes, const splat_options *opt,
                                 void *stream);

/* splat_composite_fwd with per-call options (pixels_per_lane_fwd, stats). */
splat_status splat_composite_fwd_opts(const splat_proj *proj, const splat_bins *bins, const splat_view *views, int V,
                                      splat_image *img, int32_t *status, const splat_options *opt, void *stream);

/* splat_composite_fwd_l1 with per-call options (pixels_per_lane_fwd, stats). */
splat_status splat_composite_fwd_l1_opts(const splat_proj *proj, const splat_bins *bins, const splat_view *views,
                                         int V, splat_image *img, const float *target, float scale, float *dL_drgb,
                                         float *loss, int32_t *status, const splat_options *opt, void *stream);

/* splat_composite_bwd with per-call options (pixels_per_lane_bwd, stats). */
splat_status splat_composite_bwd_opts(const splat_proj *proj, const splat_bins *bins, const splat_view *views, int V,
                                      const splat_image *img, const float *dL_drgb, const splat_g3 *g3,
                                      const splat_g4 *g4, splat_grads3 *dg3, splat_grads4 *dg4, float *dproj,
                                      uint32_t flags, int32_t *status, void *workspace, size_t workspace_bytes,
                                      const splat_options *opt, void *stream);

/* Human-readable name of a status code (static string). */
const char *splat_status_string(int32_t code);

/*
 * Test knob: maximum polling iterations of every bounded device-side wait
 * (decoupled look-back of the scans and sorts).  0 gives up at the first
 * not-yet-published predecessor.  Default 1 << 22.  Host-side global: the
 * library default that splat_options.spin_limit = -1 takes.
 */
void splat_set_spin_limit(int64_t iterations);

/*
 * Tuning knob of the compositing kernels: pixels each lane owns (2, 4 or 8,
 * evaluated in pairs; one warp covers 32 x that many pixels of a 16x16
 * tile).  Other values are ignored.  Default 8 / 8.  Host-side global (the library default
 * of splat_options.pixels_per_lane_*); the results do not depend
 * on it beyond floating-point summation order of the gradients.
 */
void splat_set_pixels_per_lane(int fwd, int bwd);

/* Number of kernels this library has launched (or enqueued into a stream
 * capture) in this process; a diagnostic counter. */
int64_t splat_launch_count(void);

/*
 * Selects how splat_bin_sort orders the instances by tile (the result is the
 * same):  0 = automatic (default), 1 = tile-digit radix passes over the
 * instance list, 2 = binned partition: the rows split by 8x8-tile super-tile,
 * then each super-tile's list filtered into its tiles' lists (used
 * automatically when every view has at most 40960 tiles; never for a view of
 * more than 1023 super-tiles in x or y or more than about 5000 in all, which
 * take the radix passes).  Host-side global (the library default of
 * splat_options.tile_sort); splat_workspace_size depends on it.
 */
void splat_set_tile_sort(int mode);

/*
 * Binned tile sort only: when on (default), a Gaussian is listed for a tile of
 * its rectangle only if its opacity footprint -- the ellipse where alpha_max
 * exp(power) can reach 1/255, enlarged by a margin covering FP32 rounding --
 * meets the tile; and each tile's list ends once the entries so far certify
 * that every pixel of the tile has stopped its walk (T below 1e-4): a lower
 * bound of each entry's alpha over the tile (alpha_max exp(-q/2), q the
 * largest quadratic form over the tile's corners, with margins for FP32
 * rounding) enters a fixed-point sum of -ln(1 - alpha), and the list ends
 * after the batch of 32 entries that takes the sum past -ln(1e-4) plus a
 * margin (checked over the first 512 entries of the tile's 8x8-tile block in
 * depth order; a tile not saturated by then keeps its whole list).  Every
 * pixel skips the dropped pairs, or stops before reaching
 * them, so images and gradients do not change; the lists (and so `last`) are
 * shorter.  Off: every tile of the rectangle, as in splat_bin_sort's key
 * definition.  Host-side global (the library default of splat_options.tile_cull).
 */
void splat_set_tile_cull(int on);

/*
 * Diagnostic: when dev_counters (device uint64[8]) is not NULL, later
 * compositing launches use an instrumented variant that adds the numbers of
 * pixel-Gaussian pairs evaluated (power computed) and blended by the forward
 * (counters 0, 1) and by the backward (2, 3), and splat_bin_sort on the
 * binned path with culling adds the number of super-tiles whose lists ended
 * in the saturation head for some of their tiles while others continue in
 * tail segments (4) and the number of tail segments (5); 6 and 7 are
 * reserved.  NULL (default) turns it off.  Host-side global (the library
 * default of splat_options.stats); the caller zeroes the counters.
 */
void splat_set_stats(unsigned long long *dev_counters);

/*
 * Diagnostic: throughput probe of one SM pipe, for the roofline of the
 * compositing kernels (bound by FP32 arithmetic and the multi-function unit,
 * not by memory).  Launches `blocks` CTAs of 256 threads on `stream`, each
 * thread running 8 independent chains of `iters` steps of one instruction:
 *   SPLAT_PROBE_FFMA   fma.rn.f32            2 FP32 operations per step
 *   SPLAT_PROBE_FFMA2  fma.rn.f32x2 (packed) 4 FP32 operations per step
 *   SPLAT_PROBE_EX2    ex2.approx.ftz.f32    1 operation per step
 *   SPLAT_PROBE_RCP    rcp.approx.ftz.f32    1 operation per step
 * Returns the number of operations the launch performs (the caller times it
 * with CUDA events), or -1 on invalid arguments or a launch failure.  `out`:
 * device float[256], written only to keep the chains from being optimised
 * away (its contents are meaningless).
 */
enum { SPLAT_PROBE_FFMA = 0, SPLAT_PROBE_FFMA2 = 1, SPLAT_PROBE_EX2 = 2, SPLAT_PROBE_RCP = 3 };
double splat_peak_probe(int kind, int blocks, int iters, float *out, void *stream);

/* Library version, e.g. 0x000100 for 0.1.0. */
int32_t splat_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SPLAT_H */
