/*
 * trips.h -- C ABI of the GB300 trilinear point splatting library (libtrips.so).
 *
 * The library renders a point cloud into a screen-space feature pyramid the
 * way TRIPS does (Franke, Rueckert, Fink, Stamminger, "TRIPS: Trilinear Point
 * Splatting for Real-Time Radiance Field Rendering", Eurographics 2024):
 *
 *   I = Phi(C, R, t, x, s_w, tau, alpha)                         (Sec. 3, Eq. 1)
 *
 * C are the camera intrinsics, (R, t) the pose, x the point positions, s_w
 * the world-space point sizes, tau the point descriptors and alpha the point
 * opacities.  The optional environment map E of Eq. 1 is not part of this
 * library.  The frame is produced by four stream-ordered calls that follow the
 * paper's three render stages (Sec. 3.6: collect, splat, sort-and-accumulate)
 * and the backward pass:
 *
 *   tp_project        project, cull and choose layers (Sec. 3.1, Eq. 2)
 *   tp_splat_forward  bin every (point, screen tile) pair of the trilinear
 *                     2x2x2 splat into per-tile lists (Sec. 3.1, Eq. 3-5;
 *                     Sec. 3.6 "counting", "offset scan", "splatting")
 *   tp_blend          per pixel: the K front-most fragments by depth, blended
 *                     front to back (Sec. 3.2, Eq. 6-7; Sec. 3.6)
 *   tp_splat_backward gradients of a loss with respect to positions, world
 *                     sizes, opacities and descriptors (Sec. 3.5, Sec. 3.6)
 *   tp_camera_backward the gradient with respect to the camera intrinsics and
 *                     pose, from one view's point gradients (Sec. 3.5)
 *   tp_init_point_sizes initial world sizes: mean distance to the 4 nearest
 *                     neighbours (Sec. 3.6)
 *   tp_merge          the decoder's layer merge in its weight-free form: the
 *                     pyramid summed into one image by bilinear upsampling
 *                     (Sec. 3.3), and tp_merge_backward, its adjoint
 *
 * Conventions shared by every call
 * --------------------------------
 * - Device pointers are CUDA device memory of the current device; host
 *   pointers are marked "host".  The caller owns every buffer, including the
 *   workspace.  The library never allocates or frees memory and never
 *   synchronises the stream, except tp_get_status.
 * - All work is enqueued on `stream` (NULL = the legacy default stream) in
 *   call order.  The calls contain no host round trip, so a frame can be
 *   captured in a CUDA graph.
 * - One frame = one (tp_config, tp_camera, n, workspace) tuple; every call of
 *   a frame must see the same values.
 * - Argument errors are found on the host and returned before anything is
 *   enqueued.  Errors found on the device are bits of a status word in the
 *   workspace (TP_FLAG_*), read with tp_get_status.
 * - A CUDA launch error is returned as TP_ERR_CUDA.
 *
 * Geometry (the readings of the paper this library implements)
 * ------------------------------------------------------------
 * - Pinhole camera, +z forward, +y down: X_c = R X_w + t,
 *   x = fx X_c/Z_c + cx, y = fy Y_c/Z_c + cy, screen size s = fx s_w / Z_c
 *   (Eq. 2), depth z = Z_c.  Points with Z_c <= znear are culled.
 * - Pyramid layer L has W_L = ceil(W / 2^L) by H_L = ceil(H / 2^L) pixels.
 *   Layer-L pixel (j, k) has its centre at ((j + 0.5) 2^L, (k + 0.5) 2^L).
 * - s < 1: layer 0 only with iota = eps + (1 - eps) s (Eq. 5, second case).
 *   1 <= s < 2^(n-1): layers floor(log2 s) and floor(log2 s) + 1 with the
 *   linear weights of Eq. 5.  s >= 2^(n-1): layer n-1 only, iota = 1.
 * - Fragments with an exactly zero bilinear or layer weight are not written;
 *   taps outside a layer are dropped.
 * - Per pixel, fragments are ordered by ascending (z, point index) and the
 *   first K are kept (Sec. 3.2 and Sec. 3.6, K = 16 in the paper).  With
 *   coarse-layer inclusion (TP_COARSE_LAYERS) a pixel's list also holds the
 *   fragments of the coarser pixels that contain it (a point's two layers
 *   then follow each other, the finer first).
 * - The projection and everything that decides an integer (culling, layer
 *   pair, taps, order) is evaluated in IEEE float32 in this fixed order, with
 *   no fused multiply-add: Xc = ((R0 X + R1 Y) + R2 Z) + t0 (likewise Yc, Zc),
 *   x = (fx Xc)/Zc + cx, y = (fy Yc)/Zc + cy, s = (fx s_w)/Zc,
 *   u = x 2^-L - 0.5, j0 = floor(u).
 *
 * Layouts
 * -------
 * - pos [n][3] float32, size_w [n], opacity [n] float32.
 * - desc [n][D] float32 or bfloat16 (tp_config.desc_dtype), row-major.
 * - point records [n][4] float32: (x, y, z, s) of each point, all zero for a
 *   culled point.
 * - pyramid [P][D] float32: layer L occupies rows
 *   [layer_offsets[L], layer_offsets[L+1]), each layer row-major (row k,
 *   column j).  P = tp_pyramid_pixels(...).
 * - kept [P][K] uint32 point indices of the kept fragments in blend order,
 *   0xFFFFFFFF past n_kept; n_kept [P] uint8; t_final [P] float32 is the
 *   transmittance left after the kept fragments; n_frag [P] uint32 is the
 *   number of candidate fragments of the pixel before the K cap.
 *
 * Sizes: n < 2^27 points (and n x views < 2^29 for batches of views: the
 * tile offsets are 32-bit), 1 <= n_layers <= 16, K in {4, 8, 16, 32},
 * 1 <= D <= 64, width and height in [1, 32768], tile_w * tile_h <= 1024 (a
 * tile whose CTA does not fit the kernel's registers returns TP_ERR_UNSUPPORTED).
 */
#ifndef TRIPS_H
#define TRIPS_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define TP_API __attribute__((visibility("default")))
#else
#define TP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t. */
typedef struct CUstream_st *tp_stream_t;

typedef enum {
    TP_OK = 0,
    TP_ERR_INVALID_ARG = 1, /* null pointer, bad size or config (host check) */
    TP_ERR_CAPACITY = 2,    /* workspace too small for the frame's tile lists */
    TP_ERR_NONFINITE = 3,   /* a point had a non-finite input or s_w < 0; it was culled */
    TP_ERR_TIMEOUT = 4,     /* a bounded device wait gave up (no current kernel waits on the device) */
    TP_ERR_CUDA = 5,        /* a CUDA runtime call or launch failed */
    TP_ERR_UNSUPPORTED = 6, /* valid but not supported by this build (e.g. K) */
    TP_ERR_BOUNDS = 7       /* checking build only: a kernel computed an out-of-range index */
} tp_status;

/* Bits of the device status word (tp_get_status).  TP_FLAG_BOUNDS is set
 * only by the checking build (libtrips_debug.so, compiled with TP_DEBUG),
 * whose kernels test every list, pyramid, workspace and shared-memory index
 * they compute and skip an out-of-range access instead of making it. */
#define TP_FLAG_NONFINITE 0x1u
#define TP_FLAG_CAPACITY 0x2u
#define TP_FLAG_TIMEOUT 0x4u
#define TP_FLAG_BOUNDS 0x8u

/* Pinhole camera; R is row-major world->camera, X_c = R X_w + t. */
typedef struct {
    float fx, fy, cx, cy;
    float R[9];
    float t[3];
    float znear;
    int32_t width, height;
} tp_camera;

enum { TP_F32 = 0, TP_BF16 = 1 };
enum { TP_STORE_LISTS = 0, TP_RECOMPUTE = 1 };

typedef struct {
    int32_t n_layers;   /* pyramid layers n (the paper uses 4-8, Tab. "layers_num") */
    int32_t K;          /* per-pixel list cap (16 in the paper, Sec. 3.2) */
    int32_t desc_dim;   /* descriptor width D (4 in the paper, Tab. "feature_num") */
    float eps;          /* minimum sub-pixel layer weight (0.25, Eq. 5) */
    int32_t desc_dtype; /* TP_F32 or TP_BF16 */
    int32_t mode;       /* TP_STORE_LISTS or TP_RECOMPUTE (see tp_splat_backward) */
    int32_t tile_w;     /* screen tile of the binning and blend kernels, in pixels */
    int32_t tile_h;     /*   of each layer; 0 = the default 16 x 8 */
    int32_t flags;      /* TP_COARSE_LAYERS | TP_GRADS_ZEROED, or 0 */
} tp_config;

/*
 * tp_config.flags.  TP_COARSE_LAYERS: coarse-layer inclusion (the paper
 * includes points from coarser layers during blending, in the usual way, so
 * that occlusion holds across large differences in point density; Sec. 3.6,
 * Implementation Details).  The list of pixel (L, j, k) then also holds, for
 * every coarser layer L' > L, the fragments of the layer-L' pixel that
 * contains it, (j >> (L'-L), k >> (L'-L)), each with its own weight gamma
 * (Eq. 3-5 at its own layer), ordered with the pixel's own fragments by
 * (depth, point index, layer); the first K are blended (Eq. 6-7) and the
 * gradients flow to every kept instance.  Supported with TP_RECOMPUTE
 * backward passes (tp_splat_backward returns TP_ERR_UNSUPPORTED for stored
 * lists, whose point indices do not say which layer's fragment was kept).
 */
#define TP_COARSE_LAYERS 0x1

/*
 * tp_config.flags.  TP_GRADS_ZEROED: the backward calls take their gradient
 * buffers as already zero (the caller cleared them, for example on another
 * stream while the forward kernels run, ordered before the call) and only
 * add to them; without it they clear the buffers first on `stream`.
 */
#define TP_GRADS_ZEROED 0x2

/*
 * Number of pyramid pixels P = sum_L W_L H_L.  If layer_offsets is not NULL
 * (host, [n_layers + 1]) it receives the first pyramid row of each layer and
 * P at the end.  Returns -1 on bad arguments.
 */
TP_API int64_t tp_pyramid_pixels(const tp_camera *cam, int32_t n_layers, int64_t *layer_offsets);

/*
 * Bytes of workspace a frame needs.  entry_capacity is the number of
 * (point, tile) pairs the tile lists can hold; <= 0 selects 8 n, which can
 * never overflow (a point touches at most 2 x 2 tiles in each of its two
 * layers).  Returns -1 on bad arguments.  The workspace must be 256-byte
 * aligned.
 */
TP_API int64_t tp_workspace_bytes(const tp_config *cfg, const tp_camera *cam, int64_t n_points, int64_t entry_capacity);

/*
 * Collect stage (Sec. 3.1 Eq. 2, Sec. 3.6 first stage): project each point,
 * cull it (Z_c <= znear, non-finite input, s_w < 0), compute its screen size
 * and layer pair, and count the (point, tile) pairs of every screen tile.
 *   pos [n][3], size_w [n] (device, read)
 *   records [n][4] (device, written): (x, y, z, s), zeros when culled
 *   ws, ws_bytes: workspace (device); this call resets its status word.
 * Non-finite inputs set TP_FLAG_NONFINITE; the point is culled and the frame
 * still renders.
 */
TP_API tp_status tp_project(const tp_config *cfg, const tp_camera *cam, int64_t n, const float *pos, const float *size_w,
                     float *records, void *ws, int64_t ws_bytes, tp_stream_t stream);

/*
 * Offset scan and splatting stages (Sec. 3.6): exclusive scan of the tile
 * counts, then every point writes its fragment key (z, i) and its payload
 * (x, y, s, alpha) into the list of each screen tile its 2x2x2 splat
 * touches (24 bytes per entry, in the workspace).  Needs tp_project of the
 * same frame first.
 *   records [n][4] (device, read; from tp_project), opacity [n] (device, read)
 * If the lists exceed the workspace's entry capacity, TP_FLAG_CAPACITY is set
 * and the frame's outputs are not valid; the splatting, blend and backward
 * kernels of that frame then skip their work.
 */
TP_API tp_status tp_splat_forward(const tp_config *cfg, const tp_camera *cam, int64_t n, const float *records,
                                  const float *opacity, void *ws, int64_t ws_bytes, tp_stream_t stream);

/*
 * Sort-and-accumulate stage (Sec. 3.2 Eq. 6-7, Sec. 3.6): for every pyramid
 * pixel, the K smallest (z, index) fragments in order, blended front to back:
 *   C = sum_m T_m gamma_m tau_m,  T_m = prod_{i<m} (1 - gamma_i),
 *   gamma = beta iota alpha (Eq. 3).
 * The fragments come from the workspace's tile lists (tp_splat_forward);
 * each kept fragment's opacity gamma is evaluated again from its point's
 * record and opacity (the same float32 operations as the lists use).
 * The call also leaves each pixel's largest kept key in the workspace, for a
 * TP_RECOMPUTE backward pass.
 *   records [n][4] (device, read; from tp_project, 16-byte aligned),
 *   opacity [n] (device, read), desc [n][D] (device, read)
 *   pyramid [P][D] (device, written; every pixel)
 *   kept [P][K], n_kept [P], t_final [P], n_frag [P] (device, written;
 *   each may be NULL).  kept and n_kept are what tp_splat_backward reads in
 *   TP_STORE_LISTS mode.
 */
TP_API tp_status tp_blend(const tp_config *cfg, const tp_camera *cam, int64_t n, const float *records,
                          const float *opacity, const void *desc, float *pyramid, uint32_t *kept, uint8_t *n_kept,
                          float *t_final, uint32_t *n_frag, void *ws, int64_t ws_bytes, tp_stream_t stream);

/*
 * Backward pass (Sec. 3.6 "for the backwards pass, the sorted per-pixel lists
 * are stored"; the paper optimises positions, sizes and descriptors,
 * Sec. 3.5).  Given G = dL/dpyramid [P][D] (device), writes
 *   grad_pos [n][3], grad_size_w [n], grad_opacity [n], grad_desc [n][D]
 * (device float32, overwritten; every entry, zero where a point has no kept
 * fragment).  With grad_size_w == NULL the position and size gradients are
 * packed: grad_pos is [n][4] rows (dL/dX, dL/dY, dL/dZ, dL/ds_w), 16-byte
 * aligned, and each kept fragment adds to its point's row with one 16-byte
 * atomic instead of four scalar ones (the same for the batch calls).  With kept and n_kept (TP_STORE_LISTS) the per-pixel lists come
 * from tp_blend.  With kept == NULL (TP_RECOMPUTE) the lists are rebuilt from
 * the workspace's tile lists and the per-pixel largest kept key that
 * tp_blend leaves in the workspace (8 bytes per pixel); the workspace must
 * still hold this frame's tp_splat_forward and tp_blend results.  The adjoint of one pixel runs back to front:
 *   R_M = 0,  dL/dgamma_m = T_m (G.tau_m - R_m),
 *   R_{m-1} = gamma_m G.tau_m + (1 - gamma_m) R_m,  dL/dtau_m = T_m gamma_m G,
 * and chains through gamma = beta iota alpha to alpha, the screen position
 * (x, y), the screen size s, and from there to X_w and s_w.
 */
TP_API tp_status tp_splat_backward(const tp_config *cfg, const tp_camera *cam, int64_t n, const float *records,
                            const float *opacity, const void *desc, const uint32_t *kept, const uint8_t *n_kept,
                            const float *grad_pyramid, float *grad_pos, float *grad_size_w, float *grad_opacity,
                            float *grad_desc, void *ws, int64_t ws_bytes, tp_stream_t stream);

/*
 * Camera adjoint (the paper optimises camera poses and intrinsics along with
 * the points: Sec. 3 pipeline figure, Sec. 3.5).  The camera enters only
 * through each point's screen position and size (Eq. 2), so its gradient
 * follows from the point gradients of one view's backward pass:
 *   dL/dX_c = (R^T)^-1 grad_pos,  Gx = dL/dX_c[0] Z_c/fx,  Gy = dL/dX_c[1] Z_c/fy,
 *   Gs = grad_size_w Z_c/fx  (the point's summed dL/dx, dL/dy, dL/ds);
 *   dL/dfx = sum Gx (x-cx)/fx + Gs s/fx,  dL/dfy = sum Gy (y-cy)/fy,
 *   dL/dcx = sum Gx,  dL/dcy = sum Gy,  dL/dt = sum dL/dX_c,
 *   dL/dR[r][c] = sum dL/dX_c[r] X_w[c]   (sums over the visible points).
 *   pos [n][3], records [n][4] (this view's tp_project output, 16-byte
 *   aligned), grad_pos [n][3], grad_size_w [n]: device, read (grad_size_w
 *   NULL: grad_pos is the packed [n][4] layout of tp_splat_backward).  The point
 *   gradients must come from a backward pass of this view alone (the batched
 *   backward sums the views' gradients).
 *   grad_camera [16] (device, float64, overwritten): dL/d(fx, fy, cx, cy,
 *   R[0..8] row-major, t[0..2]) -- the order of tp_camera's fields.
 * R must be invertible (TP_ERR_INVALID_ARG otherwise); for a rotation
 * (R^T)^-1 = R.
 */
TP_API tp_status tp_camera_backward(const tp_camera *cam, int64_t n, const float *pos, const float *records,
                                    const float *grad_pos, const float *grad_size_w, double *grad_camera,
                                    tp_stream_t stream);

/*
 * Pyramid merge (the decoder's layer merge, Sec. 3.3: every layer but the
 * finest is upsampled bilinearly and merged with the next finer one), in its
 * fixed form without trained weights -- a sum:
 *   M_{n-1} = P_{n-1},   M_L = P_L + up2(M_{L+1}),
 * where up2 samples layer L+1 at the centres of layer L's pixels: pixel j of
 * layer L reads layer L+1 at r = max((j + 0.5)/2 - 0.5, 0) with taps
 * floor(r), min(floor(r) + 1, W_{L+1} - 1) and weights 1 - (r - floor r),
 * r - floor r (the same along y).
 *   pyramid [P][D] (device, read), merged [P][D] (device, written): merged
 *   layer L is M_L in the pyramid layout, so rows [0, W H) are the merged
 *   full-resolution image.  merged may be the pyramid itself (in place).
 * tp_merge_backward: from dL/d(image) grad_image [W H][D] (device), writes
 *   grad_pyramid [P][D] = dL/dP (dL/dP_L = dL/dM_L, dL/dM_{L+1} =
 *   up2^T dL/dM_L).  grad_image may be grad_pyramid's first rows.
 * 1 <= D <= 64.  tp_merge out of place on up to 2^23 values of layer 0
 * (W H D) is one kernel launch (each CTA merges a 32 x 32 tile of the image
 * and the coarser pixels above it, recomputing a one-pixel halo); larger or
 * in place, and tp_merge_backward, one launch per layer.  Both forms give the
 * same bits.
 */
TP_API tp_status tp_merge(const tp_camera *cam, int32_t n_layers, int32_t D, const float *pyramid, float *merged,
                          tp_stream_t stream);

TP_API tp_status tp_merge_backward(const tp_camera *cam, int32_t n_layers, int32_t D, const float *grad_image,
                                   float *grad_pyramid, tp_stream_t stream);

/*
 * Point-size initialisation (Sec. 3.6): size_w[i] = the mean distance from
 * point i to its 4 nearest other points (exact, float32 distances).  A
 * point's own index is never its neighbour; duplicates at distance 0 are.
 * With fewer than 5 finite points the mean runs over the others (0 for one
 * point); points with a non-finite coordinate are nobody's neighbour and get
 * size 0.  Coordinates are expected below 1e18 in magnitude.
 *   pos [n][3] (device, read), size_w [n] (device, written).
 *   ws: device workspace of tp_init_sizes_workspace_bytes(n) bytes, 256-byte
 *   aligned (about 32 n + 8 T bytes, T the power of two >= 2 n).
 * Method: hashed uniform grids of cell c_m = c0 8^m, m = 0..5 (c0 = box
 * extent / (8 max(64, 4 n^(1/3)))), each filled by a counting sort by a
 * locality-preserving cell hash; each point searches rings of cells around
 * its own until its 4th distance is within the searched radius, moving to
 * the next coarser grid after 3 rings (the last grid covers the whole box).
 * All on the device; no host synchronisation.
 */
TP_API int64_t tp_init_sizes_workspace_bytes(int64_t n_points);

TP_API tp_status tp_init_point_sizes(int64_t n, const float *pos, float *size_w, void *ws, int64_t ws_bytes,
                                     tp_stream_t stream);

/*
 * Spatial order of a point cloud (a one-time relabeling of the points; not a
 * step of the render path, and the paper has no counterpart).  The render
 * kernels touch a point's data at every stage -- its tile counters and
 * tile-list appends, its descriptor row, its gradient rows -- and the points
 * that meet in one screen tile are neighbours in space; stored along a
 * space-filling curve they share cache lines and DRAM pages.  A caller that
 * owns the cloud's storage can relabel it once (and again after large
 * position updates); every result is the same up to the relabeling, except
 * that fragments at exactly equal depth are ordered by the new indices.
 *
 * tp_spatial_order: perm [n] (device, uint32, written) lists the point
 *   indices sorted stably by the Morton code of each point's cell in a
 *   1024^3 grid over the bounding box of the finite points: with
 *   lo = the box minimum, e = its largest side and s = 1023 / e (float32),
 *   the cell coordinate along each axis is q = clamp((int)((p - lo) * s),
 *   0, 1023) in float32 (0 for a box of one position), and the code
 *   interleaves the bits of qx, qy, qz, x in the lowest bit of each triple.
 *   Points with a non-finite coordinate come last.  pos [n][3] (device).
 *   ws: device workspace of tp_spatial_order_workspace_bytes(n) bytes,
 *   256-byte aligned (about 16 n bytes).  n < 2^31.
 * tp_permute_rows: dst row k = src row perm[k] for k < n, rows of row_bytes
 *   bytes (a multiple of 4); src, dst (device, 4-byte aligned, distinct),
 *   perm [n] (device).  Apply it to every per-point array (positions, sizes,
 *   opacities, descriptors) with the same perm.
 */
TP_API int64_t tp_spatial_order_workspace_bytes(int64_t n_points);

TP_API tp_status tp_spatial_order(int64_t n, const float *pos, uint32_t *perm, void *ws, int64_t ws_bytes,
                                  tp_stream_t stream);

TP_API tp_status tp_permute_rows(int64_t n, int32_t row_bytes, const void *src, const uint32_t *perm, void *dst,
                                 tp_stream_t stream);

/* ------------------------------------------------------------------------
 * Batches of views.  Up to TP_MAX_VIEWS cameras (each with its own
 * resolution and screen tile) are rendered from one point cloud by the same
 * launches: each of the four stages is one kernel launch over all views, so
 * a whole frame batch can be captured as one CUDA graph.  The calls mirror
 * the single-view ones with these differences:
 *   cams [n_views] (host): one camera per view; all views share cfg.
 *   tiles [n_views][2] (host, nullable): tile_w, tile_h of each view (0 = the
 *     default); NULL uses cfg->tile_w / cfg->tile_h for every view.
 *   records [n_views][n][4]: the projection of every point in every view.
 *   pyramid, grad_pyramid [P_total][D], kept [P_total][K] ...: the views'
 *     pyramids concatenated in view order; view v starts at row
 *     view_offsets[v] of tp_batch_pixels.
 *   grad_* [n][...]: the gradient of the sum of the views' losses.
 * The workspace is sized by tp_batch_workspace_bytes (default capacity
 * 8 n n_views tile-list entries, which cannot overflow).
 * ------------------------------------------------------------------------ */
#define TP_MAX_VIEWS 16

TP_API int64_t tp_batch_pixels(const tp_camera *cams, int32_t n_views, int32_t n_layers, int64_t *view_offsets);

TP_API int64_t tp_batch_workspace_bytes(const tp_config *cfg, const tp_camera *cams, const int32_t *tiles,
                                        int32_t n_views, int64_t n_points, int64_t entry_capacity);

TP_API tp_status tp_batch_project(const tp_config *cfg, const tp_camera *cams, const int32_t *tiles, int32_t n_views,
                                  int64_t n, const float *pos, const float *size_w, float *records, void *ws,
                                  int64_t ws_bytes, tp_stream_t stream);

TP_API tp_status tp_batch_splat_forward(const tp_config *cfg, const tp_camera *cams, const int32_t *tiles,
                                        int32_t n_views, int64_t n, const float *records, const float *opacity,
                                        void *ws, int64_t ws_bytes, tp_stream_t stream);

TP_API tp_status tp_batch_blend(const tp_config *cfg, const tp_camera *cams, const int32_t *tiles, int32_t n_views,
                                int64_t n, const float *records, const float *opacity, const void *desc,
                                float *pyramid, uint32_t *kept, uint8_t *n_kept, float *t_final, uint32_t *n_frag,
                                void *ws, int64_t ws_bytes, tp_stream_t stream);

TP_API tp_status tp_batch_splat_backward(const tp_config *cfg, const tp_camera *cams, const int32_t *tiles,
                                         int32_t n_views, int64_t n, const float *records, const float *opacity,
                                         const void *desc, const uint32_t *kept, const uint8_t *n_kept,
                                         const float *grad_pyramid, float *grad_pos, float *grad_size_w,
                                         float *grad_opacity, float *grad_desc, void *ws, int64_t ws_bytes,
                                         tp_stream_t stream);

/*
 * Clears the gradient buffers of tp_splat_backward (the same layouts: with
 * grad_size_w NULL grad_pos is the packed [n][4] form) on `stream`, so that a
 * caller can clear them on a second stream while the forward kernels run and
 * call the backward with TP_GRADS_ZEROED.  cudaMemsetAsync only; no kernel.
 */
TP_API tp_status tp_zero_gradients(const tp_config *cfg, int64_t n, float *grad_pos, float *grad_size_w,
                                   float *grad_opacity, float *grad_desc, tp_stream_t stream);

/*
 * The batch backward (lists recomputed) that also returns the gradient of
 * every view's camera, as the paper optimises all training cameras with the
 * points (Sec. 3.5).  Point gradients are those of tp_batch_splat_backward
 * (summed over the views); grad_cameras [n_views][16] (device, float64,
 * written) holds per view dL/d(fx, fy, cx, cy, R[0..8], t[0..2]) in the
 * order and meaning of tp_camera_backward, accumulated per fragment from its
 * screen-space gradient (dL/dx, dL/dy, dL/ds), its camera-space gradient
 * dL/dX_c and the point's world position pos [n][3] (device, read):
 *   dL/dfx += (dL/dx (x - cx) + dL/ds s) / fx,  dL/dfy += dL/dy (y - cy) / fy,
 *   dL/dcx += dL/dx,  dL/dcy += dL/dy,  dL/dt += dL/dX_c,
 *   dL/dR[a][b] += dL/dX_c[a] X_w[b].
 * Float32 per-CTA sums, added into float64 with one atomic each.  Returns
 * TP_ERR_INVALID_ARG when grad_cameras or (for n > 0) pos is NULL.
 */
TP_API tp_status tp_batch_splat_backward_cameras(const tp_config *cfg, const tp_camera *cams, const int32_t *tiles,
                                                 int32_t n_views, int64_t n, const float *pos, const float *records,
                                                 const float *opacity, const void *desc, const float *grad_pyramid,
                                                 float *grad_pos, float *grad_size_w, float *grad_opacity,
                                                 float *grad_desc, double *grad_cameras, void *ws, int64_t ws_bytes,
                                                 tp_stream_t stream);

/* ------------------------------------------------------------------------
 * Forward render with no caller workspace.  The paper has no counterpart:
 * this entry point exists for callers that may not allocate device memory
 * at run time, such as a plug-in inside a host application that owns every
 * CUDA allocation through its own pool, or a real-time frame loop that must
 * not call cudaMalloc (which can synchronise the whole device) once it runs.
 *
 * It enqueues the same kernels as tp_project, tp_splat_forward and tp_blend
 * (without kept lists or statistics) on `stream`, but keeps the frame's
 * workspace in an array that the library reserves in device memory: a fixed
 * TP_STATIC_WORKSPACE_BYTES on every GPU that loads the library, held until
 * the process exits.  The call itself allocates and frees nothing.
 *
 *   records [n][4] (device, 16-byte aligned): written as by tp_project.
 *   pyramid [P][D] (device): written as by tp_blend.
 *   device_flags (device, nullable): if not NULL, one uint32 that receives
 *     the frame's TP_FLAG_* bits (stream-ordered; no host synchronisation).
 *
 * - Returns TP_ERR_CAPACITY, before enqueuing anything, when the frame's
 *   workspace, tp_workspace_bytes(cfg, cam, n, 0), is larger than
 *   TP_STATIC_WORKSPACE_BYTES: about 190 bytes per point plus 8 per pyramid
 *   pixel, so some 340 thousand points at 256 x 256 with 4 layers and 200
 *   thousand at 1920 x 1080 with 8 layers.
 * - The first call on a device, with that device current, loads the
 *   library's module on that device (with CUDA's default lazy loading this
 *   is when the array is reserved, so that first call can fail for lack of
 *   device memory, as TP_ERR_CUDA) and looks up the array's device address
 *   once; make that first call at start-up, before any stream capture
 *   begins.  A cudaDeviceReset voids the looked-up address: call nothing
 *   here on a device after resetting it.
 * - Every call on a device uses the same array, and each call starts by
 *   resetting the parts that must begin at zero.  Calls that can run at the
 *   same time on the GPU (unordered streams, several host threads) race on
 *   the array and corrupt each other's results: order them on one stream.
 * ------------------------------------------------------------------------ */
#define TP_STATIC_WORKSPACE_BYTES ((int64_t)64 << 20)

TP_API tp_status tp_render_forward_static(const tp_config *cfg, const tp_camera *cam, int64_t n, const float *pos,
                                          const float *size_w, const float *opacity, const void *desc,
                                          float *records, float *pyramid, uint32_t *device_flags,
                                          tp_stream_t stream);

/*
 * Synchronises `stream` and reads the workspace's device status word into
 * *device_flags (host; TP_FLAG_* bits).  Returns TP_ERR_CAPACITY,
 * TP_ERR_BOUNDS, TP_ERR_TIMEOUT or TP_ERR_NONFINITE for the first set bit in that order,
 * TP_OK if none is set.
 */
TP_API tp_status tp_get_status(const void *ws, tp_stream_t stream, int32_t *device_flags);

/* Static string for a status code. */
TP_API const char *tp_status_string(tp_status status);

/* Library version, 100 * major + minor. */
TP_API int32_t tp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TRIPS_H */
