/*
 * dashgs.h -- C ABI of the GB300 (sm_103a) differentiable tile rasterizer
 * for DashGaussian's scheduled 3DGS optimisation (arXiv 2503.18402).
 *
 * The paper's problem statement (Sec. 3 "Preliminary"): given posed images,
 * optimise P Gaussians {p_i, Sigma_i, o_i, c_i} by rendering them with Eq. 1
 * and back-propagating a photometric loss.  Its method (Sec. 4) schedules the
 * rendering resolution and the primitive count around that rasterizer.  The
 * calls below are the steps of one optimisation iteration:
 *   dg_project -> dg_bin_count -> dg_bin_sort -> dg_render_fwd ->
 *   dg_loss_l1 -> dg_render_bwd -> dg_project_bwd -> dg_adam_step
 * plus the schedule (dg_schedule_*) and densification (dg_densify_*) calls.
 *
 * Conventions for every call:
 *   - All array arguments are DEVICE pointers owned by the caller unless the
 *     comment says "host".  The library allocates no device memory: scratch
 *     is a caller-provided workspace whose size a *_workspace_size query
 *     returns.
 *   - Every call is asynchronous on `stream` (a cudaStream_t; NULL = the
 *     legacy default stream) unless stated otherwise.
 *   - Return value: DG_OK (0) or a negative dg_status; the call then has
 *     launched nothing, and dg_last_error() returns a thread-local message.
 *     Device-side conditions that cannot be known at launch time (pair
 *     capacity overflow) are reported through device status words.
 *   - Gaussian parameters are float32, planar: row r of Gaussian i is at
 *     params[r * stride + i], stride >= P, rows:
 *        0..2  mean p (world)          3..5  log scale (Sigma = R S S^T R^T,
 *        6..9  quaternion (w,x,y,z),         S = diag(exp(log scale)))
 *        10    opacity logit (o = sigmoid)
 *        11..58 SH coefficients, 11 + 3*k + channel, k = l*l + l + m, l <= 3
 *   - Readings where the paper is silent (fixed in this ABI): near plane and
 *     2D dilation from dg_raster_opts; Jacobian frustum guard 1.3 x half-FOV
 *     tangent; radius ceil(3 sqrt(lambda_max)); pixel (x, y) sampled at
 *     (x + 0.5, y + 0.5); tile rect [floor((u-r)/B), floor((u+r)/B)+1)
 *     clipped to the grid; alpha = min(0.99, o exp(power)), Gaussians with
 *     power > 0 or alpha < 1/255 skipped, compositing stops before a
 *     Gaussian that would take T below 1e-4; colour = SH + 0.5 clamped at 0.
 */
#ifndef DASHGS_H
#define DASHGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Every entry point is exported from the shared library (built with hidden
 * default visibility). */
#if defined(__GNUC__)
#define DG_API __attribute__((visibility("default")))
#else
#define DG_API
#endif

typedef int32_t dg_status;
#define DG_OK 0
#define DG_ERR_ARG (-1)       /* invalid argument (null pointer, size, alignment) */
#define DG_ERR_CAPACITY (-2)  /* caller buffer or workspace too small */
#define DG_ERR_TIMEOUT (-3)   /* a bounded device wait gave up */
#define DG_ERR_CUDA (-4)      /* a CUDA launch or runtime call failed */

#define DG_NPARAM 59
#define DG_FEAT_FLOATS 12     /* floats per projected record, see dg_project */
#define DG_MAX_VIEWS 16       /* views per batched call */

typedef void* dg_stream;      /* cudaStream_t */

/* Pinhole camera.  viewmat = world-to-camera [R | t], row-major 3x4:
 * x_cam = R x_world + t; x right, y down, z forward.  Pixel coordinates
 * u = fx x/z + cx, v = fy y/z + cy.  width, height: image size in pixels. */
typedef struct dg_camera {
    float viewmat[12];
    float fx, fy, cx, cy;
    int32_t width, height;
} dg_camera;

/* Rasterizer options.  tile: tile edge B in pixels (16; the render kernels
 * take 8 or 16); sh_degree: 0..3; near_plane: Gaussians with camera z <=
 * near_plane are culled (0.2); eps2d: dilation added to the 2D covariance
 * diagonal, px^2 (0.3); bg: background colour composited with the final
 * transmittance; pixels_per_thread: pixels each render thread owns (1, 2 or
 * 4 with tile 16, 1 or 2 with tile 8; 0 = the library's default per pass);
 * split_len: list splitting of the render passes: a tile whose sorted list is longer than L
 * entries is composited as ceil(n/L) chunks in parallel (Eq. 1 composes over
 * chunks through the transmittance product); 0 = automatic (split when the
 * batch has fewer tiles than twice the resident CTAs, L = max(64, M / resident
 * CTAs)), > 0 = always split with that L (raised where the workspace needs
 * it), < 0 = never split.
 * pixels_per_thread and split_len change the launch shape only, not the
 * result beyond float rounding order.  record: format of the records the
 * render calls read: 0 = the float32 records of dg_project, 1 = the
 * mixed-precision records of dg_pack_records (float16 conic and opacity,
 * bfloat16 colour; transmittance, colour sums and gradients stay float32).
 * mip2d: 0 = the eps2d dilation; > 0 = Mip-Splatting's 2D filter (a backbone
 * variant of the supplementary): the 2D covariance gets + mip2d I instead of
 * + eps2d I and the opacity of the record is scaled by
 * sqrt(det(S2) / det(S2 + mip2d I)) (0 when det(S2) <= 0); dg_project_bwd
 * differentiates the factor.
 * tight_bins: 0 = each Gaussian's pair list covers every tile of its rect
 * (Sec. 2's tile binning as written); 1 = dg_project leaves out the tiles of
 * a rect of at most 8 x 8 tiles (radius at most 4 tiles) whose pixel centres
 * all lie outside the ellipse where the Gaussian's alpha reaches 1/255 (the
 * ellipse's x-interval on each tile row, in closed form, widened beyond
 * float32 rounding), for the record format opts->record names (render with
 * the same format).  Such an entry is skipped by every pixel of that tile in
 * both compositing passes, so images, transmittances and gradients are the
 * same; the lists are shorter (list positions in `last` count the entries of
 * the shorter lists). */
typedef struct dg_raster_opts {
    int32_t tile;
    int32_t sh_degree;
    float near_plane;
    float eps2d;
    float bg[3];
    int32_t pixels_per_thread;
    int32_t split_len;
    int32_t record;
    float mip2d;
    int32_t tight_bins;
} dg_raster_opts;

/* Thread-local message of the last failing call on this thread ("" if none). */
DG_API const char* dg_last_error(void);
/* ABI version of this header (incremented on incompatible changes). */
DG_API int32_t dg_abi_version(void);
/* Number of CUDA kernels this library has launched in this process (host
 * counter, for launch accounting in benchmarks). */
DG_API int64_t dg_kernel_launches(void);

/* ---------------------------------------------------------------------- */
/* Several views per call.  The projection, binning, render and adjoint calls
 * take a host array of n_views (1..DG_MAX_VIEWS) cameras.  A "record" is a
 * (view, Gaussian) pair with index r = v * P + i; per-record arrays are
 * view-major [n_views][P].  Tiles of all views share one range table: view v's
 * tiles are ids toff[v] .. toff[v+1]-1 with toff the running sum of
 * ceil(W_v/B) * ceil(H_v/B).  Per-pixel arrays concatenate the views: images
 * [v][3][H_v][W_v] from element 3 * poff[v], T/last from poff[v], poff the
 * running sum of W_v * H_v.
 * cams_dev (projection and its adjoint): nullable device copy of the same
 * n_views cameras.  When given, the kernels read each camera's pose and
 * intrinsics from it when they run (so a call captured once in a CUDA graph
 * can be replayed with new cameras written to that buffer); the image sizes
 * and tile grids are always those of the host array. */

/* Projection (EWA splatting of Sec. 3, "2D Gaussian splatted to the image
 * plane", and the SH colour of the colour coefficients c_i).
 * In:  params [59][stride] planar float32, P Gaussians, cams[n_views], *opts (host).
 * Out (per record r = v * P + i):
 *      feat   [P][12] float32, 16-byte aligned, per record
 *              (u, v, A, B | C, o, r, g | b, m0, m1, 0): pixel mean, conic
 *              (A, B, C) = inverse 2D covariance (power = -A dx^2/2 - C dy^2/2
 *              - B dx dy), opacity, colour; m0, m1 (uint32 bits): with
 *              opts->tight_bins, the low and high words of the 64-bit mask of
 *              the rect's tiles kept in the pair list (bit 8 ry + rx for tile
 *              (x0 + rx, y0 + ry)), 0 for "every tile of the rect" (always
 *              without tight_bins, and for rects wider or taller than 8 tiles);
 *      depth  [P] camera-space z;
 *      radius [P] int32, 0 when culled (near plane, singular, empty rect);
 *      tiles  [P] int32, number of pair-list tiles: the tiles in the rect, or
 *              the kept tiles of the mask (0 when culled);
 *      clamp  [P] uint8, bit c set when colour channel c was clamped at 0.
 * Errors: DG_ERR_ARG for null pointers, P < 0, stride < P, sh_degree
 * outside 0..3, tile < 1, non-positive image size or focal length. */
DG_API dg_status dg_project(const float* params, int64_t stride, int64_t P, const dg_camera* cams,
                     const dg_camera* cams_dev, int32_t n_views, const dg_raster_opts* opts, float* feat,
                     float* depth, int32_t* radius, int32_t* tiles, uint8_t* clamp, dg_stream stream);

/* ---------------------------------------------------------------------- */
/* Tile binning and ordering (the tile-based "GPU-friendly rendering
 * pipeline" of Sec. 2 that evaluates Eq. 1 front to back).  The pair list of
 * a view holds one (tile, Gaussian) entry per tile in each Gaussian's rect
 * (per kept tile with opts->tight_bins),
 * ordered by (tile id = ty * TX + tx, depth as float bits, Gaussian index).
 *
 * Bytes of device workspace needed to bin P Gaussians in n_views views into
 * at most M_cap pairs (host call, no device work). */
DG_API size_t dg_bin_workspace_size(int64_t P, int32_t n_views, int64_t M_cap);

/* Phase 1: orders the visible records by (view, depth bits, index) and
 * computes each one's first pair slot.  Writes the total pair count M to
 * *M_out (device int64).  The caller reads M (or checks it against its
 * capacity) before phase 2.  ws/ws_bytes: workspace from
 * dg_bin_workspace_size with the same P and n_views; its content carries
 * over to dg_bin_sort (a workspace laid out for another M_cap is fine as
 * long as phase 1 ran in it). */
DG_API dg_status dg_bin_count(const float* depth, const int32_t* tiles, int64_t P, int32_t n_views, void* ws,
                       size_t ws_bytes, int64_t M_cap, int64_t* M_out, dg_stream stream);

/* Phase 2: emits the pairs in (view, depth) order and stably sorts them by
 * global tile id.  A record whose feat holds a tile mask (opts->tight_bins
 * of dg_project) gets pairs only for the mask's tiles.
 * Out: gid    [M_cap] uint32, record index v * P + i of each sorted pair;
 *      ranges [2 * total tiles] uint32, [start, end) of each tile's list;
 *      status (device int32): 0, or DG_ERR_CAPACITY when M > M_cap, in which
 *              case gid is untouched and every range is empty, or
 *              DG_ERR_TIMEOUT when a bounded wait between thread blocks of
 *              phase 1 gave up (lists not valid; does not happen when the
 *              device runs the launch to completion).
 * feat/radius are dg_project's outputs for the same P and cameras. */
DG_API dg_status dg_bin_sort(const float* feat, const int32_t* radius, int64_t P, const dg_camera* cams,
                      int32_t n_views, int32_t tile, void* ws, size_t ws_bytes, int64_t M_cap, uint32_t* gid,
                      uint32_t* ranges, int32_t* status, dg_stream stream);

/* Diagnostic: runs, in one device thread, the bounded look-back wait that the
 * depth-order passes of dg_bin_count use between thread blocks (decoupled
 * look-back, Merrill & Garland 2016; the paper's rasterizer needs the sort of
 * Sec. 3, the wait is this library's), so that its give-up path can be tested
 * without starving a real pass.
 * In:  look [tile][stride] uint64 look-back words (device): top two bits 0 =
 *      not published, 1 = the tile's own count, 2 = the inclusive prefix up
 *      to that tile, low 62 bits the count; the wait sums column `digit` of
 *      tiles tile-1, tile-2, ... down to the nearest inclusive word;
 *      max_polls: re-reads of an unpublished word before giving up
 *      (0..2^20; the passes use 2^20, about a second).
 * Out: *sum (device uint64): the counts summed (partial after a give-up);
 *      *err (device int32): 0, or DG_ERR_TIMEOUT when the wait gave up.
 * Errors: DG_ERR_ARG for null pointers, tile < 0, stride < 1, digit outside
 * 0..stride-1, max_polls outside its range. */
DG_API dg_status dg_lookback_probe(const uint64_t* look, int64_t tile, int32_t stride, int32_t digit,
                                   int32_t max_polls, uint64_t* sum, int32_t* err, dg_stream stream);

/* Mixed-precision records for the render calls (opts->record = 1): each
 * float32 record of dg_project becomes 24 bytes, u and v float32 (pixel
 * positions need the full mantissa at 1600 px), conic A, B, C and opacity
 * float16 (round to nearest), colour r, g, b bfloat16 (round to nearest),
 * two bytes of zero padding.  packed: n_records * 24 bytes, 8-byte aligned.
 * Binning keeps reading the float32 records, so the pair lists are those of
 * the float32 path. */
#define DG_PACKED_RECORD_BYTES 24
DG_API dg_status dg_pack_records(const float* feat, int64_t n_records, void* packed, dg_stream stream);

/* ---------------------------------------------------------------------- */
/* Render workspace for these cameras and options and up to M_cap pairs: work
 * counters of the persistent launches, unless opts->split_len < 0 the split
 * plan and per-pixel chunk state (about 40 MB plus 40 bytes per tile), and one
 * byte per pair in which the forward records whether some pixel of the pair's
 * tile blended it (the backward then stages only those entries; pairs beyond
 * the bytes a smaller workspace holds fall back to the tile test).  Returns 0
 * for invalid arguments.  The workspace must be 256-byte aligned.
 * dg_render_bwd must get the workspace, cameras, tile and split_len of the
 * dg_render_fwd of the same batch, unmodified in between. */
DG_API size_t dg_render_workspace_size(const dg_camera* cams, int32_t n_views, const dg_raster_opts* opts,
                                       int64_t M_cap);

/* Forward compositing, Eq. 1: per pixel, front to back over its tile's list,
 * C = sum_i T_i alpha_i c_i + T_N bg.  One persistent launch covers every
 * tile of every view (work items taken from a counter in ws).
 * Out: img [3][H][W] float32 (planar RGB), T_final [H][W] float32,
 *      last [H][W] int32 = 1-based list position of the last blended Gaussian
 *      (0 if none), examined [H][W] int32 (nullable) = list entries visited
 *      including the one that stopped compositing, blended [H][W] int32
 *      (nullable) = entries blended into the pixel. */
DG_API dg_status dg_render_fwd(const float* feat, const uint32_t* gid, const uint32_t* ranges,
                        const dg_camera* cams, int32_t n_views, const dg_raster_opts* opts, float* img,
                        float* T_final, int32_t* last, int32_t* examined, int32_t* blended, void* ws,
                        size_t ws_bytes, dg_stream stream);

/* Adjoint of Eq. 1 ("fully differentiable", Sec. 3).  Recomputes each
 * pixel's transmittance back to front from T_final and last (no per-pair
 * state), with dC/dc_j = alpha_j T_j and
 * dC/dalpha_j = T_j c_j - S_j / (1 - alpha_j), S_j the colour behind j
 * including T_N bg.
 * In:  dL_dimg, laid out like the images.
 * Out: grad2d [n_records][12] float32 (n_records = n_views * P), 16-byte
 *      aligned, zeroed by this call, then accumulated per record:
 *      (dL/du, dL/dv, dL/dA, dL/dB | dL/dC, dL/do, dL/dr, dL/dg | dL/db, 0, 0, 0). */
DG_API dg_status dg_render_bwd(const float* feat, const uint32_t* gid, const uint32_t* ranges,
                        const dg_camera* cams, int32_t n_views, const dg_raster_opts* opts, const float* T_final,
                        const int32_t* last, const float* dL_dimg, int64_t n_records, float* grad2d, void* ws,
                        size_t ws_bytes, dg_stream stream);

/* Adjoint of dg_project: from grad2d (all views) to the gradient of every
 * parameter row, summed over the views.
 * Out: grads [59][stride] planar float32, overwritten for Gaussians 0..P-1
 *      (zero where culled in every view; rows above the SH degree are zero). */
DG_API dg_status dg_project_bwd(const float* params, int64_t stride, int64_t P, const dg_camera* cams,
                         const dg_camera* cams_dev, int32_t n_views, const dg_raster_opts* opts,
                         const int32_t* radius, const uint8_t* clamp, const float* grad2d, float* grads,
                         dg_stream stream);

/* dg_project_bwd fused with dg_adam_step: the gradient of each parameter row
 * goes straight into the Adam update of that row (same arithmetic and result
 * as the two calls in sequence), so it is never stored and reloaded and the
 * parameters are read once (1.47 kB instead of 2.18 kB of HBM traffic per
 * Gaussian).  grads: nullable; when given, the gradient is also written there.
 * params, m, v: planar [59][stride], updated in place; lr: host float[59]. */
DG_API dg_status dg_project_bwd_adam(float* params, int64_t stride, int64_t P, const dg_camera* cams,
                                     const dg_camera* cams_dev, int32_t n_views, const dg_raster_opts* opts,
                                     const int32_t* radius, const uint8_t* clamp, const float* grad2d, float* grads,
                                     float* m, float* v, const float* lr, float beta1, float beta2, float eps,
                                     int64_t step, dg_stream stream);

/* ---------------------------------------------------------------------- */
/* L1 photometric loss of the 3DGS backbone the paper keeps (Sec. 5):
 * loss = mean |img - target| over n values; dL_dimg = sign(img - target)/n
 * (0 at a tie).  loss: one device float32, written.  ws: workspace of
 * dg_loss_workspace_size(n) bytes. */
DG_API size_t dg_loss_workspace_size(int64_t n);
DG_API dg_status dg_loss_l1(const float* img, const float* target, int64_t n, float* dL_dimg,
                     float* loss, void* ws, size_t ws_bytes, dg_stream stream);

/* Training loss of the 3DGS backbone the paper keeps unchanged (Sec. 5):
 * L_v = (1 - lambda) mean|img - target| + lambda (1 - SSIM) per view, SSIM of
 * Wang et al. 2004 (11 x 11 Gaussian window, sigma 1.5, C1 = 0.01^2,
 * C2 = 0.03^2, zero padding, mean over pixels and channels); the backbone
 * uses lambda = 0.2.
 * In:  img, target: n_views planar images [3][H_v][W_v] concatenated (the
 *      render layout); wh: host int32 [n_views][2] = (W_v, H_v).
 * Out: dL_dimg (same layout) = gradient of the mean over views of L_v;
 *      loss: device float32 [n_views + 1] = L_0 .. L_{n-1}, then the mean.
 * ws: dg_ssim_workspace_size(wh, n_views) bytes (36 bytes per pixel plus
 * per-block sums); 0 is returned for invalid sizes. */
DG_API size_t dg_ssim_workspace_size(const int32_t* wh, int32_t n_views);
DG_API dg_status dg_loss_l1_dssim(const float* img, const float* target, const int32_t* wh, int32_t n_views,
                                  float lambda, float* dL_dimg, float* loss, void* ws, size_t ws_bytes,
                                  dg_stream stream);

/* Mean squared error of two arrays (held-out PSNR = -10 log10(mse) for images
 * in [0, 1]; Sec. 5 "Metrics").  ws: dg_loss_workspace_size(n) bytes. */
DG_API dg_status dg_mse(const float* a, const float* b, int64_t n, float* mse, void* ws, size_t ws_bytes,
                        dg_stream stream);

/* Opacity reset of the 3DGS backbone (kept unchanged by the paper, Sec. 5):
 * opacity logit <- min(logit, logit(max_opacity)) and its Adam moments set
 * to zero, for Gaussians 0..P-1 of the planar arrays. */
DG_API dg_status dg_opacity_reset(float* params, float* m, float* v, int64_t stride, int64_t P, float max_opacity,
                                  dg_stream stream);

/* L1 loss for callers that cannot allocate device memory (the paper has no
 * counterpart).  Some callers cannot call cudaMalloc: plugins whose host
 * application owns every device allocation, and real-time loops that forbid
 * allocator calls after start-up.  Call it from an ordinary host thread (never
 * from a host function or callback enqueued on a stream, where no CUDA call is
 * allowed).  Same result as
 * dg_loss_l1, but the per-block partial sums live in a fixed 4 KiB device array
 * inside this library (DG_L1_NOALLOC_BLOCKS floats), so no workspace is passed
 * and nothing is allocated.  n <= DG_L1_NOALLOC_MAX_N (2^28 values: at most
 * 1024 values summed per thread), else DG_ERR_ARG.  The first call on a device
 * (and again after that device's context was destroyed and recreated) looks up
 * the array's device address with that device current; make that first call
 * before any stream capture: if `stream` is capturing and no address is known
 * yet for the current context, the call returns DG_ERR_ARG and launches
 * nothing.  Every call shares the array: calls queued on one stream run in
 * order, calls that overlap on the GPU (unordered streams) race on it. */
#define DG_L1_NOALLOC_BLOCKS 1024
#define DG_L1_NOALLOC_MAX_N (1024LL * 256LL * 1024LL)
DG_API dg_status dg_loss_l1_noalloc(const float* img, const float* target, int64_t n, float* dL_dimg,
                                    float* loss, dg_stream stream);

/* Adam (the optimiser of the 3DGS backbone, supplementary Sec. "Equipping
 * DashGaussian to Backbones"), float32, on all P Gaussians of the planar
 * arrays params/grads/m/v [59][stride].  lr: host array of 59 per-row
 * learning rates; step >= 1 is the 1-based step count used in the bias
 * corrections. */
DG_API dg_status dg_adam_step(float* params, const float* grads, float* m, float* v, int64_t stride,
                       int64_t P, const float* lr, float beta1, float beta2, float eps,
                       int64_t step, dg_stream stream);

/* Sparse Adam of the Taming-3DGS backbone (supplementary, "Equipping
 * DashGaussian to Backbones"): the Adam update of dg_adam_step applied only to
 * the Gaussians whose visible[i] != 0; the others keep their parameters and
 * their moments (no decay).  The bias corrections use the global step.
 * visible: device uint8 [P], e.g. from dg_visibility. */
DG_API dg_status dg_sparse_adam_step(float* params, const float* grads, float* m, float* v, int64_t stride,
                                     int64_t P, const float* lr, float beta1, float beta2, float eps,
                                     int64_t step, const uint8_t* visible, dg_stream stream);

/* visible[i] = 1 if Gaussian i has a non-zero radius in any of the n_views
 * views of a dg_project call (radius: [n_views][P] int32), else 0. */
DG_API dg_status dg_visibility(const int32_t* radius, int64_t P, int32_t n_views, uint8_t* visible,
                               dg_stream stream);

/* Adam hyper-parameters of one step, in the layout the kernels read: per-row
 * learning rates, betas, bias corrections bc1 = 1 - beta1^step and
 * bc2_sqrt = sqrt(1 - beta2^step) (computed in FP64, rounded once), eps. */
typedef struct dg_adam_hparams {
    float lr[DG_NPARAM];
    float beta1, beta2;
    float bc1, bc2_sqrt;
    float eps;
} dg_adam_hparams;

/* Host: fills *out for step `step` (>= 1) exactly as dg_adam_step uses it. */
DG_API dg_status dg_adam_hparams_fill(const float* lr, float beta1, float beta2, float eps, int64_t step,
                                      dg_adam_hparams* out);

/* dg_adam_step with the hyper-parameters read from device memory at execution
 * time (hp_dev: one dg_adam_hparams), for a step captured once in a CUDA graph
 * and replayed with a new learning rate and step count.  skip_if: nullable
 * device int32; when it holds a non-zero value (e.g. the binning status of the
 * same step reporting a pair-list overflow) the update is skipped. */
DG_API dg_status dg_adam_step_dev(float* params, const float* grads, float* m, float* v, int64_t stride,
                                  int64_t P, const dg_adam_hparams* hp_dev, const int32_t* skip_if,
                                  dg_stream stream);

/* dg_project_bwd_adam with the hyper-parameters read from device memory when
 * the kernel runs (hp_dev: one dg_adam_hparams, e.g. filled by
 * dg_adam_hparams_fill and copied) and the update skipped when *skip_if != 0
 * (skip_if: nullable device int32, e.g. dg_bin_sort's status), for a step
 * captured once in a CUDA graph and replayed (cf. dg_adam_step_dev).  The
 * adjoint (and grads, when given) is computed either way. */
DG_API dg_status dg_project_bwd_adam_dev(float* params, int64_t stride, int64_t P, const dg_camera* cams,
                                         const dg_camera* cams_dev, int32_t n_views, const dg_raster_opts* opts,
                                         const int32_t* radius, const uint8_t* clamp, const float* grad2d,
                                         float* grads, float* m, float* v, const dg_adam_hparams* hp_dev,
                                         const int32_t* skip_if, dg_stream stream);

/* ---------------------------------------------------------------------- */
/* Scheduled densification (supplementary "Densification of DashGaussian"):
 * prune first (N'), then clone or split the Gaussians that meet the 3DGS
 * condition (mean view-space positional gradient >= grad_thresh) and have a
 * top-(P_i - N') score; P_i comes from dg_schedule_densify (Eq. 4/5).
 * Selected Gaussians whose largest scale exceeds percent_dense * extent are
 * split into two samples (scales / 1.6, means drawn with caller-provided
 * standard normal noise), the others are cloned.  All integer decisions are
 * float32 comparisons against float32 thresholds (logit of min_opacity, log
 * of the scale limits).  Ties in the top-k go to the lower index; survivors
 * keep their order, new Gaussians follow in index order of their source and
 * start with zero Adam moments. */
typedef struct dg_densify_opts {
    float grad_thresh;        /* 0.0002 */
    float min_opacity;        /* 0.005: pruned below */
    float percent_dense;      /* 0.01 */
    float extent;             /* scene extent */
    float max_screen_radius;  /* > 0: also prune when the largest radius seen exceeds it */
    float max_world_scale;    /* > 0: also prune when the largest scale exceeds it */
} dg_densify_opts;

/* After rendering: for each view v and Gaussian with radius[v*P+i] > 0,
 * grad_accum += |(dL/du W_v/2, dL/dv H_v/2)| (the NDC-space gradient norm),
 * denom += 1, max_radius = max(max_radius, radius).  grad_accum, denom,
 * max_radius: [P] float32. */
DG_API dg_status dg_densify_stats(const float* grad2d, const int32_t* radius, int64_t P, const dg_camera* cams,
                                  int32_t n_views, float* grad_accum, float* denom, float* max_radius,
                                  dg_stream stream);
DG_API size_t dg_densify_workspace_size(int64_t P);
/* Phase 1: prune/candidate/split flags into ws; counts (device int64[2]) =
 * {N' kept, candidates}.  The caller reads the counts (Eq. 5's P_add is the
 * candidate count) before phase 2 with the same ws. */
DG_API dg_status dg_densify_mark(const float* params, int64_t stride, int64_t P, const float* grad_accum,
                                 const float* denom, const float* max_radius, const dg_densify_opts* opts,
                                 void* ws, size_t ws_bytes, int64_t* counts, dg_stream stream);
/* Phase 2: selects min(n_cand, budget) candidates, writes survivors and new
 * Gaussians to dst (planar [59][dst_stride], dst_stride >= P + min(n_cand,
 * budget)) and their Adam moments; noise [min(n_cand,budget)][2][3] standard
 * normals for the j-th selected Gaussian (index order); *P_out (device int64)
 * = N' + number selected.  Sources and destinations must not overlap. */
DG_API dg_status dg_densify_apply(const float* params, const float* m, const float* v, int64_t stride, int64_t P,
                                  int64_t n_cand, int64_t budget, const float* noise, void* ws, size_t ws_bytes,
                                  float* dst_params, float* dst_m, float* dst_v, int64_t dst_stride,
                                  int64_t* P_out, dg_stream stream);

/* ---------------------------------------------------------------------- */
/* Resolution schedule (Sec. 4.1-4.2, Eq. 2, supplementary Eq. 6/7, floor
 * modulation of Sec. 5) and primitive schedule (Sec. 4.3, Eq. 4/5).
 *
 * Spectrum of the training views (once per scene, FP64 sums on the GPU):
 *   for each view: dg_spectrum_accumulate(view [3][H][W] float32, ...) adds
 *   sum over RGB of |DFT2(view_c)| into acc [H][W] float64 (caller zeroes acc
 *   before the first view); then dg_spectrum_finalize divides by n_views,
 *   moves DC to (H/2, W/2) into shifted [H][W] float64 and writes the summed-
 *   area table sat [(H+1)][(W+1)] float64 (sat[y][x] = sum of shifted over
 *   rows < y, columns < x).  ws: dg_spectrum_workspace_size(H, W) bytes. */
DG_API size_t dg_spectrum_workspace_size(int32_t H, int32_t W);
DG_API dg_status dg_spectrum_accumulate(const float* view, int32_t H, int32_t W, double* acc, void* ws,
                                        size_t ws_bytes, dg_stream stream);
DG_API dg_status dg_spectrum_finalize(const double* acc, int32_t n_views, int32_t H, int32_t W,
                                      double* shifted, double* sat, dg_stream stream);

/* Anti-aliased ground-truth downsampling (supplementary "Ground Truth
 * Downsampling"), read as area resampling with exact coverage weights:
 * src [C][H][W] -> dst [C][h][w], h <= H, w <= W. */
DG_API dg_status dg_downsample_area(const float* src, int32_t C, int32_t H, int32_t W, float* dst,
                                    int32_t h, int32_t w, dg_stream stream);

#define DG_SCHED_MAX_LEVELS 64

/* Host-side schedule parameters.  S: total iterations; a: X(F_rm) = X(F)/a
 * (4); m: number of levels (<= 0: ceil(r_m)); gamma, eta: Eq. 5 (0.98, 1);
 * P_init: initial primitive count; P_cap: hard cap on the primitive target
 * (<= 0: none); lr_pos_init/final: position learning rate held, then decayed
 * from the first full-resolution iteration to S. */
typedef struct dg_sched_params {
    int64_t S;
    double a;
    int32_t m;
    double gamma, eta;
    double P_init, P_cap;
    double lr_pos_init, lr_pos_final;
} dg_sched_params;

/* Schedule state (host struct).  X[i], r[i], s[i] for i = 0..m: level
 * significance, downsampling factor and anchor iteration (s[0] = S, s[m] = 0);
 * k_full: first iteration with floor(r) = 1; P_fin: Eq. 5 state. */
typedef struct dg_schedule {
    dg_sched_params p;
    int32_t H, W, m;
    double X0, Xm, r_m;
    double X[DG_SCHED_MAX_LEVELS + 1], r[DG_SCHED_MAX_LEVELS + 1], s[DG_SCHED_MAX_LEVELS + 1];
    int64_t k_full;
    double P_fin;
} dg_schedule;

/* Per-iteration outputs: continuous and floored factor, render size
 * (floor(H/r_mod), floor(W/r_mod)), position learning rate, Eq. 4 target. */
typedef struct dg_sched_out {
    double r_cont;
    int32_t r_mod, height, width;
    double lr_pos;
    double P_target;
} dg_sched_out;

/* Builds the schedule from the HOST copy of the summed-area table (host call,
 * no device work): X(r) = centred (floor(H/r) x floor(W/r)) crop sum / (H W)
 * (Eq. 2 with a pixel-normalised DFT, which absorbs the 1/r^2 of Sec. 4.1);
 * r_m = inf{r : X(r) <= X(1)/a}; X_i linear between X(1) and X(1)/a;
 * r_i = inf{r : X(r) <= X_i}; s_i = S ln(X_i/X_m) / ln(X_0/X_m) (Eq. 7);
 * P_fin = 5 P_init. */
DG_API dg_status dg_schedule_init(const double* sat_host, int32_t H, int32_t W, const dg_sched_params* p,
                                  dg_schedule* out);
/* Rendering factor, size, learning rate and Eq. 4 target at `iter` (host). */
DG_API dg_status dg_schedule_step(const dg_schedule* s, int64_t iter, dg_sched_out* out);
/* Densification step: Eq. 5 update of P_fin with P_add, then as
 * dg_schedule_step (host). */
DG_API dg_status dg_schedule_densify(dg_schedule* s, int64_t iter, int64_t P_add, dg_sched_out* out);

/* The plain (unscheduled) arm as a schedule (host call): full resolution at
 * every iteration (m = 0, r = 1, k_full = 0), so dg_schedule_step returns the
 * full size and the backbone's position learning rate decaying log-linearly
 * from lr_pos_init at iteration 0 to lr_pos_final at S (3DGS backbone, kept
 * by the paper, Sec. 5 "Implementation Details"). */
DG_API dg_status dg_schedule_init_plain(int32_t H, int32_t W, const dg_sched_params* p, dg_schedule* out);

/* Number of Gaussians a densification step may add (host call).
 * s non-null (primitive schedule, Sec. 4.3): Eq. 5 with P_add = n_cand (the
 * Gaussians meeting the backbone's densification threshold), then Eq. 4's
 * target P_k at `iter`, written to *out; budget = floor(P_k) - n_keep.
 * s null (3DGS backbone): budget = n_cand (out untouched).
 * Then, with P_cap > 0, budget <= P_cap - n_keep; finally budget >= 0.
 * n_keep: Gaussians left after pruning. */
DG_API dg_status dg_densify_budget(dg_schedule* s, int64_t iter, int64_t n_keep, int64_t n_cand, int64_t P_cap,
                                   int64_t* budget, dg_sched_out* out);

/* Camera of a render at width x height of the full-resolution camera `full`
 * (host call): fx, cx scaled by width / full->width, fy, cy by height /
 * full->height (in double, rounded once to float); the pose is unchanged.
 * This is how the schedule's reduced-resolution renders (floor(H/r),
 * floor(W/r)) see the scene (Sec. 4.2). */
DG_API dg_status dg_camera_scale(const dg_camera* full, int32_t width, int32_t height, dg_camera* out);

/* Adam hyper-parameters for V views per step (host call; the paper trains one
 * view per iteration and has no counterpart): the batch-size rules of
 * Grendel-GS (Zhao et al. 2024, "On Scaling Up 3D Gaussian Splatting
 * Training"): every learning rate times sqrt(V), beta1 <- beta1^V,
 * beta2 <- beta2^V, so that one step over V views moves the parameters about
 * as far as V single-view steps.  lr: host float[59], in place. */
DG_API dg_status dg_batch_adam_scale(int32_t views_per_step, float* lr, float* beta1, float* beta2);

#ifdef __cplusplus
}
#endif
#endif /* DASHGS_H */
