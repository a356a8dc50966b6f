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

typedef void* dg_stream;      /* cudaStream_t */

/* Pinhole camera.  viewmat = world-to-camera [R | t], row-major 3x4:
 * x_cam = R x_world + t; x right, y down, z forward.  Pixel coordinates
 * u = fx x/z + cx, v = fy y/z + cy.  width, height: image size in pixels. */
typedef struct dg_camera {
    float viewmat[12];
    float fx, fy, cx, cy;
    int32_t width, height;
} dg_camera;

/* Rasterizer options.  tile: tile edge B in pixels (16); sh_degree: 0..3;
 * near_plane: Gaussians with camera z <= near_plane are culled (0.2);
 * eps2d: dilation added to the 2D covariance diagonal, px^2 (0.3);
 * bg: background colour composited with the final transmittance. */
typedef struct dg_raster_opts {
    int32_t tile;
    int32_t sh_degree;
    float near_plane;
    float eps2d;
    float bg[3];
} dg_raster_opts;

/* Thread-local message of the last failing call on this thread ("" if none). */
DG_API const char* dg_last_error(void);
/* ABI version of this header (incremented on incompatible changes). */
DG_API int32_t dg_abi_version(void);
/* Number of CUDA kernels this library has launched in this process (host
 * counter, for launch accounting in benchmarks). */
DG_API int64_t dg_kernel_launches(void);

/* ---------------------------------------------------------------------- */
/* Projection (EWA splatting of Sec. 3, "2D Gaussian splatted to the image
 * plane", and the SH colour of the colour coefficients c_i).
 * In:  params [59][stride] planar float32, P Gaussians, *cam, *opts (host).
 * Out: feat   [P][12] float32, 16-byte aligned, per Gaussian
 *              (u, v, A, B | C, o, r, g | b, 0, 0, 0): pixel mean, conic
 *              (A, B, C) = inverse 2D covariance (power = -A dx^2/2 - C dy^2/2
 *              - B dx dy), opacity, colour;
 *      depth  [P] camera-space z;
 *      radius [P] int32, 0 when culled (near plane, singular, empty rect);
 *      tiles  [P] int32, number of tiles in the rect (0 when culled);
 *      clamp  [P] uint8, bit c set when colour channel c was clamped at 0.
 * Errors: DG_ERR_ARG for null pointers, P < 0, stride < P, sh_degree
 * outside 0..3, tile < 1, non-positive image size or focal length. */
DG_API dg_status dg_project(const float* params, int64_t stride, int64_t P, const dg_camera* cam,
                     const dg_raster_opts* opts, float* feat, float* depth, int32_t* radius,
                     int32_t* tiles, uint8_t* clamp, dg_stream stream);

/* ---------------------------------------------------------------------- */
/* Tile binning and ordering (the tile-based "GPU-friendly rendering
 * pipeline" of Sec. 2 that evaluates Eq. 1 front to back).  The pair list of
 * a view holds one (tile, Gaussian) entry per tile in each Gaussian's rect,
 * ordered by (tile id = ty * TX + tx, depth as float bits, Gaussian index).
 *
 * Bytes of device workspace needed to bin P Gaussians into at most M_cap
 * pairs over n_tiles tiles (host call, no device work). */
DG_API size_t dg_bin_workspace_size(int64_t P, int64_t M_cap, int32_t n_tiles);

/* Phase 1: orders the visible Gaussians by (depth bits, index) and computes
 * each one's first pair slot.  Writes the total pair count M to *M_out
 * (device int64).  The caller reads M (or checks it against its capacity)
 * before phase 2.  ws/ws_bytes: workspace from dg_bin_workspace_size with
 * the same P; its content carries over to dg_bin_sort. */
DG_API dg_status dg_bin_count(const float* depth, const int32_t* tiles, int64_t P, void* ws,
                       size_t ws_bytes, int64_t M_cap, int32_t n_tiles, int64_t* M_out,
                       dg_stream stream);

/* Phase 2: emits the pairs in depth order and stably sorts them by tile.
 * Out: gid    [M_cap] uint32, Gaussian index of each sorted pair;
 *      ranges [2 * n_tiles] uint32, [start, end) of each tile's list;
 *      status (device int32): 0, or DG_ERR_CAPACITY when M > M_cap, in which
 *              case gid is untouched and every range is empty.
 * feat/radius are dg_project's outputs for the same P. */
DG_API dg_status dg_bin_sort(const float* feat, const int32_t* radius, int64_t P, const dg_camera* cam,
                      int32_t tile, void* ws, size_t ws_bytes, int64_t M_cap, uint32_t* gid,
                      uint32_t* ranges, int32_t* status, dg_stream stream);

/* ---------------------------------------------------------------------- */
/* Forward compositing, Eq. 1: per pixel, front to back over its tile's list,
 * C = sum_i T_i alpha_i c_i + T_N bg.
 * Out: img [3][H][W] float32 (planar RGB), T_final [H][W] float32,
 *      last [H][W] int32 = 1-based list position of the last blended Gaussian
 *      (0 if none), examined [H][W] int32 (nullable) = list entries visited
 *      including the one that stopped compositing. */
DG_API dg_status dg_render_fwd(const float* feat, const uint32_t* gid, const uint32_t* ranges,
                        const dg_camera* cam, const dg_raster_opts* opts, float* img,
                        float* T_final, int32_t* last, int32_t* examined, dg_stream stream);

/* Adjoint of Eq. 1 ("fully differentiable", Sec. 3).  Recomputes each
 * pixel's transmittance back to front from T_final and last (no per-pair
 * state), with dC/dc_j = alpha_j T_j and
 * dC/dalpha_j = T_j c_j - S_j / (1 - alpha_j), S_j the colour behind j
 * including T_N bg.
 * In:  dL_dimg [3][H][W] float32.
 * Out: grad2d [P][12] float32, 16-byte aligned, zeroed by this call, then
 *      accumulated: (dL/du, dL/dv, dL/dA, dL/dB | dL/dC, dL/do, dL/dr, dL/dg |
 *      dL/db, 0, 0, 0). */
DG_API dg_status dg_render_bwd(const float* feat, const uint32_t* gid, const uint32_t* ranges,
                        const dg_camera* cam, const dg_raster_opts* opts, const float* T_final,
                        const int32_t* last, const float* dL_dimg, int64_t P, float* grad2d,
                        dg_stream stream);

/* Adjoint of dg_project: from grad2d to the gradient of every parameter row.
 * Out: grads [59][stride] planar float32, overwritten for Gaussians 0..P-1
 *      (zero for culled ones; rows above the SH degree are zero). */
DG_API dg_status dg_project_bwd(const float* params, int64_t stride, int64_t P, const dg_camera* cam,
                         const dg_raster_opts* opts, const int32_t* radius, const uint8_t* clamp,
                         const float* grad2d, float* grads, dg_stream stream);

/* ---------------------------------------------------------------------- */
/* L1 photometric loss of the 3DGS backbone the paper keeps (Sec. 5):
 * loss = mean |img - target| over n values; dL_dimg = sign(img - target)/n
 * (0 at a tie).  loss: one device float32, written.  ws: workspace of
 * dg_loss_workspace_size(n) bytes. */
DG_API size_t dg_loss_workspace_size(int64_t n);
DG_API dg_status dg_loss_l1(const float* img, const float* target, int64_t n, float* dL_dimg,
                     float* loss, void* ws, size_t ws_bytes, dg_stream stream);

/* L1 loss for callers that cannot allocate device memory (the paper has no
 * counterpart).  Some callers cannot call cudaMalloc: code inside graph-node or
 * stream host callbacks, plugins whose host application owns every device
 * allocation, loops that forbid allocator calls after start-up.  Same result as
 * dg_loss_l1, but the per-block partial sums live in a fixed 4 KiB device array
 * inside this library (DG_L1_NOALLOC_BLOCKS floats), so no workspace is passed
 * and nothing is allocated.  n <= DG_L1_NOALLOC_MAX_N (2^28 values: at most
 * 1024 values summed per thread), else DG_ERR_ARG.  The first call on a device
 * looks up the array's device address with that device current (make that
 * first call before any stream capture).  Every call shares the array: calls
 * that overlap on the GPU (unordered streams) race on it. */
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

#ifdef __cplusplus
}
#endif
#endif /* DASHGS_H */
