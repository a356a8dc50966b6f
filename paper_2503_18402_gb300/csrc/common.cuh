// common.cuh -- shared device-side definitions of the CUDA rasterizer library.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/dashgs.h"

namespace dg {

// Thresholds of the compositing rule (fixed readings of the ABI, see dashgs.h):
// alpha clamp, skip threshold and early-stop transmittance.
constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTMin = 1e-4f;
constexpr float kFrustumGuard = 1.3f;
constexpr float kGuardPx = 1073741824.0f;  // 2^30: footprints or centres beyond are culled

// Camera in registers: world-to-camera rotation (row-major), translation,
// intrinsics and image size.
struct Cam {
    float r[9];
    float t[3];
    float fx, fy, cx, cy;
    int w, h;
};

__host__ __device__ inline Cam make_cam(const dg_camera& c)
{
    Cam k;
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) k.r[3 * i + j] = c.viewmat[4 * i + j];
        k.t[i] = c.viewmat[4 * i + 3];
    }
    k.fx = c.fx; k.fy = c.fy; k.cx = c.cx; k.cy = c.cy;
    k.w = c.width; k.h = c.height;
    return k;
}

// Camera centre in world coordinates, -R^T t, with explicit fused multiply-adds
// so that host and device give the same bits.
__host__ __device__ inline void cam_centre(const Cam& c, float out[3])
{
    for (int k = 0; k < 3; ++k) out[k] = -fmaf(c.r[k], c.t[0], fmaf(c.r[3 + k], c.t[1], c.r[6 + k] * c.t[2]));
}

// Tile rect [x0, x1) x [y0, y1) of a footprint centred at (u, v) with integer
// radius r: floor((u -/+ r)/B) computed exactly as the floor of (floor(u) -/+ r) / B,
// clamped to [0, TX] (x1 after adding 1).  The numerator is clamped to
// [-1, TX B] first, which changes no clamped result (a negative numerator
// gives a negative quotient, one from TX B on a quotient from TX on), so the
// division runs in 32 bits instead of a 64-bit division and remainder.
struct Rect { int x0, y0, x1, y1; };

__device__ inline int floor_div_clamped(long long a, int B, int hi)  // B > 0; -1 for a < 0
{
    if (a < 0) return -1;
    const long long lim = (long long)hi * B;
    const long long c = a < lim ? a : lim;
    return c <= 0x7fffffffLL ? (int)c / B : (int)(c / B);
}

__device__ inline Rect tile_rect(float u, float v, int r, int B, int TX, int TY)
{
    const long long fu = (long long)floorf(u), fv = (long long)floorf(v);
    const int x0 = floor_div_clamped(fu - r, B, TX), x1 = floor_div_clamped(fu + r, B, TX) + 1;
    const int y0 = floor_div_clamped(fv - r, B, TY), y1 = floor_div_clamped(fv + r, B, TY) + 1;
    Rect q;
    q.x0 = x0 < 0 ? 0 : (x0 > TX ? TX : x0);
    q.x1 = x1 < 0 ? 0 : (x1 > TX ? TX : x1);
    q.y0 = y0 < 0 ? 0 : (y0 > TY ? TY : y0);
    q.y1 = y1 < 0 ? 0 : (y1 > TY ? TY : y1);
    return q;
}

// Adam hyper-parameters of one step (the public dg_adam_hparams): per-row
// learning rate, betas, bias corrections 1 - b1^t and sqrt(1 - b2^t), epsilon.
using AdamHp = dg_adam_hparams;

// Per-row constants of the update: step size lr / (1 - b1^t) and 1 / sqrt(1 - b2^t).
struct AdamRowK { float step, inv_bc2; };
__device__ __forceinline__ AdamRowK adam_row(float lr, const AdamHp& h)
{
    return AdamRowK{lr / h.bc1, 1.f / h.bc2_sqrt};
}

// One Adam update of a scalar parameter (shared by the standalone and the fused
// kernels so that both give the same bits):
//   m <- b1 m + (1 - b1) g,  v <- b2 v + (1 - b2) g^2,
//   p <- p - step * m / (sqrt(v) / sqrt(1 - b2^t) + eps).
// The square root and the division use the hardware approximations (a few ulp;
// the update is a ratio of float32 moment estimates, far coarser than that):
// the exact-rounded forms cost most of the kernel's issue slots.
__device__ __forceinline__ void adam_update(float& p, float& m, float& v, float g, const AdamRowK& r,
                                            const AdamHp& h)
{
    m = fmaf(h.beta1, m, (1.f - h.beta1) * g);
    v = fmaf(h.beta2, v, (1.f - h.beta2) * (g * g));
    const float sv = v >= 1e-30f ? v * rsqrtf(v) : sqrtf(v);  // exact path for tiny (also subnormal) v
    p -= __fdividef(r.step * m, fmaf(sv, r.inv_bc2, h.eps));
}

// Smallest value of A dx^2 + 2 B dx dy + C dy^2 over dx in [dxl, dxh], dy in [dyl, dyh]
// (positive-definite form; 0 when the box contains the origin), less a bound
// on its float32 rounding (a multiple of the magnitude of the summed terms).
__device__ inline float quad_min_box(float A, float B, float C, float dxl, float dxh, float dyl, float dyh)
{
    if (dxl <= 0.f && dxh >= 0.f && dyl <= 0.f && dyh >= 0.f) return 0.f;
    float best = 3.4e38f;
    // edges dx = const: minimiser dy* = -B dx / C, clamped; then dy = const
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        float dx, dy;
        // (the minimiser only has to be near the edge's minimum: the form is
        // flat there, so the fast division changes f by a second-order amount)
        if (e < 2) {
            dx = e ? dxh : dxl;
            dy = fminf(fmaxf(__fdividef(-B * dx, C), dyl), dyh);
        } else {
            dy = (e & 1) ? dyh : dyl;
            dx = fminf(fmaxf(__fdividef(-B * dy, A), dxl), dxh);
        }
        const float f = A * dx * dx + 2.f * B * dx * dy + C * dy * dy;
        const float mag = A * dx * dx + 2.f * fabsf(B * dx * dy) + C * dy * dy;
        best = fminf(best, f - 1e-5f * mag);
    }
    return best;
}

// True when no pixel centre of the rectangle [px0, px1] x [py0, py1] can give
// the Gaussian of record (a, b) = (u, v, A, B | C, o, ...) an alpha >= 1/255.
// The render passes drop such entries per tile or pixel block when they stage
// a batch.
__device__ inline bool tile_skip(const float4& a, const float4& b, float px0, float px1, float py0, float py1)
{
    const float o = b.y;
    if (!(o >= kAlphaMin)) return true;  // alpha <= o < 1/255 everywhere
    const float fmin = quad_min_box(a.z, a.w, b.x, a.x - px1, a.x - px0, a.y - py1, a.y - py0);
    // alpha = o exp(-fmin/2) < 1/255  <=>  fmin > 2 ln(255 o); 0.02 absorbs the
    // per-pixel rounding of the power and of exp
    return fmin > 2.f * __logf(255.f * o) + 0.02f;
}

// Two float32 values in one 64-bit register for the packed float32 operations
// of sm_100 and later (PTX .f32x2): one instruction does the operation on both
// halves, each rounded exactly as the scalar operation (fma: one rounding), so
// packed and scalar code give the same bits.  Low half = first value.
using f32x2 = unsigned long long;

__device__ __forceinline__ f32x2 f2_pack(float lo, float hi)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ void f2_unpack(f32x2 v, float& lo, float& hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

__device__ __forceinline__ f32x2 f2_fma(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ f32x2 f2_mul(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f32x2 f2_add(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// The two floats at x (8-byte aligned) as one packed register.
__device__ __forceinline__ f32x2 f2_ld(const float& x) { return *(const f32x2*)&x; }

}  // namespace dg

// Host-side error reporting shared by the C-ABI entry points.
void dg_set_error(const char* fmt, ...);
// Counts kernel launches issued by this library (read by dg_kernel_launches).
void dg_note_launch(int n = 1);
dg_status dg_check_launch(const char* what);
// Adam hyper-parameters of step `step` (bias corrections in FP64, rounded once).
dg::AdamHp dg_adam_hp(const float* lr, float beta1, float beta2, float eps, int64_t step);
