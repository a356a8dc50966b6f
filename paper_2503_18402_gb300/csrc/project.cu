// project.cu -- EWA projection + SH colour (forward) and its adjoint, for one
// or several views per launch.
//
// One thread per Gaussian.  Parameters are planar [59][stride], so every row a
// warp reads is one coalesced 128-byte line.  The view-independent part (3D
// covariance from scale and rotation, SH coefficients) is computed once per
// Gaussian and kept in registers; the thread then loops over the views, so
// with V views the parameters are read once instead of V times.  Records are
// laid out view-major: record r = v * P + i, three 16-byte stores each.
//
// Forward (Sec. 3: the 3D Gaussian is splatted to a 2D Gaussian on the image
// plane; colour from the colour coefficients c_i):
//   t = R p + t_c;  Sigma = (Rq S)(Rq S)^T, S = diag(exp(log scale));
//   J = d(pinhole)/dt at t with t_x/t_z, t_y/t_z clamped to 1.3 x half-FOV;
//   Sigma2 = J R Sigma R^T J^T + eps I;  conic = Sigma2^-1;
//   radius = ceil(3 sqrt(lambda_max(Sigma2)));  colour = SH(dir) + 0.5, >= 0.
// Adjoint: per view, the 2D gradients are pulled back to dL/dt, dL/dSigma and
// the colour terms; dL/dSigma is summed over the views and pushed through
// Sigma = M M^T, M = Rq S and the quaternion normalisation once.
#include <cuda_fp16.h>

#include "common.cuh"

namespace dg {

// Real orthonormal SH up to degree 3 at a unit direction, index l*l + l + m,
// Cartesian polynomial form without the Condon-Shortley phase.
struct ShK {
    static constexpr float k0 = 0.28209479177387814f;   // 1/(2 sqrt(pi))
    static constexpr float k1 = 0.4886025119029199f;    // sqrt(3/(4 pi))
    static constexpr float k2a = 1.0925484305920792f;   // sqrt(15/pi)/2
    static constexpr float k20 = 0.31539156525252005f;  // sqrt(5/pi)/4
    static constexpr float k22 = 0.5462742152960396f;   // sqrt(15/pi)/4
    static constexpr float k33 = 0.5900435899266435f;   // sqrt(35/(2 pi))/4
    static constexpr float k32a = 2.890611442640554f;   // sqrt(105/pi)/2
    static constexpr float k31 = 0.4570457994644658f;   // sqrt(21/(2 pi))/4
    static constexpr float k30 = 0.3731763325901154f;   // sqrt(7/pi)/4
    static constexpr float k32b = 1.445305721320277f;   // sqrt(105/pi)/4
};

__device__ inline void sh_values(float x, float y, float z, float Y[16])
{
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[0] = ShK::k0;
    Y[1] = ShK::k1 * y;
    Y[2] = ShK::k1 * z;
    Y[3] = ShK::k1 * x;
    Y[4] = ShK::k2a * x * y;
    Y[5] = ShK::k2a * y * z;
    Y[6] = ShK::k20 * (3.f * zz - 1.f);
    Y[7] = ShK::k2a * x * z;
    Y[8] = ShK::k22 * (xx - yy);
    Y[9] = ShK::k33 * y * (3.f * xx - yy);
    Y[10] = ShK::k32a * x * y * z;
    Y[11] = ShK::k31 * y * (5.f * zz - 1.f);
    Y[12] = ShK::k30 * z * (5.f * zz - 3.f);
    Y[13] = ShK::k31 * x * (5.f * zz - 1.f);
    Y[14] = ShK::k32b * z * (xx - yy);
    Y[15] = ShK::k33 * x * (xx - 3.f * yy);
}

// d/d(x,y,z) of each basis polynomial above.
__device__ inline void sh_partials(float x, float y, float z, float D[16][3])
{
    const float xx = x * x, yy = y * y, zz = z * z;
#pragma unroll
    for (int k = 0; k < 16; ++k) D[k][0] = D[k][1] = D[k][2] = 0.f;
    D[1][1] = ShK::k1;
    D[2][2] = ShK::k1;
    D[3][0] = ShK::k1;
    D[4][0] = ShK::k2a * y;  D[4][1] = ShK::k2a * x;
    D[5][1] = ShK::k2a * z;  D[5][2] = ShK::k2a * y;
    D[6][2] = ShK::k20 * 6.f * z;
    D[7][0] = ShK::k2a * z;  D[7][2] = ShK::k2a * x;
    D[8][0] = ShK::k22 * 2.f * x;  D[8][1] = -ShK::k22 * 2.f * y;
    D[9][0] = ShK::k33 * 6.f * x * y;  D[9][1] = ShK::k33 * 3.f * (xx - yy);
    D[10][0] = ShK::k32a * y * z;  D[10][1] = ShK::k32a * x * z;  D[10][2] = ShK::k32a * x * y;
    D[11][1] = ShK::k31 * (5.f * zz - 1.f);  D[11][2] = ShK::k31 * 10.f * y * z;
    D[12][2] = ShK::k30 * (15.f * zz - 3.f);
    D[13][0] = ShK::k31 * (5.f * zz - 1.f);  D[13][2] = ShK::k31 * 10.f * x * z;
    D[14][0] = ShK::k32b * 2.f * x * z;  D[14][1] = -ShK::k32b * 2.f * y * z;  D[14][2] = ShK::k32b * (xx - yy);
    D[15][0] = ShK::k33 * 3.f * (xx - yy);  D[15][1] = -ShK::k33 * 6.f * x * y;
}

// View-independent part of one Gaussian.
struct G3 {
    float p[3];
    float qn[4], qinv;      // normalised quaternion and 1/|q|
    float rq[9], s[3], m[9];
    float sig[6];           // Sigma: xx xy xz yy yz zz
};

__device__ inline void gauss3d(const float* __restrict__ prm, long long stride, int i, G3& g)
{
    g.p[0] = prm[i]; g.p[1] = prm[stride + i]; g.p[2] = prm[2 * stride + i];
    const float q0 = prm[6 * stride + i], q1 = prm[7 * stride + i], q2 = prm[8 * stride + i], q3 = prm[9 * stride + i];
    g.qinv = 1.f / sqrtf(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
    const float w = q0 * g.qinv, x = q1 * g.qinv, y = q2 * g.qinv, z = q3 * g.qinv;
    g.qn[0] = w; g.qn[1] = x; g.qn[2] = y; g.qn[3] = z;
    float* R = g.rq;
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
    g.s[0] = expf(prm[3 * stride + i]);
    g.s[1] = expf(prm[4 * stride + i]);
    g.s[2] = expf(prm[5 * stride + i]);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) g.m[3 * r + c] = R[3 * r + c] * g.s[c];
    const float* M = g.m;
    g.sig[0] = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
    g.sig[1] = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
    g.sig[2] = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
    g.sig[3] = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
    g.sig[4] = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
    g.sig[5] = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
}

// One view's projection of a Gaussian.
struct Splat {
    float t[3];
    bool gx, gy;            // frustum guard active on x / y
    float lx, ly;           // signed guard value when active
    float t2[6];            // J R, 2 x 3
    float a, b, c, det;     // 2D covariance (with dilation or 2D filter) and determinant
    float A, B, C;          // conic
    float det0, comp;       // 2D filter: undilated determinant, opacity factor sqrt(det0 / det)
};

// mip2d > 0: Mip-Splatting's 2D filter, S2 + mip2d I in place of the dilation,
// with the opacity scaled by sqrt(det(S2) / det(S2 + mip2d I)); else the eps2d dilation.
__device__ inline bool splat(const G3& g, const Cam& cam, float near_plane, float eps2d, float mip2d, Splat& S)
{
    S.t[0] = cam.r[0] * g.p[0] + cam.r[1] * g.p[1] + cam.r[2] * g.p[2] + cam.t[0];
    S.t[1] = cam.r[3] * g.p[0] + cam.r[4] * g.p[1] + cam.r[5] * g.p[2] + cam.t[1];
    S.t[2] = cam.r[6] * g.p[0] + cam.r[7] * g.p[1] + cam.r[8] * g.p[2] + cam.t[2];
    if (!(S.t[2] > near_plane)) return false;
    const float tz = S.t[2];
    const float limx = kFrustumGuard * 0.5f * (float)cam.w / cam.fx;
    const float limy = kFrustumGuard * 0.5f * (float)cam.h / cam.fy;
    const float txtz = S.t[0] / tz, tytz = S.t[1] / tz;
    S.gx = txtz < -limx || txtz > limx;
    S.gy = tytz < -limy || tytz > limy;
    S.lx = txtz < 0.f ? -limx : limx;
    S.ly = tytz < 0.f ? -limy : limy;
    const float txc = S.gx ? S.lx * tz : S.t[0];
    const float tyc = S.gy ? S.ly * tz : S.t[1];
    const float j00 = cam.fx / tz, j02 = -cam.fx * txc / (tz * tz);
    const float j11 = cam.fy / tz, j12 = -cam.fy * tyc / (tz * tz);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        S.t2[c] = j00 * cam.r[c] + j02 * cam.r[6 + c];
        S.t2[3 + c] = j11 * cam.r[3 + c] + j12 * cam.r[6 + c];
    }
    // Sigma2 = T2 Sigma T2^T
    const float* sg = g.sig;
    float u0[3], u1[3];  // Sigma T2_row^T
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float* tr = S.t2 + 3 * k;
        float* u = k == 0 ? u0 : u1;
        u[0] = sg[0] * tr[0] + sg[1] * tr[1] + sg[2] * tr[2];
        u[1] = sg[1] * tr[0] + sg[3] * tr[1] + sg[4] * tr[2];
        u[2] = sg[2] * tr[0] + sg[4] * tr[1] + sg[5] * tr[2];
    }
    const float a0 = S.t2[0] * u0[0] + S.t2[1] * u0[1] + S.t2[2] * u0[2];
    S.b = S.t2[0] * u1[0] + S.t2[1] * u1[1] + S.t2[2] * u1[2];
    const float c0 = S.t2[3] * u1[0] + S.t2[4] * u1[1] + S.t2[5] * u1[2];
    const float dil = mip2d > 0.f ? mip2d : eps2d;
    S.a = a0 + dil;
    S.c = c0 + dil;
    S.det = fmaf(S.a, S.c, -S.b * S.b);
    if (!(S.det > 0.f)) return false;
    S.comp = 1.f;
    S.det0 = 0.f;
    if (mip2d > 0.f) {
        S.det0 = fmaf(a0, c0, -S.b * S.b);
        S.comp = S.det0 > 0.f ? sqrtf(S.det0 / S.det) : 0.f;
    }
    const float inv = 1.f / S.det;
    S.A = S.c * inv;
    S.B = -S.b * inv;
    S.C = S.a * inv;
    return true;
}

struct ViewSet {
    int n;
    Cam cam[DG_MAX_VIEWS];
    float campos[DG_MAX_VIEWS][3];
    int TX[DG_MAX_VIEWS], TY[DG_MAX_VIEWS];
};

// The cameras a kernel uses: the by-value set built on the host, or, when the
// caller passes a device copy of the cameras (read at execution time, e.g. on
// every replay of a captured graph), the same set rebuilt from it in shared
// memory (sizes and tile grids stay those of the host set).  Call with the
// whole block; ends with a barrier when cdev is given.
__device__ inline const ViewSet& block_views(const ViewSet& vs, const dg_camera* cdev, ViewSet* s_vs)
{
    if (!cdev) return vs;
    for (int v = threadIdx.x; v < vs.n; v += blockDim.x) {
        s_vs->cam[v] = make_cam(cdev[v]);
        s_vs->cam[v].w = vs.cam[v].w;
        s_vs->cam[v].h = vs.cam[v].h;
        cam_centre(s_vs->cam[v], s_vs->campos[v]);
        s_vs->TX[v] = vs.TX[v];
        s_vs->TY[v] = vs.TY[v];
    }
    if (threadIdx.x == 0) s_vs->n = vs.n;
    __syncthreads();
    return *s_vs;
}

// Resident 128-thread CTAs per SM requested from the compiler (a register
// bound: 5 gives 96 registers; measured 0.132 -> 0.128 ms at 2M Gaussians,
// 6 no better).
// Square root on the special-function unit (sqrt.approx: a few ulps).
__device__ inline float sqrt_approx(float x)
{
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// x as a float16 holds it (round to nearest): the conic and opacity of the
// mixed-precision records.
__device__ inline float round_f16(float x) { return __half2float(__float2half_rn(x)); }

// Tiles of the rect q where a record with pixel mean (u, v), conic (A, B, C)
// and opacity o may blend: bit 8 ry + rx for the tile (q.x0 + rx, q.y0 + ry).
// A pixel centre d from the mean blends only when f = A dx^2 + 2 B dx dy +
// C dy^2 <= 2 ln(255 o).  That ellipse meets the band of a tile row's pixel
// centres in one x-interval: its ends lie where the ellipse's rightmost
// (leftmost) point, clamped to the band, sits, with the half-width
// sqrt(det(S)/Syy (t - dy^2/Syy)) around the centre line dx = (Sxy/Syy) dy of
// the covariance S = conic^-1 (the 2x2 determinant in Kahan's fma form).  The
// threshold and the interval are widened (1e-3 relative, 0.02 absolute on f;
// 0.01 px and 1e-3 relative on x) beyond the float32 rounding of the render's
// per-pixel test: a radius of at most 4 tiles bounds the Gaussian's extent
// and so the conditioning of f (at most 3e-4 relative error there).  False
// (no mask) when the rect is wider or taller than 8 tiles or the radius r
// exceeds 4 tiles (a large Gaussian whose rect was clipped by the image).
__device__ inline bool tile_mask(float u, float v, float A, float B, float C, float o, int r, const Rect& q, int Bt,
                                 uint64_t* mask)
{
    if (q.x1 - q.x0 > 8 || q.y1 - q.y0 > 8 || r > 4 * Bt) return false;
    uint64_t m = 0;
    if (o >= kAlphaMin) {
        // (the fast log, reciprocals and square roots err by a few ulps, far
        // inside the margins)
        const float t = fmaf(2.f * __logf(255.f * o), 1.001f, 0.02f);
        const float bb = B * B;
        const float det = fmaf(A, C, -bb) - fmaf(B, B, -bb);  // A C - B^2
        const float id = __fdividef(1.f, det);                 // det(S)
        const float sa = C * id, sb = -B * id, sc = A * id;    // S = [[sa, sb], [sb, sc]]
        const float isc = __fdividef(1.f, sc);
        const float ky = sb * isc;                             // centre line dx = ky dy
        const float w2 = id * isc;                             // det(S) / Syy
        const float ry = fmaf(sqrt_approx(t * sc), 1.001f, 0.01f);  // dy half-extent of the ellipse
        const float dyr = sb * sqrt_approx(t * __fdividef(1.f, sa));  // dy of the rightmost point
        const float fb = (float)Bt, ifb = __fdividef(1.f, fb);
        for (int ty = q.y0; ty < q.y1; ++ty) {
            const float yl = fmaf((float)ty, fb, 0.5f) - v;
            const float lo = fmaxf(yl, -ry), hi = fminf(yl + (fb - 1.f), ry);
            if (lo > hi) continue;
            const float d1 = fminf(fmaxf(dyr, lo), hi), d2 = fminf(fmaxf(-dyr, lo), hi);
            const float xr = fmaf(ky, d1, sqrt_approx(fmaxf(0.f, w2 * fmaf(-d1 * d1, isc, t))));
            const float xl = fmaf(ky, d2, -sqrt_approx(fmaxf(0.f, w2 * fmaf(-d2 * d2, isc, t))));
            const float eta = fmaf(1e-3f, fabsf(xl) + fabsf(xr), 0.01f);
            // tiles whose pixel-centre columns [tx B + 0.5, tx B + B - 0.5] meet [u + xl, u + xr]
            const int ta = max(q.x0, (int)ceilf((u + xl - eta - (fb - 0.5f)) * ifb));
            const int tb = min(q.x1 - 1, (int)floorf((u + xr + eta - 0.5f) * ifb));
            if (ta > tb) continue;
            m |= ((2ull << (tb - ta)) - 1ull) << (8 * (ty - q.y0) + (ta - q.x0));
        }
    }
    *mask = m;
    return true;
}

#ifndef DG_PROJECT_FWD_MINB
#define DG_PROJECT_FWD_MINB 5
#endif
#ifndef DG_PROJECT_FWD_MINB_LATE
#define DG_PROJECT_FWD_MINB_LATE 8
#endif
// LATE_SH (one view per launch): the colour coefficients are loaded where the
// colour is formed instead of before the view loop, so they are not live
// across the projection and the kernel fits more resident warps.
template <int NB, bool LATE_SH>
__global__ void __launch_bounds__(128, LATE_SH ? DG_PROJECT_FWD_MINB_LATE : DG_PROJECT_FWD_MINB)
k_project_fwd(const float* __restrict__ prm, long long stride, int P, ViewSet vs_host, const dg_camera* cdev, int B,
              float near_plane, float eps2d, float mip2d, int tight, float4* __restrict__ feat, float* __restrict__ depth,
              int* __restrict__ radius, int* __restrict__ tiles, uint8_t* __restrict__ clampm)
{
    __shared__ ViewSet s_vs;
    const ViewSet& vs = block_views(vs_host, cdev, &s_vs);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    G3 g;
    gauss3d(prm, stride, i, g);
    float sh[NB][3];
    if (!LATE_SH) {
#pragma unroll
        for (int k = 0; k < NB; ++k)
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) sh[k][ch] = prm[(11 + 3 * k + ch) * stride + i];
    }
    const float osig = 1.f / (1.f + expf(-prm[10 * stride + i]));
    for (int v = 0; v < vs.n; ++v) {
        const Cam& cam = vs.cam[v];
        const size_t r = (size_t)v * P + i;
        Splat S;
        float4 f0 = make_float4(0.f, 0.f, 0.f, 0.f), f1 = f0, f2 = f0;
        int rad = 0, nt = 0;
        uint8_t cm = 0;
        const bool ok = splat(g, cam, near_plane, eps2d, mip2d, S);
        if (ok) {
            const float tz = S.t[2];
            const float lam = 0.5f * (S.a + S.c) + sqrtf(0.25f * (S.a - S.c) * (S.a - S.c) + S.b * S.b);
            const float r3 = 3.f * sqrtf(lam);
            const float u = cam.fx * S.t[0] / tz + cam.cx;
            const float vv = cam.fy * S.t[1] / tz + cam.cy;
            if (r3 <= kGuardPx && fabsf(u) <= kGuardPx && fabsf(vv) <= kGuardPx) {
                const int rr = (int)ceilf(r3);
                const Rect q = tile_rect(u, vv, rr, B, vs.TX[v], vs.TY[v]);
                if (q.x0 < q.x1 && q.y0 < q.y1) {
                    float d0 = g.p[0] - vs.campos[v][0], d1 = g.p[1] - vs.campos[v][1], d2 = g.p[2] - vs.campos[v][2];
                    const float dinv = 1.f / sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
                    d0 *= dinv; d1 *= dinv; d2 *= dinv;
                    float Y[16];
                    sh_values(d0, d1, d2, Y);
                    float col[3];
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) {
                        float acc = 0.f;
#pragma unroll
                        for (int k = 0; k < NB; ++k)
                            acc += Y[k] * (LATE_SH ? prm[(11 + 3 * k + ch) * stride + i] : sh[k][ch]);
                        acc += 0.5f;
                        if (acc < 0.f) { cm |= (uint8_t)(1u << ch); acc = 0.f; }
                        col[ch] = acc;
                    }
                    rad = rr;
                    nt = (q.x1 - q.x0) * (q.y1 - q.y0);
                    f0 = make_float4(u, vv, S.A, S.B);
                    f1 = make_float4(S.C, osig * S.comp, col[0], col[1]);
                    f2 = make_float4(col[2], 0.f, 0.f, 0.f);
                    uint64_t m;
                    const bool r16 = tight > 1;  // the render reads float16 conic and opacity
                    if (tight && tile_mask(u, vv, r16 ? round_f16(S.A) : S.A, r16 ? round_f16(S.B) : S.B,
                                           r16 ? round_f16(S.C) : S.C, r16 ? round_f16(f1.y) : f1.y, rr, q, B, &m)) {
                        nt = __popcll(m);  // 0: no tile of the rect can blend the record
                        f2.y = __uint_as_float((uint32_t)m);
                        f2.z = __uint_as_float((uint32_t)(m >> 32));
                    }
                }
            }
        }
        depth[r] = S.t[2];
        feat[3 * r] = f0;
        feat[3 * r + 1] = f1;
        feat[3 * r + 2] = f2;
        radius[r] = rad;
        tiles[r] = nt;
        clampm[r] = cm;
    }
}

// Loads the parameters of the Gaussians c0 .. c0 + 31 (rows 0..58 of the planar
// [59][stride] array) into columns 32 w .. 32 w + 31 of the shared tile t: 8
// lanes per row and 16 bytes per lane when `vec` (16-byte aligned rows), all 15
// loads of a lane issued before its first shared store; 4-byte loads at the end
// of P.  Columns from P on are left as zeros.
__device__ inline void stage_params(const float* __restrict__ prm, long long stride, long long c0, long long P,
                                    bool vec, float (*t)[128], int w, int lane)
{
    const int rr = lane >> 3, cc = 4 * (lane & 7);
    const long long c = c0 + cc;
    float4 x[15];
#pragma unroll
    for (int k = 0; k < 15; ++k) {
        const int r = 4 * k + rr;
        x[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r < DG_NPARAM) {
            const float* a = prm + (long long)r * stride + c;
            if (vec && c + 3 < P) {
                x[k] = *(const float4*)a;
            } else {
                if (c < P) x[k].x = a[0];
                if (c + 1 < P) x[k].y = a[1];
                if (c + 2 < P) x[k].z = a[2];
                if (c + 3 < P) x[k].w = a[3];
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 15; ++k) {
        const int r = 4 * k + rr;
        if (r < DG_NPARAM) *(float4*)&t[r][32 * w + cc] = x[k];
    }
    __syncwarp();
}

// Adjoint of the projection, summed over the views.  Each parameter-row
// gradient goes to `grads` (when given) and, with ADAM, to shared memory; the
// CTA then runs the Adam update of its 128 Gaussians row by row, so the fused
// form never stores or reloads the gradient.  Each thread owns one Gaussian
// (one column of every row), so the in-place update races with nothing.
// At most 128 registers (four 128-thread CTAs per SM), 96 when fused with
// Adam for one view (five CTAs, measured 0.664 -> 0.648 ms at 2M Gaussians; six were
// slower): the adjoint streams 0.5-1.5 kB per Gaussian, and the extra resident
// warps hide more memory latency than the few spilled values cost.
template <int NB, bool ADAM, bool SINGLE>
__global__ void __launch_bounds__(128, ADAM && SINGLE ? 5 : 4)
k_project_bwd(float* __restrict__ prm, long long stride, int P, ViewSet vs_host, const dg_camera* cdev,
              float near_plane, float eps2d, float mip2d, const int* __restrict__ radius, const uint8_t* __restrict__ clampm,
              const float4* __restrict__ grad2d, float* __restrict__ grads, float* __restrict__ am,
              float* __restrict__ av, AdamHp hp_val, const AdamHp* __restrict__ hp_dev,
              const int* __restrict__ skip_if, int vec)
{
    __shared__ ViewSet s_vs;
    __shared__ __align__(16) float s_g[ADAM ? DG_NPARAM : 1][128];  // ADAM: this CTA's gradients, for the row sweep
    __shared__ AdamHp s_hp;                            // ADAM: this step's hyper-parameters
    __shared__ AdamRowK s_rk[ADAM ? DG_NPARAM : 1];    // ADAM: per-row step and 1 / sqrt(1 - b2^t)
    if (ADAM) {
        // from device memory when given (a captured step reads the values of the replay)
        const float* src = (const float*)(hp_dev ? hp_dev : &hp_val);
        for (int k = threadIdx.x; k < (int)(sizeof(AdamHp) / sizeof(float)); k += blockDim.x)
            ((float*)&s_hp)[k] = src[k];
    }
    const ViewSet& vs = block_views(vs_host, cdev, &s_vs);
    if (ADAM) {
        __syncthreads();  // s_hp complete (block_views has no barrier without device cameras)
        if (threadIdx.x < DG_NPARAM) s_rk[threadIdx.x] = adam_row(s_hp.lr[threadIdx.x], s_hp);
        // (published by the barrier before the Adam sweep)
    }
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    // ADAM: each warp stages its 32 Gaussians' parameters in the gradient tile
    // (16-byte loads); a thread reads its own column there and overwrites each
    // row with the row's gradient after its last read of that row
    if (ADAM)
        stage_params(prm, stride, (long long)blockIdx.x * blockDim.x + 32 * (threadIdx.x >> 5), P, vec, s_g,
                     threadIdx.x >> 5, threadIdx.x & 31);
    const float* src = ADAM ? &s_g[0][0] : prm;  // the thread's parameters: src[row * sst + si]
    const long long sst = ADAM ? 128 : stride;
    const int si = ADAM ? (int)threadIdx.x : i;
    auto put = [&](int row, float gval) {
        if (grads) grads[(long long)row * stride + i] = gval;
        if (ADAM) s_g[row][threadIdx.x] = gval;
    };
    auto adjoint = [&]() {
        G3 g;
        gauss3d(src, sst, si, g);
        const float osig = 1.f / (1.f + expf(-src[10 * sst + si]));
        float dp[3] = {0.f, 0.f, 0.f};
        float dsg[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // dL/dSigma (xx xy xz yy yz zz), off-diagonals counted once
        float dop = 0.f;
        // SH-coefficient gradients: summed over the views in registers, or, with a
        // single view (SINGLE), emitted row by row as they are formed (no 48-float
        // accumulator held across the kernel)
        float dsh[SINGLE ? 1 : NB][3];
    #pragma unroll
        for (int k = 0; k < (SINGLE ? 1 : NB); ++k) dsh[k][0] = dsh[k][1] = dsh[k][2] = 0.f;
        bool any = false;
        for (int v = 0; v < vs.n; ++v) {
            const size_t r = (size_t)v * P + i;
            if (radius[r] == 0) continue;
            const Cam& cam = vs.cam[v];
            Splat S;
            if (!splat(g, cam, near_plane, eps2d, mip2d, S)) continue;
            any = true;
            const float4 g0 = grad2d[3 * r], g1 = grad2d[3 * r + 1], g2 = grad2d[3 * r + 2];
            const float dLu = g0.x, dLv = g0.y, dLA = g0.z, dLB = g0.w, dLC = g1.x;
            dop += g1.y * S.comp;  // record opacity = sigmoid * comp
            const uint8_t cm = clampm[r];
            const float dcol[3] = {(cm & 1u) ? 0.f : g1.z, (cm & 2u) ? 0.f : g1.w, (cm & 4u) ? 0.f : g2.x};
            // colour: SH coefficients and the view direction
            {
                float d0 = g.p[0] - vs.campos[v][0], d1 = g.p[1] - vs.campos[v][1], d2 = g.p[2] - vs.campos[v][2];
                const float len = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
                const float linv = 1.f / len;
                d0 *= linv; d1 *= linv; d2 *= linv;
                float Y[16], D[16][3];
                sh_values(d0, d1, d2, Y);
                sh_partials(d0, d1, d2, D);
                float gd[3] = {0.f, 0.f, 0.f};
    #pragma unroll
                for (int k = 0; k < NB; ++k)
    #pragma unroll
                    for (int ch = 0; ch < 3; ++ch) {
                        const float cw = dcol[ch] * src[(11 + 3 * k + ch) * sst + si];
                        gd[0] += cw * D[k][0];
                        gd[1] += cw * D[k][1];
                        gd[2] += cw * D[k][2];
                        if (SINGLE) put(11 + 3 * k + ch, Y[k] * dcol[ch]);  // after the coefficient was read
                        else dsh[SINGLE ? 0 : k][ch] += Y[k] * dcol[ch];
                    }
                const float dd = d0 * gd[0] + d1 * gd[1] + d2 * gd[2];
                dp[0] += (gd[0] - d0 * dd) * linv;
                dp[1] += (gd[1] - d1 * dd) * linv;
                dp[2] += (gd[2] - d2 * dd) * linv;
            }
            const float tx = S.t[0], ty = S.t[1], tz = S.t[2];
            const float iz = 1.f / tz, iz2 = iz * iz;
            float dt[3];
            dt[0] = dLu * cam.fx * iz;
            dt[1] = dLv * cam.fy * iz;
            dt[2] = -(dLu * cam.fx * tx + dLv * cam.fy * ty) * iz2;
            // conic -> 2D covariance: Gm = -K Gk K, Gk = [[dA, dB/2], [dB/2, dC]]
            const float A = S.A, B = S.B, C = S.C;
            const float k00 = A * dLA + 0.5f * B * dLB, k01 = 0.5f * A * dLB + B * dLC;
            const float k10 = B * dLA + 0.5f * C * dLB, k11 = 0.5f * B * dLB + C * dLC;
            float gm00 = -(k00 * A + k01 * B);
            float gm01 = -(k00 * B + k01 * C);
            float gm11 = -(k10 * B + k11 * C);
            if (mip2d > 0.f && S.det0 > 0.f) {
                // 2D filter: d sqrt(det0 / det) per covariance entry (det0 of the
                // undilated, det of the filtered matrix; the off-diagonal entry
                // carries half of the derivative in b)
                const float h = 0.5f * S.comp * g1.y * osig;
                const float a0 = S.a - mip2d, c0 = S.c - mip2d;
                const float i0 = 1.f / S.det0, i1 = 1.f / S.det;
                gm00 += h * (c0 * i0 - S.c * i1);
                gm11 += h * (a0 * i0 - S.a * i1);
                gm01 += h * (S.b * i1 - S.b * i0);
            }
            // Sigma2 = T2 Sigma T2^T:  dSigma = T2^T Gm T2,  dT2 = 2 Gm T2 Sigma
            const float* t2 = S.t2;
            float gt[6];  // Gm T2
    #pragma unroll
            for (int c = 0; c < 3; ++c) {
                gt[c] = gm00 * t2[c] + gm01 * t2[3 + c];
                gt[3 + c] = gm01 * t2[c] + gm11 * t2[3 + c];
            }
            // symmetric dSigma accumulated as 6 unique entries of the full-matrix gradient
            dsg[0] += t2[0] * gt[0] + t2[3] * gt[3];
            dsg[1] += t2[0] * gt[1] + t2[3] * gt[4];
            dsg[2] += t2[0] * gt[2] + t2[3] * gt[5];
            dsg[3] += t2[1] * gt[1] + t2[4] * gt[4];
            dsg[4] += t2[1] * gt[2] + t2[4] * gt[5];
            dsg[5] += t2[2] * gt[2] + t2[5] * gt[5];
            const float* sg = g.sig;
            const float sgm[9] = {sg[0], sg[1], sg[2], sg[1], sg[3], sg[4], sg[2], sg[4], sg[5]};
            float dt2[6];
    #pragma unroll
            for (int rr = 0; rr < 2; ++rr)
    #pragma unroll
                for (int c = 0; c < 3; ++c)
                    dt2[3 * rr + c] = 2.f * (gt[3 * rr] * sgm[c] + gt[3 * rr + 1] * sgm[3 + c] + gt[3 * rr + 2] * sgm[6 + c]);
            // T2 = J Rc
            const float* rc = cam.r;
            const float dj00 = dt2[0] * rc[0] + dt2[1] * rc[1] + dt2[2] * rc[2];
            const float dj02 = dt2[0] * rc[6] + dt2[1] * rc[7] + dt2[2] * rc[8];
            const float dj11 = dt2[3] * rc[3] + dt2[4] * rc[4] + dt2[5] * rc[5];
            const float dj12 = dt2[3] * rc[6] + dt2[4] * rc[7] + dt2[5] * rc[8];
            dt[2] -= (dj00 * cam.fx + dj11 * cam.fy) * iz2;
            if (!S.gx) {
                dt[0] -= dj02 * cam.fx * iz2;
                dt[2] += dj02 * 2.f * cam.fx * tx * iz2 * iz;
            } else {
                dt[2] += dj02 * cam.fx * S.lx * iz2;
            }
            if (!S.gy) {
                dt[1] -= dj12 * cam.fy * iz2;
                dt[2] += dj12 * 2.f * cam.fy * ty * iz2 * iz;
            } else {
                dt[2] += dj12 * cam.fy * S.ly * iz2;
            }
            // t = Rc p + t_c
    #pragma unroll
            for (int c = 0; c < 3; ++c) dp[c] += rc[c] * dt[0] + rc[3 + c] * dt[1] + rc[6 + c] * dt[2];
        }
        if (!any) {
            for (int rr = 0; rr < DG_NPARAM; ++rr) put(rr, 0.f);
            return;
        }
        put(0, dp[0]);
        put(1, dp[1]);
        put(2, dp[2]);
        put(10, dop * osig * (1.f - osig));
    #pragma unroll
        for (int k = SINGLE ? NB : 0; k < 16; ++k)
    #pragma unroll
            for (int ch = 0; ch < 3; ++ch) put(11 + 3 * k + ch, k < NB ? dsh[SINGLE ? 0 : k][ch] : 0.f);
        // Sigma = M M^T:  dM = 2 dSigma M;  M = Rq diag(s)
        const float ds[9] = {dsg[0], dsg[1], dsg[2], dsg[1], dsg[3], dsg[4], dsg[2], dsg[4], dsg[5]};
        float dR[9];
    #pragma unroll
        for (int c = 0; c < 3; ++c) {
            float dsc = 0.f;
    #pragma unroll
            for (int rr = 0; rr < 3; ++rr) {
                const float dm = 2.f * (ds[3 * rr] * g.m[c] + ds[3 * rr + 1] * g.m[3 + c] + ds[3 * rr + 2] * g.m[6 + c]);
                dsc += dm * g.rq[3 * rr + c];
                dR[3 * rr + c] = dm * g.s[c];
            }
            put(3 + c, dsc * g.s[c]);
        }
        const float w = g.qn[0], x = g.qn[1], y = g.qn[2], z = g.qn[3];
        float dq[4];
        dq[0] = 2.f * (z * (dR[3] - dR[1]) + y * (dR[2] - dR[6]) + x * (dR[7] - dR[5]));
        dq[1] = 2.f * (y * (dR[1] + dR[3]) + z * (dR[2] + dR[6]) + w * (dR[7] - dR[5]) - 2.f * x * (dR[4] + dR[8]));
        dq[2] = 2.f * (x * (dR[1] + dR[3]) + w * (dR[2] - dR[6]) + z * (dR[5] + dR[7]) - 2.f * y * (dR[0] + dR[8]));
        dq[3] = 2.f * (w * (dR[3] - dR[1]) + x * (dR[2] + dR[6]) + y * (dR[5] + dR[7]) - 2.f * z * (dR[0] + dR[4]));
        const float qd = w * dq[0] + x * dq[1] + y * dq[2] + z * dq[3];
    #pragma unroll
        for (int c = 0; c < 4; ++c) put(6 + c, (dq[c] - g.qn[c] * qd) * g.qinv);

    };
    if (i < P) adjoint();
    if (ADAM) {
        // Adam over the CTA's [59][128] tile: warp w takes the rows w, w + 4,
        // ..., lane l the four Gaussians 4 l .. 4 l + 3 of a row, one 16-byte
        // access per array when `vec` (16-byte aligned rows), else four
        // 4-byte ones (also for the lanes at the end of P).  The loads of RBV
        // rows are issued before the first store.  Measured at 2M Gaussians:
        // 0.642 ms with one thread per Gaussian and 4-byte accesses, 0.571 ms
        // so (the sweep alone 0.610 -> 0.427 ms, 98% of the copy bandwidth).
        constexpr int RBV = 4;
        __syncthreads();  // gradients of the whole tile (lanes read other threads' columns)
        const AdamHp& hp = s_hp;
        // (skip_if: e.g. the step's pair list overflowed; then no update)
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        const long long c = (long long)blockIdx.x * 128 + 4 * lane;  // the lane's first Gaussian
        const long long nc = (long long)P - c;                        // of its four, those below P
        if (nc > 0 && !(skip_if && *skip_if != 0)) {
            const bool full = vec && nc >= 4;
            for (int q0 = w; q0 < DG_NPARAM; q0 += 4 * RBV) {
                float4 p[RBV], mm[RBV], vv[RBV];
#pragma unroll
                for (int j = 0; j < RBV; ++j) {
                    const int r = q0 + 4 * j;
                    if (r < DG_NPARAM) {
                        const long long o = (long long)r * stride + c;
                        if (full) {
                            p[j] = *(const float4*)(prm + o);
                            mm[j] = *(const float4*)(am + o);
                            vv[j] = *(const float4*)(av + o);
                        } else {
                            float* pp = &p[j].x;
                            float* mp = &mm[j].x;
                            float* vp = &vv[j].x;
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                if (k < nc) {
                                    pp[k] = prm[o + k];
                                    mp[k] = am[o + k];
                                    vp[k] = av[o + k];
                                }
                            }
                        }
                    }
                }
#pragma unroll
                for (int j = 0; j < RBV; ++j) {
                    const int r = q0 + 4 * j;
                    if (r < DG_NPARAM) {
                        const float4 g = *(const float4*)&s_g[r][4 * lane];
                        const long long o = (long long)r * stride + c;
                        const AdamRowK& rk = s_rk[r];
                        if (full) {
                            adam_update(p[j].x, mm[j].x, vv[j].x, g.x, rk, hp);
                            adam_update(p[j].y, mm[j].y, vv[j].y, g.y, rk, hp);
                            adam_update(p[j].z, mm[j].z, vv[j].z, g.z, rk, hp);
                            adam_update(p[j].w, mm[j].w, vv[j].w, g.w, rk, hp);
                            *(float4*)(prm + o) = p[j];
                            *(float4*)(am + o) = mm[j];
                            *(float4*)(av + o) = vv[j];
                        } else {
                            float* pp = &p[j].x;
                            float* mp = &mm[j].x;
                            float* vp = &vv[j].x;
                            const float* gp = &g.x;
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                if (k < nc) {
                                    adam_update(pp[k], mp[k], vp[k], gp[k], rk, hp);
                                    prm[o + k] = pp[k];
                                    am[o + k] = mp[k];
                                    av[o + k] = vp[k];
                                }
                            }
                        }
                    }
                }
            }
        }
    }
}

}  // namespace dg

// ---------------------------------------------------------------------------
bool dg_check_cameras(const dg_camera* cams, int n_views)
{
    if (!cams) { dg_set_error("cameras are null"); return false; }
    if (n_views < 1 || n_views > DG_MAX_VIEWS) { dg_set_error("n_views %d outside 1..%d", n_views, DG_MAX_VIEWS); return false; }
    for (int v = 0; v < n_views; ++v) {
        const dg_camera* c = cams + v;
        if (c->width <= 0 || c->height <= 0) { dg_set_error("view %d: image size %dx%d", v, c->width, c->height); return false; }
        if (!(c->fx > 0.f) || !(c->fy > 0.f)) { dg_set_error("view %d: focal length must be positive", v); return false; }
    }
    return true;
}

static bool check_opts(const dg_raster_opts* o)
{
    if (!o) { dg_set_error("opts is null"); return false; }
    if (o->tile < 1 || o->tile > 64) { dg_set_error("tile %d outside 1..64", o->tile); return false; }
    if (o->sh_degree < 0 || o->sh_degree > 3) { dg_set_error("sh_degree %d outside 0..3", o->sh_degree); return false; }
    if (!(o->mip2d >= 0.f)) { dg_set_error("mip2d must be >= 0"); return false; }
    return true;
}

static dg::ViewSet make_views(const dg_camera* cams, int n, int B)
{
    dg::ViewSet vs;
    vs.n = n;
    for (int v = 0; v < n; ++v) {
        const dg::Cam c = dg::make_cam(cams[v]);
        vs.cam[v] = c;
        dg::cam_centre(c, vs.campos[v]);
        vs.TX[v] = (cams[v].width + B - 1) / B;
        vs.TY[v] = (cams[v].height + B - 1) / B;
    }
    return vs;
}

extern "C" dg_status dg_project(const float* params, int64_t stride, int64_t P, const dg_camera* cams,
                                const dg_camera* cams_dev, int32_t n_views, const dg_raster_opts* opts, float* feat,
                                float* depth, int32_t* radius, int32_t* tiles, uint8_t* clamp, dg_stream stream)
{
    if (!dg_check_cameras(cams, n_views) || !check_opts(opts)) return DG_ERR_ARG;
    if (P < 0 || P > INT32_MAX || stride < P || (long long)P * n_views > (long long)UINT32_MAX) {
        dg_set_error("bad P=%lld stride=%lld", (long long)P, (long long)stride);
        return DG_ERR_ARG;
    }
    if (P == 0) return DG_OK;
    if (!params || !feat || !depth || !radius || !tiles || !clamp) { dg_set_error("null buffer"); return DG_ERR_ARG; }
    if (((uintptr_t)feat) & 15u) { dg_set_error("feat must be 16-byte aligned"); return DG_ERR_ARG; }
    const dg::ViewSet vs = make_views(cams, n_views, opts->tile);
    const int threads = 128;
    const int blocks = (int)((P + threads - 1) / threads);
    cudaStream_t s = (cudaStream_t)stream;
    const int tight = opts->tight_bins ? 1 + (opts->record == 1) : 0;
    auto go = [&](auto kern) {
        kern<<<blocks, threads, 0, s>>>(params, (long long)stride, (int)P, vs, cams_dev, opts->tile, opts->near_plane,
                                        opts->eps2d, opts->mip2d, tight, (float4*)feat, depth, radius, tiles, clamp);
    };
    const bool one = n_views == 1;
    switch (opts->sh_degree) {
    case 0: one ? go(dg::k_project_fwd<1, true>) : go(dg::k_project_fwd<1, false>); break;
    case 1: one ? go(dg::k_project_fwd<4, true>) : go(dg::k_project_fwd<4, false>); break;
    case 2: one ? go(dg::k_project_fwd<9, true>) : go(dg::k_project_fwd<9, false>); break;
    default: one ? go(dg::k_project_fwd<16, true>) : go(dg::k_project_fwd<16, false>); break;
    }
    dg_note_launch();
    return dg_check_launch("project_fwd");
}

template <bool ADAM, bool SINGLE>
static void launch_project_bwd(int nb, int blocks, int threads, cudaStream_t s, float* params, long long st, int P,
                               const dg::ViewSet& vs, const dg_camera* cams_dev, const dg_raster_opts* opts,
                               const int32_t* radius, const uint8_t* clamp, const float4* g2, float* grads, float* m,
                               float* v, const dg::AdamHp& hp, const dg::AdamHp* hp_dev, const int* skip_if)
{
    const float np = opts->near_plane, e2 = opts->eps2d, mp = opts->mip2d;
    // 16-byte row accesses in the Adam sweep: rows of params, m and v start on
    // 16-byte boundaries
    const int vec = ADAM && st % 4 == 0 && ((uintptr_t)params & 15u) == 0 && ((uintptr_t)m & 15u) == 0 &&
                    ((uintptr_t)v & 15u) == 0;
    switch (nb) {
    case 1: dg::k_project_bwd<1, ADAM, SINGLE><<<blocks, threads, 0, s>>>(params, st, P, vs, cams_dev, np, e2, mp, radius, clamp, g2, grads, m, v, hp, hp_dev, skip_if, vec); break;
    case 4: dg::k_project_bwd<4, ADAM, SINGLE><<<blocks, threads, 0, s>>>(params, st, P, vs, cams_dev, np, e2, mp, radius, clamp, g2, grads, m, v, hp, hp_dev, skip_if, vec); break;
    case 9: dg::k_project_bwd<9, ADAM, SINGLE><<<blocks, threads, 0, s>>>(params, st, P, vs, cams_dev, np, e2, mp, radius, clamp, g2, grads, m, v, hp, hp_dev, skip_if, vec); break;
    default: dg::k_project_bwd<16, ADAM, SINGLE><<<blocks, threads, 0, s>>>(params, st, P, vs, cams_dev, np, e2, mp, radius, clamp, g2, grads, m, v, hp, hp_dev, skip_if, vec); break;
    }
}

template <bool ADAM>
static dg_status project_bwd(float* params, int64_t stride, int64_t P, const dg_camera* cams,
                             const dg_camera* cams_dev, int32_t n_views,
                             const dg_raster_opts* opts, const int32_t* radius, const uint8_t* clamp,
                             const float* grad2d, float* grads, float* m, float* v, const dg::AdamHp& hp,
                             const dg::AdamHp* hp_dev, const int* skip_if, dg_stream stream)
{
    if (!dg_check_cameras(cams, n_views) || !check_opts(opts)) return DG_ERR_ARG;
    if (P < 0 || P > INT32_MAX || stride < P || (long long)P * n_views > (long long)UINT32_MAX) {
        dg_set_error("bad P=%lld stride=%lld", (long long)P, (long long)stride);
        return DG_ERR_ARG;
    }
    if (P == 0) return DG_OK;
    if (!params || !radius || !clamp || !grad2d || (!ADAM && !grads) || (ADAM && (!m || !v))) {
        dg_set_error("null buffer");
        return DG_ERR_ARG;
    }
    if (((uintptr_t)grad2d) & 15u) { dg_set_error("grad2d must be 16-byte aligned"); return DG_ERR_ARG; }
    const dg::ViewSet vs = make_views(cams, n_views, opts->tile);
    const int threads = 128;
    const int blocks = (int)((P + threads - 1) / threads);
    cudaStream_t s = (cudaStream_t)stream;
    const long long st = (long long)stride;
    const float4* g2 = (const float4*)grad2d;
    const int nb = opts->sh_degree == 0 ? 1 : opts->sh_degree == 1 ? 4 : opts->sh_degree == 2 ? 9 : 16;
    if (n_views == 1) launch_project_bwd<ADAM, true>(nb, blocks, threads, s, params, st, (int)P, vs, cams_dev, opts, radius, clamp, g2, grads, m, v, hp, hp_dev, skip_if);
    else launch_project_bwd<ADAM, false>(nb, blocks, threads, s, params, st, (int)P, vs, cams_dev, opts, radius, clamp, g2, grads, m, v, hp, hp_dev, skip_if);
    dg_note_launch();
    return dg_check_launch(ADAM ? "project_bwd_adam" : "project_bwd");
}

extern "C" dg_status dg_project_bwd(const float* params, int64_t stride, int64_t P, const dg_camera* cams,
                                    const dg_camera* cams_dev, int32_t n_views, const dg_raster_opts* opts,
                                    const int32_t* radius, const uint8_t* clamp, const float* grad2d, float* grads,
                                    dg_stream stream)
{
    // the non-Adam instantiation never writes params
    return project_bwd<false>(const_cast<float*>(params), stride, P, cams, cams_dev, n_views, opts, radius, clamp,
                              grad2d, grads, nullptr, nullptr, dg::AdamHp{}, nullptr, nullptr, stream);
}

extern "C" dg_status dg_project_bwd_adam(float* params, int64_t stride, int64_t P, const dg_camera* cams,
                                         const dg_camera* cams_dev, int32_t n_views, const dg_raster_opts* opts,
                                         const int32_t* radius, const uint8_t* clamp, const float* grad2d,
                                         float* grads, float* m, float* v, const float* lr, float beta1, float beta2,
                                         float eps, int64_t step, dg_stream stream)
{
    if (step < 1 || !lr) { dg_set_error("step must be >= 1 and lr given"); return DG_ERR_ARG; }
    return project_bwd<true>(params, stride, P, cams, cams_dev, n_views, opts, radius, clamp, grad2d, grads, m, v,
                             dg_adam_hp(lr, beta1, beta2, eps, step), nullptr, nullptr, stream);
}

extern "C" dg_status dg_project_bwd_adam_dev(float* params, int64_t stride, int64_t P, const dg_camera* cams,
                                             const dg_camera* cams_dev, int32_t n_views, const dg_raster_opts* opts,
                                             const int32_t* radius, const uint8_t* clamp, const float* grad2d,
                                             float* grads, float* m, float* v, const dg_adam_hparams* hp_dev,
                                             const int32_t* skip_if, dg_stream stream)
{
    if (!hp_dev) { dg_set_error("hp_dev is null"); return DG_ERR_ARG; }
    return project_bwd<true>(params, stride, P, cams, cams_dev, n_views, opts, radius, clamp, grad2d, grads, m, v,
                             dg::AdamHp{}, hp_dev, skip_if, stream);
}
