// project.cu -- EWA projection + SH colour (forward) and its adjoint.
//
// One thread per Gaussian.  Parameters are planar [59][stride], so every row
// read by a warp is one coalesced 128-byte transaction; the projected record
// is written as three 16-byte stores per Gaussian (the render kernels gather
// it by Gaussian index).
//
// Forward (Sec. 3: the 3D Gaussian is splatted to a 2D Gaussian on the image
// plane; colour from the colour coefficients c_i):
//   t = R p + t_c;  Sigma = (Rq S)(Rq S)^T, S = diag(exp(log scale));
//   J = d(pinhole)/dt at t with t_x/t_z, t_y/t_z clamped to 1.3 x half-FOV;
//   Sigma2 = J R Sigma R^T J^T + eps I;  conic = Sigma2^-1;
//   radius = ceil(3 sqrt(lambda_max(Sigma2)));  colour = SH(dir) + 0.5, >= 0.
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

// Everything the forward computes for one Gaussian, kept for the adjoint.
struct Splat {
    float t[3];
    float qn[4], qinv;      // normalised quaternion and 1/|q|
    float rq[9], s[3], m[9];
    float sig[6];           // Sigma: xx xy xz yy yz zz
    bool gx, gy;            // frustum guard active on x / y
    float lx, ly;           // signed guard value when active
    float t2[6];            // J R, 2 x 3
    float a, b, c, det;     // 2D covariance (with dilation) and determinant
    float A, B, C;          // conic
};

__device__ inline bool splat(const float* __restrict__ prm, long long stride, int i, const Cam& cam,
                             float near_plane, float eps2d, Splat& S)
{
    const float p0 = prm[i], p1 = prm[stride + i], p2 = prm[2 * stride + i];
    S.t[0] = cam.r[0] * p0 + cam.r[1] * p1 + cam.r[2] * p2 + cam.t[0];
    S.t[1] = cam.r[3] * p0 + cam.r[4] * p1 + cam.r[5] * p2 + cam.t[1];
    S.t[2] = cam.r[6] * p0 + cam.r[7] * p1 + cam.r[8] * p2 + cam.t[2];
    if (!(S.t[2] > near_plane)) return false;
    const float tz = S.t[2];

    float q0 = prm[6 * stride + i], q1 = prm[7 * stride + i], q2 = prm[8 * stride + i], q3 = prm[9 * stride + i];
    S.qinv = 1.f / sqrtf(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
    const float w = q0 * S.qinv, x = q1 * S.qinv, y = q2 * S.qinv, z = q3 * S.qinv;
    S.qn[0] = w; S.qn[1] = x; S.qn[2] = y; S.qn[3] = z;
    float* R = S.rq;
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
    S.s[0] = expf(prm[3 * stride + i]);
    S.s[1] = expf(prm[4 * stride + i]);
    S.s[2] = expf(prm[5 * stride + i]);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) S.m[3 * r + c] = R[3 * r + c] * S.s[c];
    const float* M = S.m;
    S.sig[0] = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
    S.sig[1] = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
    S.sig[2] = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
    S.sig[3] = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
    S.sig[4] = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
    S.sig[5] = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];

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
    const float* g = S.sig;
    float u0[3], u1[3];  // Sigma T2_row^T
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float* tr = S.t2 + 3 * k;
        float* u = k == 0 ? u0 : u1;
        u[0] = g[0] * tr[0] + g[1] * tr[1] + g[2] * tr[2];
        u[1] = g[1] * tr[0] + g[3] * tr[1] + g[4] * tr[2];
        u[2] = g[2] * tr[0] + g[4] * tr[1] + g[5] * tr[2];
    }
    S.a = S.t2[0] * u0[0] + S.t2[1] * u0[1] + S.t2[2] * u0[2] + eps2d;
    S.b = S.t2[0] * u1[0] + S.t2[1] * u1[1] + S.t2[2] * u1[2];
    S.c = S.t2[3] * u1[0] + S.t2[4] * u1[1] + S.t2[5] * u1[2] + eps2d;
    S.det = fmaf(S.a, S.c, -S.b * S.b);
    if (!(S.det > 0.f)) return false;
    const float inv = 1.f / S.det;
    S.A = S.c * inv;
    S.B = -S.b * inv;
    S.C = S.a * inv;
    return true;
}

__global__ void __launch_bounds__(256)
k_project_fwd(const float* __restrict__ prm, long long stride, int P, Cam cam, float3 campos,
              int B, int TX, int TY, int nb, float near_plane, float eps2d,
              float4* __restrict__ feat, float* __restrict__ depth, int* __restrict__ radius,
              int* __restrict__ tiles, uint8_t* __restrict__ clampm)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    Splat S;
    float4 f0 = make_float4(0.f, 0.f, 0.f, 0.f), f1 = f0, f2 = f0;
    int rad = 0, nt = 0;
    uint8_t cm = 0;
    const bool ok = splat(prm, stride, i, cam, near_plane, eps2d, S);
    depth[i] = S.t[2];
    if (ok) {
        const float tz = S.t[2];
        const float lam = 0.5f * (S.a + S.c) + sqrtf(0.25f * (S.a - S.c) * (S.a - S.c) + S.b * S.b);
        const float r3 = 3.f * sqrtf(lam);
        const float u = cam.fx * S.t[0] / tz + cam.cx;
        const float v = cam.fy * S.t[1] / tz + cam.cy;
        if (r3 <= kGuardPx && fabsf(u) <= kGuardPx && fabsf(v) <= kGuardPx) {
            const int r = (int)ceilf(r3);
            const Rect q = tile_rect(u, v, r, B, TX, TY);
            if (q.x0 < q.x1 && q.y0 < q.y1) {
                float d0 = prm[i] - campos.x, d1 = prm[stride + i] - campos.y, d2 = prm[2 * stride + i] - campos.z;
                const float dinv = 1.f / sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
                d0 *= dinv; d1 *= dinv; d2 *= dinv;
                float Y[16];
                sh_values(d0, d1, d2, Y);
                float col[3];
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    float acc = 0.f;
                    for (int k = 0; k < nb; ++k) acc += Y[k] * prm[(11 + 3 * k + ch) * stride + i];
                    acc += 0.5f;
                    if (acc < 0.f) { cm |= (uint8_t)(1u << ch); acc = 0.f; }
                    col[ch] = acc;
                }
                const float o = 1.f / (1.f + expf(-prm[10 * stride + i]));
                rad = r;
                nt = (q.x1 - q.x0) * (q.y1 - q.y0);
                f0 = make_float4(u, v, S.A, S.B);
                f1 = make_float4(S.C, o, col[0], col[1]);
                f2 = make_float4(col[2], 0.f, 0.f, 0.f);
            }
        }
    }
    feat[3 * (size_t)i] = f0;
    feat[3 * (size_t)i + 1] = f1;
    feat[3 * (size_t)i + 2] = f2;
    radius[i] = rad;
    tiles[i] = nt;
    clampm[i] = cm;
}

__global__ void __launch_bounds__(128)
k_project_bwd(const float* __restrict__ prm, long long stride, int P, Cam cam, float3 campos, int nb,
              float near_plane, float eps2d, const int* __restrict__ radius,
              const uint8_t* __restrict__ clampm, const float4* __restrict__ grad2d,
              float* __restrict__ grads)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    Splat S;
    if (radius[i] == 0 || !splat(prm, stride, i, cam, near_plane, eps2d, S)) {
        for (int r = 0; r < DG_NPARAM; ++r) grads[r * stride + i] = 0.f;
        return;
    }
    const float4 g0 = grad2d[3 * (size_t)i], g1 = grad2d[3 * (size_t)i + 1], g2 = grad2d[3 * (size_t)i + 2];
    const float dLu = g0.x, dLv = g0.y, dLA = g0.z, dLB = g0.w, dLC = g1.x, dLo = g1.y;
    const uint8_t cm = clampm[i];
    const float dcol[3] = {(cm & 1u) ? 0.f : g1.z, (cm & 2u) ? 0.f : g1.w, (cm & 4u) ? 0.f : g2.x};

    float dp[3] = {0.f, 0.f, 0.f};
    // colour: SH coefficients and the view direction
    {
        float d0 = prm[i] - campos.x, d1 = prm[stride + i] - campos.y, d2 = prm[2 * stride + i] - campos.z;
        const float len = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
        const float linv = 1.f / len;
        d0 *= linv; d1 *= linv; d2 *= linv;
        float Y[16], D[16][3];
        sh_values(d0, d1, d2, Y);
        sh_partials(d0, d1, d2, D);
        float gd[3] = {0.f, 0.f, 0.f};
        for (int k = 0; k < 16; ++k) {
            const bool on = k < nb;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                const long long row = (long long)(11 + 3 * k + ch) * stride + i;
                grads[row] = on ? Y[k] * dcol[ch] : 0.f;
                if (on) {
                    const float cw = dcol[ch] * prm[row];
                    gd[0] += cw * D[k][0];
                    gd[1] += cw * D[k][1];
                    gd[2] += cw * D[k][2];
                }
            }
        }
        const float dd = d0 * gd[0] + d1 * gd[1] + d2 * gd[2];
        dp[0] += (gd[0] - d0 * dd) * linv;
        dp[1] += (gd[1] - d1 * dd) * linv;
        dp[2] += (gd[2] - d2 * dd) * linv;
    }
    // opacity through the sigmoid
    {
        const float o = 1.f / (1.f + expf(-prm[10 * stride + i]));
        grads[10 * stride + i] = dLo * o * (1.f - o);
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
    const float gm00 = -(k00 * A + k01 * B);
    const float gm01 = -(k00 * B + k01 * C);
    const float gm11 = -(k10 * B + k11 * C);

    // Sigma2 = T2 Sigma T2^T:  dSigma = T2^T Gm T2,  dT2 = 2 Gm T2 Sigma
    const float* t2 = S.t2;
    float gt[6];  // Gm T2
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        gt[c] = gm00 * t2[c] + gm01 * t2[3 + c];
        gt[3 + c] = gm01 * t2[c] + gm11 * t2[3 + c];
    }
    float ds[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) ds[3 * r + c] = t2[r] * gt[c] + t2[3 + r] * gt[3 + c];
    const float* g = S.sig;
    const float sg[9] = {g[0], g[1], g[2], g[1], g[3], g[4], g[2], g[4], g[5]};
    float dt2[6];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            dt2[3 * r + c] = 2.f * (gt[3 * r] * sg[c] + gt[3 * r + 1] * sg[3 + c] + gt[3 * r + 2] * sg[6 + c]);
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
    grads[i] = dp[0];
    grads[stride + i] = dp[1];
    grads[2 * stride + i] = dp[2];

    // Sigma = M M^T:  dM = 2 dSigma M;  M = Rq diag(s)
    float dR[9];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float dsc = 0.f;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const float dm = 2.f * (ds[3 * r] * S.m[c] + ds[3 * r + 1] * S.m[3 + c] + ds[3 * r + 2] * S.m[6 + c]);
            dsc += dm * S.rq[3 * r + c];
            dR[3 * r + c] = dm * S.s[c];
        }
        grads[(3 + c) * stride + i] = dsc * S.s[c];
    }
    const float w = S.qn[0], x = S.qn[1], y = S.qn[2], z = S.qn[3];
    float dq[4];
    dq[0] = 2.f * (z * (dR[3] - dR[1]) + y * (dR[2] - dR[6]) + x * (dR[7] - dR[5]));
    dq[1] = 2.f * (y * (dR[1] + dR[3]) + z * (dR[2] + dR[6]) + w * (dR[7] - dR[5]) - 2.f * x * (dR[4] + dR[8]));
    dq[2] = 2.f * (x * (dR[1] + dR[3]) + w * (dR[2] - dR[6]) + z * (dR[5] + dR[7]) - 2.f * y * (dR[0] + dR[8]));
    dq[3] = 2.f * (w * (dR[3] - dR[1]) + x * (dR[2] + dR[6]) + y * (dR[5] + dR[7]) - 2.f * z * (dR[0] + dR[4]));
    const float qd = w * dq[0] + x * dq[1] + y * dq[2] + z * dq[3];
#pragma unroll
    for (int c = 0; c < 4; ++c) grads[(6 + c) * stride + i] = (dq[c] - S.qn[c] * qd) * S.qinv;
}

}  // namespace dg

// ---------------------------------------------------------------------------
static bool check_cam(const dg_camera* cam)
{
    if (!cam) { dg_set_error("camera is null"); return false; }
    if (cam->width <= 0 || cam->height <= 0) { dg_set_error("image size %dx%d", cam->width, cam->height); return false; }
    if (!(cam->fx > 0.f) || !(cam->fy > 0.f)) { dg_set_error("focal length must be positive"); return false; }
    return true;
}

static bool check_opts(const dg_raster_opts* o)
{
    if (!o) { dg_set_error("opts is null"); return false; }
    if (o->tile < 1 || o->tile > 64) { dg_set_error("tile %d outside 1..64", o->tile); return false; }
    if (o->sh_degree < 0 || o->sh_degree > 3) { dg_set_error("sh_degree %d outside 0..3", o->sh_degree); return false; }
    return true;
}

static float3 camera_centre(const dg::Cam& c)
{
    return make_float3(-(c.r[0] * c.t[0] + c.r[3] * c.t[1] + c.r[6] * c.t[2]),
                       -(c.r[1] * c.t[0] + c.r[4] * c.t[1] + c.r[7] * c.t[2]),
                       -(c.r[2] * c.t[0] + c.r[5] * c.t[1] + c.r[8] * c.t[2]));
}

extern "C" dg_status dg_project(const float* params, int64_t stride, int64_t P, const dg_camera* cam,
                                const dg_raster_opts* opts, float* feat, float* depth, int32_t* radius,
                                int32_t* tiles, uint8_t* clamp, dg_stream stream)
{
    if (!check_cam(cam) || !check_opts(opts)) return DG_ERR_ARG;
    if (P < 0 || P > INT32_MAX || stride < P) { dg_set_error("bad P=%lld stride=%lld", (long long)P, (long long)stride); return DG_ERR_ARG; }
    if (P == 0) return DG_OK;
    if (!params || !feat || !depth || !radius || !tiles || !clamp) { dg_set_error("null buffer"); return DG_ERR_ARG; }
    if (((uintptr_t)feat) & 15u) { dg_set_error("feat must be 16-byte aligned"); return DG_ERR_ARG; }
    const dg::Cam c = dg::make_cam(*cam);
    const int B = opts->tile;
    const int TX = (cam->width + B - 1) / B, TY = (cam->height + B - 1) / B;
    const int nb = (opts->sh_degree + 1) * (opts->sh_degree + 1);
    const int threads = 256;
    const int blocks = (int)((P + threads - 1) / threads);
    dg::k_project_fwd<<<blocks, threads, 0, (cudaStream_t)stream>>>(
        params, (long long)stride, (int)P, c, camera_centre(c), B, TX, TY, nb, opts->near_plane,
        opts->eps2d, (float4*)feat, depth, radius, tiles, clamp);
    dg_note_launch();
    return dg_check_launch("project_fwd");
}

extern "C" dg_status dg_project_bwd(const float* params, int64_t stride, int64_t P, const dg_camera* cam,
                                    const dg_raster_opts* opts, const int32_t* radius, const uint8_t* clamp,
                                    const float* grad2d, float* grads, dg_stream stream)
{
    if (!check_cam(cam) || !check_opts(opts)) return DG_ERR_ARG;
    if (P < 0 || P > INT32_MAX || stride < P) { dg_set_error("bad P=%lld stride=%lld", (long long)P, (long long)stride); return DG_ERR_ARG; }
    if (P == 0) return DG_OK;
    if (!params || !radius || !clamp || !grad2d || !grads) { dg_set_error("null buffer"); return DG_ERR_ARG; }
    if (((uintptr_t)grad2d) & 15u) { dg_set_error("grad2d must be 16-byte aligned"); return DG_ERR_ARG; }
    const dg::Cam c = dg::make_cam(*cam);
    const int nb = (opts->sh_degree + 1) * (opts->sh_degree + 1);
    const int threads = 128;
    const int blocks = (int)((P + threads - 1) / threads);
    dg::k_project_bwd<<<blocks, threads, 0, (cudaStream_t)stream>>>(
        params, (long long)stride, (int)P, c, camera_centre(c), nb, opts->near_plane, opts->eps2d,
        radius, clamp, (const float4*)grad2d, grads);
    dg_note_launch();
    return dg_check_launch("project_bwd");
}
