// render.cu -- Eq. 1 compositing per tile (forward) and its adjoint (backward).
//
// One CTA per B x B tile, one pixel per thread.  The tile's sorted list is
// streamed through shared memory in batches of B*B records (one coalesced
// gather per thread per batch).  Forward: front to back, a CTA stops as soon
// as every pixel has terminated (__syncthreads_count).  Backward: back to
// front from each pixel's last contributor, transmittance recovered as
// T_j = T_{j+1} / (1 - alpha_j) from the stored final T; per-Gaussian partial
// gradients are summed across the warp with shuffles and added with one
// 16-byte vector atomic per 4 floats (3 atomics per Gaussian per warp), and
// warps with no contributing pixel skip the reduction entirely.
#include "common.cuh"

namespace dg {

template <int B>
__global__ void __launch_bounds__(B * B)
k_render_fwd(const float4* __restrict__ feat, const uint32_t* __restrict__ gid,
             const uint2* __restrict__ ranges, int W, int H, int TX, float bg0, float bg1, float bg2,
             float* __restrict__ img, float* __restrict__ Tout, int* __restrict__ lastout,
             int* __restrict__ exout)
{
    constexpr int NT = B * B;
    __shared__ float4 s_a[NT];  // u, v, A, B
    __shared__ float4 s_b[NT];  // C, o, r, g
    __shared__ float s_c[NT];   // b
    const int tile = blockIdx.x;
    const int tx = tile % TX, ty = tile / TX;
    const int x = tx * B + (int)(threadIdx.x % B), y = ty * B + (int)(threadIdx.x / B);
    const bool inside = x < W && y < H;
    const float pxc = (float)x + 0.5f, pyc = (float)y + 0.5f;
    const uint2 rg = ranges[tile];
    const int n = (int)(rg.y - rg.x);
    float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
    int last = 0, ex = 0;
    bool done = !inside;
    for (int base = 0; base < n; base += NT) {
        if (__syncthreads_count(done) == NT) break;
        const int j = base + (int)threadIdx.x;
        if (j < n) {
            const uint32_t g = gid[rg.x + j];
            s_a[threadIdx.x] = feat[3 * (size_t)g];
            s_b[threadIdx.x] = feat[3 * (size_t)g + 1];
            s_c[threadIdx.x] = feat[3 * (size_t)g + 2].x;
        }
        __syncthreads();
        const int cnt = min(NT, n - base);
        for (int k = 0; k < cnt && !done; ++k) {
            ++ex;
            const float4 a = s_a[k];
            const float4 b = s_b[k];
            const float dx = a.x - pxc, dy = a.y - pyc;
            const float power = -0.5f * (a.z * dx * dx + b.x * dy * dy) - a.w * dx * dy;
            if (power > 0.f) continue;
            const float alpha = fminf(kAlphaMax, b.y * __expf(power));
            if (alpha < kAlphaMin) continue;
            const float Tn = T * (1.f - alpha);
            if (Tn < kTMin) { done = true; break; }
            const float w = alpha * T;
            c0 += w * b.z;
            c1 += w * b.w;
            c2 += w * s_c[k];
            T = Tn;
            last = base + k + 1;
        }
    }
    if (inside) {
        const size_t pix = (size_t)y * W + x, HW = (size_t)W * H;
        img[pix] = c0 + T * bg0;
        img[HW + pix] = c1 + T * bg1;
        img[2 * HW + pix] = c2 + T * bg2;
        Tout[pix] = T;
        lastout[pix] = last;
        if (exout) exout[pix] = ex;
    }
}

__device__ inline float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int B>
__global__ void __launch_bounds__(B * B)
k_render_bwd(const float4* __restrict__ feat, const uint32_t* __restrict__ gid,
             const uint2* __restrict__ ranges, int W, int H, int TX, float bg0, float bg1, float bg2,
             const float* __restrict__ Tfin, const int* __restrict__ lastin,
             const float* __restrict__ dLdimg, float4* __restrict__ grad2d)
{
    constexpr int NT = B * B;
    __shared__ float4 s_a[NT];
    __shared__ float4 s_b[NT];
    __shared__ float s_c[NT];
    __shared__ uint32_t s_g[NT];
    __shared__ int s_n;
    const int tile = blockIdx.x;
    const int tx = tile % TX, ty = tile / TX;
    const int x = tx * B + (int)(threadIdx.x % B), y = ty * B + (int)(threadIdx.x / B);
    const bool inside = x < W && y < H;
    const float pxc = (float)x + 0.5f, pyc = (float)y + 0.5f;
    const uint2 rg = ranges[tile];
    const size_t pix = (size_t)y * W + x, HW = (size_t)W * H;
    float T = 1.f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
    int lastp = 0;
    if (inside) {
        T = Tfin[pix];
        lastp = lastin[pix];
        g0 = dLdimg[pix];
        g1 = dLdimg[HW + pix];
        g2 = dLdimg[2 * HW + pix];
    }
    float S0 = T * bg0, S1 = T * bg1, S2 = T * bg2;  // colour behind the current entry
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    if (lastp > 0) atomicMax(&s_n, lastp);
    __syncthreads();
    // never walk past the tile's own list, whatever `last` holds
    const int n = min(s_n, (int)(rg.y - rg.x));
    const int lane = threadIdx.x & 31;
    for (int base = ((n - 1) / NT) * NT; n > 0 && base >= 0; base -= NT) {
        const int j = base + (int)threadIdx.x;
        if (j < n) {
            const uint32_t g = gid[rg.x + j];
            s_g[threadIdx.x] = g;
            s_a[threadIdx.x] = feat[3 * (size_t)g];
            s_b[threadIdx.x] = feat[3 * (size_t)g + 1];
            s_c[threadIdx.x] = feat[3 * (size_t)g + 2].x;
        }
        __syncthreads();
        const int cnt = min(NT, n - base);
        for (int k = cnt - 1; k >= 0; --k) {
            const float4 a = s_a[k];
            const float4 b = s_b[k];
            const float dx = a.x - pxc, dy = a.y - pyc;
            bool act = base + k < lastp;
            float power = 0.f, G = 0.f, alpha = 0.f;
            bool clamped = false;
            if (act) {
                power = -0.5f * (a.z * dx * dx + b.x * dy * dy) - a.w * dx * dy;
                if (power > 0.f) {
                    act = false;
                } else {
                    G = __expf(power);
                    const float raw = b.y * G;
                    clamped = raw > kAlphaMax;
                    alpha = fminf(kAlphaMax, raw);
                    if (alpha < kAlphaMin) act = false;
                }
            }
            if (!__any_sync(0xffffffffu, act)) continue;
            float du = 0.f, dv = 0.f, dA = 0.f, dB = 0.f, dC = 0.f, dop = 0.f, dr = 0.f, dgc = 0.f, db = 0.f;
            if (act) {
                const float inv = 1.f / (1.f - alpha);
                T *= inv;  // transmittance in front of this entry
                const float wT = alpha * T;
                const float cr = b.z, cg = b.w, cb = s_c[k];
                dr = wT * g0;
                dgc = wT * g1;
                db = wT * g2;
                const float dLda = g0 * (T * cr - S0 * inv) + g1 * (T * cg - S1 * inv) + g2 * (T * cb - S2 * inv);
                S0 += wT * cr;
                S1 += wT * cg;
                S2 += wT * cb;
                if (!clamped) {
                    dop = dLda * G;
                    const float dp = dLda * alpha;
                    du = -dp * (a.z * dx + a.w * dy);
                    dv = -dp * (a.w * dx + b.x * dy);
                    dA = -0.5f * dp * dx * dx;
                    dB = -dp * dx * dy;
                    dC = -0.5f * dp * dy * dy;
                }
            }
            du = warp_sum(du); dv = warp_sum(dv); dA = warp_sum(dA); dB = warp_sum(dB);
            dC = warp_sum(dC); dop = warp_sum(dop); dr = warp_sum(dr); dgc = warp_sum(dgc);
            db = warp_sum(db);
            if (lane == 0) {
                float4* dst = grad2d + 3 * (size_t)s_g[k];
                atomicAdd(dst, make_float4(du, dv, dA, dB));
                atomicAdd(dst + 1, make_float4(dC, dop, dr, dgc));
                atomicAdd(&dst[2].x, db);
            }
        }
        __syncthreads();
    }
}

}  // namespace dg

template <int B>
static void launch_fwd(const float* feat, const uint32_t* gid, const uint32_t* ranges, const dg_camera* cam,
                       const dg_raster_opts* o, float* img, float* T, int* last, int* ex, cudaStream_t s)
{
    const int TX = (cam->width + B - 1) / B, TY = (cam->height + B - 1) / B;
    dg::k_render_fwd<B><<<TX * TY, B * B, 0, s>>>((const float4*)feat, gid, (const uint2*)ranges, cam->width,
                                                  cam->height, TX, o->bg[0], o->bg[1], o->bg[2], img, T, last, ex);
    dg_note_launch();
}

template <int B>
static void launch_bwd(const float* feat, const uint32_t* gid, const uint32_t* ranges, const dg_camera* cam,
                       const dg_raster_opts* o, const float* T, const int* last, const float* dL, float* g2,
                       cudaStream_t s)
{
    const int TX = (cam->width + B - 1) / B, TY = (cam->height + B - 1) / B;
    dg::k_render_bwd<B><<<TX * TY, B * B, 0, s>>>((const float4*)feat, gid, (const uint2*)ranges, cam->width,
                                                  cam->height, TX, o->bg[0], o->bg[1], o->bg[2], T, last, dL,
                                                  (float4*)g2);
    dg_note_launch();
}

static bool render_args(const dg_camera* cam, const dg_raster_opts* opts)
{
    if (!cam || !opts) { dg_set_error("camera/opts null"); return false; }
    if (cam->width <= 0 || cam->height <= 0) { dg_set_error("bad image size"); return false; }
    if (opts->tile != 8 && opts->tile != 16) { dg_set_error("render supports tile 8 or 16, got %d", opts->tile); return false; }
    return true;
}

extern "C" dg_status dg_render_fwd(const float* feat, const uint32_t* gid, const uint32_t* ranges,
                                   const dg_camera* cam, const dg_raster_opts* opts, float* img,
                                   float* T_final, int32_t* last, int32_t* examined, dg_stream stream)
{
    if (!render_args(cam, opts)) return DG_ERR_ARG;
    if (!ranges || !img || !T_final || !last) { dg_set_error("null buffer"); return DG_ERR_ARG; }
    if (feat && (((uintptr_t)feat) & 15u)) { dg_set_error("feat must be 16-byte aligned"); return DG_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    if (opts->tile == 16) launch_fwd<16>(feat, gid, ranges, cam, opts, img, T_final, last, examined, s);
    else launch_fwd<8>(feat, gid, ranges, cam, opts, img, T_final, last, examined, s);
    return dg_check_launch("render_fwd");
}

extern "C" dg_status dg_render_bwd(const float* feat, const uint32_t* gid, const uint32_t* ranges,
                                   const dg_camera* cam, const dg_raster_opts* opts, const float* T_final,
                                   const int32_t* last, const float* dL_dimg, int64_t P, float* grad2d,
                                   dg_stream stream)
{
    if (!render_args(cam, opts)) return DG_ERR_ARG;
    if (P < 0) { dg_set_error("P < 0"); return DG_ERR_ARG; }
    if (!ranges || !T_final || !last || !dL_dimg || (P > 0 && !grad2d)) { dg_set_error("null buffer"); return DG_ERR_ARG; }
    if (grad2d && (((uintptr_t)grad2d) & 15u)) { dg_set_error("grad2d must be 16-byte aligned"); return DG_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    if (P > 0) cudaMemsetAsync(grad2d, 0, sizeof(float) * DG_FEAT_FLOATS * (size_t)P, s);
    if (opts->tile == 16) launch_bwd<16>(feat, gid, ranges, cam, opts, T_final, last, dL_dimg, grad2d, s);
    else launch_bwd<8>(feat, gid, ranges, cam, opts, T_final, last, dL_dimg, grad2d, s);
    return dg_check_launch("render_bwd");
}
