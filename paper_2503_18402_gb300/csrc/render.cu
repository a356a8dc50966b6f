// render.cu -- Eq. 1 compositing per tile (forward) and its adjoint (backward).
//
// One CTA per B x B tile; each thread owns PPT pixels of one column of the
// tile (rows ly, ly + B/PPT, ...).  The tile's sorted list is streamed through
// shared memory in batches of B*B/PPT records (one coalesced 48-byte gather per
// thread per batch); every staged record is then evaluated for the thread's
// PPT pixels, so shared-memory loads and loop control are shared by PPT
// evaluations.
//   Forward: front to back; a CTA stops once every pixel has terminated
//   (__syncthreads_count).
//   Backward: back to front from each pixel's last contributor; the
//   transmittance in front of entry j is recovered as T_j = T_{j+1} / (1 - a_j)
//   from the stored final T.  A thread first sums its PPT pixels' partial
//   gradients, the warp then sums the nine values by recursive halving (12
//   shuffles) and nine lanes add the totals with one atomic instruction; warps
//   with no contributing pixel skip the reduction.  Larger PPT divides the reduction
//   and atomic cost per evaluated (pixel, Gaussian) entry.
// Tile-level skip: while a batch is staged, each entry is tested once against
// the whole tile: the minimum of its quadratic form over the rectangle of the
// tile's pixel centres (closed form on the four edges when the mean lies
// outside).  If even that maximum alpha is below 1/255 (with a margin that
// absorbs float32 rounding of the per-pixel evaluation), every pixel would
// skip the entry, so it is dropped from the batch (stable compaction; the
// original list position is kept for `last`).  Results are unchanged.
#include "common.cuh"

namespace dg {

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
        if (e < 2) {
            dx = e ? dxh : dxl;
            dy = fminf(fmaxf(-B * dx / C, dyl), dyh);
        } else {
            dy = (e & 1) ? dyh : dyl;
            dx = fminf(fmaxf(-B * dy / A, dxl), dxh);
        }
        const float f = A * dx * dx + 2.f * B * dx * dy + C * dy * dy;
        const float mag = A * dx * dx + 2.f * fabsf(B * dx * dy) + C * dy * dy;
        best = fminf(best, f - 1e-5f * mag);
    }
    return best;
}

// True when no pixel centre of the tile [px0, px1] x [py0, py1] can give the
// Gaussian an alpha >= 1/255.
__device__ inline bool tile_skip(const float4& a, const float4& b, float px0, float px1, float py0, float py1)
{
    const float o = b.y;
    if (!(o >= kAlphaMin)) return true;  // alpha <= o < 1/255 everywhere
    const float fmin = quad_min_box(a.z, a.w, b.x, a.x - px1, a.x - px0, a.y - py1, a.y - py0);
    // alpha = o exp(-fmin/2) < 1/255  <=>  fmin > 2 ln(255 o); 0.02 absorbs the
    // per-pixel rounding of the power and of exp
    return fmin > 2.f * logf(255.f * o) + 0.02f;
}

// Stable block-wide compaction index of `keep`; *total = number kept.  Ends with a barrier.
template <int NT>
__device__ inline int compact_index(bool keep, int* s_w, int* total)
{
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) s_w[w] = __popc(bal);
    __syncthreads();
    int pre = 0, tot = 0;
#pragma unroll
    for (int i = 0; i < NW; ++i) {
        const int c = s_w[i];
        pre += i < w ? c : 0;
        tot += c;
    }
    *total = tot;
    __syncthreads();
    return pre + __popc(bal & ((1u << lane) - 1u));
}

template <int B, int PPT>
__global__ void __launch_bounds__(B * B / PPT)
k_render_fwd(const float4* __restrict__ feat, const uint32_t* __restrict__ gid,
             const uint2* __restrict__ ranges, int W, int H, int TX, float bg0, float bg1, float bg2,
             float* __restrict__ img, float* __restrict__ Tout, int* __restrict__ lastout,
             int* __restrict__ exout, int* __restrict__ blout)
{
    constexpr int NT = B * B / PPT;
    constexpr int RSTEP = B / PPT;  // row step between a thread's pixels
    __shared__ float4 s_a[NT];  // u, v, A, B
    __shared__ float4 s_b[NT];  // C, o, r, g
    __shared__ float s_c[NT];   // b
    __shared__ int s_pos[NT];   // list position
    __shared__ int s_w[NT / 32];
    const int tile = blockIdx.x;
    const int tx = tile % TX, ty = tile / TX;
    const int x = tx * B + (int)(threadIdx.x % B);
    const int y0 = ty * B + (int)(threadIdx.x / B);
    const float pxc = (float)x + 0.5f;
    const float tpx0 = (float)(tx * B) + 0.5f, tpx1 = tpx0 + (float)(B - 1);
    const float tpy0 = (float)(ty * B) + 0.5f, tpy1 = tpy0 + (float)(B - 1);
    float pyc[PPT], T[PPT], c0[PPT], c1[PPT], c2[PPT];
    int last[PPT], stop[PPT], nbl[PPT];
    bool done[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int y = y0 + k * RSTEP;
        pyc[k] = (float)y + 0.5f;
        T[k] = 1.f; c0[k] = c1[k] = c2[k] = 0.f;
        last[k] = 0; stop[k] = -1; nbl[k] = 0;
        done[k] = !(x < W && y < H);
    }
    bool alldone = true;
#pragma unroll
    for (int k = 0; k < PPT; ++k) alldone = alldone && done[k];
    const uint2 rg = ranges[tile];
    const int n = (int)(rg.y - rg.x);
    for (int base = 0; base < n; base += NT) {
        if (__syncthreads_count(alldone) == NT) break;
        const int j = base + (int)threadIdx.x;
        bool keep = false;
        float4 ga, gb;
        float gc = 0.f;
        if (j < n) {
            const uint32_t g = gid[rg.x + j];
            ga = feat[3 * (size_t)g];
            gb = feat[3 * (size_t)g + 1];
            gc = feat[3 * (size_t)g + 2].x;
            keep = !tile_skip(ga, gb, tpx0, tpx1, tpy0, tpy1);
        }
        int cnt;
        const int slot = compact_index<NT>(keep, s_w, &cnt);
        if (keep) {
            s_a[slot] = ga;
            s_b[slot] = gb;
            s_c[slot] = gc;
            s_pos[slot] = j;
        }
        __syncthreads();
        for (int kk = 0; kk < cnt && !alldone; ++kk) {
            const float4 a = s_a[kk];
            const float4 b = s_b[kk];
            const float cb = s_c[kk];
            const int pos = s_pos[kk];
            const float dx = a.x - pxc;
            alldone = true;
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                if (!done[k]) {
                    const float dy = a.y - pyc[k];
                    const float power = -0.5f * (a.z * dx * dx + b.x * dy * dy) - a.w * dx * dy;
                    const float alpha = fminf(kAlphaMax, b.y * __expf(power));
                    if (power <= 0.f && alpha >= kAlphaMin) {
                        const float Tn = T[k] * (1.f - alpha);
                        if (Tn < kTMin) {
                            done[k] = true;
                            stop[k] = pos;
                        } else {
                            const float w = alpha * T[k];
                            c0[k] += w * b.z;
                            c1[k] += w * b.w;
                            c2[k] += w * cb;
                            T[k] = Tn;
                            last[k] = pos + 1;
                            ++nbl[k];
                        }
                    }
                }
                alldone = alldone && done[k];
            }
        }
    }
    const size_t HW = (size_t)W * H;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int y = y0 + k * RSTEP;
        if (x < W && y < H) {
            const size_t pix = (size_t)y * W + x;
            img[pix] = c0[k] + T[k] * bg0;
            img[HW + pix] = c1[k] + T[k] * bg1;
            img[2 * HW + pix] = c2[k] + T[k] * bg2;
            Tout[pix] = T[k];
            lastout[pix] = last[k];
            // entries visited: up to and including the one that stopped compositing
            if (exout) exout[pix] = stop[k] >= 0 ? stop[k] + 1 : n;
            if (blout) blout[pix] = nbl[k];
        }
    }
}

// Sum of 9 per-lane values over the warp by recursive halving: at each step a
// lane keeps half of its values and receives its partner's partial sums of
// that half (12 shuffles instead of 45).  Returns the total of value `*idx`
// (0..8) on the lanes where *idx is valid (*idx = -1 elsewhere); both lanes of
// each final pair hold it, only the even one reports it.
__device__ inline float warp_sum9(const float v[9], int lane, int* idx)
{
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
    float a1[6];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const float lo = v[i], hi = i + 5 < 9 ? v[i + 5] : 0.f;
        const float keep = b4 ? hi : lo, send = b4 ? lo : hi;
        a1[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    a1[5] = 0.f;
    float a2[4];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float keep = b3 ? a1[i + 3] : a1[i], send = b3 ? a1[i] : a1[i + 3];
        a2[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    a2[3] = 0.f;
    float a3[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float keep = b2 ? a2[i + 2] : a2[i], send = b2 ? a2[i] : a2[i + 2];
        a3[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    float a4;
    {
        const float keep = b1 ? a3[1] : a3[0], send = b1 ? a3[0] : a3[1];
        a4 = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
    a4 += __shfl_xor_sync(0xffffffffu, a4, 1);
    const int i2 = (b2 ? 2 : 0) + (b1 ? 1 : 0);        // index into a2 (3 = padding)
    const int i1 = (b3 ? 3 : 0) + i2;                   // index into a1 (5 = padding)
    const int i0 = (b4 ? 5 : 0) + i1;                   // original index (9 = padding)
    *idx = ((lane & 1) == 0 && i2 < 3 && i1 < 5 && i0 < 9) ? i0 : -1;
    return a4;
}

template <int B, int PPT>
__global__ void __launch_bounds__(B * B / PPT)
k_render_bwd(const float4* __restrict__ feat, const uint32_t* __restrict__ gid,
             const uint2* __restrict__ ranges, int W, int H, int TX, float bg0, float bg1, float bg2,
             const float* __restrict__ Tfin, const int* __restrict__ lastin,
             const float* __restrict__ dLdimg, float4* __restrict__ grad2d)
{
    constexpr int NT = B * B / PPT;
    constexpr int RSTEP = B / PPT;
    __shared__ float4 s_a[NT];
    __shared__ float4 s_b[NT];
    __shared__ float s_c[NT];
    __shared__ uint32_t s_g[NT];
    __shared__ int s_pos[NT];
    __shared__ int s_w[NT / 32];
    __shared__ int s_n;
    const int tile = blockIdx.x;
    const int tx = tile % TX, ty = tile / TX;
    const int x = tx * B + (int)(threadIdx.x % B);
    const int y0 = ty * B + (int)(threadIdx.x / B);
    const float pxc = (float)x + 0.5f;
    const float tpx0 = (float)(tx * B) + 0.5f, tpx1 = tpx0 + (float)(B - 1);
    const float tpy0 = (float)(ty * B) + 0.5f, tpy1 = tpy0 + (float)(B - 1);
    const uint2 rg = ranges[tile];
    const size_t HW = (size_t)W * H;
    float pyc[PPT], T[PPT], g0[PPT], g1[PPT], g2[PPT], S0[PPT], S1[PPT], S2[PPT];
    int lastp[PPT];
    int mylast = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int y = y0 + k * RSTEP;
        pyc[k] = (float)y + 0.5f;
        T[k] = 1.f; g0[k] = g1[k] = g2[k] = 0.f; lastp[k] = 0;
        if (x < W && y < H) {
            const size_t pix = (size_t)y * W + x;
            T[k] = Tfin[pix];
            lastp[k] = lastin[pix];
            g0[k] = dLdimg[pix];
            g1[k] = dLdimg[HW + pix];
            g2[k] = dLdimg[2 * HW + pix];
        }
        S0[k] = T[k] * bg0; S1[k] = T[k] * bg1; S2[k] = T[k] * bg2;  // colour behind the current entry
        mylast = max(mylast, lastp[k]);
    }
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    if (mylast > 0) atomicMax(&s_n, mylast);
    __syncthreads();
    // never walk past the tile's own list, whatever `last` holds
    const int n = min(s_n, (int)(rg.y - rg.x));
    const int lane = threadIdx.x & 31;
    for (int base = ((n - 1) / NT) * NT; n > 0 && base >= 0; base -= NT) {
        const int j = base + (int)threadIdx.x;
        bool keep = false;
        float4 ga, gb;
        float gc = 0.f;
        uint32_t g = 0;
        if (j < n) {
            g = gid[rg.x + j];
            ga = feat[3 * (size_t)g];
            gb = feat[3 * (size_t)g + 1];
            gc = feat[3 * (size_t)g + 2].x;
            keep = !tile_skip(ga, gb, tpx0, tpx1, tpy0, tpy1);
        }
        int cnt;
        const int slot = compact_index<NT>(keep, s_w, &cnt);
        if (keep) {
            s_g[slot] = g;
            s_a[slot] = ga;
            s_b[slot] = gb;
            s_c[slot] = gc;
            s_pos[slot] = j;
        }
        __syncthreads();
        for (int kk = cnt - 1; kk >= 0; --kk) {
            const int pos = s_pos[kk];
            if (!__any_sync(0xffffffffu, pos < mylast)) continue;
            const float4 a = s_a[kk];
            const float4 b = s_b[kk];
            const float cr = b.z, cg = b.w, cb = s_c[kk];
            const float dx = a.x - pxc;
            float du = 0.f, dv = 0.f, dA = 0.f, dB = 0.f, dC = 0.f, dop = 0.f, dr = 0.f, dgc = 0.f, db = 0.f;
            bool any = false;
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                if (pos < lastp[k]) {
                    const float dy = a.y - pyc[k];
                    const float power = -0.5f * (a.z * dx * dx + b.x * dy * dy) - a.w * dx * dy;
                    const float G = __expf(power);
                    const float raw = b.y * G;
                    const float alpha = fminf(kAlphaMax, raw);
                    if (power <= 0.f && alpha >= kAlphaMin) {
                        any = true;
                        const float inv = 1.f / (1.f - alpha);
                        T[k] *= inv;  // transmittance in front of this entry
                        const float wT = alpha * T[k];
                        dr += wT * g0[k];
                        dgc += wT * g1[k];
                        db += wT * g2[k];
                        const float dLda = g0[k] * (T[k] * cr - S0[k] * inv) + g1[k] * (T[k] * cg - S1[k] * inv) +
                                           g2[k] * (T[k] * cb - S2[k] * inv);
                        S0[k] += wT * cr;
                        S1[k] += wT * cg;
                        S2[k] += wT * cb;
                        if (raw <= kAlphaMax) {
                            dop += dLda * G;
                            const float dp = dLda * alpha;
                            du -= dp * (a.z * dx + a.w * dy);
                            dv -= dp * (a.w * dx + b.x * dy);
                            dA -= 0.5f * dp * dx * dx;
                            dB -= dp * dx * dy;
                            dC -= 0.5f * dp * dy * dy;
                        }
                    }
                }
            }
            if (!__any_sync(0xffffffffu, any)) continue;
            const float vals[9] = {du, dv, dA, dB, dC, dop, dr, dgc, db};
            int idx;
            const float tot = warp_sum9(vals, lane, &idx);
            if (idx >= 0) atomicAdd((float*)(grad2d + 3 * (size_t)s_g[kk]) + idx, tot);
        }
        __syncthreads();
    }
}

}  // namespace dg

template <int B, int PPT>
static void launch_fwd(const float* feat, const uint32_t* gid, const uint32_t* ranges, const dg_camera* cam,
                       const dg_raster_opts* o, float* img, float* T, int* last, int* ex, int* bl, cudaStream_t s)
{
    const int TX = (cam->width + B - 1) / B, TY = (cam->height + B - 1) / B;
    dg::k_render_fwd<B, PPT><<<TX * TY, B * B / PPT, 0, s>>>((const float4*)feat, gid, (const uint2*)ranges,
                                                             cam->width, cam->height, TX, o->bg[0], o->bg[1],
                                                             o->bg[2], img, T, last, ex, bl);
    dg_note_launch();
}

template <int B, int PPT>
static void launch_bwd(const float* feat, const uint32_t* gid, const uint32_t* ranges, const dg_camera* cam,
                       const dg_raster_opts* o, const float* T, const int* last, const float* dL, float* g2,
                       cudaStream_t s)
{
    const int TX = (cam->width + B - 1) / B, TY = (cam->height + B - 1) / B;
    dg::k_render_bwd<B, PPT><<<TX * TY, B * B / PPT, 0, s>>>((const float4*)feat, gid, (const uint2*)ranges,
                                                             cam->width, cam->height, TX, o->bg[0], o->bg[1],
                                                             o->bg[2], T, last, dL, (float4*)g2);
    dg_note_launch();
}

// Pixels per thread used for (tile, request): tile 16 -> 1, 2 or 4 (0 selects
// the default of each pass), tile 8 -> 1.
static int resolve_ppt(const dg_raster_opts* o, bool backward)
{
    if (o->tile == 8) return 1;
    const int req = o->pixels_per_thread;
    if (req == 1 || req == 2 || req == 4) return req;
    return backward ? 4 : 2;
}

static bool render_args(const dg_camera* cam, const dg_raster_opts* opts)
{
    if (!cam || !opts) { dg_set_error("camera/opts null"); return false; }
    if (cam->width <= 0 || cam->height <= 0) { dg_set_error("bad image size"); return false; }
    if (opts->tile != 8 && opts->tile != 16) { dg_set_error("render supports tile 8 or 16, got %d", opts->tile); return false; }
    const int p = opts->pixels_per_thread;
    if (p != 0 && p != 1 && p != 2 && p != 4) { dg_set_error("pixels_per_thread must be 0, 1, 2 or 4, got %d", p); return false; }
    return true;
}

extern "C" dg_status dg_render_fwd(const float* feat, const uint32_t* gid, const uint32_t* ranges,
                                   const dg_camera* cam, const dg_raster_opts* opts, float* img,
                                   float* T_final, int32_t* last, int32_t* examined, int32_t* blended,
                                   dg_stream stream)
{
    if (!render_args(cam, opts)) return DG_ERR_ARG;
    if (!ranges || !img || !T_final || !last) { dg_set_error("null buffer"); return DG_ERR_ARG; }
    if (feat && (((uintptr_t)feat) & 15u)) { dg_set_error("feat must be 16-byte aligned"); return DG_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    const int ppt = resolve_ppt(opts, false);
    if (opts->tile == 8) launch_fwd<8, 1>(feat, gid, ranges, cam, opts, img, T_final, last, examined, blended, s);
    else if (ppt == 1) launch_fwd<16, 1>(feat, gid, ranges, cam, opts, img, T_final, last, examined, blended, s);
    else if (ppt == 2) launch_fwd<16, 2>(feat, gid, ranges, cam, opts, img, T_final, last, examined, blended, s);
    else launch_fwd<16, 4>(feat, gid, ranges, cam, opts, img, T_final, last, examined, blended, s);
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
    const int ppt = resolve_ppt(opts, true);
    if (opts->tile == 8) launch_bwd<8, 1>(feat, gid, ranges, cam, opts, T_final, last, dL_dimg, grad2d, s);
    else if (ppt == 1) launch_bwd<16, 1>(feat, gid, ranges, cam, opts, T_final, last, dL_dimg, grad2d, s);
    else if (ppt == 2) launch_bwd<16, 2>(feat, gid, ranges, cam, opts, T_final, last, dL_dimg, grad2d, s);
    else launch_bwd<16, 4>(feat, gid, ranges, cam, opts, T_final, last, dL_dimg, grad2d, s);
    return dg_check_launch("render_bwd");
}
