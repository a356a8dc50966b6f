// render.cu -- Eq. 1 compositing per tile (forward) and its adjoint (backward).
//
// Persistent launch over all views: one CTA per resident slot, each taking
// (view, tile) work items from an atomic counter until none are left, so
// tiles of very different cost (list lengths differ by orders of magnitude)
// balance across the SMs and all views of a batch share one launch.  A work
// item is a B x B tile; each thread owns PPT pixels of one column of the
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

// 2^x on the MUFU unit (ex2.approx, flush-to-zero).
__device__ inline float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

constexpr float kLog2e = 1.4426950408889634f;

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

// Views of one launch: image sizes, tile grids and where each view's tiles and
// pixels start in the global tile range table and the concatenated images.
struct RViews {
    int n;
    int total;                      // work items = tiles of all views
    int W[DG_MAX_VIEWS], H[DG_MAX_VIEWS], TX[DG_MAX_VIEWS];
    int toff[DG_MAX_VIEWS + 1];
    long long poff[DG_MAX_VIEWS];   // first pixel of each view
    float bg0, bg1, bg2;
};

struct Item { int tile, v, tx, ty, W, H; long long poff; };

// Next work item of this CTA (item.tile < 0: none left).  Ends with a barrier.
__device__ inline Item next_item(int* counter, const RViews& rv, int* s_item)
{
    if (threadIdx.x == 0) *s_item = atomicAdd(counter, 1);
    __syncthreads();
    Item it;
    it.tile = *s_item;
    __syncthreads();
    if (it.tile >= rv.total) { it.tile = -1; return it; }
    int v = 0;
    while (v + 1 < rv.n && it.tile >= rv.toff[v + 1]) ++v;
    const int t = it.tile - rv.toff[v];
    it.v = v;
    it.tx = t % rv.TX[v];
    it.ty = t / rv.TX[v];
    it.W = rv.W[v];
    it.H = rv.H[v];
    it.poff = rv.poff[v];
    return it;
}

template <int B, int PPT>
__global__ void __launch_bounds__(B * B / PPT)
k_render_fwd(const float4* __restrict__ feat, const uint32_t* __restrict__ gid,
             const uint2* __restrict__ ranges, RViews rv, int* __restrict__ counter,
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
    __shared__ int s_item;
    for (;;) {
    const Item it = next_item(counter, rv, &s_item);
    if (it.tile < 0) break;
    const int tile = it.tile, tx = it.tx, ty = it.ty, W = it.W, H = it.H;
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
            // prescaled: p = log2(e) * power = dx (a' dx + b' dy) + c' dy^2, alpha = 2^(p + log2 o)
            s_a[slot] = make_float4(ga.x, ga.y, -0.5f * kLog2e * ga.z, -kLog2e * ga.w);
            s_b[slot] = make_float4(-0.5f * kLog2e * gb.x, __log2f(gb.y), gb.z, gb.w);
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
            const float adx = a.z * dx;
            alldone = true;
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                if (!done[k]) {
                    const float dy = a.y - pyc[k];
                    const float p = fmaf(dx, fmaf(a.w, dy, adx), b.x * dy * dy);
                    const float alpha = fminf(kAlphaMax, ex2_approx(p + b.y));
                    if (p <= 0.f && alpha >= kAlphaMin) {
                        const float Tn = fmaf(-alpha, T[k], T[k]);
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
    float* im = img + 3 * it.poff;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int y = y0 + k * RSTEP;
        if (x < W && y < H) {
            const size_t pix = (size_t)y * W + x;
            im[pix] = c0[k] + T[k] * rv.bg0;
            im[HW + pix] = c1[k] + T[k] * rv.bg1;
            im[2 * HW + pix] = c2[k] + T[k] * rv.bg2;
            Tout[it.poff + pix] = T[k];
            lastout[it.poff + pix] = last[k];
            // entries visited: up to and including the one that stopped compositing
            if (exout) exout[it.poff + pix] = stop[k] >= 0 ? stop[k] + 1 : n;
            if (blout) blout[it.poff + pix] = nbl[k];
        }
    }
    }  // work items
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
             const uint2* __restrict__ ranges, RViews rv, int* __restrict__ counter,
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
    __shared__ int s_item;
    const float bg0 = rv.bg0, bg1 = rv.bg1, bg2 = rv.bg2;
    for (;;) {
    const Item it = next_item(counter, rv, &s_item);
    if (it.tile < 0) break;
    const int tile = it.tile, tx = it.tx, ty = it.ty, W = it.W, H = it.H;
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
            const float* dl = dLdimg + 3 * it.poff;
            T[k] = Tfin[it.poff + pix];
            lastp[k] = lastin[it.poff + pix];
            g0[k] = dl[pix];
            g1[k] = dl[HW + pix];
            g2[k] = dl[2 * HW + pix];
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
    }  // work items
}

}  // namespace dg

static dg::RViews make_rviews(const dg_camera* cams, int n, int B, const dg_raster_opts* o)
{
    dg::RViews rv;
    rv.n = n;
    int tiles = 0;
    long long pix = 0;
    for (int v = 0; v < n; ++v) {
        rv.W[v] = cams[v].width;
        rv.H[v] = cams[v].height;
        rv.TX[v] = (cams[v].width + B - 1) / B;
        rv.toff[v] = tiles;
        rv.poff[v] = pix;
        tiles += rv.TX[v] * ((cams[v].height + B - 1) / B);
        pix += (long long)cams[v].width * cams[v].height;
    }
    rv.toff[n] = tiles;
    rv.total = tiles;
    rv.bg0 = o->bg[0]; rv.bg1 = o->bg[1]; rv.bg2 = o->bg[2];
    return rv;
}

// CTAs of a persistent launch: every resident slot of the device, at most one per item.
template <typename Kern>
static int persistent_grid(Kern kern, int threads, int items)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0);
    long long g = (long long)(sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
    if (g > items) g = items;
    return (int)(g > 0 ? g : 1);
}

template <int B, int PPT>
static void launch_fwd(const float* feat, const uint32_t* gid, const uint32_t* ranges, const dg::RViews& rv,
                       int* counter, float* img, float* T, int* last, int* ex, int* bl, cudaStream_t s)
{
    auto kern = dg::k_render_fwd<B, PPT>;
    const int grid = persistent_grid(kern, B * B / PPT, rv.total);
    kern<<<grid, B * B / PPT, 0, s>>>((const float4*)feat, gid, (const uint2*)ranges, rv, counter, img, T, last, ex, bl);
    dg_note_launch();
}

template <int B, int PPT>
static void launch_bwd(const float* feat, const uint32_t* gid, const uint32_t* ranges, const dg::RViews& rv,
                       int* counter, const float* T, const int* last, const float* dL, float* g2, cudaStream_t s)
{
    auto kern = dg::k_render_bwd<B, PPT>;
    const int grid = persistent_grid(kern, B * B / PPT, rv.total);
    kern<<<grid, B * B / PPT, 0, s>>>((const float4*)feat, gid, (const uint2*)ranges, rv, counter, T, last, dL,
                                      (float4*)g2);
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

bool dg_check_cameras(const dg_camera* cams, int n_views);

static bool render_args(const dg_camera* cams, int n_views, const dg_raster_opts* opts, void* ws, size_t ws_bytes)
{
    if (!dg_check_cameras(cams, n_views)) return false;
    if (!opts) { dg_set_error("opts null"); return false; }
    if (opts->tile != 8 && opts->tile != 16) { dg_set_error("render supports tile 8 or 16, got %d", opts->tile); return false; }
    const int p = opts->pixels_per_thread;
    if (p != 0 && p != 1 && p != 2 && p != 4) { dg_set_error("pixels_per_thread must be 0, 1, 2 or 4, got %d", p); return false; }
    if (!ws || ws_bytes < dg_render_workspace_size()) { dg_set_error("render workspace missing or too small"); return false; }
    return true;
}

extern "C" size_t dg_render_workspace_size(void) { return 256; }

extern "C" dg_status dg_render_fwd(const float* feat, const uint32_t* gid, const uint32_t* ranges,
                                   const dg_camera* cams, int32_t n_views, const dg_raster_opts* opts, float* img,
                                   float* T_final, int32_t* last, int32_t* examined, int32_t* blended, void* ws,
                                   size_t ws_bytes, dg_stream stream)
{
    if (!render_args(cams, n_views, opts, ws, ws_bytes)) return DG_ERR_ARG;
    if (!ranges || !img || !T_final || !last) { dg_set_error("null buffer"); return DG_ERR_ARG; }
    if (feat && (((uintptr_t)feat) & 15u)) { dg_set_error("feat must be 16-byte aligned"); return DG_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    const dg::RViews rv = make_rviews(cams, n_views, opts->tile, opts);
    int* counter = (int*)ws;
    cudaMemsetAsync(counter, 0, sizeof(int), s);
    const int ppt = resolve_ppt(opts, false);
    if (opts->tile == 8) launch_fwd<8, 1>(feat, gid, ranges, rv, counter, img, T_final, last, examined, blended, s);
    else if (ppt == 1) launch_fwd<16, 1>(feat, gid, ranges, rv, counter, img, T_final, last, examined, blended, s);
    else if (ppt == 2) launch_fwd<16, 2>(feat, gid, ranges, rv, counter, img, T_final, last, examined, blended, s);
    else launch_fwd<16, 4>(feat, gid, ranges, rv, counter, img, T_final, last, examined, blended, s);
    return dg_check_launch("render_fwd");
}

extern "C" dg_status dg_render_bwd(const float* feat, const uint32_t* gid, const uint32_t* ranges,
                                   const dg_camera* cams, int32_t n_views, const dg_raster_opts* opts,
                                   const float* T_final, const int32_t* last, const float* dL_dimg, int64_t n_records,
                                   float* grad2d, void* ws, size_t ws_bytes, dg_stream stream)
{
    if (!render_args(cams, n_views, opts, ws, ws_bytes)) return DG_ERR_ARG;
    if (n_records < 0) { dg_set_error("n_records < 0"); return DG_ERR_ARG; }
    if (!ranges || !T_final || !last || !dL_dimg || (n_records > 0 && !grad2d)) { dg_set_error("null buffer"); return DG_ERR_ARG; }
    if (grad2d && (((uintptr_t)grad2d) & 15u)) { dg_set_error("grad2d must be 16-byte aligned"); return DG_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    if (n_records > 0) cudaMemsetAsync(grad2d, 0, sizeof(float) * DG_FEAT_FLOATS * (size_t)n_records, s);
    const dg::RViews rv = make_rviews(cams, n_views, opts->tile, opts);
    int* counter = (int*)ws;
    cudaMemsetAsync(counter, 0, sizeof(int), s);
    const int ppt = resolve_ppt(opts, true);
    if (opts->tile == 8) launch_bwd<8, 1>(feat, gid, ranges, rv, counter, T_final, last, dL_dimg, grad2d, s);
    else if (ppt == 1) launch_bwd<16, 1>(feat, gid, ranges, rv, counter, T_final, last, dL_dimg, grad2d, s);
    else if (ppt == 2) launch_bwd<16, 2>(feat, gid, ranges, rv, counter, T_final, last, dL_dimg, grad2d, s);
    else launch_bwd<16, 4>(feat, gid, ranges, rv, counter, T_final, last, dL_dimg, grad2d, s);
    return dg_check_launch("render_bwd");
}
