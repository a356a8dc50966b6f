// ssim.cu -- the backbone's photometric loss (1 - lambda) L1 + lambda (1 - SSIM)
// and its gradient, for one or several views per call.
//
// SSIM (Wang et al. 2004): per channel, window sums under an 11 x 11 Gaussian
// (sigma 1.5, normalised, zero padding outside the image) give mu_x, mu_y and
// a = E[x^2], b = E[y^2], c = E[xy]; per pixel
//   S = (2 mu_x mu_y + C1)(2 (c - mu_x mu_y) + C2)
//       / ((mu_x^2 + mu_y^2 + C1)((a - mu_x^2) + (b - mu_y^2) + C2)).
// Its gradient is the adjoint of the window sums applied to three per-pixel
// partial derivatives of S (with respect to mu_x, a and c):
//   dS/dx(q) = F[dS/dmu_x](q) + 2 x(q) F[dS/da](q) + y(q) F[dS/dc](q),
// F the same symmetric, zero-padded window.
//
// Two passes over 32 x 32 output tiles (256 threads, 4 rows each): the
// forward stages the tile and a 5-pixel halo of x and y in shared memory,
// runs the horizontal then the vertical 11-tap sums of four statistics (mu_x,
// mu_y, a + b, c: S uses a and b only through their sum),
// and writes the three partial-derivative maps plus per-block sums of S and
// |x - y|; the backward stages the maps with their halo, filters them the same
// way and writes dL/dx including the L1 term.  A last one-block kernel sums
// the block partials per view in a fixed order (FP64).
// HBM per pixel and channel: forward reads x, y (8 B) and writes 3 maps
// (12 B); backward reads the maps and x, y (20 B) and writes dL/dx (4 B).
#include <math.h>

#include "common.cuh"

namespace dg {
namespace {

constexpr int SS_T = 32;             // output tile edge
constexpr int SS_R = 5;              // window radius
constexpr int SS_E = SS_T + 2 * SS_R; // staged edge (42)
constexpr int SS_THREADS = 256;      // 32 x 8
constexpr float kC1 = 0.01f * 0.01f;
constexpr float kC2 = 0.03f * 0.03f;

struct Win { float w[2 * SS_R + 1]; };

struct SViews {
    int n;
    int W[DG_MAX_VIEWS], H[DG_MAX_VIEWS], TX[DG_MAX_VIEWS], TY[DG_MAX_VIEWS];
    int boff[DG_MAX_VIEWS + 1];    // first block of each view (3 channels x tiles)
    long long poff[DG_MAX_VIEWS];  // first pixel of each view
};

struct Blk { int v, ch, tx, ty, W, H; long long plane; };

__device__ inline Blk decode(const SViews& sv)
{
    Blk b;
    const int i = blockIdx.x;
    int v = 0;
    while (v + 1 < sv.n && i >= sv.boff[v + 1]) ++v;
    const int r = i - sv.boff[v];
    const int per = sv.TX[v] * sv.TY[v];
    b.v = v;
    b.ch = r / per;
    const int t = r % per;
    b.tx = t % sv.TX[v];
    b.ty = t / sv.TX[v];
    b.W = sv.W[v];
    b.H = sv.H[v];
    b.plane = 3 * sv.poff[v] + (long long)b.ch * b.W * b.H;  // first element of this channel plane
    return b;
}

// Stage plane[y0 - R .. y0 + T + R) x [x0 - R ..) into s (zero outside the image).
// Thread t < 252 keeps column t % 42 and takes the rows t / 42 + 6 k (k < 7),
// so its column test and offsets are formed once; all of its loads are issued
// before its first shared store.
constexpr int SS_SR = SS_THREADS / SS_E;  // staged rows per pass (6)
static_assert(SS_E % SS_SR == 0, "the staged rows split evenly into passes");
__device__ inline void stage(const float* __restrict__ plane, int W, int H, int x0, int y0, float (*s)[SS_E + 1])
{
    constexpr int NR = SS_E / SS_SR;
    const int t = threadIdx.x;
    if (t >= SS_SR * SS_E) return;
    const int c = t % SS_E, r0 = t / SS_E;
    const int x = x0 - SS_R + c;
    const bool xok = x >= 0 && x < W;
    const int ys = y0 - SS_R + r0;
    float v[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        const int y = ys + SS_SR * k;
        v[k] = (xok && y >= 0 && y < H) ? plane[(size_t)y * W + x] : 0.f;
    }
#pragma unroll
    for (int k = 0; k < NR; ++k) s[r0 + SS_SR * k][c] = v[k];
}

// Work split of the two window passes: the horizontal pass gives each thread
// SS_SL adjacent outputs of one staged row (one load per input, reused by the
// SS_SL sums), the vertical pass SS_SL adjacent output rows of one column.
constexpr int SS_SL = 4;
static_assert((SS_THREADS / 32) * SS_SL == SS_T && SS_T / SS_SL == 8, "vertical: one warp per SS_SL rows; horizontal: 8 groups per row");

__global__ void __launch_bounds__(SS_THREADS)
k_ssim_fwd(const float* __restrict__ img, const float* __restrict__ tgt, SViews sv, Win win,
           float* __restrict__ dm, float* __restrict__ da, float* __restrict__ dc, float2* __restrict__ part)
{
    __shared__ float sx[SS_E][SS_E + 1];
    __shared__ float sy[SS_E][SS_E + 1];
    // horizontal sums: mu_x, mu_y, a + b, c (S needs E[x^2] and E[y^2] only
    // through their sum, so one window sum serves both)
    __shared__ float hs[4][SS_E][SS_T];
    __shared__ float red[2][SS_THREADS / 32];
    const Blk b = decode(sv);
    const int x0 = b.tx * SS_T, y0 = b.ty * SS_T;
    stage(img + b.plane, b.W, b.H, x0, y0, sx);
    stage(tgt + b.plane, b.W, b.H, x0, y0, sy);
    __syncthreads();
    // (lanes: 8 groups of SS_SL columns x 4 rows per warp; banks all distinct)
    for (int it = threadIdx.x; it < SS_E * (SS_T / SS_SL); it += SS_THREADS) {
        const int r = it / (SS_T / SS_SL), c0 = (it % (SS_T / SS_SL)) * SS_SL;
        float xv[SS_SL + 2 * SS_R], yv[SS_SL + 2 * SS_R];
#pragma unroll
        for (int q = 0; q < SS_SL + 2 * SS_R; ++q) { xv[q] = sx[r][c0 + q]; yv[q] = sy[r][c0 + q]; }
#pragma unroll
        for (int o = 0; o < SS_SL; ++o) {
            float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
            for (int k = 0; k <= 2 * SS_R; ++k) {
                const float x = xv[o + k], y = yv[o + k], w = win.w[k];
                s0 = fmaf(w, x, s0);
                s1 = fmaf(w, y, s1);
                s2 = fmaf(w, fmaf(x, x, y * y), s2);
                s3 = fmaf(w, x * y, s3);
            }
            hs[0][r][c0 + o] = s0; hs[1][r][c0 + o] = s1; hs[2][r][c0 + o] = s2;
            hs[3][r][c0 + o] = s3;
        }
    }
    __syncthreads();
    // vertical pass: lane = column, warp w = output rows SS_SL w .. SS_SL w + SS_SL - 1
    const int c = threadIdx.x & 31, rb = (threadIdx.x >> 5) * SS_SL;
    float st[4][SS_SL];  // window sums of the four statistics at this thread's outputs
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        float col[SS_SL + 2 * SS_R];
#pragma unroll
        for (int q = 0; q < SS_SL + 2 * SS_R; ++q) col[q] = hs[t][rb + q][c];
#pragma unroll
        for (int j = 0; j < SS_SL; ++j) {
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k <= 2 * SS_R; ++k) acc = fmaf(win.w[k], col[j + k], acc);
            st[t][j] = acc;
        }
    }
    float ssum = 0.f, l1sum = 0.f;
#pragma unroll
    for (int j = 0; j < SS_SL; ++j) {
        const int r = rb + j;
        const int x = x0 + c, y = y0 + r;
        if (x >= b.W || y >= b.H) continue;
        const float mx = st[0][j], my = st[1][j], ab = st[2][j], cc = st[3][j];
        const float A1 = 2.f * mx * my + kC1;
        const float A2 = 2.f * (cc - mx * my) + kC2;
        const float B1 = mx * mx + my * my + kC1;
        const float B2 = (ab - mx * mx - my * my) + kC2;
        const float inv = 1.f / (B1 * B2);
        const float S = A1 * A2 * inv;
        const size_t o = (size_t)b.plane + (size_t)y * b.W + x;
        dm[o] = 2.f * my * (A2 - A1) * inv - 2.f * mx * S * (B2 - B1) * inv;
        da[o] = -S * B1 * inv;
        dc[o] = 2.f * A1 * inv;
        ssum += S;
        l1sum += fabsf(sx[r + SS_R][c + SS_R] - sy[r + SS_R][c + SS_R]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ssum += __shfl_xor_sync(0xffffffffu, ssum, o);
        l1sum += __shfl_xor_sync(0xffffffffu, l1sum, o);
    }
    if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = ssum; red[1][threadIdx.x >> 5] = l1sum; }
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f, l = 0.f;
        for (int w = 0; w < SS_THREADS / 32; ++w) { s += red[0][w]; l += red[1][w]; }
        part[blockIdx.x] = make_float2(s, l);
    }
}

__global__ void __launch_bounds__(SS_THREADS, 4)
k_ssim_bwd(const float* __restrict__ img, const float* __restrict__ tgt, SViews sv, Win win,
           const float* __restrict__ dm, const float* __restrict__ da, const float* __restrict__ dc,
           float lam, float* __restrict__ grad)
{
    __shared__ float s0[SS_E][SS_E + 1];
    __shared__ float s1[SS_E][SS_E + 1];
    __shared__ float s2[SS_E][SS_E + 1];
    __shared__ float hs[3][SS_E][SS_T];
    const Blk b = decode(sv);
    const int x0 = b.tx * SS_T, y0 = b.ty * SS_T;
    // this thread's outputs (column c, rows rb ..): their x and y are loaded
    // first, so the loads' latency passes during the window sums
    const int c = threadIdx.x & 31, rb = (threadIdx.x >> 5) * SS_SL;
    float xo[SS_SL], yo[SS_SL];
#pragma unroll
    for (int j = 0; j < SS_SL; ++j) {
        const int x = x0 + c, y = y0 + rb + j;
        const bool in = x < b.W && y < b.H;
        const size_t o = (size_t)b.plane + (size_t)(in ? y : 0) * b.W + (in ? x : 0);
        xo[j] = in ? img[o] : 0.f;
        yo[j] = in ? tgt[o] : 0.f;
    }
    stage(dm + b.plane, b.W, b.H, x0, y0, s0);
    stage(da + b.plane, b.W, b.H, x0, y0, s1);
    stage(dc + b.plane, b.W, b.H, x0, y0, s2);
    __syncthreads();
    for (int it = threadIdx.x; it < SS_E * (SS_T / SS_SL); it += SS_THREADS) {
        const int r = it / (SS_T / SS_SL), c0 = (it % (SS_T / SS_SL)) * SS_SL;
        float v0[SS_SL + 2 * SS_R], v1[SS_SL + 2 * SS_R], v2[SS_SL + 2 * SS_R];
#pragma unroll
        for (int q = 0; q < SS_SL + 2 * SS_R; ++q) { v0[q] = s0[r][c0 + q]; v1[q] = s1[r][c0 + q]; v2[q] = s2[r][c0 + q]; }
#pragma unroll
        for (int o = 0; o < SS_SL; ++o) {
            float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
            for (int k = 0; k <= 2 * SS_R; ++k) {
                const float w = win.w[k];
                a0 = fmaf(w, v0[o + k], a0);
                a1 = fmaf(w, v1[o + k], a1);
                a2 = fmaf(w, v2[o + k], a2);
            }
            hs[0][r][c0 + o] = a0; hs[1][r][c0 + o] = a1; hs[2][r][c0 + o] = a2;
        }
    }
    __syncthreads();
    // d/dx of the mean over views of (1 - lam) mean|x - y| + lam (1 - mean S)
    const float scale = 1.f / ((float)sv.n * 3.f * (float)b.W * (float)b.H);
    float fs[3][SS_SL];  // filtered partial-derivative maps at this thread's outputs
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        float col[SS_SL + 2 * SS_R];
#pragma unroll
        for (int q = 0; q < SS_SL + 2 * SS_R; ++q) col[q] = hs[t][rb + q][c];
#pragma unroll
        for (int j = 0; j < SS_SL; ++j) {
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k <= 2 * SS_R; ++k) acc = fmaf(win.w[k], col[j + k], acc);
            fs[t][j] = acc;
        }
    }
#pragma unroll
    for (int j = 0; j < SS_SL; ++j) {
        const int r = rb + j;
        const int x = x0 + c, y = y0 + r;
        if (x >= b.W || y >= b.H) continue;
        const float f0 = fs[0][j], f1 = fs[1][j], f2 = fs[2][j];
        const size_t o = (size_t)b.plane + (size_t)y * b.W + x;
        const float xv = xo[j], yv = yo[j];
        const float dS = f0 + 2.f * xv * f1 + yv * f2;
        const float d = xv - yv;
        const float sg = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
        grad[o] = scale * ((1.f - lam) * sg - lam * dS);
    }
}

// loss[v] = (1 - lam) l1_v + lam (1 - ssim_v); loss[n] = mean over views.
// One block of four warps per view (at most 32 warps; at 16 views two per
// view): each warp sums a fixed stride of its view's block partials in FP64,
// and the warps' sums and then the views' losses are added in a fixed order,
// so the result does not depend on timing.  (One block of 32 warps for any
// view count made the one-view sum slower: 12 -> 19 us.)
constexpr int SS_FINAL_THREADS = 1024;
__host__ __device__ inline int ssim_final_warps(int n_views) { return 4 * n_views < 32 ? 4 * n_views : 32; }
__global__ void __launch_bounds__(SS_FINAL_THREADS)
k_ssim_final(const float2* __restrict__ part, SViews sv, float lam, float* __restrict__ loss)
{
    constexpr int NWMAX = SS_FINAL_THREADS / 32;
    __shared__ double sm[2][NWMAX];
    __shared__ double lv_s[DG_MAX_VIEWS];
    const int nv = sv.n;
    const int wpv = ssim_final_warps(nv) / nv;  // warps per view
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int v = w / wpv;
    double s = 0.0, l = 0.0;
    if (v < nv) {
        // eight loads in flight per round, added in index order
        const int step = 32 * wpv, end = sv.boff[v + 1];
        for (int i0 = sv.boff[v] + 32 * (w % wpv) + lane; i0 < end; i0 += 8 * step) {
            float2 p[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) p[u] = i0 + u * step < end ? part[i0 + u * step] : make_float2(0.f, 0.f);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                s += (double)p[u].x;
                l += (double)p[u].y;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        l += __shfl_xor_sync(0xffffffffu, l, o);
    }
    if (lane == 0) { sm[0][w] = s; sm[1][w] = l; }
    __syncthreads();
    if ((int)threadIdx.x < nv) {
        const int vv = threadIdx.x;
        double S = 0.0, Lv = 0.0;
        for (int q = 0; q < wpv; ++q) { S += sm[0][vv * wpv + q]; Lv += sm[1][vv * wpv + q]; }
        const double n = 3.0 * (double)sv.W[vv] * (double)sv.H[vv];
        const double lv = (1.0 - (double)lam) * (Lv / n) + (double)lam * (1.0 - S / n);
        loss[vv] = (float)lv;
        lv_s[vv] = lv;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double mean = 0.0;
        for (int q = 0; q < nv; ++q) mean += lv_s[q];
        loss[nv] = (float)(mean / nv);
    }
}

}  // namespace
}  // namespace dg

static bool ssim_views(const int32_t* wh, int n_views, dg::SViews* sv, long long* npix)
{
    if (!wh) { dg_set_error("wh is null"); return false; }
    if (n_views < 1 || n_views > DG_MAX_VIEWS) { dg_set_error("n_views %d outside 1..%d", n_views, DG_MAX_VIEWS); return false; }
    sv->n = n_views;
    long long blocks = 0, pix = 0;
    for (int v = 0; v < n_views; ++v) {
        const int W = wh[2 * v], H = wh[2 * v + 1];
        if (W <= 0 || H <= 0 || W > (1 << 16) || H > (1 << 16)) { dg_set_error("view %d: image size %dx%d", v, W, H); return false; }
        sv->W[v] = W; sv->H[v] = H;
        sv->TX[v] = (W + dg::SS_T - 1) / dg::SS_T;
        sv->TY[v] = (H + dg::SS_T - 1) / dg::SS_T;
        sv->boff[v] = (int)blocks;
        sv->poff[v] = pix;
        blocks += 3LL * sv->TX[v] * sv->TY[v];
        pix += (long long)W * H;
    }
    if (blocks >= (1LL << 31)) { dg_set_error("images too large"); return false; }
    sv->boff[n_views] = (int)blocks;
    *npix = pix;
    return true;
}

static size_t ssim_ws_bytes(const dg::SViews& sv, long long npix)
{
    const size_t maps = ((size_t)3 * 3 * npix * sizeof(float) + 255) & ~(size_t)255;
    return maps + sizeof(float2) * (size_t)sv.boff[sv.n];
}

extern "C" size_t dg_ssim_workspace_size(const int32_t* wh, int32_t n_views)
{
    dg::SViews sv;
    long long npix = 0;
    if (!ssim_views(wh, n_views, &sv, &npix)) return 0;
    return ssim_ws_bytes(sv, npix);
}

extern "C" dg_status dg_loss_l1_dssim(const float* img, const float* target, const int32_t* wh, int32_t n_views,
                                      float lambda, float* dL_dimg, float* loss, void* ws, size_t ws_bytes,
                                      dg_stream stream)
{
    dg::SViews sv;
    long long npix = 0;
    if (!ssim_views(wh, n_views, &sv, &npix)) return DG_ERR_ARG;
    if (!img || !target || !dL_dimg || !loss) { dg_set_error("null buffer"); return DG_ERR_ARG; }
    if (!(lambda >= 0.f && lambda <= 1.f)) { dg_set_error("lambda must be in [0, 1]"); return DG_ERR_ARG; }
    const size_t need = ssim_ws_bytes(sv, npix);
    if (!ws || ws_bytes < need) { dg_set_error("ssim workspace missing or too small (%zu < %zu bytes)", ws_bytes, need); return DG_ERR_ARG; }
    dg::Win win;
    double sum = 0.0, w[2 * dg::SS_R + 1];
    for (int k = 0; k <= 2 * dg::SS_R; ++k) {
        const double x = (double)(k - dg::SS_R);
        w[k] = exp(-x * x / (2.0 * 1.5 * 1.5));
        sum += w[k];
    }
    for (int k = 0; k <= 2 * dg::SS_R; ++k) win.w[k] = (float)(w[k] / sum);
    float* dm = (float*)ws;
    float* da = dm + 3 * npix;
    float* dc = da + 3 * npix;
    float2* part = (float2*)((char*)ws + (((size_t)3 * 3 * npix * sizeof(float) + 255) & ~(size_t)255));
    cudaStream_t s = (cudaStream_t)stream;
    const int nb = sv.boff[sv.n];
    dg::k_ssim_fwd<<<nb, dg::SS_THREADS, 0, s>>>(img, target, sv, win, dm, da, dc, part);
    dg::k_ssim_bwd<<<nb, dg::SS_THREADS, 0, s>>>(img, target, sv, win, dm, da, dc, lambda, dL_dimg);
    dg::k_ssim_final<<<1, 32 * dg::ssim_final_warps(sv.n), 0, s>>>(part, sv, lambda, loss);
    dg_note_launch(3);
    return dg_check_launch("loss_l1_dssim");
}
