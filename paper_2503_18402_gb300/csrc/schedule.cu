// schedule.cu -- DashGaussian's resolution and primitive schedules.
//
// Device part (once per scene): the significance of Eq. 2 needs, for every
// training view, the DFT magnitude summed over RGB.  Each channel's 2D DFT is
// two dense complex products, F = T_H (I T_W^T), computed with FP32 tiled
// kernels; the twiddle of index product k*x is taken from a table at
// (k*x mod N), so every twiddle is exact to the table's rounding and the
// angle never grows.  |F| is accumulated per view into an FP64 buffer, the
// view mean is moved to DC-centred order and turned into an FP64 summed-area
// table, from which any centred crop sum is four lookups.
//
// Host part: X(r) = (crop sum of floor(H/r) x floor(W/r)) / (H W): Eq. 2 with
// the DFT normalised by the pixel count, under which the 1/r^2 of Sec. 4.1
// cancels (with unnormalised transforms X(r) <= X(1)/r^2 would cap r_m at
// sqrt(a)); r_m where X = X(1)/a;
// m levels spaced linearly in X (Sec. 4.2); anchors by Eq. 7; 1/r^2 linear in
// the iteration between anchors; floor(r) rendering factor (Sec. 5); the
// position learning-rate rule (supplementary "Learning Rate"); Eq. 5 budget
// and Eq. 4 primitive target.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace dg {

constexpr int DFT_TILE = 64;   // output tile edge
constexpr int DFT_K = 16;      // reduction chunk
constexpr int DFT_THREADS = 256;

__global__ void k_twiddle(int N, float2* tab)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double s, c;
    sincospi(-2.0 * (double)i / (double)N, &s, &c);
    tab[i] = make_float2((float)c, (float)s);
}

// G[y][kx] = sum_x I[y][x] * tw_W[(kx*x) mod W]   (real input, complex output)
__global__ void __launch_bounds__(DFT_THREADS)
k_dft_rows(const float* __restrict__ img, int H, int W, const float2* __restrict__ twW, float2* __restrict__ G)
{
    __shared__ float sI[DFT_TILE][DFT_K + 1];      // [y][x]
    __shared__ float2 sT[DFT_K][DFT_TILE + 1];     // [x][kx]
    const int y0 = blockIdx.y * DFT_TILE, k0 = blockIdx.x * DFT_TILE;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    float2 acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = make_float2(0.f, 0.f);
    for (int x0 = 0; x0 < W; x0 += DFT_K) {
        for (int e = threadIdx.x; e < DFT_TILE * DFT_K; e += DFT_THREADS) {
            const int yy = e / DFT_K, xx = e % DFT_K;
            const int y = y0 + yy, x = x0 + xx;
            sI[yy][xx] = (y < H && x < W) ? img[(size_t)y * W + x] : 0.f;
            const int xk = e / DFT_TILE, kk = e % DFT_TILE;
            const int x2 = x0 + xk, k = k0 + kk;
            sT[xk][kk] = (x2 < W && k < W) ? twW[(int)(((long long)k * x2) % W)] : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll
        for (int xx = 0; xx < DFT_K; ++xx) {
            float iv[4];
            float2 tv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) iv[a] = sI[ty + 16 * a][xx];
#pragma unroll
            for (int b = 0; b < 4; ++b) tv[b] = sT[xx][tx + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    acc[a][b].x = fmaf(iv[a], tv[b].x, acc[a][b].x);
                    acc[a][b].y = fmaf(iv[a], tv[b].y, acc[a][b].y);
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int y = y0 + ty + 16 * a, k = k0 + tx + 16 * b;
            if (y < H && k < W) G[(size_t)y * W + k] = acc[a][b];
        }
}

// F[ky][kx] = sum_y tw_H[(ky*y) mod H] * G[y][kx];  acc[ky][kx] += |F|  (FP64)
__global__ void __launch_bounds__(DFT_THREADS)
k_dft_cols_mag(const float2* __restrict__ G, int H, int W, const float2* __restrict__ twH,
               double* __restrict__ acc_out)
{
    __shared__ float2 sT[DFT_TILE][DFT_K + 1];     // [ky][y]
    __shared__ float2 sG[DFT_K][DFT_TILE + 1];     // [y][kx]
    const int ky0 = blockIdx.y * DFT_TILE, kx0 = blockIdx.x * DFT_TILE;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    float2 acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = make_float2(0.f, 0.f);
    for (int y0 = 0; y0 < H; y0 += DFT_K) {
        for (int e = threadIdx.x; e < DFT_TILE * DFT_K; e += DFT_THREADS) {
            const int kk = e / DFT_K, yy = e % DFT_K;
            const int ky = ky0 + kk, y = y0 + yy;
            sT[kk][yy] = (ky < H && y < H) ? twH[(int)(((long long)ky * y) % H)] : make_float2(0.f, 0.f);
            const int y2 = y0 + e / DFT_TILE, kx = kx0 + e % DFT_TILE;
            sG[e / DFT_TILE][e % DFT_TILE] = (y2 < H && kx < W) ? G[(size_t)y2 * W + kx] : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll
        for (int yy = 0; yy < DFT_K; ++yy) {
            float2 tv[4], gv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) tv[a] = sT[ty + 16 * a][yy];
#pragma unroll
            for (int b = 0; b < 4; ++b) gv[b] = sG[yy][tx + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    acc[a][b].x = fmaf(tv[a].x, gv[b].x, fmaf(-tv[a].y, gv[b].y, acc[a][b].x));
                    acc[a][b].y = fmaf(tv[a].x, gv[b].y, fmaf(tv[a].y, gv[b].x, acc[a][b].y));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int ky = ky0 + ty + 16 * a, kx = kx0 + tx + 16 * b;
            if (ky < H && kx < W) {
                const double re = acc[a][b].x, im = acc[a][b].y;
                acc_out[(size_t)ky * W + kx] += sqrt(re * re + im * im);
            }
        }
}

// mean over views, DC moved to (H/2, W/2): out[(ky + H/2) % H][(kx + W/2) % W] = acc[ky][kx] / N
__global__ void k_spec_shift(const double* __restrict__ acc, int H, int W, double inv_n, double* __restrict__ sh)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= H * W) return;
    const int ky = i / W, kx = i % W;
    sh[(size_t)((ky + H / 2) % H) * W + (kx + W / 2) % W] = acc[i] * inv_n;
}

// inclusive 2D prefix sums into sat[(H+1)][(W+1)] with a zero first row/column
__global__ void k_sat_rows(const double* __restrict__ sh, int H, int W, double* __restrict__ sat)
{
    const int y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y > H) return;
    double run = 0.0;
    sat[(size_t)y * (W + 1)] = 0.0;
    for (int x = 0; x < W; ++x) {
        if (y > 0) run += sh[(size_t)(y - 1) * W + x];
        sat[(size_t)y * (W + 1) + x + 1] = run;
    }
}

__global__ void k_sat_cols(int H, int W, double* __restrict__ sat)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x > W) return;
    double run = 0.0;
    for (int y = 0; y <= H; ++y) {
        run += sat[(size_t)y * (W + 1) + x];
        sat[(size_t)y * (W + 1) + x] = run;
    }
}

// Area resampling with exact coverage: output pixel i covers input rows
// [i H/h, (i+1) H/h); scaled by h the bounds are the integers i*H and (i+1)*H,
// so each overlap (in units of 1/h) is an integer and the weight of input row y
// is ov_y / H.
__global__ void k_downsample_area(const float* __restrict__ src, int C, int H, int W, float* __restrict__ dst,
                                  int h, int w)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)C * h * w) return;
    const int j = (int)(idx % w), i = (int)((idx / w) % h), c = (int)(idx / ((long long)w * h));
    const long long ay = (long long)i * H, by = (long long)(i + 1) * H;   // row bounds x h
    const long long ax = (long long)j * W, bx = (long long)(j + 1) * W;   // col bounds x w
    const int y_lo = (int)(ay / h), y_hi = (int)((by + h - 1) / h);
    const int x_lo = (int)(ax / w), x_hi = (int)((bx + w - 1) / w);
    const float* s = src + (size_t)c * H * W;
    double acc = 0.0;
    for (int y = y_lo; y < y_hi; ++y) {
        const long long ov_y = std::min(by, (long long)(y + 1) * h) - std::max(ay, (long long)y * h);
        if (ov_y <= 0) continue;
        double row = 0.0;
        for (int x = x_lo; x < x_hi; ++x) {
            const long long ov_x = std::min(bx, (long long)(x + 1) * w) - std::max(ax, (long long)x * w);
            if (ov_x > 0) row += (double)ov_x * (double)s[(size_t)y * W + x];
        }
        acc += (double)ov_y * row;
    }
    dst[idx] = (float)(acc / ((double)H * (double)W));
}

}  // namespace dg

// ---------------------------------------------------------------------------
static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

extern "C" size_t dg_spectrum_workspace_size(int32_t H, int32_t W)
{
    if (H <= 0 || W <= 0) return 0;
    return al256(sizeof(float2) * (size_t)H * W) + al256(sizeof(float2) * H) + al256(sizeof(float2) * W);
}

extern "C" dg_status dg_spectrum_accumulate(const float* view, int32_t H, int32_t W, double* acc, void* ws,
                                            size_t ws_bytes, dg_stream stream)
{
    if (H <= 0 || W <= 0) { dg_set_error("bad size %dx%d", W, H); return DG_ERR_ARG; }
    if (!view || !acc || !ws) { dg_set_error("null buffer"); return DG_ERR_ARG; }
    if (ws_bytes < dg_spectrum_workspace_size(H, W)) { dg_set_error("spectrum workspace too small"); return DG_ERR_CAPACITY; }
    char* base = (char*)ws;
    float2* G = (float2*)base;
    float2* twH = (float2*)(base + al256(sizeof(float2) * (size_t)H * W));
    float2* twW = (float2*)((char*)twH + al256(sizeof(float2) * H));
    cudaStream_t s = (cudaStream_t)stream;
    dg::k_twiddle<<<(H + 255) / 256, 256, 0, s>>>(H, twH);
    dg_note_launch();
    dg::k_twiddle<<<(W + 255) / 256, 256, 0, s>>>(W, twW);
    dg_note_launch();
    const dim3 gr((W + dg::DFT_TILE - 1) / dg::DFT_TILE, (H + dg::DFT_TILE - 1) / dg::DFT_TILE);
    for (int c = 0; c < 3; ++c) {
        dg::k_dft_rows<<<gr, dg::DFT_THREADS, 0, s>>>(view + (size_t)c * H * W, H, W, twW, G);
        dg_note_launch();
        dg::k_dft_cols_mag<<<gr, dg::DFT_THREADS, 0, s>>>(G, H, W, twH, acc);
        dg_note_launch();
    }
    return dg_check_launch("spectrum_accumulate");
}

extern "C" dg_status dg_spectrum_finalize(const double* acc, int32_t n_views, int32_t H, int32_t W,
                                          double* shifted, double* sat, dg_stream stream)
{
    if (H <= 0 || W <= 0 || n_views <= 0) { dg_set_error("bad sizes"); return DG_ERR_ARG; }
    if (!acc || !shifted || !sat) { dg_set_error("null buffer"); return DG_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    const int n = H * W;
    dg::k_spec_shift<<<(n + 255) / 256, 256, 0, s>>>(acc, H, W, 1.0 / (double)n_views, shifted);
    dg_note_launch();
    dg::k_sat_rows<<<(H + 1 + 127) / 128, 128, 0, s>>>(shifted, H, W, sat);
    dg_note_launch();
    dg::k_sat_cols<<<(W + 1 + 127) / 128, 128, 0, s>>>(H, W, sat);
    dg_note_launch();
    return dg_check_launch("spectrum_finalize");
}

extern "C" dg_status dg_downsample_area(const float* src, int32_t C, int32_t H, int32_t W, float* dst, int32_t h,
                                        int32_t w, dg_stream stream)
{
    if (C <= 0 || H <= 0 || W <= 0 || h <= 0 || w <= 0 || h > H || w > W) {
        dg_set_error("bad sizes C=%d %dx%d -> %dx%d", C, W, H, w, h);
        return DG_ERR_ARG;
    }
    if (!src || !dst) { dg_set_error("null buffer"); return DG_ERR_ARG; }
    const long long n = (long long)C * h * w;
    dg::k_downsample_area<<<(int)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(src, C, H, W, dst, h, w);
    dg_note_launch();
    return dg_check_launch("downsample_area");
}

// --------------------------------------------------------------------------- host schedule
namespace {

struct Frac { long long num, den; };  // r = num / den > 0

// centred crop sum from the (H+1) x (W+1) summed-area table of the DC-centred spectrum
double crop_sum(const double* sat, int H, int W, int h, int w)
{
    if (h <= 0 || w <= 0) return 0.0;
    const int cy = H / 2, cx = W / 2;
    const int y0 = cy - h / 2, y1 = cy + (h + 1) / 2;  // [y0, y1)
    const int x0 = cx - w / 2, x1 = cx + (w + 1) / 2;
    const size_t S = (size_t)W + 1;
    return sat[(size_t)y1 * S + x1] - sat[(size_t)y0 * S + x1] - sat[(size_t)y1 * S + x0] + sat[(size_t)y0 * S + x0];
}

// inf{r >= 1 : X(r) <= target}; on (lo, hi] between consecutive breakpoints
// the crop is that of hi, X is constant there and the infimum is lo.
double solve_r(const double* sat, int H, int W, const std::vector<Frac>& bps, double target)
{
    const double norm = 1.0 / ((double)H * (double)W);
    if (crop_sum(sat, H, W, H, W) * norm <= target) return 1.0;
    double lo = 1.0;
    for (const Frac& b : bps) {
        const int h = (int)((long long)H * b.den / b.num), w = (int)((long long)W * b.den / b.num);
        if (crop_sum(sat, H, W, h, w) * norm <= target) return lo;
        lo = (double)b.num / (double)b.den;
    }
    return lo;
}

}  // namespace

extern "C" dg_status dg_schedule_init(const double* sat_host, int32_t H, int32_t W, const dg_sched_params* p,
                                      dg_schedule* out)
{
    if (!sat_host || !p || !out) { dg_set_error("null argument"); return DG_ERR_ARG; }
    if (H <= 0 || W <= 0 || p->S <= 0 || !(p->a > 1.0)) { dg_set_error("bad schedule parameters"); return DG_ERR_ARG; }
    // breakpoints r = H/n, W/n (> 1), sorted ascending, exact rational compare
    std::vector<Frac> bps;
    for (int n = 1; n < H; ++n) bps.push_back(Frac{H, n});
    for (int n = 1; n < W; ++n) bps.push_back(Frac{W, n});
    std::sort(bps.begin(), bps.end(), [](const Frac& a, const Frac& b) { return a.num * b.den < b.num * a.den; });
    bps.erase(std::unique(bps.begin(), bps.end(), [](const Frac& a, const Frac& b) { return a.num * b.den == b.num * a.den; }),
              bps.end());
    dg_schedule s;
    memset(&s, 0, sizeof s);
    s.p = *p;
    s.H = H;
    s.W = W;
    s.X0 = crop_sum(sat_host, H, W, H, W) / ((double)H * (double)W);
    if (!(s.X0 > 0.0)) { dg_set_error("spectrum has no energy"); return DG_ERR_ARG; }
    s.Xm = s.X0 / p->a;
    s.r_m = solve_r(sat_host, H, W, bps, s.Xm);
    int m = p->m > 0 ? p->m : (int)ceil(s.r_m);
    if (m < 1) m = 1;
    if (m > DG_SCHED_MAX_LEVELS) m = DG_SCHED_MAX_LEVELS;
    s.m = m;
    const double den = log(s.X0 / s.Xm);
    for (int i = 0; i <= m; ++i) {
        s.X[i] = s.X0 + ((double)i / (double)m) * (s.Xm - s.X0);
        s.r[i] = i == 0 ? 1.0 : solve_r(sat_host, H, W, bps, s.X[i]);
        s.s[i] = (double)p->S * log(s.X[i] / s.Xm) / den;
    }
    s.P_fin = 5.0 * p->P_init;  // P_fin(0) = 5 P_init (Sec. 4.3)
    // first iteration rendered at full resolution
    s.k_full = p->S;
    for (int64_t k = 0; k <= p->S; ++k) {
        dg_sched_out o;
        dg_schedule_step(&s, k, &o);
        if (o.r_mod == 1) { s.k_full = k; break; }
    }
    *out = s;
    return DG_OK;
}

extern "C" dg_status dg_schedule_step(const dg_schedule* s, int64_t iter, dg_sched_out* out)
{
    if (!s || !out) { dg_set_error("null argument"); return DG_ERR_ARG; }
    const double k = (double)iter;
    double r;
    if (k <= s->s[s->m]) {
        r = s->r[s->m];
    } else {
        r = s->r[0];
        for (int i = s->m; i > 0; --i) {
            const double si = s->s[i], sp = s->s[i - 1];
            if (k <= sp) {
                const double t = sp > si ? (k - si) / (sp - si) : 1.0;
                const double inv2 = (1.0 - t) / (s->r[i] * s->r[i]) + t / (s->r[i - 1] * s->r[i - 1]);
                r = 1.0 / sqrt(inv2);
                break;
            }
        }
    }
    out->r_cont = r;
    int rm = (int)floor(r);
    out->r_mod = rm < 1 ? 1 : rm;
    out->height = s->H / out->r_mod;
    out->width = s->W / out->r_mod;
    const dg_sched_params* p = &s->p;
    if (iter <= s->k_full || p->S <= s->k_full) {
        out->lr_pos = p->lr_pos_init;
    } else {
        double t = (double)(iter - s->k_full) / (double)(p->S - s->k_full);
        if (t > 1.0) t = 1.0;
        out->lr_pos = exp((1.0 - t) * log(p->lr_pos_init) + t * log(p->lr_pos_final));
    }
    out->P_target = p->P_init + (s->P_fin - p->P_init) / pow((double)out->r_mod, 2.0 - k / (double)p->S);
    if (p->P_cap > 0.0 && out->P_target > p->P_cap) out->P_target = p->P_cap;
    return DG_OK;
}

extern "C" dg_status dg_schedule_densify(dg_schedule* s, int64_t iter, int64_t P_add, dg_sched_out* out)
{
    if (!s || !out || P_add < 0) { dg_set_error("bad argument"); return DG_ERR_ARG; }
    const double upd = s->p.gamma * s->P_fin + s->p.eta * (double)P_add;  // Eq. 5
    if (upd > s->P_fin) s->P_fin = upd;
    return dg_schedule_step(s, iter, out);
}

extern "C" dg_status dg_schedule_init_plain(int32_t H, int32_t W, const dg_sched_params* p, dg_schedule* out)
{
    if (!p || !out) { dg_set_error("null argument"); return DG_ERR_ARG; }
    if (H <= 0 || W <= 0 || p->S <= 0) { dg_set_error("bad schedule parameters"); return DG_ERR_ARG; }
    dg_schedule s;
    memset(&s, 0, sizeof s);
    s.p = *p;
    s.H = H;
    s.W = W;
    s.m = 0;
    s.X0 = s.Xm = 1.0;
    s.r_m = 1.0;
    s.X[0] = 1.0;
    s.r[0] = 1.0;
    s.s[0] = (double)p->S;
    s.k_full = 0;  // full resolution from the start: the position LR decays from iteration 0
    s.P_fin = 5.0 * p->P_init;
    *out = s;
    return DG_OK;
}

extern "C" dg_status dg_densify_budget(dg_schedule* s, int64_t iter, int64_t n_keep, int64_t n_cand, int64_t P_cap,
                                       int64_t* budget, dg_sched_out* out)
{
    if (!budget || n_keep < 0 || n_cand < 0 || P_cap < 0 || (s && !out)) {
        dg_set_error("bad argument");
        return DG_ERR_ARG;
    }
    int64_t b = n_cand;  // 3DGS backbone: every candidate
    if (s) {
        // Eq. 5 with P_add = the candidate count, then Eq. 4's target; the
        // budget is what the target leaves after the kept Gaussians
        const dg_status st = dg_schedule_densify(s, iter, n_cand, out);
        if (st != DG_OK) return st;
        b = (int64_t)floor(out->P_target) - n_keep;
    }
    if (P_cap > 0 && b > P_cap - n_keep) b = P_cap - n_keep;
    *budget = b > 0 ? b : 0;
    return DG_OK;
}

extern "C" dg_status dg_camera_scale(const dg_camera* full, int32_t width, int32_t height, dg_camera* out)
{
    if (!full || !out) { dg_set_error("null argument"); return DG_ERR_ARG; }
    if (width <= 0 || height <= 0 || full->width <= 0 || full->height <= 0) {
        dg_set_error("bad image size %dx%d (full %dx%d)", width, height, full->width, full->height);
        return DG_ERR_ARG;
    }
    const double sx = (double)width / (double)full->width, sy = (double)height / (double)full->height;
    dg_camera c = *full;
    c.fx = (float)((double)full->fx * sx);
    c.cx = (float)((double)full->cx * sx);
    c.fy = (float)((double)full->fy * sy);
    c.cy = (float)((double)full->cy * sy);
    c.width = width;
    c.height = height;
    *out = c;
    return DG_OK;
}

extern "C" dg_status dg_batch_adam_scale(int32_t views_per_step, float* lr, float* beta1, float* beta2)
{
    if (views_per_step < 1 || !lr || !beta1 || !beta2) { dg_set_error("bad argument"); return DG_ERR_ARG; }
    const double V = (double)views_per_step;
    const double f = sqrt(V);
    for (int i = 0; i < DG_NPARAM; ++i) lr[i] = (float)((double)lr[i] * f);
    *beta1 = (float)pow((double)*beta1, V);
    *beta2 = (float)pow((double)*beta2, V);
    return DG_OK;
}
