// densify.cu -- DashGaussian's scheduled densification (supplementary
// "Densification of DashGaussian"): prune first, then clone or split the
// top-(P_i - N'_GS) Gaussians by densification score among those meeting the
// backbone's condition (3DGS: mean view-space positional gradient >= thresh).
//
// Every decision that yields an integer (prune, candidate, split, selection)
// is taken on float32 values against float32 thresholds computed once on the
// host, so the result does not depend on transcendental rounding: opacity is
// tested as logit < logit(min_opacity), scales as max log-scale > log(t).
// Selection is a stable radix sort of the candidates on the bit-inverted
// float score (descending score, ties by lower index); survivors keep their
// order and appended Gaussians follow in index order of their source.
#include <math.h>

#include "radix.cuh"

namespace dg {

enum : uint8_t { F_KEEP = 1, F_CAND = 2, F_SPLIT = 4, F_SEL = 8 };

struct HalfSizes {
    int n;
    float hw[DG_MAX_VIEWS], hh[DG_MAX_VIEWS];
};

__global__ void k_dstats(const float4* __restrict__ grad2d, const int* __restrict__ radius, int P, HalfSizes hs,
                         float* __restrict__ accum, float* __restrict__ denom, float* __restrict__ maxr)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    float acc = 0.f, den = 0.f, mr = maxr[i];
    for (int v = 0; v < hs.n; ++v) {
        const size_t r = (size_t)v * P + i;
        const int rad = radius[r];
        if (rad <= 0) continue;
        const float4 g = grad2d[3 * r];
        const float gx = g.x * hs.hw[v], gy = g.y * hs.hh[v];
        acc += sqrtf(gx * gx + gy * gy);
        den += 1.f;
        mr = fmaxf(mr, (float)rad);
    }
    if (den > 0.f) {
        accum[i] += acc;
        denom[i] += den;
        maxr[i] = mr;
    }
}

struct DThresh {
    float grad, logit_min_op, log_split, max_screen, log_max_world;
    int use_screen, use_world;
};

__global__ void k_dmark(const float* __restrict__ prm, long long stride, int P, const float* __restrict__ accum,
                        const float* __restrict__ denom, const float* __restrict__ maxr, DThresh t,
                        uint8_t* __restrict__ flags, float* __restrict__ score, long long* counts)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool keep = false, cand = false;
    if (i < P) {
        const float logit = prm[10 * stride + i];
        const float ls = fmaxf(prm[3 * stride + i], fmaxf(prm[4 * stride + i], prm[5 * stride + i]));
        bool prune = logit < t.logit_min_op;
        if (t.use_screen) prune = prune || (maxr[i] > t.max_screen);
        if (t.use_world) prune = prune || (ls > t.log_max_world);
        keep = !prune;
        const float den = denom[i];
        const float sc = den > 0.f ? accum[i] / den : 0.f;
        cand = keep && den > 0.f && sc >= t.grad;
        flags[i] = (uint8_t)((keep ? F_KEEP : 0) | (cand ? F_CAND : 0) | (ls > t.log_split ? F_SPLIT : 0));
        score[i] = sc;
    }
    const unsigned nk = __popc(__ballot_sync(0xffffffffu, keep));
    const unsigned nc = __popc(__ballot_sync(0xffffffffu, cand));
    if ((threadIdx.x & 31) == 0) {
        if (nk) atomicAdd((unsigned long long*)&counts[0], (unsigned long long)nk);
        if (nc) atomicAdd((unsigned long long*)&counts[1], (unsigned long long)nc);
    }
}

struct LoadFlag {  // 1 where all bits of `mask` are set and none of `nmask`
    const uint8_t* f;
    uint8_t mask, nmask;
    __device__ uint64_t operator()(long long i) const { return ((f[i] & mask) == mask) && !(f[i] & nmask); }
};
struct LoadKeep {  // survivor: kept and not a selected split
    const uint8_t* f;
    __device__ uint64_t operator()(long long i) const
    {
        const uint8_t x = f[i];
        return (x & F_KEEP) && !((x & F_SEL) && (x & F_SPLIT));
    }
};
struct LoadAppend {  // entries appended for a selected Gaussian
    const uint8_t* f;
    __device__ uint64_t operator()(long long i) const
    {
        const uint8_t x = f[i];
        return (x & F_SEL) ? ((x & F_SPLIT) ? 2u : 1u) : 0u;
    }
};

__global__ void k_cand_keys(const uint8_t* __restrict__ flags, const float* __restrict__ score,
                            const uint32_t* __restrict__ cpos, int P, uint32_t* __restrict__ keys,
                            uint32_t* __restrict__ vals)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P || !(flags[i] & F_CAND)) return;
    const uint32_t p = cpos[i];
    keys[p] = ~__float_as_uint(score[i]);  // score >= 0: ascending key = descending score
    vals[p] = (uint32_t)i;
}

__global__ void k_mark_selected(const uint32_t* __restrict__ order, long long n_sel, uint8_t* __restrict__ flags)
{
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n_sel) flags[order[r]] |= F_SEL;
}

__global__ void k_mark_all_candidates(uint8_t* __restrict__ flags, int P)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < P && (flags[i] & F_CAND)) flags[i] |= F_SEL;
}

__device__ inline void quat_rot(float q0, float q1, float q2, float q3, float R[9])
{
    const float inv = 1.f / sqrtf(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
    const float w = q0 * inv, x = q1 * inv, y = q2 * inv, z = q3 * inv;
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
}

__global__ void k_densify_write(const float* __restrict__ prm, const float* __restrict__ m, const float* __restrict__ v,
                                long long stride, int P, const uint8_t* __restrict__ flags,
                                const uint32_t* __restrict__ keep_pos, const uint32_t* __restrict__ app_pos,
                                const uint32_t* __restrict__ sel_rank, const long long* n_keep,
                                const float* __restrict__ noise, float log_div, float* __restrict__ dp,
                                float* __restrict__ dm, float* __restrict__ dv, long long dstride)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const uint8_t f = flags[i];
    const bool sel = f & F_SEL, split = f & F_SPLIT;
    if ((f & F_KEEP) && !(sel && split)) {
        const long long o = keep_pos[i];
        for (int r = 0; r < DG_NPARAM; ++r) {
            dp[r * dstride + o] = prm[r * stride + i];
            dm[r * dstride + o] = m[r * stride + i];
            dv[r * dstride + o] = v[r * stride + i];
        }
    }
    if (!sel) return;
    const long long base = *n_keep + app_pos[i];
    if (!split) {
        for (int r = 0; r < DG_NPARAM; ++r) {
            dp[r * dstride + base] = prm[r * stride + i];
            dm[r * dstride + base] = 0.f;
            dv[r * dstride + base] = 0.f;
        }
        return;
    }
    float R[9];
    quat_rot(prm[6 * stride + i], prm[7 * stride + i], prm[8 * stride + i], prm[9 * stride + i], R);
    float s[3], mu[3];
    for (int c = 0; c < 3; ++c) {
        s[c] = expf(prm[(3 + c) * stride + i]);
        mu[c] = prm[c * stride + i];
    }
    const float* eps = noise + 6 * (size_t)sel_rank[i];
    for (int k = 0; k < 2; ++k) {
        const long long o = base + k;
        const float e0 = s[0] * eps[3 * k], e1 = s[1] * eps[3 * k + 1], e2 = s[2] * eps[3 * k + 2];
        for (int c = 0; c < 3; ++c) dp[c * dstride + o] = mu[c] + R[3 * c] * e0 + R[3 * c + 1] * e1 + R[3 * c + 2] * e2;
        for (int c = 0; c < 3; ++c) dp[(3 + c) * dstride + o] = prm[(3 + c) * stride + i] - log_div;
        for (int r = 6; r < DG_NPARAM; ++r) dp[r * dstride + o] = prm[r * stride + i];
        for (int r = 0; r < DG_NPARAM; ++r) {
            dm[r * dstride + o] = 0.f;
            dv[r * dstride + o] = 0.f;
        }
    }
}

__global__ void k_store_total(const long long* a, const long long* b, long long* out)
{
    *out = *a + *b;
}

struct DensWs {
    uint8_t* flags;
    float* score;
    uint32_t *cpos, *keep_pos, *app_pos, *sel_rank;
    uint32_t *k0, *v0, *k1, *v1;
    uint32_t* hist;
    uint64_t* bsum;
    long long *n_cand, *n_keep, *n_app, *n_sel;
    size_t bytes;
};

static size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

static DensWs dens_layout(char* b, long long P)
{
    DensWs w;
    size_t o = 0;
    auto take = [&](size_t n) { char* p = b + o; o += al(n); return p; };
    w.flags = (uint8_t*)take(P);
    w.score = (float*)take(4 * P);
    w.cpos = (uint32_t*)take(4 * P);
    w.keep_pos = (uint32_t*)take(4 * P);
    w.app_pos = (uint32_t*)take(4 * P);
    w.sel_rank = (uint32_t*)take(4 * P);
    w.k0 = (uint32_t*)take(4 * P); w.v0 = (uint32_t*)take(4 * P);
    w.k1 = (uint32_t*)take(4 * P); w.v1 = (uint32_t*)take(4 * P);
    const long long nblk = (P + RS_TILE - 1) / RS_TILE;
    const long long nh = (long long)(1 << RS_MAXBITS) * nblk;
    w.hist = (uint32_t*)take(4 * nh);
    const long long ns = nh > P ? nh : P;
    w.bsum = (uint64_t*)take(8 * ((ns + SCAN_TILE - 1) / SCAN_TILE + 1));
    w.n_cand = (long long*)take(8);
    w.n_keep = (long long*)take(8);
    w.n_app = (long long*)take(8);
    w.n_sel = (long long*)take(8);
    w.bytes = o;
    return w;
}

static bool thresholds(const dg_densify_opts* o, DThresh* t)
{
    if (!(o->grad_thresh >= 0.f) || !(o->min_opacity > 0.f && o->min_opacity < 1.f) ||
        !(o->percent_dense > 0.f) || !(o->extent > 0.f))
        return false;
    t->grad = o->grad_thresh;
    t->logit_min_op = (float)log((double)o->min_opacity / (1.0 - (double)o->min_opacity));
    t->log_split = (float)log((double)o->percent_dense * (double)o->extent);
    t->use_screen = o->max_screen_radius > 0.f;
    t->max_screen = o->max_screen_radius;
    t->use_world = o->max_world_scale > 0.f;
    t->log_max_world = t->use_world ? (float)log((double)o->max_world_scale) : 0.f;
    return true;
}

}  // namespace dg

bool dg_check_cameras(const dg_camera* cams, int n_views);

extern "C" dg_status dg_densify_stats(const float* grad2d, const int32_t* radius, int64_t P, const dg_camera* cams,
                                      int32_t n_views, float* grad_accum, float* denom, float* max_radius,
                                      dg_stream stream)
{
    if (!dg_check_cameras(cams, n_views)) return DG_ERR_ARG;
    if (P < 0 || P > INT32_MAX) { dg_set_error("bad sizes"); return DG_ERR_ARG; }
    if (P == 0) return DG_OK;
    if (!grad2d || !radius || !grad_accum || !denom || !max_radius) { dg_set_error("null buffer"); return DG_ERR_ARG; }
    dg::HalfSizes hs;
    hs.n = n_views;
    for (int v = 0; v < n_views; ++v) {
        hs.hw[v] = 0.5f * cams[v].width;
        hs.hh[v] = 0.5f * cams[v].height;
    }
    dg::k_dstats<<<(int)((P + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        (const float4*)grad2d, radius, (int)P, hs, grad_accum, denom, max_radius);
    dg_note_launch();
    return dg_check_launch("densify_stats");
}

extern "C" size_t dg_densify_workspace_size(int64_t P)
{
    if (P < 0) return 0;
    return dg::dens_layout(nullptr, P).bytes;
}

extern "C" dg_status dg_densify_mark(const float* params, int64_t stride, int64_t P, const float* grad_accum,
                                     const float* denom, const float* max_radius, const dg_densify_opts* opts,
                                     void* ws, size_t ws_bytes, int64_t* counts, dg_stream stream)
{
    dg::DThresh t;
    if (!opts || !dg::thresholds(opts, &t)) { dg_set_error("bad densify options"); return DG_ERR_ARG; }
    if (P < 0 || P > INT32_MAX || stride < P) { dg_set_error("bad P/stride"); return DG_ERR_ARG; }
    if (!ws || !counts || (P > 0 && (!params || !grad_accum || !denom || !max_radius))) {
        dg_set_error("null buffer");
        return DG_ERR_ARG;
    }
    const dg::DensWs w = dg::dens_layout((char*)ws, P);
    if (ws_bytes < w.bytes) { dg_set_error("densify workspace too small"); return DG_ERR_CAPACITY; }
    cudaStream_t s = (cudaStream_t)stream;
    cudaMemsetAsync(counts, 0, 2 * sizeof(int64_t), s);
    if (P == 0) return dg_check_launch("densify_mark");
    dg::k_dmark<<<(int)((P + 255) / 256), 256, 0, s>>>(params, (long long)stride, (int)P, grad_accum, denom,
                                                       max_radius, t, w.flags, w.score, (long long*)counts);
    dg_note_launch();
    return dg_check_launch("densify_mark");
}

extern "C" dg_status dg_densify_apply(const float* params, const float* m, const float* v, int64_t stride, int64_t P,
                                      int64_t n_cand, int64_t budget, const float* noise, void* ws, size_t ws_bytes,
                                      float* dst_params, float* dst_m, float* dst_v, int64_t dst_stride,
                                      int64_t* P_out, dg_stream stream)
{
    if (P < 0 || P > INT32_MAX || stride < P || n_cand < 0 || n_cand > P || budget < 0) {
        dg_set_error("bad sizes");
        return DG_ERR_ARG;
    }
    const long long n_sel = n_cand < budget ? n_cand : budget;
    if (!ws || !P_out || !dst_params || !dst_m || !dst_v || (P > 0 && (!params || !m || !v)) || (n_sel > 0 && !noise)) {
        dg_set_error("null buffer");
        return DG_ERR_ARG;
    }
    const dg::DensWs w = dg::dens_layout((char*)ws, P);
    if (ws_bytes < w.bytes) { dg_set_error("densify workspace too small"); return DG_ERR_CAPACITY; }
    if (dst_stride < P + n_sel) {
        dg_set_error("dst_stride %lld below the largest possible count %lld", (long long)dst_stride, (long long)(P + n_sel));
        return DG_ERR_CAPACITY;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (P == 0) {
        cudaMemsetAsync(P_out, 0, sizeof(int64_t), s);
        return dg_check_launch("densify_apply");
    }
    const int gb = (int)((P + 255) / 256);
    if (n_sel > 0) {
        if (n_cand > budget) {
            // compact the candidates, order them by descending score (ties: lower index)
            dg::exclusive_scan(dg::LoadFlag{w.flags, dg::F_CAND, 0}, P, w.cpos, w.bsum, w.n_cand, s);
            dg::k_cand_keys<<<gb, 256, 0, s>>>(w.flags, w.score, w.cpos, (int)P, w.k0, w.v0);
            dg_note_launch();
            dg::SortBufs sb{w.hist, w.bsum};
            const dg::KV r = dg::radix_sort(w.k0, w.v0, w.k1, w.v1, nullptr, nullptr, nullptr, n_cand, 32, sb, s);
            dg::k_mark_selected<<<(int)((n_sel + 255) / 256), 256, 0, s>>>(r.v, n_sel, w.flags);
            dg_note_launch();
        } else {
            dg::k_mark_all_candidates<<<gb, 256, 0, s>>>(w.flags, (int)P);
            dg_note_launch();
        }
    }
    dg::exclusive_scan(dg::LoadKeep{w.flags}, P, w.keep_pos, w.bsum, w.n_keep, s);
    dg::exclusive_scan(dg::LoadAppend{w.flags}, P, w.app_pos, w.bsum, w.n_app, s);
    dg::exclusive_scan(dg::LoadFlag{w.flags, dg::F_SEL, 0}, P, w.sel_rank, w.bsum, w.n_sel, s);
    dg::k_densify_write<<<gb, 256, 0, s>>>(params, m, v, (long long)stride, (int)P, w.flags, w.keep_pos, w.app_pos,
                                           w.sel_rank, w.n_keep, noise, (float)log(1.6), dst_params, dst_m, dst_v,
                                           (long long)dst_stride);
    dg_note_launch();
    dg::k_store_total<<<1, 1, 0, s>>>(w.n_keep, w.n_app, (long long*)P_out);
    dg_note_launch();
    return dg_check_launch("densify_apply");
}
