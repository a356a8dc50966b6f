// optim.cu -- L1 photometric loss (+ its gradient) and the Adam update.
#include <math.h>

#include "common.cuh"

namespace dg {

constexpr int LOSS_THREADS = 256;
constexpr int LOSS_BLOCKS_MAX = 1024;

// Grid-stride: grad = sign(img - target) / n; per-block partial sum of |d|.
__global__ void __launch_bounds__(LOSS_THREADS)
k_l1(const float* __restrict__ img, const float* __restrict__ tgt, long long n, float inv_n,
     float* __restrict__ grad, float* __restrict__ partial)
{
    __shared__ float sm[LOSS_THREADS / 32];
    float acc = 0.f;
    for (long long i = (long long)blockIdx.x * LOSS_THREADS + threadIdx.x; i < n;
         i += (long long)gridDim.x * LOSS_THREADS) {
        const float d = img[i] - tgt[i];
        acc += fabsf(d);
        grad[i] = d > 0.f ? inv_n : (d < 0.f ? -inv_n : 0.f);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < LOSS_THREADS / 32; ++w) s += sm[w];
        partial[blockIdx.x] = s;
    }
}

// Deterministic final sum of the block partials (fixed order, FP64 accumulator).
__global__ void k_l1_final(const float* __restrict__ partial, int nb, float inv_n, float* loss)
{
    __shared__ double sm[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += (double)partial[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sm[w];
        *loss = (float)(s * (double)inv_n);
    }
}

// Sum of squared differences, per-block partials (deterministic final sum).
__global__ void __launch_bounds__(LOSS_THREADS)
k_sqdiff(const float* __restrict__ a, const float* __restrict__ b, long long n, float* __restrict__ partial)
{
    __shared__ float sm[LOSS_THREADS / 32];
    float acc = 0.f;
    for (long long i = (long long)blockIdx.x * LOSS_THREADS + threadIdx.x; i < n;
         i += (long long)gridDim.x * LOSS_THREADS) {
        const float d = a[i] - b[i];
        acc = fmaf(d, d, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < LOSS_THREADS / 32; ++w) s += sm[w];
        partial[blockIdx.x] = s;
    }
}

// Opacity reset of the 3DGS backbone: logit <- min(logit, cap); its Adam moments cleared.
__global__ void k_opacity_reset(float* __restrict__ prm, float* __restrict__ m, float* __restrict__ v,
                                long long stride, long long P, float cap)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const long long o = 10 * stride + i;
    prm[o] = fminf(prm[o], cap);
    m[o] = 0.f;
    v[o] = 0.f;
}

// One thread per 4 consecutive Gaussians of one parameter row (float4 when the
// row start is 16-byte aligned, scalar otherwise).
__global__ void __launch_bounds__(256)
k_adam(float* __restrict__ prm, const float* __restrict__ grd, float* __restrict__ m,
       float* __restrict__ v, long long stride, long long P, AdamHp hp_val, const AdamHp* __restrict__ hp_dev,
       const int* __restrict__ skip_if, const uint8_t* __restrict__ vis)
{
    const int row = blockIdx.y;
    const long long i0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (i0 >= P) return;
    if (skip_if && *skip_if != 0) return;  // e.g. the step's pair list overflowed: no update
    const AdamHp& hp = hp_dev ? *hp_dev : hp_val;
    const AdamRowK lr = adam_row(hp.lr[row], hp);
    const long long o = (long long)row * stride + i0;
    const bool vec = ((o & 3) == 0) && (i0 + 3 < P) && ((((uintptr_t)prm) & 15u) == 0) &&
                     ((((uintptr_t)grd) & 15u) == 0) && ((((uintptr_t)m) & 15u) == 0) &&
                     ((((uintptr_t)v) & 15u) == 0);
    // sparse Adam: Gaussians outside the visibility mask keep parameters and moments
    uint8_t on[4] = {1, 1, 1, 1};
    if (vis) {
        for (int c = 0; c < 4; ++c) on[c] = i0 + c < P ? vis[i0 + c] : 0;
        if (!(on[0] | on[1] | on[2] | on[3])) return;
    }
    if (vec) {
        float4 p = *(float4*)(prm + o), g = *(const float4*)(grd + o);
        float4 mm = *(float4*)(m + o), vv = *(float4*)(v + o);
        float* pp = &p.x; const float* gg = &g.x; float* mp = &mm.x; float* vp = &vv.x;
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (on[c]) adam_update(pp[c], mp[c], vp[c], gg[c], lr, hp);
        *(float4*)(prm + o) = p;
        *(float4*)(m + o) = mm;
        *(float4*)(v + o) = vv;
    } else {
        for (int c = 0; c < 4 && i0 + c < P; ++c) {
            if (!on[c]) continue;
            const long long k = o + c;
            float pc = prm[k], mc = m[k], vc = v[k];
            adam_update(pc, mc, vc, grd[k], lr, hp);
            prm[k] = pc;
            m[k] = mc;
            v[k] = vc;
        }
    }
}

}  // namespace dg

dg::AdamHp dg_adam_hp(const float* lr, float beta1, float beta2, float eps, int64_t step)
{
    dg::AdamHp h;
    for (int i = 0; i < DG_NPARAM; ++i) h.lr[i] = lr[i];
    h.beta1 = beta1;
    h.beta2 = beta2;
    h.bc1 = (float)(1.0 - pow((double)beta1, (double)step));
    h.bc2_sqrt = (float)sqrt(1.0 - pow((double)beta2, (double)step));
    h.eps = eps;
    return h;
}

extern "C" dg_status dg_adam_hparams_fill(const float* lr, float beta1, float beta2, float eps, int64_t step,
                                          dg_adam_hparams* out)
{
    if (!lr || !out || step < 1) { dg_set_error("lr/out null or step < 1"); return DG_ERR_ARG; }
    *out = dg_adam_hp(lr, beta1, beta2, eps, step);
    return DG_OK;
}

extern "C" dg_status dg_adam_step_dev(float* params, const float* grads, float* m, float* v, int64_t stride,
                                      int64_t P, const dg_adam_hparams* hp_dev, const int32_t* skip_if,
                                      dg_stream stream)
{
    if (P < 0 || stride < P) { dg_set_error("bad P/stride"); return DG_ERR_ARG; }
    if (P == 0) return DG_OK;
    if (!params || !grads || !m || !v || !hp_dev) { dg_set_error("null buffer"); return DG_ERR_ARG; }
    const long long per = 256 * 4;
    dim3 grid((unsigned)((P + per - 1) / per), DG_NPARAM);
    dg::k_adam<<<grid, 256, 0, (cudaStream_t)stream>>>(params, grads, m, v, stride, P, dg::AdamHp{}, hp_dev, skip_if,
                                                        nullptr);
    dg_note_launch();
    return dg_check_launch("adam_dev");
}

extern "C" size_t dg_loss_workspace_size(int64_t n)
{
    (void)n;
    return sizeof(float) * dg::LOSS_BLOCKS_MAX;
}

extern "C" dg_status dg_loss_l1(const float* img, const float* target, int64_t n, float* dL_dimg,
                                float* loss, void* ws, size_t ws_bytes, dg_stream stream)
{
    if (n <= 0) { dg_set_error("n must be positive"); return DG_ERR_ARG; }
    if (!img || !target || !dL_dimg || !loss || !ws) { dg_set_error("null buffer"); return DG_ERR_ARG; }
    if (ws_bytes < dg_loss_workspace_size(n)) { dg_set_error("loss workspace too small"); return DG_ERR_CAPACITY; }
    long long nb = (n + dg::LOSS_THREADS - 1) / dg::LOSS_THREADS;
    if (nb > dg::LOSS_BLOCKS_MAX) nb = dg::LOSS_BLOCKS_MAX;
    cudaStream_t s = (cudaStream_t)stream;
    const float inv_n = (float)(1.0 / (double)n);
    dg::k_l1<<<(int)nb, dg::LOSS_THREADS, 0, s>>>(img, target, n, inv_n, dL_dimg, (float*)ws);
    dg_note_launch();
    dg::k_l1_final<<<1, 256, 0, s>>>((const float*)ws, (int)nb, (float)(1.0 / (double)n), loss);
    dg_note_launch();
    return dg_check_launch("loss_l1");
}

extern "C" dg_status dg_adam_step(float* params, const float* grads, float* m, float* v, int64_t stride,
                                  int64_t P, const float* lr, float beta1, float beta2, float eps,
                                  int64_t step, dg_stream stream)
{
    if (P < 0 || stride < P || step < 1) { dg_set_error("bad P/stride/step"); return DG_ERR_ARG; }
    if (P == 0) return DG_OK;
    if (!params || !grads || !m || !v || !lr) { dg_set_error("null buffer"); return DG_ERR_ARG; }
    const dg::AdamHp hp = dg_adam_hp(lr, beta1, beta2, eps, step);
    const long long per = 256 * 4;
    dim3 grid((unsigned)((P + per - 1) / per), DG_NPARAM);
    dg::k_adam<<<grid, 256, 0, (cudaStream_t)stream>>>(params, grads, m, v, stride, P, hp, nullptr, nullptr, nullptr);
    dg_note_launch();
    return dg_check_launch("adam");
}

namespace dg {
__global__ void k_visibility(const int* __restrict__ radius, long long P, int n_views, uint8_t* __restrict__ vis)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    uint8_t on = 0;
    for (int v = 0; v < n_views; ++v) on |= radius[(long long)v * P + i] > 0;
    vis[i] = on;
}
}  // namespace dg

extern "C" dg_status dg_visibility(const int32_t* radius, int64_t P, int32_t n_views, uint8_t* visible,
                                   dg_stream stream)
{
    if (P < 0 || n_views < 1 || n_views > DG_MAX_VIEWS) { dg_set_error("bad P/n_views"); return DG_ERR_ARG; }
    if (P == 0) return DG_OK;
    if (!radius || !visible) { dg_set_error("null buffer"); return DG_ERR_ARG; }
    dg::k_visibility<<<(unsigned)((P + 255) / 256), 256, 0, (cudaStream_t)stream>>>(radius, P, n_views, visible);
    dg_note_launch();
    return dg_check_launch("visibility");
}

extern "C" dg_status dg_sparse_adam_step(float* params, const float* grads, float* m, float* v, int64_t stride,
                                         int64_t P, const float* lr, float beta1, float beta2, float eps,
                                         int64_t step, const uint8_t* visible, dg_stream stream)
{
    if (P < 0 || stride < P || step < 1) { dg_set_error("bad P/stride/step"); return DG_ERR_ARG; }
    if (P == 0) return DG_OK;
    if (!params || !grads || !m || !v || !lr || !visible) { dg_set_error("null buffer"); return DG_ERR_ARG; }
    const dg::AdamHp hp = dg_adam_hp(lr, beta1, beta2, eps, step);
    const long long per = 256 * 4;
    dim3 grid((unsigned)((P + per - 1) / per), DG_NPARAM);
    dg::k_adam<<<grid, 256, 0, (cudaStream_t)stream>>>(params, grads, m, v, stride, P, hp, nullptr, nullptr, visible);
    dg_note_launch();
    return dg_check_launch("sparse_adam");
}

extern "C" dg_status dg_mse(const float* a, const float* b, int64_t n, float* mse, void* ws, size_t ws_bytes,
                            dg_stream stream)
{
    if (n <= 0) { dg_set_error("n must be positive"); return DG_ERR_ARG; }
    if (!a || !b || !mse || !ws) { dg_set_error("null buffer"); return DG_ERR_ARG; }
    if (ws_bytes < dg_loss_workspace_size(n)) { dg_set_error("workspace too small"); return DG_ERR_CAPACITY; }
    long long nb = (n + dg::LOSS_THREADS - 1) / dg::LOSS_THREADS;
    if (nb > dg::LOSS_BLOCKS_MAX) nb = dg::LOSS_BLOCKS_MAX;
    cudaStream_t s = (cudaStream_t)stream;
    dg::k_sqdiff<<<(int)nb, dg::LOSS_THREADS, 0, s>>>(a, b, n, (float*)ws);
    dg_note_launch();
    dg::k_l1_final<<<1, 256, 0, s>>>((const float*)ws, (int)nb, (float)(1.0 / (double)n), mse);
    dg_note_launch();
    return dg_check_launch("mse");
}

extern "C" dg_status dg_opacity_reset(float* params, float* m, float* v, int64_t stride, int64_t P, float max_opacity,
                                      dg_stream stream)
{
    if (P < 0 || stride < P || !(max_opacity > 0.f && max_opacity < 1.f)) { dg_set_error("bad arguments"); return DG_ERR_ARG; }
    if (P == 0) return DG_OK;
    if (!params || !m || !v) { dg_set_error("null buffer"); return DG_ERR_ARG; }
    const float cap = (float)log((double)max_opacity / (1.0 - (double)max_opacity));
    dg::k_opacity_reset<<<(int)((P + 255) / 256), 256, 0, (cudaStream_t)stream>>>(params, m, v, stride, P, cap);
    dg_note_launch();
    return dg_check_launch("opacity_reset");
}
