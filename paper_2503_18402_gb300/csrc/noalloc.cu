// noalloc.cu -- L1 loss entry point for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: plugins whose host application
// owns every device allocation, or real-time loops that forbid allocator calls
// after start-up.  dg_loss_l1 needs a caller workspace for its per-block partial
// sums; this variant keeps those partials in a fixed device array that lives in
// the library's own module instead.  It is called from an ordinary host thread
// (host functions enqueued on a stream may not make CUDA calls).
//
// The array is DG_L1_NOALLOC_BLOCKS floats (4 KiB).  Every GPU that loads the
// library holds it until the process exits.  All calls share it: calls queued
// on one stream run in order, two calls that overlap on the GPU (different
// streams, no ordering between them) race on it.  Each call overwrites every
// partial it later reads, so nothing needs clearing.
#include <mutex>

#include "common.cuh"

namespace dg {
constexpr int L1_THREADS = 256;
constexpr int L1_BLOCKS = DG_L1_NOALLOC_BLOCKS;
// defined in optim.cu
__global__ void k_l1(const float* __restrict__ img, const float* __restrict__ tgt, long long n, float inv_n,
                     float* __restrict__ grad, float* __restrict__ partial);
__global__ void k_l1_final(const float* __restrict__ partial, int nb, float inv_n, float* loss);
}  // namespace dg

static __device__ __align__(256) float g_l1_scratch[DG_L1_NOALLOC_BLOCKS];

// Device address of g_l1_scratch per device, looked up with that device current
// and remembered together with the context it belongs to: after the device's
// context is destroyed and recreated (cudaDeviceReset) the module is loaded
// anew, so a changed context means the address is looked up again.
static constexpr int kMaxDevices = 64;
struct ScratchEntry {
    void* ctx;
    float* ptr;
};
static ScratchEntry g_scratch[kMaxDevices] = {};
static std::mutex g_scratch_mu;

// cuCtxGetCurrent through the runtime's driver entry-point query (no link
// against the driver library, so the library still loads on hosts without one).
typedef int (*CtxGetCurrentFn)(void**);
static CtxGetCurrentFn ctx_get_current()
{
    static CtxGetCurrentFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return (CtxGetCurrentFn)p;
    }();
    return fn;
}

static dg_status scratch_for_current_device(cudaStream_t stream, float** out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { dg_set_error("cudaGetDevice: %s", cudaGetErrorString(e)); return DG_ERR_CUDA; }
    if (dev < 0 || dev >= kMaxDevices) { dg_set_error("device ordinal %d out of range", dev); return DG_ERR_ARG; }
    CtxGetCurrentFn get = ctx_get_current();
    if (!get) { dg_set_error("cannot query the current CUDA context"); return DG_ERR_CUDA; }
    // null before this thread's first runtime call made the primary context current
    void* ctx = nullptr;
    if (get(&ctx) != 0) ctx = nullptr;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    ScratchEntry& ent = g_scratch[dev];
    if (ctx && ent.ptr && ent.ctx == ctx) {
        *out = ent.ptr;
        return DG_OK;
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(stream, &cap);
    if (e != cudaSuccess) { dg_set_error("cudaStreamIsCapturing: %s", cudaGetErrorString(e)); return DG_ERR_CUDA; }
    if (cap != cudaStreamCaptureStatusNone) {
        dg_set_error("dg_loss_l1_noalloc: the first call on device %d (or after its context was recreated) "
                     "must come before stream capture",
                     dev);
        return DG_ERR_ARG;
    }
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_l1_scratch);
    if (e != cudaSuccess || !p) {
        dg_set_error("cudaGetSymbolAddress(l1 scratch): %s", cudaGetErrorString(e));
        return DG_ERR_CUDA;
    }
    if (get(&ctx) != 0 || !ctx) { dg_set_error("no current CUDA context"); return DG_ERR_CUDA; }
    ent.ctx = ctx;
    ent.ptr = (float*)p;
    *out = ent.ptr;
    return DG_OK;
}

extern "C" dg_status dg_loss_l1_noalloc(const float* img, const float* target, int64_t n, float* dL_dimg,
                                        float* loss, dg_stream stream)
{
    if (n <= 0) { dg_set_error("n must be positive"); return DG_ERR_ARG; }
    if (n > DG_L1_NOALLOC_MAX_N) {
        dg_set_error("n = %lld exceeds the no-allocation limit of %lld values", (long long)n,
                     (long long)DG_L1_NOALLOC_MAX_N);
        return DG_ERR_ARG;
    }
    if (!img || !target || !dL_dimg || !loss) { dg_set_error("null buffer"); return DG_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    float* scratch = nullptr;
    const dg_status st = scratch_for_current_device(s, &scratch);
    if (st != DG_OK) return st;
    long long nb = (n + dg::L1_THREADS - 1) / dg::L1_THREADS;
    if (nb > dg::L1_BLOCKS) nb = dg::L1_BLOCKS;
    const float inv_n = (float)(1.0 / (double)n);
    dg::k_l1<<<(int)nb, dg::L1_THREADS, 0, s>>>(img, target, n, inv_n, dL_dimg, scratch);
    dg_note_launch();
    dg::k_l1_final<<<1, 256, 0, s>>>(scratch, (int)nb, inv_n, loss);
    dg_note_launch();
    return dg_check_launch("loss_l1_noalloc");
}
