// pack.cu -- mixed-precision projected records for the render passes: float16
// conic and opacity, bfloat16 colour, float32 pixel position (24 bytes instead
// of 48 per record; the render kernels widen them to float32 when staging).
#include <string.h>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"

namespace dg {
namespace {

__global__ void __launch_bounds__(256)
k_pack_records(const float4* __restrict__ feat, long long n, uint2* __restrict__ out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 a = feat[3 * i], b = feat[3 * i + 1];
    const float c = feat[3 * i + 2].x;
    const __half2 ab = __floats2half2_rn(a.z, a.w);
    const __half2 co = __floats2half2_rn(b.x, b.y);
    const __nv_bfloat162 rg = __floats2bfloat162_rn(b.z, b.w);
    const __nv_bfloat16 bb = __float2bfloat16_rn(c);
    uint2 w1, w2;
    memcpy(&w1.x, &ab, 4);
    memcpy(&w1.y, &co, 4);
    memcpy(&w2.x, &rg, 4);
    unsigned short bbits;
    memcpy(&bbits, &bb, 2);
    w2.y = (unsigned)bbits;
    out[3 * i] = make_uint2(__float_as_uint(a.x), __float_as_uint(a.y));
    out[3 * i + 1] = w1;
    out[3 * i + 2] = w2;
}

}  // namespace
}  // namespace dg

extern "C" dg_status dg_pack_records(const float* feat, int64_t n_records, void* packed, dg_stream stream)
{
    if (n_records < 0) { dg_set_error("n_records < 0"); return DG_ERR_ARG; }
    if (n_records == 0) return DG_OK;
    if (!feat || !packed) { dg_set_error("null buffer"); return DG_ERR_ARG; }
    if ((((uintptr_t)feat) & 15u) || (((uintptr_t)packed) & 7u)) {
        dg_set_error("feat must be 16-byte and packed 8-byte aligned");
        return DG_ERR_ARG;
    }
    const long long nb = (n_records + 255) / 256;
    dg::k_pack_records<<<(unsigned)nb, 256, 0, (cudaStream_t)stream>>>((const float4*)feat, n_records, (uint2*)packed);
    dg_note_launch();
    return dg_check_launch("pack_records");
}
