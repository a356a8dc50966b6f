// capi.cu -- error reporting and version entry points of the C ABI.
#include <stdarg.h>
#include <stdio.h>

#include <atomic>

#include "common.cuh"

static thread_local char g_err[512] = "";
static std::atomic<long long> g_launches{0};

void dg_note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

extern "C" int64_t dg_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

void dg_set_error(const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

// Reports (and clears) a launch-configuration error of the last launch.
dg_status dg_check_launch(const char* what)
{
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        dg_set_error("%s: %s", what, cudaGetErrorString(e));
        return DG_ERR_CUDA;
    }
    return DG_OK;
}

extern "C" const char* dg_last_error(void) { return g_err; }

extern "C" int32_t dg_abi_version(void) { return 7; }
