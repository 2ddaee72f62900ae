// hp_div_norms_noalloc: the divergence-norm reduction with its scratch in a
// fixed device array of this library instead of memory from cudaMalloc.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdio.h>

#include <mutex>

#include "hproj_internal.cuh"

namespace {

// Scratch of hp_div_norms_noalloc: one 8-byte partial (the FP32 sum and max
// of |div|) per 256-cell segment.  Every device that loads the library holds
// this array until the process exits.
static __device__ __align__(256) double g_noalloc_partial[HP_NOALLOC_MAX_BLOCKS];

// The device address of a __device__ array belongs to the CUDA context that
// loaded this library's module, not to the device: after cudaDeviceReset, or
// with another (non-primary) context current, the array sits elsewhere.  The
// address is therefore cached per context, keyed by the driver's context id
// (unique for the life of the process, never reused).  In host code the array
// name is a host-side stand-in, never a device address.
struct ScratchAddr {
    unsigned long long ctx_id;
    double* partial;
};
constexpr int kCacheSlots = 16;
std::mutex g_setup_mu;
ScratchAddr g_cache[kCacheSlots] = {};
int g_cache_next = 0;

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

// The two driver calls are reached through the runtime's entry-point lookup,
// so that the library does not link the driver library itself (it must load
// on machines without a GPU driver, where every call then reports an error).
hp_status resolve_driver_calls()
{
    if (g_ctx_get_current && g_ctx_get_id) return HP_OK;
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000,
                                                     cudaEnableDefault, &q1);
    if (e == cudaSuccess)
        e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
    if (e != cudaSuccess) { hp::set_cuda_error(e); return HP_ERR_CUDA; }
    if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
        return HP_ERR_CUDA;
    g_ctx_get_current = (CtxGetCurrentFn)f1;
    g_ctx_get_id = (CtxGetIdFn)f2;
    return HP_OK;
}

// Id of the context current on this thread; 0 when there is none yet.
hp_status current_ctx_id(unsigned long long* id)
{
    CUcontext ctx = nullptr;
    *id = 0;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS) return HP_ERR_CUDA;
    if (!ctx) return HP_OK;
    if (g_ctx_get_id(ctx, id) != CUDA_SUCCESS) return HP_ERR_CUDA;
    return HP_OK;
}

hp_status scratch_for_current_context(double** partial)
{
    std::lock_guard<std::mutex> lock(g_setup_mu);
    hp_status rc = resolve_driver_calls();
    if (rc != HP_OK) return rc;
    unsigned long long id = 0;
    if ((rc = current_ctx_id(&id)) != HP_OK) return rc;
    for (int k = 0; id && k < kCacheSlots; ++k) {
        if (g_cache[k].ctx_id == id) {
            *partial = g_cache[k].partial;
            return HP_OK;
        }
    }
    // Set-up for this context: look the array up with it current (the
    // runtime makes the device's primary context current first if no context
    // is; the id is then read again).
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partial);
    if (e != cudaSuccess) { hp::set_cuda_error(e); return HP_ERR_CUDA; }
    if (!id && ((rc = current_ctx_id(&id)) != HP_OK || !id)) return HP_ERR_CUDA;
    g_cache[g_cache_next] = {id, (double*)p};
    g_cache_next = (g_cache_next + 1) % kCacheSlots;
    *partial = (double*)p;
    return HP_OK;
}

}  // namespace

extern "C" hp_status hp_div_norms_noalloc(const float* u, const float* v, const uint8_t* flags,
                                          double* e1_out, double* einf_out, hp_shape s,
                                          void* stream)
{
    if (!u || !v || !flags || !e1_out || !einf_out || !hp::shape_ok(s)) return HP_ERR_INVALID_ARG;
    const size_t blocks = (size_t)s.batch * (size_t)s.ny * (size_t)((s.nx + 255) / 256);
    if (s.batch > HP_NOALLOC_MAX_BATCH || blocks > (size_t)HP_NOALLOC_MAX_BLOCKS) {
        return HP_ERR_INVALID_ARG;
    }
    double* partial = nullptr;
    hp_status rc = scratch_for_current_context(&partial);
    if (rc != HP_OK) return rc;
    return hp::launch_div_norms_scratch(u, v, flags, partial, e1_out, einf_out, s,
                                        (cudaStream_t)stream);
}
