// hp_div_norms_noalloc: the divergence-norm reduction with its scratch in a
// fixed device array of this library instead of memory from cudaMalloc.
#include <cuda_runtime.h>
#include <stdio.h>

#include <mutex>

#include "hproj_internal.cuh"

namespace {

// Scratch of hp_div_norms_noalloc.  Every device that loads the library holds
// these arrays until the process exits.
static __device__ __align__(256) double g_noalloc_partial[HP_NOALLOC_MAX_BLOCKS];
static __device__ __align__(256) uint32_t g_noalloc_einf[HP_NOALLOC_MAX_BATCH];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
// Device addresses of the arrays, looked up once per device.  In host code
// the array names are host-side stand-ins, never device addresses.
double* g_partial_addr[kMaxDevices] = {};
uint32_t* g_einf_addr[kMaxDevices] = {};

hp_status scratch_for_current_device(double** partial, uint32_t** einf)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { hp::set_cuda_error(e); return HP_ERR_CUDA; }
    if (dev < 0 || dev >= kMaxDevices) return HP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_partial_addr[dev]) {
        void* p = nullptr;
        void* q = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partial);
        if (e != cudaSuccess) { hp::set_cuda_error(e); return HP_ERR_CUDA; }
        e = cudaGetSymbolAddress(&q, g_noalloc_einf);
        if (e != cudaSuccess) { hp::set_cuda_error(e); return HP_ERR_CUDA; }
        g_einf_addr[dev] = (uint32_t*)q;
        g_partial_addr[dev] = (double*)p;
    }
    *partial = g_partial_addr[dev];
    *einf = g_einf_addr[dev];
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
    uint32_t* einf = nullptr;
    hp_status rc = scratch_for_current_device(&partial, &einf);
    if (rc != HP_OK) return rc;
    return hp::launch_div_norms_scratch(u, v, flags, partial, einf, 1, e1_out, einf_out, s,
                                        (cudaStream_t)stream);
}
