// C ABI of the projection library: context, argument checks, entry points.
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "hproj_internal.cuh"

namespace hp {

static thread_local char g_cuda_err[256] = "";

void set_cuda_error(cudaError_t e)
{
    snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", cudaGetErrorName(e),
             cudaGetErrorString(e));
}

hp_status check_launch()
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_cuda_error(e);
        return HP_ERR_CUDA;
    }
    return HP_OK;
}

// Kernels cover rows and grids with one CUDA grid dimension each (at most
// 65535 blocks), some with one row or grid more than the shape.
bool shape_ok(hp_shape s)
{
    return s.batch > 0 && s.ny > 0 && s.nx > 0 && s.batch <= HP_MAX_BATCH && s.ny <= HP_MAX_NY;
}

static bool fits(const hp_ctx* c, hp_shape s)
{
    return shape_ok(s) && s.batch <= c->max_shape.batch && s.ny <= c->max_shape.ny &&
           s.nx <= c->max_shape.nx;
}

bool project_args_ok(const hp_ctx* c, const float* u, const float* v, const uint8_t* flags,
                     hp_shape s, const hp_project_params* prm, const int32_t* iters_out,
                     const double* e_hist, int32_t hist_len)
{
    if (!c || !u || !v || !flags || !prm || !iters_out || !fits(c, s)) return false;
    if (prm->max_iters < 0 || prm->fixed_iters < 0 || prm->temporal_block < 0 ||
        prm->temporal_block > kMaxBlock || !(prm->threshold >= 0.0) || !(prm->dt > 0.0f) ||
        !(prm->rho0 > 0.0f) || prm->sweep_kernel < 0 || prm->sweep_kernel > 4)
        return false;
    if (prm->open_top != 0 && prm->open_top != 1) return false;
    if (prm->inflow_x1 > prm->inflow_x0 && (prm->inflow_x0 < 0 || prm->inflow_x1 > s.nx))
        return false;
    return (e_hist == nullptr) == (hist_len <= 0);
}

cudaError_t guarded_malloc(void** p, size_t bytes, Guards* g)
{
    *p = nullptr;
    cudaError_t e = cudaMalloc(p, bytes + kGuardBytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return e;
    }
    unsigned char* b = (unsigned char*)*p;
    e = cudaMemset(b, 0, bytes);
    if (e == cudaSuccess) e = cudaMemset(b + bytes, kGuardByte, kGuardBytes);
    if (e == cudaSuccess && g) g->zones.push_back(b + bytes);
    return e;
}

hp_status check_guards(const Guards& g)
{
    cudaError_t e = cudaDeviceSynchronize();
    unsigned char buf[kGuardBytes];
    for (size_t k = 0; e == cudaSuccess && k < g.zones.size(); ++k) {
        e = cudaMemcpy(buf, g.zones[k], kGuardBytes, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) break;
        for (size_t i = 0; i < kGuardBytes; ++i)
            if (buf[i] != (unsigned char)kGuardByte) return HP_ERR_GUARD;
    }
    if (e != cudaSuccess) {
        set_cuda_error(e);
        return HP_ERR_CUDA;
    }
    return HP_OK;
}

template <typename T>
static hp_status dalloc(T** p, size_t n, Guards* g)
{
    cudaError_t e = guarded_malloc((void**)p, n * sizeof(T), g);
    if (e != cudaSuccess) {
        set_cuda_error(e);
        return e == cudaErrorMemoryAllocation ? HP_ERR_OOM : HP_ERR_CUDA;
    }
    return HP_OK;
}

}  // namespace hp

using namespace hp;

extern "C" {

const char* hp_status_string(hp_status s)
{
    switch (s) {
    case HP_OK: return "ok";
    case HP_ERR_INVALID_ARG: return "invalid argument";
    case HP_ERR_CUDA: return "CUDA error";
    case HP_ERR_NONFINITE: return "non-finite input";
    case HP_ERR_OOM: return "out of device memory";
    case HP_ERR_UNSUPPORTED: return "unsupported";
    case HP_ERR_TIMEOUT: return "a tensor-core wait timed out";
    case HP_ERR_IO: return "checkpoint file error";
    case HP_ERR_GUARD: return "a workspace guard zone was overwritten";
    case HP_WARN_CNN_NONFINITE:
        return "warning: a network guess was not finite; its grids started from zero";
    }
    return "unknown status";
}

const char* hp_last_cuda_error(void) { return g_cuda_err; }

void hp_ctx_destroy(hp_ctx* c)
{
    if (!c) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(c->device);
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    cudaFree(c->mask);
    cudaFree(c->div);
    cudaFree(c->phi[0]);
    cudaFree(c->phi[1]);
    cudaFree(c->ckpt);
    cudaFree(c->partial);
    cudaFree(c->partial2);
    cudaFree(c->gs);
    cudaFree(c->ls);
    if (c->host_flag) cudaFreeHost(c->host_flag);
    if (prev >= 0) cudaSetDevice(prev);
    delete c;
}

hp_status hp_ctx_create(hp_ctx** out, hp_shape mx, int device)
{
    if (!out || !shape_ok(mx)) return HP_ERR_INVALID_ARG;
    *out = nullptr;
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) { set_cuda_error(e); return HP_ERR_CUDA; }
    if (prop.major != 10 || prop.minor != 3) {
        snprintf(g_cuda_err, sizeof(g_cuda_err),
                 "device %d is sm_%d%d; this library is built for sm_103a only", device,
                 prop.major, prop.minor);
        return HP_ERR_CUDA;
    }
    e = cudaSetDevice(device);
    if (e != cudaSuccess) { set_cuda_error(e); return HP_ERR_CUDA; }
    hp_ctx* c = new hp_ctx();
    c->device = device;
    c->num_sms = prop.multiProcessorCount;
    c->max_shape = mx;
    c->max_cells = (size_t)mx.batch * mx.ny * mx.nx;
    const int nct = ctas_per_grid(mx.ny, mx.nx, kMaxBlock) > ctas_per_grid(mx.ny, mx.nx, 4)
                        ? ctas_per_grid(mx.ny, mx.nx, kMaxBlock)
                        : ctas_per_grid(mx.ny, mx.nx, 4);
    c->partial_len = (size_t)mx.batch * kMaxBlock * nct;
    {
        // the streaming sweep keeps two partials (sweep parity) per 16 x 128 block
        const size_t s1 = (size_t)mx.batch * 2 * ((mx.nx + 127) / 128) * ((mx.ny + 15) / 16);
        if (s1 > c->partial_len) c->partial_len = s1;
    }
    c->partial2_len = (size_t)mx.batch * ((mx.nx + 255) / 256) * mx.ny;
    hp_status rc;
    if ((rc = dalloc(&c->mask, c->max_cells, &c->guards)) != HP_OK ||
        (rc = dalloc(&c->div, c->max_cells, &c->guards)) != HP_OK ||
        (rc = dalloc(&c->phi[0], c->max_cells, &c->guards)) != HP_OK ||
        (rc = dalloc(&c->phi[1], c->max_cells, &c->guards)) != HP_OK ||
        (rc = dalloc(&c->ckpt, c->max_cells, &c->guards)) != HP_OK ||
        (rc = dalloc(&c->partial, c->partial_len, &c->guards)) != HP_OK ||
        (rc = dalloc(&c->partial2, c->partial2_len, &c->guards)) != HP_OK ||
        (rc = dalloc(&c->gs, (size_t)mx.batch, &c->guards)) != HP_OK ||
        (rc = dalloc(&c->ls, 1, &c->guards)) != HP_OK) {
        hp_ctx_destroy(c);
        return rc;
    }
    e = cudaMallocHost((void**)&c->host_flag, sizeof(int32_t));
    if (e != cudaSuccess) {
        set_cuda_error(e);
        hp_ctx_destroy(c);
        return HP_ERR_CUDA;
    }
    // zero the workspaces once so that no kernel ever reads uninitialised
    // memory (the phi buffers are read in halo cells of ragged tiles)
    cudaMemset(c->phi[0], 0, c->max_cells * sizeof(float));
    cudaMemset(c->phi[1], 0, c->max_cells * sizeof(float));
    cudaMemset(c->gs, 0, (size_t)mx.batch * sizeof(GridState));
    cudaMemset(c->ls, 0, sizeof(LoopState));
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        set_cuda_error(e);
        hp_ctx_destroy(c);
        return HP_ERR_CUDA;
    }
    *out = c;
    return HP_OK;
}

hp_status hp_ctx_check(hp_ctx* c)
{
    if (!c) return HP_ERR_INVALID_ARG;
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) { set_cuda_error(e); return HP_ERR_CUDA; }
    return check_guards(c->guards);
}

hp_status hp_face_mask(const uint8_t* flags, uint8_t* mask_out, hp_shape s, void* stream)
{
    if (!flags || !mask_out || !shape_ok(s)) return HP_ERR_INVALID_ARG;
    return launch_mask(flags, mask_out, s, (cudaStream_t)stream);
}

hp_status hp_divergence(const float* u, const float* v, const uint8_t* flags, float* div_out,
                        hp_shape s, void* stream)
{
    if (!u || !v || !flags || !div_out || !shape_ok(s)) return HP_ERR_INVALID_ARG;
    return launch_mask_div(u, v, flags, nullptr, div_out, s, (cudaStream_t)stream);
}

hp_status hp_div_norms(hp_ctx* c, const float* u, const float* v, const uint8_t* flags,
                       double* e1_out, double* einf_out, hp_shape s, void* stream)
{
    if (!c || !u || !v || !flags || !fits(c, s)) return HP_ERR_INVALID_ARG;
    return launch_div_norms(u, v, flags, c->partial2, (int)(c->partial2_len / s.batch), e1_out,
                            einf_out, s, (cudaStream_t)stream);
}

hp_status hp_project(hp_ctx* c, float* u, float* v, const uint8_t* flags, hp_shape s,
                     const hp_project_params* prm, const float* phi0, float* p_out,
                     int32_t* iters_out, double* e1_out, double* einf_out, uint8_t* conv_out,
                     double* e_hist, int32_t hist_len, void* stream)
{
    if (!project_args_ok(c, u, v, flags, s, prm, iters_out, e_hist, hist_len))
        return HP_ERR_INVALID_ARG;
    return project_impl(c, u, v, flags, s, prm, phi0, p_out, iters_out, e1_out, einf_out, conv_out,
                        e_hist, hist_len, (cudaStream_t)stream, nullptr);
}

hp_status hp_jacobi_sweeps(hp_ctx* c, const float* phi_in, const float* div,
                           const uint8_t* flags, float* phi_out, int32_t n, double* e_out,
                           hp_shape s, void* stream)
{
    if (!c || !phi_in || !div || !flags || !phi_out || n < 1 || !fits(c, s) || phi_in == phi_out)
        return HP_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t cells = (size_t)s.batch * s.ny * s.nx;
    // geometry from the flags, right-hand side copied into the workspace
    hp_status rc = launch_mask(flags, c->mask, s, st);
    if (rc != HP_OK) return rc;
    cudaError_t e = cudaMemcpyAsync(c->div, div, cells * sizeof(float), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) { set_cuda_error(e); return HP_ERR_CUDA; }
    hp_project_params prm = {};
    prm.fixed_iters = n;
    prm.dt = 1.0f;
    prm.rho0 = 1.0f;
    prm.use_graph = 1;
    return project_impl(c, nullptr, nullptr, flags, s, &prm, phi_in, nullptr, nullptr, nullptr,
                        nullptr, nullptr, e_out, e_out ? n : 0, st, phi_out);
}

hp_status hp_jacobi_target(hp_ctx* c, const float* div, const uint8_t* flags, int32_t n,
                           float* target_out, hp_shape s, void* stream)
{
    if (!c || !div || !flags || !target_out || n < 0 || !fits(c, s)) return HP_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t cells = (size_t)s.batch * s.ny * s.nx;
    hp_status rc = launch_mask(flags, c->mask, s, st);
    if (rc != HP_OK) return rc;
    cudaError_t e =
        cudaMemcpyAsync(c->div, div, cells * sizeof(float), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) { set_cuda_error(e); return HP_ERR_CUDA; }
    // phi_n into the checkpoint workspace (free once the sweeps are done)
    if (n > 0) {
        hp_project_params prm = {};
        prm.fixed_iters = n;
        prm.dt = 1.0f;
        prm.rho0 = 1.0f;
        prm.use_graph = 1;
        rc = project_impl(c, nullptr, nullptr, flags, s, &prm, nullptr, nullptr, nullptr, nullptr,
                          nullptr, nullptr, nullptr, 0, st, c->ckpt);
        if (rc != HP_OK) return rc;
    } else {
        e = cudaMemsetAsync(c->ckpt, 0, cells * sizeof(float), st);
        if (e != cudaSuccess) { set_cuda_error(e); return HP_ERR_CUDA; }
    }
    return launch_mean_sweep(c->ckpt, c->div, c->mask, target_out, s, st);
}

}  // extern "C"
