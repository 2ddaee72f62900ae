// Adjoint of the fixed-count projection (Sec. 3.2: the gradient of the
// correction of Eq. 2 is known, so the network can be trained through the
// solver).  Forward: div = D(Z u*), phi_k = k masked Jacobi sweeps from
// phi_0, u = Z u* - G phi_k, p = phi_k rho0 / dt.  With W the open-face
// adjacency and n the open-face count, one sweep is phi' = n^-1 (W phi - div);
// its transpose needs no stored iterate (the map is affine):
//   lam_k = D(g_u) + (rho0/dt) g_p            (G^T = -D on open faces)
//   mu_t  = n^-1 lam_t,  lam_{t-1} = W mu_t    for t = k .. 1
//   dL/dphi_0 = lam_0,  dL/ddiv = -sum_{t=1..k} mu_t
//   dL/du* = Z g_u - G dL/ddiv
// and mu_{t-1} = n^-1 W mu_t is the forward sweep with a zero right-hand side.
#include <cuda_runtime.h>

#include "hproj_internal.cuh"

namespace hp {

namespace {

__device__ __forceinline__ float inv_open(uint32_t m)
{
    const int n = __popc(m & 15u);
    return n == 4 ? 0.25f : n == 3 ? (1.0f / 3.0f) : n == 2 ? 0.5f : n == 1 ? 1.0f : 0.0f;
}

// sum of q over the open-face neighbours of cell c
__device__ __forceinline__ float open_sum(const float* q, uint32_t m, size_t c, int nx)
{
    float s = 0.0f;
    if (m & 1u) s += q[c - 1];
    if (m & 2u) s += q[c + 1];
    if (m & 4u) s += q[c - nx];
    if (m & 8u) s += q[c + nx];
    return s;
}

// lam_k = D(g) + scale * g_p; mu_k = lam_k / n (k > 0) or g_phi0 = lam_k (k = 0)
__global__ void adj_init_kernel(const float* __restrict__ gu, const float* __restrict__ gv,
                                const float* __restrict__ gp, const uint8_t* __restrict__ mask,
                                float scale, float* __restrict__ mu, float* __restrict__ acc,
                                int k, int ny, int nx)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    const int b = blockIdx.z;
    if (i >= nx) return;
    const size_t q = (size_t)b * ny * nx + (size_t)j * nx + i;
    const uint32_t m = mask[q];
    const float* ub = gu + (size_t)b * ny * (nx + 1) + (size_t)j * (nx + 1);
    const float* vb = gv + (size_t)b * (ny + 1) * nx;
    const float ue = (m & 2u) ? ub[i + 1] : 0.0f;
    const float uw = (m & 1u) ? ub[i] : 0.0f;
    const float vs = (m & 8u) ? vb[(size_t)(j + 1) * nx + i] : 0.0f;
    const float vn = (m & 4u) ? vb[(size_t)j * nx + i] : 0.0f;
    float lam = (ue - uw) + (vs - vn);
    if (gp) lam += scale * gp[q];
    if (!(m & 15u)) lam = 0.0f;
    mu[q] = k > 0 ? lam * inv_open(m) : lam;
    acc[q] = 0.0f;
}

// acc += mu_t; mu_{t-1} = n^-1 W mu_t, or on the last step g_phi0 = W mu_1
__global__ void adj_sweep_kernel(const float* __restrict__ mu_in, float* __restrict__ out,
                                 float* __restrict__ acc, const uint8_t* __restrict__ mask,
                                 int last, int ny, int nx)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    const int b = blockIdx.z;
    if (i >= nx) return;
    const size_t base = (size_t)b * ny * nx;
    const size_t c = (size_t)j * nx + i;
    const uint32_t m = mask[base + c];
    acc[base + c] += mu_in[base + c];
    const float s = open_sum(mu_in + base, m, c, nx);
    out[base + c] = last ? s : s * inv_open(m);
}

// g_u* = g_u + (acc_c - acc_nb) on open faces, 0 on closed faces
__global__ void adj_correct_kernel(const float* __restrict__ gu, const float* __restrict__ gv,
                                   const float* __restrict__ acc, const uint8_t* __restrict__ mask,
                                   float* __restrict__ gus, float* __restrict__ gvs, int ny, int nx)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    const int b = blockIdx.z;
    if (i >= nx) return;
    const size_t base = (size_t)b * ny * nx;
    const size_t c = (size_t)j * nx + i;
    const uint32_t m = mask[base + c];
    const size_t uo = (size_t)b * ny * (nx + 1) + (size_t)j * (nx + 1);
    const size_t vo = (size_t)b * (ny + 1) * nx;
    float uw = 0.0f, vn = 0.0f;
    if (m & 1u) uw = gu[uo + i] + (acc[base + c] - acc[base + c - 1]);
    if (m & 4u) vn = gv[vo + (size_t)j * nx + i] + (acc[base + c] - acc[base + c - nx]);
    gus[uo + i] = uw;
    gvs[vo + (size_t)j * nx + i] = vn;
    if (i == nx - 1) gus[uo + nx] = 0.0f;
    if (j == ny - 1) gvs[vo + (size_t)ny * nx + i] = 0.0f;
}

}  // namespace

}  // namespace hp

using namespace hp;

extern "C" hp_status hp_project_adjoint(hp_ctx* ctx, const float* gu, const float* gv,
                                        const float* gp, const uint8_t* flags, hp_shape s,
                                        int32_t k, float dt, float rho0, float* gu_star,
                                        float* gv_star, float* g_phi0, void* stream)
{
    if (!ctx || !gu || !gv || !flags || !gu_star || !gv_star || !g_phi0 || k < 0 ||
        !shape_ok(s) || s.batch > ctx->max_shape.batch || s.ny > ctx->max_shape.ny ||
        s.nx > ctx->max_shape.nx || !(dt > 0.0f))
        return HP_ERR_INVALID_ARG;
    if (gu_star == gu || gv_star == gv) return HP_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    hp_status rc = launch_mask(flags, ctx->mask, s, st);
    if (rc != HP_OK) return rc;
    dim3 blk(256), grd((s.nx + 255) / 256, s.ny, s.batch);
    float* acc = ctx->div;
    float* bufs[2] = {ctx->phi[0], ctx->phi[1]};
    adj_init_kernel<<<grd, blk, 0, st>>>(gu, gv, gp, ctx->mask, rho0 / dt, k > 0 ? bufs[0] : g_phi0,
                                         acc, k, s.ny, s.nx);
    if ((rc = check_launch()) != HP_OK) return rc;
    for (int t = k; t >= 1; --t) {
        const int cur = (k - t) & 1;
        float* out = t == 1 ? g_phi0 : bufs[cur ^ 1];
        adj_sweep_kernel<<<grd, blk, 0, st>>>(bufs[cur], out, acc, ctx->mask, t == 1, s.ny, s.nx);
        if ((rc = check_launch()) != HP_OK) return rc;
    }
    adj_correct_kernel<<<grd, blk, 0, st>>>(gu, gv, acc, ctx->mask, gu_star, gv_star, s.ny, s.nx);
    return check_launch();
}
