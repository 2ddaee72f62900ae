// Plume driver step for sm_103a: inlet source, first-order semi-Lagrangian
// advection of rho (cell centres) and u, v (faces) with the start-of-step
// velocity, Boussinesq buoyancy on the v faces (forward Euler), closed faces
// zeroed.  This produces u* for the projection (Sec. 2.2: advection, then
// external forces, then the pressure projection).
//
// Positions: cell (i, j) centred at (i + 1/2, j + 1/2); u face (j, i) at
// (i, j + 1/2); v face (j, i) at (i + 1/2, j); row 0 is the top of the image.
#include <cuda_runtime.h>
#include <math.h>

#include "hproj_internal.cuh"

namespace hp {

namespace {

struct Field {
    const float* q;  // [My][Mx]
    int Mx, My;
    float ox, oy;    // position of sample (0, 0)
};

// Bilinear sample at (x, y); the position is clamped to the sample span.
__device__ __forceinline__ float sample(const Field& f, float x, float y)
{
    const float tx = fminf(fmaxf(x - f.ox, 0.0f), (float)(f.Mx - 1));
    const float ty = fminf(fmaxf(y - f.oy, 0.0f), (float)(f.My - 1));
    int i0 = (int)floorf(tx), j0 = (int)floorf(ty);
    i0 = min(i0, max(f.Mx - 2, 0));
    j0 = min(j0, max(f.My - 2, 0));
    const float fx = tx - (float)i0, fy = ty - (float)j0;
    const int i1 = min(i0 + 1, f.Mx - 1), j1 = min(j0 + 1, f.My - 1);
    const float q00 = f.q[(size_t)j0 * f.Mx + i0], q01 = f.q[(size_t)j0 * f.Mx + i1];
    const float q10 = f.q[(size_t)j1 * f.Mx + i0], q11 = f.q[(size_t)j1 * f.Mx + i1];
    const float top = q00 * (1.0f - fx) + q01 * fx;
    const float bot = q10 * (1.0f - fx) + q11 * fx;
    return top * (1.0f - fy) + bot * fy;
}

// Density field with the inlet applied: rho_in on the inlet cells.
struct Rho {
    const float* q;
    int nx, ny, x0, x1;
    float rho_in;
    __device__ float at(int i, int j) const
    {
        return (j == ny - 1 && i >= x0 && i < x1) ? rho_in : q[(size_t)j * nx + i];
    }
};

__device__ __forceinline__ float sample_rho(const Rho& r, float x, float y)
{
    const float tx = fminf(fmaxf(x - 0.5f, 0.0f), (float)(r.nx - 1));
    const float ty = fminf(fmaxf(y - 0.5f, 0.0f), (float)(r.ny - 1));
    int i0 = (int)floorf(tx), j0 = (int)floorf(ty);
    i0 = min(i0, max(r.nx - 2, 0));
    j0 = min(j0, max(r.ny - 2, 0));
    const float fx = tx - (float)i0, fy = ty - (float)j0;
    const int i1 = min(i0 + 1, r.nx - 1), j1 = min(j0 + 1, r.ny - 1);
    const float top = r.at(i0, j0) * (1.0f - fx) + r.at(i1, j0) * fx;
    const float bot = r.at(i0, j1) * (1.0f - fx) + r.at(i1, j1) * fx;
    return top * (1.0f - fy) + bot * fy;
}

__device__ __forceinline__ bool fluid(const uint8_t* fl, int nx, int i, int j)
{
    return fl[(size_t)j * nx + i] == 0;
}

// New density of cell (i, j).
__device__ __forceinline__ float rho_new_at(const Rho& r, const Field& fu, const Field& fv,
                                            float dt, int i, int j)
{
    const float x = i + 0.5f, y = j + 0.5f;
    const float vx = sample(fu, x, y), vy = sample(fv, x, y);
    return sample_rho(r, x - dt * vx, y - dt * vy);
}

// One thread per (i, j) in [0, nx] x [0, ny]: cell (i, j) density, u face
// (j, i), v face (j, i) with buoyancy.
__global__ void advect_kernel(const float* __restrict__ u, const float* __restrict__ v,
                              const float* __restrict__ rho, const uint8_t* __restrict__ flags,
                              float* __restrict__ u_out, float* __restrict__ v_out,
                              float* __restrict__ rho_out, int ny, int nx, hp_plume_params p)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    const int b = blockIdx.z;
    if (i > nx) return;
    const size_t cells = (size_t)ny * nx;
    const Field fu = {u + (size_t)b * ny * (nx + 1), nx + 1, ny, 0.0f, 0.5f};
    const Field fv = {v + (size_t)b * (ny + 1) * nx, nx, ny + 1, 0.5f, 0.0f};
    const Rho r = {rho + b * cells, nx, ny, p.inlet_x0, p.inlet_x1, p.rho_in};
    const uint8_t* fl = flags + b * cells;
    const float dt = p.dt;

    if (i < nx && j < ny) rho_out[b * cells + (size_t)j * nx + i] = rho_new_at(r, fu, fv, dt, i, j);

    if (j < ny) {
        const bool open = i > 0 && i < nx && fluid(fl, nx, i - 1, j) && fluid(fl, nx, i, j);
        float val = 0.0f;
        if (open) {
            const float x = (float)i, y = j + 0.5f;
            const float vx = sample(fu, x, y), vy = sample(fv, x, y);
            val = sample(fu, x - dt * vx, y - dt * vy);
        }
        u_out[(size_t)b * ny * (nx + 1) + (size_t)j * (nx + 1) + i] = val;
    }
    if (i < nx) {
        const bool open = j > 0 && j < ny && fluid(fl, nx, i, j - 1) && fluid(fl, nx, i, j);
        float val = 0.0f;
        if (open) {
            const float x = i + 0.5f, y = (float)j;
            const float vx = sample(fu, x, y), vy = sample(fv, x, y);
            val = sample(fv, x - dt * vx, y - dt * vy);
            const float rf = 0.5f * (rho_new_at(r, fu, fv, dt, i, j - 1) +
                                     rho_new_at(r, fu, fv, dt, i, j));
            val += dt * p.gravity * (rf - p.rho_amb);
        }
        v_out[(size_t)b * (ny + 1) * nx + (size_t)j * nx + i] = val;
    }
}

}  // namespace

hp_status launch_advect(const float* u, const float* v, const float* rho, const uint8_t* flags,
                        float* u_out, float* v_out, float* rho_out, hp_shape s,
                        const hp_plume_params& p, cudaStream_t st)
{
    dim3 blk(128), grd((s.nx + 1 + 127) / 128, s.ny + 1, s.batch);
    advect_kernel<<<grd, blk, 0, st>>>(u, v, rho, flags, u_out, v_out, rho_out, s.ny, s.nx, p);
    return check_launch();
}

}  // namespace hp

extern "C" hp_status hp_advect_step(const float* u, const float* v, const float* rho,
                                    const uint8_t* flags, float* u_out, float* v_out,
                                    float* rho_out, hp_shape s, const hp_plume_params* p,
                                    void* stream)
{
    if (!u || !v || !rho || !flags || !u_out || !v_out || !rho_out || !p || !hp::shape_ok(s))
        return HP_ERR_INVALID_ARG;
    if (u_out == u || v_out == v || rho_out == rho || !(p->dt >= 0.0f)) return HP_ERR_INVALID_ARG;
    return hp::launch_advect(u, v, rho, flags, u_out, v_out, rho_out, s, *p, (cudaStream_t)stream);
}
