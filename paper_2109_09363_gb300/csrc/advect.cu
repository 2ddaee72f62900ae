// Plume driver step for sm_103a: inlet source, semi-Lagrangian advection of
// rho (cell centres) and u, v (faces) with the start-of-step velocity,
// first order or MacCormack, Boussinesq buoyancy on the v faces (forward
// Euler), closed faces zeroed.  This produces u* for the projection
// (Sec. 2.2: advection, then external forces, then the pressure projection).
//
// MacCormack (the scheme Sec. 2.2 names, after Selle et al. 2008): q_f, the
// forward semi-Lagrangian value, q_b, the forward field sampled backwards at
// x + dt vel(x), and q_f + (q - q_b) / 2 clamped to the range of the four
// samples the forward step interpolated.  The forward field is not stored
// in global memory: each CTA evaluates it on a window around its tile in
// shared memory (and evaluates a corner outside the window where it needs
// it), so the step needs no workspace.
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
    __device__ float at(int i, int j) const { return __ldg(q + (size_t)j * Mx + i); }
};

// Velocity at sample (i, j) of a quantity whose samples sit at (i + ox,
// j + oy): cell centres (1/2, 1/2), u faces (0, 1/2) or v faces (1/2, 0).
// There the bilinear sample of each component has weights 0, 1 or 1/2 on a
// row or column pair (pairs clamped to the field at its borders), so it is a
// copy or the mean of two or four values; for finite inputs the result is
// the same FP32 value as the general bilinear sample of sample_range()
// (products by 1/2 are exact, and the one rounding of each weighted sum is
// the rounding of the plain sum, halved).
__device__ __forceinline__ void vel_at_sample(const Field& fu, const Field& fv, float ox,
                                              float oy, int i, int j, float& vx, float& vy)
{
    const int su = fu.Mx, nx = fv.Mx, ny = fu.My;  // u rows hold nx + 1 faces
    const float* u = fu.q;
    const float* v = fv.q;
    if (ox != 0.0f && oy != 0.0f) {  // cell (i, j)
        const float* ur = u + (size_t)j * su;
        vx = 0.5f * (__ldg(ur + i) + __ldg(ur + i + 1));
        vy = 0.5f * (__ldg(v + (size_t)j * nx + i) + __ldg(v + (size_t)(j + 1) * nx + i));
    } else if (ox == 0.0f) {  // u face (j, i), i in [0, nx]
        vx = __ldg(u + (size_t)j * su + i);
        const int c0 = max(i - 1, 0), c1 = min(i, nx - 1);
        const float* v0 = v + (size_t)j * nx;
        const float* v1 = v0 + nx;
        vy = 0.5f * (0.5f * (__ldg(v0 + c0) + __ldg(v0 + c1)) +
                     0.5f * (__ldg(v1 + c0) + __ldg(v1 + c1)));
    } else {  // v face (j, i), j in [0, ny]
        vy = __ldg(v + (size_t)j * nx + i);
        const int r0 = max(j - 1, 0), r1 = min(j, ny - 1);
        const float* u0 = u + (size_t)r0 * su;
        const float* u1 = u + (size_t)r1 * su;
        vx = 0.5f * (0.5f * (__ldg(u0 + i) + __ldg(u0 + i + 1)) +
                     0.5f * (__ldg(u1 + i) + __ldg(u1 + i + 1)));
    }
}

// Density field with the inlet applied: rho_in on the inlet cells.
struct Rho {
    const float* q;
    int nx, ny, x0, x1;
    float rho_in;
    __device__ float at(int i, int j) const
    {
        return (j == ny - 1 && i >= x0 && i < x1) ? rho_in : __ldg(q + (size_t)j * nx + i);
    }
};

// Generic quantity view: Mx x My samples, sample (0, 0) at (ox, oy).
template <class Q>
struct View {
    const Q& q;
    int Mx, My;
    float ox, oy;
};

// Bilinear sample of a view at (x, y) (position clamped to the sample span),
// with the range of the four samples it interpolates.
template <class V>
__device__ __forceinline__ float sample_range(const V& f, float x, float y, float* lo, float* hi)
{
    const float tx = fminf(fmaxf(x - f.ox, 0.0f), (float)(f.Mx - 1));
    const float ty = fminf(fmaxf(y - f.oy, 0.0f), (float)(f.My - 1));
    int i0 = (int)floorf(tx), j0 = (int)floorf(ty);
    i0 = min(i0, max(f.Mx - 2, 0));
    j0 = min(j0, max(f.My - 2, 0));
    const float fx = tx - (float)i0, fy = ty - (float)j0;
    const int i1 = min(i0 + 1, f.Mx - 1), j1 = min(j0 + 1, f.My - 1);
    const float q00 = f.q.at(i0, j0), q01 = f.q.at(i1, j0);
    const float q10 = f.q.at(i0, j1), q11 = f.q.at(i1, j1);
    if (lo) {
        *lo = fminf(fminf(q00, q01), fminf(q10, q11));
        *hi = fmaxf(fmaxf(q00, q01), fmaxf(q10, q11));
    }
    const float top = q00 * (1.0f - fx) + q01 * fx;
    const float bot = q10 * (1.0f - fx) + q11 * fx;
    return top * (1.0f - fy) + bot * fy;
}

// The forward semi-Lagrangian field of a quantity, evaluated on demand at
// its own samples.
template <class Q>
struct Forward {
    const Q& q;
    const Field& fu;
    const Field& fv;
    int Mx, My;
    float ox, oy, dt;
    // the forward value at sample (i, j), with the velocity (vx, vy) there
    __device__ float at_vel(int i, int j, float& vx, float& vy) const
    {
        const float x = (float)i + ox, y = (float)j + oy;
        vel_at_sample(fu, fv, ox, oy, i, j, vx, vy);
        const View<Q> w = {q, Mx, My, ox, oy};
        return sample_range(w, x - dt * vx, y - dt * vy, nullptr, nullptr);
    }
    __device__ float at(int i, int j) const
    {
        float vx, vy;
        return at_vel(i, j, vx, vy);
    }
};

// New value of sample (i, j) of quantity q (Mx x My samples at (ox, oy)).
template <bool MC, class Q>
__device__ __forceinline__ float advected(const Q& q, int Mx, int My, float ox, float oy,
                                          const Field& fu, const Field& fv, float dt, int i,
                                          int j)
{
    const float x = (float)i + ox, y = (float)j + oy;
    float vx, vy;
    vel_at_sample(fu, fv, ox, oy, i, j, vx, vy);
    const View<Q> w = {q, Mx, My, ox, oy};
    if constexpr (!MC) {
        return sample_range(w, x - dt * vx, y - dt * vy, nullptr, nullptr);
    } else {
        float lo, hi;
        const float qf = sample_range(w, x - dt * vx, y - dt * vy, &lo, &hi);
        const Forward<Q> fwd = {q, fu, fv, Mx, My, ox, oy, dt};
        const View<Forward<Q>> wf = {fwd, Mx, My, ox, oy};
        const float qb = sample_range(wf, x + dt * vx, y + dt * vy, nullptr, nullptr);
        return fminf(fmaxf(qf + 0.5f * (q.at(i, j) - qb), lo), hi);
    }
}

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
template <bool MC>
__device__ __forceinline__ float rho_new_at(const Rho& r, const Field& fu, const Field& fv,
                                            float dt, int i, int j)
{
    if constexpr (!MC) {
        const float x = i + 0.5f, y = j + 0.5f;
        float vx, vy;
        vel_at_sample(fu, fv, 0.5f, 0.5f, i, j, vx, vy);
        return sample_rho(r, x - dt * vx, y - dt * vy);
    } else {
        return advected<true>(r, r.nx, r.ny, 0.5f, 0.5f, fu, fv, dt, i, j);
    }
}

// Tiles of the fused step: a CTA produces the outputs of kAdvTX x adv_ty(MC)
// indices (i, j) of [0, nx] x [0, ny] (cell (i, j) density, u face (j, i),
// v face (j, i)): 16 rows for MacCormack, whose windows (below) then cost
// 1.48 forward values per output, 32 for the first-order scheme, which has
// none.  MacCormack's backward sample reads the forward field at
// four corners within kAdvH samples of its own index whenever the
// displacement dt |vel| is below kAdvH cells; the CTA evaluates the forward
// field of each quantity once on its tile widened by kAdvH (and one row more
// above, for the density of the row above the tile that the buoyancy of the
// tile's top v faces reads) and keeps it in shared memory.  A corner outside
// that window (a faster flow) is evaluated where it is needed, with the same
// arithmetic, so the result does not depend on the window.
constexpr int kAdvTX = 32, kAdvH = 2, kAdvThreads = 256;
__host__ __device__ constexpr int adv_ty(bool mc) { return mc ? 16 : 32; }
constexpr int kFW = kAdvTX + 2 * kAdvH;          // columns of a forward-field window
constexpr int kFH = adv_ty(true) + 2 * kAdvH + 1;  // rows: tile rows - 1 - kAdvH .. + kAdvH

// Forward field of quantity Q on its window (sample (ci, cj) at entry 0),
// evaluated where it is not in the window.
template <class Q>
struct WindowedForward {
    Forward<Q> f;
    const float* s;
    int ci, cj;
    __device__ float at(int i, int j) const
    {
        const int a = i - ci, b = j - cj;
        if (a >= 0 && a < kFW && b >= 0 && b < kFH) return s[b * kFW + a];
        return f.at(i, j);
    }
};

// Fills the window of quantity q (Mx x My samples at (ox, oy)) with the
// forward values and the velocities at the samples: the samples of the field
// only (entries outside it are never read: every corner of a bilinear sample
// lies in the field, and so does every output sample).
template <class Q>
__device__ __forceinline__ void fill_window(float* s, float* svx, float* svy, const Forward<Q>& f,
                                            int ci, int cj)
{
    for (int t = threadIdx.x; t < kFH * kFW; t += kAdvThreads) {
        const int b = t / kFW, a = t - b * kFW;
        const int i = ci + a, j = cj + b;
        if (i >= 0 && i < f.Mx && j >= 0 && j < f.My) {
            float vx, vy;
            s[t] = f.at_vel(i, j, vx, vy);
            svx[t] = vx;
            svy[t] = vy;
        }
    }
}

// New value of sample (i, j) of quantity q: as advected<MC>, MacCormack's
// backward sample and the velocity at (i, j) taken from the window.
template <bool MC, class Q>
__device__ __forceinline__ float advected_w(const Q& q, int Mx, int My, float ox, float oy,
                                            const Field& fu, const Field& fv, float dt,
                                            const float* win, const float* wvx,
                                            const float* wvy, int ci, int cj, int i, int j)
{
    if constexpr (!MC) {
        return advected<false>(q, Mx, My, ox, oy, fu, fv, dt, i, j);
    } else {
        const float x = (float)i + ox, y = (float)j + oy;
        const int t = (j - cj) * kFW + (i - ci);
        const float vx = wvx[t], vy = wvy[t];
        const View<Q> w = {q, Mx, My, ox, oy};
        float lo, hi;
        const float qf = sample_range(w, x - dt * vx, y - dt * vy, &lo, &hi);
        const WindowedForward<Q> fwd = {{q, fu, fv, Mx, My, ox, oy, dt}, win, ci, cj};
        const View<WindowedForward<Q>> wf = {fwd, Mx, My, ox, oy};
        const float qb = sample_range(wf, x + dt * vx, y + dt * vy, nullptr, nullptr);
        return fminf(fmaxf(qf + 0.5f * (q.at(i, j) - qb), lo), hi);
    }
}

// One CTA per tile: (MacCormack) the three forward-field windows; the new
// density of the tile's rows and the row above, kept in shared memory for
// the buoyancy; then the u and v faces.
template <bool MC>
__global__ void __launch_bounds__(kAdvThreads) advect_kernel(
    const float* __restrict__ u, const float* __restrict__ v, const float* __restrict__ rho,
    const uint8_t* __restrict__ flags, float* __restrict__ u_out, float* __restrict__ v_out,
    float* __restrict__ rho_out, int ny, int nx, hp_plume_params p)
{
    // forward rho, u, v and the velocity at their samples
    __shared__ float s_win[MC ? 3 : 1][MC ? kFH * kFW : 1];
    __shared__ float s_vx[MC ? 3 : 1][MC ? kFH * kFW : 1];
    __shared__ float s_vy[MC ? 3 : 1][MC ? kFH * kFW : 1];
    constexpr int kAdvTY = adv_ty(MC);
    __shared__ float s_rho[(kAdvTY + 1) * kAdvTX];  // new rho, rows j0 - 1 ..
    const int i0 = blockIdx.x * kAdvTX, j0 = blockIdx.y * kAdvTY, b = blockIdx.z;
    const size_t cells = (size_t)ny * nx;
    const Field fu = {u + (size_t)b * ny * (nx + 1), nx + 1, ny, 0.0f, 0.5f};
    const Field fv = {v + (size_t)b * (ny + 1) * nx, nx, ny + 1, 0.5f, 0.0f};
    const Rho r = {rho + b * cells, nx, ny, p.inlet_x0, p.inlet_x1, p.rho_in};
    const uint8_t* fl = flags + b * cells;
    const float dt = p.dt;
    const int ci = i0 - kAdvH, cj = j0 - 1 - kAdvH;  // sample at entry 0 of a window

    if constexpr (MC) {
        fill_window(s_win[0], s_vx[0], s_vy[0], Forward<Rho>{r, fu, fv, nx, ny, 0.5f, 0.5f, dt},
                    ci, cj);
        fill_window(s_win[1], s_vx[1], s_vy[1],
                    Forward<Field>{fu, fu, fv, nx + 1, ny, 0.0f, 0.5f, dt}, ci, cj);
        fill_window(s_win[2], s_vx[2], s_vy[2],
                    Forward<Field>{fv, fu, fv, nx, ny + 1, 0.5f, 0.0f, dt}, ci, cj);
        __syncthreads();
    }
    constexpr int kU = MC ? 1 : 0, kV = MC ? 2 : 0;

    for (int t = threadIdx.x; t < (kAdvTY + 1) * kAdvTX; t += kAdvThreads) {
        const int rr = t / kAdvTX, c = t - rr * kAdvTX;
        const int i = i0 + c, j = j0 - 1 + rr;
        if (i < nx && j >= 0 && j < ny) {
            float val;
            if constexpr (MC)
                val = advected_w<true>(r, nx, ny, 0.5f, 0.5f, fu, fv, dt, s_win[0], s_vx[0],
                                       s_vy[0], ci, cj, i, j);
            else
                val = rho_new_at<false>(r, fu, fv, dt, i, j);
            s_rho[t] = val;
            if (rr > 0) rho_out[b * cells + (size_t)j * nx + i] = val;
        }
    }
    __syncthreads();

    for (int t = threadIdx.x; t < kAdvTY * kAdvTX; t += kAdvThreads) {
        const int rr = t / kAdvTX, c = t - rr * kAdvTX;
        const int i = i0 + c, j = j0 + rr;
        if (i > nx || j > ny) continue;
        if (j < ny) {
            const bool open = i > 0 && i < nx && fluid(fl, nx, i - 1, j) && fluid(fl, nx, i, j);
            float val = 0.0f;
            if (open)
                val = advected_w<MC>(fu, nx + 1, ny, 0.0f, 0.5f, fu, fv, dt, s_win[kU], s_vx[kU],
                                     s_vy[kU], ci, cj, i, j);
            u_out[(size_t)b * ny * (nx + 1) + (size_t)j * (nx + 1) + i] = val;
        }
        if (i < nx) {
            const bool interior = j > 0 && j < ny && fluid(fl, nx, i, j - 1) && fluid(fl, nx, i, j);
            // an open top keeps (advects) its faces; buoyancy acts on interior faces
            const bool top = j == 0 && p.open_top && fluid(fl, nx, i, 0);
            float val = 0.0f;
            if (interior || top)
                val = advected_w<MC>(fv, nx, ny + 1, 0.5f, 0.0f, fu, fv, dt, s_win[kV], s_vx[kV],
                                     s_vy[kV], ci, cj, i, j);
            if (interior) {
                // new density of cells (i, j - 1) and (i, j): rows rr and rr + 1
                const float rf = 0.5f * (s_rho[rr * kAdvTX + c] + s_rho[(rr + 1) * kAdvTX + c]);
                val += dt * p.gravity * (rf - p.rho_amb);
            }
            // injection through the inlet faces of the bottom boundary (upwards)
            if (j == ny && i >= p.inlet_x0 && i < p.inlet_x1 && fluid(fl, nx, i, ny - 1))
                val = -p.u_in;
            v_out[(size_t)b * (ny + 1) * nx + (size_t)j * nx + i] = val;
        }
    }
}

__global__ void plume_head_init_kernel(int32_t* __restrict__ out, int B, int ny, int nx)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    out[3 * b + 0] = ny;
    out[3 * b + 1] = nx;
    out[3 * b + 2] = -1;
}

// Smallest row, smallest and largest column of the cells whose density
// contrast reaches the threshold: CTA (slice, grid) reduces its slice of
// rows and merges with atomicMin / atomicMax (integers: order independent).
__global__ void __launch_bounds__(512) plume_head_kernel(const float* __restrict__ rho, int ny,
                                                         int nx, float rho_amb, float contrast,
                                                         int32_t* __restrict__ out)
{
    __shared__ int s_min_row[16], s_min_col[16], s_max_col[16];
    const int b = blockIdx.y;
    const int r0 = (int)((long)ny * blockIdx.x / gridDim.x);
    const int r1 = (int)((long)ny * (blockIdx.x + 1) / gridDim.x);
    const float* r = rho + (size_t)b * ny * nx;
    int min_row = ny, min_col = nx, max_col = -1;
    for (long c = (long)r0 * nx + threadIdx.x; c < (long)r1 * nx; c += blockDim.x) {
        if (fabsf(r[c] - rho_amb) >= contrast) {
            const int j = (int)(c / nx), i = (int)(c - (long)j * nx);
            min_row = min(min_row, j);
            min_col = min(min_col, i);
            max_col = max(max_col, i);
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        min_row = min(min_row, __shfl_down_sync(0xffffffffu, min_row, off));
        min_col = min(min_col, __shfl_down_sync(0xffffffffu, min_col, off));
        max_col = max(max_col, __shfl_down_sync(0xffffffffu, max_col, off));
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        s_min_row[warp] = min_row;
        s_min_col[warp] = min_col;
        s_max_col[warp] = max_col;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            min_row = min(min_row, s_min_row[w]);
            min_col = min(min_col, s_min_col[w]);
            max_col = max(max_col, s_max_col[w]);
        }
        if (max_col >= 0) {
            atomicMin(&out[3 * b + 0], min_row);
            atomicMin(&out[3 * b + 1], min_col);
            atomicMax(&out[3 * b + 2], max_col);
        }
    }
}

}  // namespace

hp_status launch_advect(const float* u, const float* v, const float* rho, const uint8_t* flags,
                        float* u_out, float* v_out, float* rho_out, hp_shape s,
                        const hp_plume_params& p, cudaStream_t st)
{
    const int ty = adv_ty(p.scheme == 1);
    dim3 blk(kAdvThreads), grd((s.nx + 1 + kAdvTX - 1) / kAdvTX, (s.ny + ty) / ty, s.batch);
    if (p.scheme == 1)
        advect_kernel<true><<<grd, blk, 0, st>>>(u, v, rho, flags, u_out, v_out, rho_out, s.ny,
                                                 s.nx, p);
    else
        advect_kernel<false><<<grd, blk, 0, st>>>(u, v, rho, flags, u_out, v_out, rho_out, s.ny,
                                                  s.nx, p);
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
    if (p->scheme != 0 && p->scheme != 1) return HP_ERR_INVALID_ARG;
    if ((p->open_top != 0 && p->open_top != 1) || !isfinite(p->u_in)) return HP_ERR_INVALID_ARG;
    return hp::launch_advect(u, v, rho, flags, u_out, v_out, rho_out, s, *p, (cudaStream_t)stream);
}

extern "C" hp_status hp_plume_head(const float* rho, hp_shape s, float rho_amb, float contrast,
                                   int32_t* out, void* stream)
{
    if (!rho || !out || !hp::shape_ok(s) || !(contrast >= 0.0f)) return HP_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    hp::plume_head_init_kernel<<<(s.batch + 127) / 128, 128, 0, st>>>(out, s.batch, s.ny, s.nx);
    // about 16 rows per CTA, at most 64 CTAs per grid
    const int slices = s.ny < 16 ? 1 : (s.ny / 16 < 64 ? s.ny / 16 : 64);
    hp::plume_head_kernel<<<dim3(slices, s.batch), 512, 0, st>>>(rho, s.ny, s.nx, rho_amb,
                                                                  contrast, out);
    return hp::check_launch();
}
