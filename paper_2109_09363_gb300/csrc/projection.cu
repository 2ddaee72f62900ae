// Pressure-projection kernels for sm_103a: face mask + divergence, temporally
// blocked masked Jacobi sweeps with a fused per-sweep E_1 reduction and an
// exact stop rule, correction, divergence norms.
//
// Method (arXiv 2109.09363): corrected velocity u = u* - (dt/rho0) grad p
// (Eq. 2); Poisson equation (dt/rho0) lap p = div u* (Eq. 3); Jacobi iteration
// X_{t+1} = D^{-1}(b - (L+U) X_t) (Sec. 2.2); stop when E_1 = mean |div u| is
// at or below the user threshold (Sec. 3.3 and 4.1).
//
// The sweep is written in increment form on phi = (dt/rho0) p:
//   r_c    = div_c - sum_open (phi_nb - phi_c)      (residual of phi_k)
//   phi'_c = phi_c - r_c / n_c                      (= Jacobi update)
// Solid cells and cells outside the grid hold phi = 0, so the sum over the four
// neighbours only has to remove the closed faces: with c = 4 - n_c,
//   sum_open (phi_nb - phi_c) = sum_all4 (phi_nb - phi_c) + c * phi_c.
// Differences of neighbouring values are formed first, which keeps the FP32
// residual accurate to the size of the pressure gradient rather than of the
// pressure itself.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>

#include "hproj_internal.cuh"

namespace hp {

// --------------------------------------------------------- mask + divergence

// One thread per cell.  mask (optional) receives the open-face bits, div
// (optional) the forward-difference divergence over open faces (Eq. 3); with
// an open top the top faces of fluid cells of row 0 are open, and the
// prescribed inflow faces of the bottom boundary enter the divergence.
__global__ void mask_div_kernel(const float* __restrict__ u, const float* __restrict__ v,
                                const uint8_t* __restrict__ flags, uint8_t* __restrict__ mask,
                                float* __restrict__ div, int ny, int nx, Boundary bc)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    const int b = blockIdx.z;
    if (i >= nx) return;
    const uint8_t* fl = flags + (size_t)b * ny * nx;
    const size_t c = (size_t)j * nx + i;
    uint32_t m = 0;
    if (fl[c] == 0) {
        if (i > 0 && fl[c - 1] == 0) m |= 1u;
        if (i < nx - 1 && fl[c + 1] == 0) m |= 2u;
        if (j > 0 ? fl[c - nx] == 0 : bc.open_top != 0) m |= 4u;
        if (j < ny - 1 && fl[c + nx] == 0) m |= 8u;
    }
    if (mask) mask[(size_t)b * ny * nx + c] = (uint8_t)m;
    if (div) {
        const float* ub = u + (size_t)b * ny * (nx + 1) + (size_t)j * (nx + 1);
        const float* vb = v + (size_t)b * (ny + 1) * nx;
        const float ue = (m & 2u) ? ub[i + 1] : 0.0f;
        const float uw = (m & 1u) ? ub[i] : 0.0f;
        const bool inflow = j == ny - 1 && i >= bc.x0 && i < bc.x1 && fl[c] == 0;
        const float vs = ((m & 8u) || inflow) ? vb[(size_t)(j + 1) * nx + i] : 0.0f;
        const float vn = (m & 4u) ? vb[(size_t)j * nx + i] : 0.0f;
        div[(size_t)b * ny * nx + c] = __fadd_rn(__fsub_rn(ue, uw), __fsub_rn(vs, vn));
    }
}

// ------------------------------------- vector paths (rows a multiple of 4)
//
// The same values as the one-cell kernels, with vector loads and stores of
// four consecutive cells of a row: flags as one 32-bit word per row (the bytes
// of the cells left and right of the four come from the adjacent lanes when
// they hold them), v and div, p, phi as float4 (16-byte aligned rows), u
// (rows of nx + 1) as scalars with the fifth face from the next lane.  The
// mask/divergence, correction and norm kernels walk column strips (a quad
// column of a few rows per thread), so each thread loads every byte it needs
// once; every lane of a warp takes part in the shuffles, lanes past the end do
// no memory access.

__device__ __forceinline__ uint32_t ld_u32(const uint8_t* p)
{
    return *reinterpret_cast<const uint32_t*>(p);
}

__device__ __forceinline__ uint32_t byte_of(uint32_t w, int q) { return (w >> (8 * q)) & 0xffu; }

__device__ __forceinline__ float face_div(uint32_t m, bool inflow, float uw, float ue, float vn,
                                          float vs)
{
    const float e = (m & 2u) ? ue : 0.0f;
    const float w = (m & 1u) ? uw : 0.0f;
    const float s = ((m & 8u) || inflow) ? vs : 0.0f;
    const float n = (m & 4u) ? vn : 0.0f;
    return __fadd_rn(__fsub_rn(e, w), __fsub_rn(s, n));
}

// Vector paths of the mask and divergence: blocks of kQuadThreads threads, a
// quad column per thread.
constexpr int kQuadThreads = 128;

// mask_div_kernel over quads of cells in column strips (rows a multiple of 4
// cells, 16-byte aligned v, flags, mask and div): grid (row quads /
// kQuadThreads, blocks of kDivRows rows, B); each thread walks down kDivRows
// rows of its quad column, keeping the flags of the row above and of its own
// row and the v faces north of the row in registers from the row before, so
// it loads each byte it needs once (one flag word, one float4 of v and the
// row's u faces per row); rows in pairs, both rows' loads issued before either
// is used (four rows at a time measured no faster, with 80 registers).  The
// open-face bits of four cells come from byte-wise comparisons of the flag
// words with their neighbours' words shifted by one byte; the flags left and
// right of the quad from the neighbouring lanes when they hold them.  (One
// quad per thread and row, reading the shared rows again through L2, took
// 167 us for the divergence of 16 x 2048^2; the strips 152 us.)
constexpr int kDivRows = 8;

__global__ void __launch_bounds__(kQuadThreads)
    mask_div_col_kernel(const float* __restrict__ u, const float* __restrict__ v,
                        const uint8_t* __restrict__ flags, uint8_t* __restrict__ mask,
                        float* __restrict__ div, int ny, int nx, Boundary bc)
{
    constexpr uint32_t kSolid = 0x01010101u;
    const int i0 = 4 * (blockIdx.x * kQuadThreads + threadIdx.x);
    const int rb = blockIdx.y, b = blockIdx.z, lane = threadIdx.x & 31;
    const bool act = i0 < nx;
    // the neighbouring quads of the row sit in the neighbouring lanes
    const bool from_left = lane > 0 && i0 > 0;
    const bool from_right = lane < 31 && i0 + 4 < nx;
    const int j0 = rb * kDivRows;
    const int j1 = min(ny, j0 + kDivRows);  // the same for the whole block
    const size_t gb = (size_t)b * ny * nx;
    const uint8_t* fl = flags + gb;
    const float* ug = div ? u + (size_t)b * ny * (nx + 1) : nullptr;
    const float* vg = div ? v + (size_t)b * (ny + 1) * nx : nullptr;
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    uint32_t fu = !act ? kSolid
                  : j0 > 0 ? ld_u32(fl + (size_t)(j0 - 1) * nx + i0)
                  : bc.open_top ? 0u : kSolid;
    uint32_t fc = act ? ld_u32(fl + (size_t)j0 * nx + i0) : kSolid;
    float4 vn = (div && act) ? *reinterpret_cast<const float4*>(vg + (size_t)j0 * nx + i0) : z;
    struct RowIn {
        float4 vs;
        float uf[4], ue;
        uint32_t fd, lb, rbt;
    };
    auto load_row = [&](int j, RowIn& in) {
        const size_t row = (size_t)j * nx;
        in.fd = (act && j < ny - 1) ? ld_u32(fl + row + nx + i0) : kSolid;
        in.lb = (!from_left && act && i0 > 0) ? (uint32_t)fl[row + i0 - 1] : 1u;
        in.rbt = (!from_right && act && i0 + 4 < nx) ? (uint32_t)fl[row + i0 + 4] : 1u;
        if (div) {
            const float* ub = ug + (size_t)j * (nx + 1);
            in.vs = act ? *reinterpret_cast<const float4*>(vg + row + nx + i0) : z;
#pragma unroll
            for (int q = 0; q < 4; ++q) in.uf[q] = act ? ub[i0 + q] : 0.0f;
            in.ue = (act && !from_right) ? ub[i0 + 4] : 0.0f;
        }
    };
    auto row_out = [&](int j, const RowIn& in) {
        const uint32_t sl = __shfl_up_sync(0xffffffffu, fc, 1);
        const uint32_t sr = __shfl_down_sync(0xffffffffu, fc, 1);
        const uint32_t left = from_left ? byte_of(sl, 3) : in.lb;
        const uint32_t right = from_right ? byte_of(sr, 0) : in.rbt;
        const uint32_t west = (fc << 8) | left;
        const uint32_t east = (fc >> 8) | (right << 24);
        const uint32_t open = (__vcmpeq4(west, 0u) & 0x01010101u) |
                              (__vcmpeq4(east, 0u) & 0x02020202u) |
                              (__vcmpeq4(fu, 0u) & 0x04040404u) |
                              (__vcmpeq4(in.fd, 0u) & 0x08080808u);
        const uint32_t mw = __vcmpeq4(fc, 0u) & open;
        float uf4 = 0.0f;
        if (div) {
            const float ush = __shfl_down_sync(0xffffffffu, in.uf[0], 1);
            uf4 = (act && !from_right) ? in.ue : ush;
        }
        if (act) {
            const size_t c = gb + (size_t)j * nx + i0;
            if (mask) *reinterpret_cast<uint32_t*>(mask + c) = mw;
            if (div) {
                const float ufq[5] = {in.uf[0], in.uf[1], in.uf[2], in.uf[3], uf4};
                const float vnq[4] = {vn.x, vn.y, vn.z, vn.w};
                const float vsq[4] = {in.vs.x, in.vs.y, in.vs.z, in.vs.w};
                float d[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int i = i0 + q;
                    const bool inflow = j == ny - 1 && i >= bc.x0 && i < bc.x1 && byte_of(fc, q) == 0;
                    d[q] = face_div(byte_of(mw, q), inflow, ufq[q], ufq[q + 1], vnq[q], vsq[q]);
                }
                *reinterpret_cast<float4*>(div + c) = make_float4(d[0], d[1], d[2], d[3]);
            }
        }
        fu = fc;
        fc = in.fd;
        if (div) vn = in.vs;
    };
#pragma unroll
    for (int r = 0; r < kDivRows; r += 2) {
        const int j = j0 + r;
        if (j >= j1) break;
        const bool two = j + 1 < j1;
        RowIn in0, in1;
        load_row(j, in0);
        if (two) load_row(j + 1, in1);
        row_out(j, in0);
        if (two) row_out(j + 1, in1);
    }
}

// The face mask alone over column strips of sixteen cells (rows a multiple
// of 16 cells, 16-byte aligned flags and mask): grid (row sixteens /
// kMask16Threads, blocks of kDivRows rows, B); each thread walks down its
// column keeping the flag words of the row above and of its own row from the
// row before, one 16-byte load (the row below) and one 16-byte store per row,
// rows in pairs; the bytes left and right of the sixteen from the
// neighbouring lanes.  The same bits as mask_div_col_kernel.  (A sixteen per
// thread and row, the three flag rows loaded each time: 0.0395 ms for
// 16 x 2048^2; a quad per thread: 0.078 ms.)
constexpr int kMask16Threads = 128;

__global__ void __launch_bounds__(kMask16Threads)
    mask16_col_kernel(const uint8_t* __restrict__ flags, uint8_t* __restrict__ mask, int ny,
                      int nx, int open_top)
{
    constexpr uint32_t kSolid = 0x01010101u;
    const int i0 = 16 * (blockIdx.x * kMask16Threads + threadIdx.x);
    const int rb = blockIdx.y, b = blockIdx.z, lane = threadIdx.x & 31;
    const bool act = i0 < nx;
    const bool from_left = lane > 0 && i0 > 0;
    const bool from_right = lane < 31 && i0 + 16 < nx;
    const int j0 = rb * kDivRows;
    const int j1 = min(ny, j0 + kDivRows);  // the same for the whole block
    const uint8_t* fl = flags + (size_t)b * ny * nx;
    uint8_t* mk = mask + (size_t)b * ny * nx;
    const uint4 solid = make_uint4(kSolid, kSolid, kSolid, kSolid);
    uint4 fu = !act ? solid
               : j0 > 0 ? *reinterpret_cast<const uint4*>(fl + (size_t)(j0 - 1) * nx + i0)
               : open_top ? make_uint4(0u, 0u, 0u, 0u) : solid;
    uint4 fc = act ? *reinterpret_cast<const uint4*>(fl + (size_t)j0 * nx + i0) : solid;
    struct RowIn {
        uint4 fd;
        uint32_t lb, rbt;
    };
    auto load_row = [&](int j, RowIn& in) {
        const size_t row = (size_t)j * nx;
        in.fd = (act && j < ny - 1) ? *reinterpret_cast<const uint4*>(fl + row + nx + i0) : solid;
        in.lb = (!from_left && act && i0 > 0) ? (uint32_t)fl[row + i0 - 1] : 1u;
        in.rbt = (!from_right && act && i0 + 16 < nx) ? (uint32_t)fl[row + i0 + 16] : 1u;
    };
    auto row_out = [&](int j, const RowIn& in) {
        const uint32_t c[4] = {fc.x, fc.y, fc.z, fc.w};
        const uint32_t up[4] = {fu.x, fu.y, fu.z, fu.w};
        const uint32_t dn[4] = {in.fd.x, in.fd.y, in.fd.z, in.fd.w};
        const uint32_t sl = __shfl_up_sync(0xffffffffu, c[3], 1);
        const uint32_t sr = __shfl_down_sync(0xffffffffu, c[0], 1);
        const uint32_t left = from_left ? byte_of(sl, 3) : in.lb;
        const uint32_t right = from_right ? byte_of(sr, 0) : in.rbt;
        uint32_t mw[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const uint32_t west = (c[h] << 8) | (h == 0 ? left : c[h - 1] >> 24);
            const uint32_t east = (c[h] >> 8) | ((h == 3 ? right : c[h + 1] & 0xffu) << 24);
            const uint32_t open = (__vcmpeq4(west, 0u) & 0x01010101u) |
                                  (__vcmpeq4(east, 0u) & 0x02020202u) |
                                  (__vcmpeq4(up[h], 0u) & 0x04040404u) |
                                  (__vcmpeq4(dn[h], 0u) & 0x08080808u);
            mw[h] = __vcmpeq4(c[h], 0u) & open;
        }
        if (act)
            *reinterpret_cast<uint4*>(mk + (size_t)j * nx + i0) =
                make_uint4(mw[0], mw[1], mw[2], mw[3]);
        fu = fc;
        fc = in.fd;
    };
#pragma unroll
    for (int r = 0; r < kDivRows; r += 2) {
        const int j = j0 + r;
        if (j >= j1) break;
        const bool two = j + 1 < j1;
        RowIn in0, in1;
        load_row(j, in0);
        if (two) load_row(j + 1, in1);
        row_out(j, in0);
        if (two) row_out(j + 1, in1);
    }
}

static bool aligned16(const void* p) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

hp_status launch_mask_div(const float* u, const float* v, const uint8_t* flags, uint8_t* mask,
                          float* div, hp_shape s, cudaStream_t st, Boundary bc)
{
    if (!div && mask && s.nx % 16 == 0 && aligned16(flags) && aligned16(mask)) {
        dim3 grd((s.nx / 16 + kMask16Threads - 1) / kMask16Threads, (s.ny + kDivRows - 1) / kDivRows,
                 s.batch);
        mask16_col_kernel<<<grd, kMask16Threads, 0, st>>>(flags, mask, s.ny, s.nx, bc.open_top);
        return check_launch();
    }
    if (s.nx % 4 == 0 && aligned16(flags) && aligned16(mask) && aligned16(div) &&
        (!div || aligned16(v))) {
        dim3 grd((s.nx / 4 + kQuadThreads - 1) / kQuadThreads, (s.ny + kDivRows - 1) / kDivRows,
                 s.batch);
        mask_div_col_kernel<<<grd, kQuadThreads, 0, st>>>(u, v, flags, mask, div, s.ny, s.nx, bc);
        return check_launch();
    }
    dim3 blk(256), grd((s.nx + 255) / 256, s.ny, s.batch);
    mask_div_kernel<<<grd, blk, 0, st>>>(u, v, flags, mask, div, s.ny, s.nx, bc);
    return check_launch();
}

hp_status launch_mask(const uint8_t* flags, uint8_t* mask, hp_shape s, cudaStream_t st)
{
    return launch_mask_div(nullptr, nullptr, flags, mask, nullptr, s, st);
}

// ------------------------------------------------------------- state reset

__global__ void reset_state_kernel(GridState* gs, LoopState* ls, int B)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) {
        GridState g = {};
        g.active = 1;
        gs[b] = g;
    }
    if (b == 0) {
        LoopState l = {};
        l.any_active = 1;
        l.n_active = B;
        *ls = l;
    }
}

// phi_0 = given guess on cells with an open face, else 0.
__global__ void init_phi_kernel(const float* __restrict__ phi0, const uint8_t* __restrict__ mask,
                                float* __restrict__ out, size_t cells)
{
    const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= cells) return;
    out[q] = (phi0 && (mask[q] & 15u)) ? phi0[q] : 0.0f;
}

// One more masked Jacobi sweep of phi (the same cell update as every sweep
// kernel, so phi' is bit-identical to theirs) and the mean of phi and phi'
// (the target of the training pairs: the mean cancels the period-2
// component that plain Jacobi never damps).
__global__ void mean_sweep_kernel(const float* __restrict__ phi, const float* __restrict__ div,
                                  const uint8_t* __restrict__ mask, float* __restrict__ out,
                                  int ny, int nx)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    const size_t gb = (size_t)blockIdx.z * ny * nx;
    if (i >= nx) return;
    const size_t c = gb + (size_t)j * nx + i;
    const float* ph = phi + gb;
    const float pc = phi[c];
    const float pw = i > 0 ? ph[(size_t)j * nx + i - 1] : 0.0f;
    const float pe = i < nx - 1 ? ph[(size_t)j * nx + i + 1] : 0.0f;
    const float pn = j > 0 ? ph[(size_t)(j - 1) * nx + i] : 0.0f;
    const float ps = j < ny - 1 ? ph[(size_t)(j + 1) * nx + i] : 0.0f;
    float res;
    const float nxt = cell_update(pc, pw, pe, pn, ps, make_const(div[c], mask[c]), res);
    out[c] = __fmul_rn(0.5f, __fadd_rn(pc, nxt));
}

hp_status launch_mean_sweep(const float* phi, const float* div, const uint8_t* mask, float* out,
                            hp_shape s, cudaStream_t st)
{
    dim3 blk(256), grd((s.nx + 255) / 256, s.ny, s.batch);
    mean_sweep_kernel<<<grd, blk, 0, st>>>(phi, div, mask, out, s.ny, s.nx);
    return check_launch();
}

// ----------------------------------------------------- blocked Jacobi sweeps

template <int H>
struct TileGeom {
    static constexpr int OW = kTileCols - 2 * H;  // owned columns per tile
    static constexpr int OH = kTileRows - 2 * H;  // owned rows per tile
};

int ctas_x(int nx, int H) { return (nx + (kTileCols - 2 * H) - 1) / (kTileCols - 2 * H); }
int ctas_y(int ny, int H) { return (ny + (kTileRows - 2 * H) - 1) / (kTileRows - 2 * H); }
int halo_for(int T) { return T <= 4 ? 4 : 8; }
int ctas_per_grid(int ny, int nx, int T)
{
    const int H = halo_for(T);
    return ctas_x(nx, H) * ctas_y(ny, H);
}

// Lane-ordered FP64 sum of n partials p[lane], p[lane + 32], ... (the same
// order as one add per iteration), eight loads in flight at a time; L2 reads
// (the partials were just written by other CTAs).
__device__ __forceinline__ double lane_sum(const double* p, int n, int lane)
{
    double s = 0.0;
    int i = lane;
    for (; i + 7 * 32 < n; i += 8 * 32) {
        double t[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) t[k] = __ldcg(p + i + 32 * k);
#pragma unroll
        for (int k = 0; k < 8; ++k) s += t[k];
    }
    for (; i < n; i += 32) s += __ldcg(p + i);
    return s;
}

// Called by the last CTA of grid b after all its CTAs wrote their per-sweep
// partial sums: E_k for the sweeps of this launch, stop decision.
__device__ void grid_decide(const SweepArgs& a, int b, int T, int k0, int src, int nct)
{
    __shared__ double s_e[kMaxBlock];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const double inv_cells = 1.0 / ((double)a.nx * (double)a.ny);
    if (wid < T) {
        const double* p = a.partial + ((size_t)b * kMaxBlock + wid) * nct;
        double s = lane_sum(p, nct, lane);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if (lane == 0) s_e[wid] = s * inv_cells;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        GridState* g = a.gs + b;
        int stop = -1, conv = 0;
        for (int t = 0; t < T; ++t) {
            const int k = k0 + t;
            const double e = s_e[t];
            if (a.e_hist && k < a.hist_len) a.e_hist[(size_t)b * a.hist_len + k] = e;
            if (e <= a.threshold) { stop = t; conv = 1; break; }
            // a non-finite E (NaN or Inf in the input) ends the grid at once
            if (k >= a.max_iters || !isfinite(e)) { stop = t; conv = 0; break; }
        }
        if (stop >= 0) {
            g->active = 0;
            g->kstar = k0 + stop;
            g->k0_stop = k0;
            g->replay = stop;
            g->src = src;
            g->final_buf = stop > 0 ? (src ^ 1) : src;
            g->converged = conv;
            g->e_stop = s_e[stop];
        }
        g->arrivals = 0u;
        __threadfence();
    }
}

// Called by the last CTA of the whole launch: advance the block counter and
// decide whether another block is needed.  The loop is bounded: once k0 is
// past max_iters + kMaxBlock nothing can still be active, and the flag is
// cleared regardless.
__device__ void launch_finish(const SweepArgs& a, int T)
{
    int any = 0;
    for (int b = threadIdx.x; b < a.B; b += blockDim.x) any |= __ldcg(&a.gs[b].active);
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) {
        LoopState* ls = a.ls;
        const int k0n = ls->k0 + T;
        if (k0n > a.max_iters + kMaxBlock) any = 0;
        ls->k0 = k0n;
        ls->blk = ls->blk + 1;
        ls->arrivals = 0u;
        ls->any_active = any;
        __threadfence();
        if (a.cond) cudaGraphSetConditional((cudaGraphConditionalHandle)a.cond, any ? 1u : 0u);
    }
}

__device__ __forceinline__ void launch_arrive(const SweepArgs& a, int T)
{
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t total = gridDim.x * gridDim.y * gridDim.z;
        s_last = atomicAdd(&a.ls->arrivals, 1u) == total - 1u;
        if (s_last) __threadfence();
    }
    __syncthreads();
    if (s_last) launch_finish(a, T);
}

// Temporally blocked sweep kernel.  Each CTA owns an (OH x OW) block of cells
// and loads it with a halo of H cells into registers: thread (warp w, lane l)
// holds rows 4w..4w+3 and columns 4l..4l+3 of the 64 x 128 tile.  Horizontal
// neighbours come from warp shuffles, vertical neighbours across warps from a
// double-buffered shared-memory row exchange (one barrier per sweep).  After T
// sweeps (T <= H) the owned cells are exact; the halo cells are discarded.
//
// mode 0 (loop block): sweeps k0..k0+T-1 of every active grid, per-sweep
//   residual partial sums, stop decision by the last CTA of each grid, block
//   counter advance by the last CTA of the launch.
// mode 1 (replay): gs[b].replay sweeps from buffer gs[b].src into the other
//   buffer, no reduction.
template <int H, int R>
__global__ void __launch_bounds__((kTileRows / R) * 32, 1) sweep_tb_kernel(SweepArgs a)
{
    constexpr int NW = kTileRows / R;  // warps; warp w holds rows R*w .. R*w + R - 1
    constexpr int OW = TileGeom<H>::OW;
    constexpr int OH = TileGeom<H>::OH;
    static_assert(H % R == 0, "halo must hold whole thread rows");
    // row exchange [parity][top/bottom][warp][lane], dynamic shared memory
    extern __shared__ float4 s_xchg[];
    __shared__ float s_wsum[kMaxBlock][NW];

    const int b = blockIdx.z;
    GridState* g = a.gs + b;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;

    int T, src, k0 = 0;
    if (a.mode == 0) {
        if (!g->active) {
            launch_arrive(a, a.T);
            return;
        }
        T = a.T;
        k0 = a.ls->k0;
        src = a.ls->blk & 1;
    } else {
        T = g->replay;
        src = g->src;
        if (T <= 0) return;
    }
    const int nx = a.nx, ny = a.ny;
    const size_t gbase = (size_t)b * ny * nx;
    const float* __restrict__ pin = (src ? a.phi1 : a.phi0) + gbase;
    float* __restrict__ pout = (src ? a.phi0 : a.phi1) + gbase;
    const float* __restrict__ dv = a.div + gbase;
    const uint8_t* __restrict__ mk = a.mask + gbase;
    const bool vec = (nx & 3) == 0;

    const int x0 = blockIdx.x * OW - H + 4 * lane;
    const int y0 = blockIdx.y * OH - H + R * wid;

    float phi[R][4];
    CellConst kc[R][4];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int y = y0 + r;
        if (y >= 0 && y < ny) {
            float dd[4];
            load_row4(pin + (size_t)y * nx, x0, nx, vec, phi[r]);
            load_row4(dv + (size_t)y * nx, x0, nx, vec, dd);
            const uint32_t m4 = load_mask4(mk + (size_t)y * nx, x0, nx, vec);
#pragma unroll
            for (int q = 0; q < 4; ++q) kc[r][q] = make_const(dd[q], (m4 >> (8 * q)) & 0xffu);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                phi[r][q] = 0.0f;
                kc[r][q] = make_const(0.0f, 0u);
            }
        }
    }

    const bool own = lane >= H / 4 && lane < 32 - H / 4 && wid >= H / R && wid < NW - H / R;

    for (int t = 0; t < T; ++t) {
        const int p = t & 1;
        float4* top = s_xchg + (p * 2 + 0) * NW * 32;
        float4* bot = s_xchg + (p * 2 + 1) * NW * 32;
        top[wid * 32 + lane] = make_float4(phi[0][0], phi[0][1], phi[0][2], phi[0][3]);
        bot[wid * 32 + lane] = make_float4(phi[R - 1][0], phi[R - 1][1], phi[R - 1][2], phi[R - 1][3]);
        __syncthreads();
        const float4 nb = wid > 0 ? bot[(wid - 1) * 32 + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 sb =
            wid < NW - 1 ? top[(wid + 1) * 32 + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float north[4] = {nb.x, nb.y, nb.z, nb.w};
        const float south[4] = {sb.x, sb.y, sb.z, sb.w};
        // each difference between two cells is formed once and negated for
        // the other cell (exact), as in the grid-resident kernel
        float dn[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) dn[q] = __fsub_rn(north[q], phi[0][q]);
        float acc = 0.0f;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float left = __shfl_up_sync(0xffffffffu, phi[r][3], 1);
            const float right = __shfl_down_sync(0xffffffffu, phi[r][0], 1);
            float ex[5];
            ex[0] = __fsub_rn(phi[r][0], left);
#pragma unroll
            for (int q = 0; q < 3; ++q) ex[q + 1] = __fsub_rn(phi[r][q + 1], phi[r][q]);
            ex[4] = __fsub_rn(right, phi[r][3]);
            float nw[4], ds[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float ps = r < R - 1 ? phi[r + 1][q] : south[q];
                ds[q] = __fsub_rn(ps, phi[r][q]);
                float res;
                nw[q] = cell_update_diff(phi[r][q], -ex[q], ex[q + 1], dn[q], ds[q], kc[r][q], res);
                acc = __fadd_rn(acc, fabsf(res));
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                dn[q] = -ds[q];
                phi[r][q] = nw[q];
            }
        }
        if (a.mode == 0) {
            if (!own) acc = 0.0f;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1)
                acc = __fadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, off));
            if (lane == 0) s_wsum[t][wid] = acc;
        }
    }

    if (own) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int y = y0 + r;
            if (y < ny) {
                float* row = pout + (size_t)y * nx;
                if (vec && x0 + 3 < nx) {
                    *reinterpret_cast<float4*>(row + x0) =
                        make_float4(phi[r][0], phi[r][1], phi[r][2], phi[r][3]);
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (x0 + q < nx) row[x0 + q] = phi[r][q];
                }
            }
        }
    }
    if (a.mode != 0) return;

    __syncthreads();
    const int nct = gridDim.x * gridDim.y;
    const int cta = blockIdx.y * gridDim.x + blockIdx.x;
    if (threadIdx.x < T) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < NW; ++w) s += (double)s_wsum[threadIdx.x][w];
        a.partial[((size_t)b * kMaxBlock + threadIdx.x) * nct + cta] = s;
        __threadfence();
    }
    __shared__ int s_last_grid;
    __syncthreads();
    if (threadIdx.x == 0) {
        s_last_grid = atomicAdd(&g->arrivals, 1u) == (uint32_t)nct - 1u;
        if (s_last_grid) __threadfence();
    }
    __syncthreads();
    if (s_last_grid) grid_decide(a, b, T, k0, src, nct);
    launch_arrive(a, T);
}

// ------------------------------------------------ streaming single sweep

// Rows and columns of one block of the streaming kernel: one warp per row,
// four consecutive cells per lane.
constexpr int kS1Rows = 16;
constexpr int kS1Cols = 128;

int s1_blocks_x(int nx) { return (nx + kS1Cols - 1) / kS1Cols; }
int s1_blocks_y(int ny) { return (ny + kS1Rows - 1) / kS1Rows; }

// E of sweep k-1 of grid b from the CTA partials (fixed order, one warp).
__device__ __forceinline__ double s1_grid_e(const SweepArgs& a, int b, int kprev, int nct)
{
    const int lane = threadIdx.x & 31;
    const double* p = a.partial + ((size_t)b * 2 + (kprev & 1)) * nct;
    double sum = lane_sum(p, nct, lane);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, off);
    return __shfl_sync(0xffffffffu, sum, 0) / ((double)a.nx * (double)a.ny);
}

__device__ __forceinline__ bool s1_stops(const SweepArgs& a, double e, int kprev)
{
    return e <= a.threshold || kprev >= a.max_iters || !isfinite(e);
}

// One Jacobi sweep per launch, no atomics on the data path.  Launch k (sweep
// phi_k -> phi_{k+1} of every active grid) first decides the stop test of
// E_{k-1}: every CTA of a grid sums the CTA partials of sweep k-1 in the same
// fixed order and gets the same answer, so a grid that stopped leaves
// phi_{k-1} untouched in its buffer; otherwise it sweeps and writes its
// partial of E_k.  k per grid is the CTA arrival count of the grid divided by
// its CTAs.  The extra control CTA (blockIdx.z == B) keeps the launch counter,
// decides for all grids whether another launch is needed and sets the
// CUDA-graph conditional.
__global__ void __launch_bounds__(kS1Rows * 32) sweep1_kernel(SweepArgs a)
{
    __shared__ float s_w[kS1Rows];
    __shared__ int s_k, s_stop;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nct = gridDim.x * gridDim.y;
    const int b = blockIdx.z;

    if (b == a.B) {  // control CTA
        if (blockIdx.x != 0 || blockIdx.y != 0) return;
        LoopState* ls = a.ls;
        const int k = ls->k0;
        int any = 0;
        if (k == 0) {
            any = 1;
        } else if (wid == 0) {
            for (int bb = 0; bb < a.B; ++bb) {
                if (!__ldcg(&a.gs[bb].active)) continue;
                const double e = s1_grid_e(a, bb, k - 1, nct);
                if (!s1_stops(a, e, k - 1)) any = 1;
            }
        }
        any = __syncthreads_or(any);
        if (threadIdx.x == 0) {
            if (k > a.max_iters + 2) any = 0;
            ls->k0 = k + 1;
            ls->any_active = any;
            if (a.cond) cudaGraphSetConditional((cudaGraphConditionalHandle)a.cond, any ? 1u : 0u);
        }
        return;
    }

    GridState* g = a.gs + b;
    if (!g->active) return;
    const int cta = blockIdx.y * gridDim.x + blockIdx.x;
    if (threadIdx.x == 0) s_k = (int)(atomicAdd(&g->arrivals, 1u) / (uint32_t)nct);
    __syncthreads();
    const int k = s_k;
    if (wid == 0) {
        int stop = 0;
        if (k > 0) {
            const double e = s1_grid_e(a, b, k - 1, nct);
            stop = s1_stops(a, e, k - 1);
            if (lane == 0 && cta == 0) {
                if (a.e_hist && k - 1 < a.hist_len) a.e_hist[(size_t)b * a.hist_len + k - 1] = e;
                if (stop) {
                    g->kstar = k - 1;
                    g->k0_stop = k - 1;
                    g->replay = 0;
                    g->src = (k - 1) & 1;
                    g->final_buf = (k - 1) & 1;
                    g->converged = e <= a.threshold;
                    g->e_stop = e;
                    g->active = 0;
                }
            }
        }
        if (lane == 0) s_stop = stop;
    }
    __syncthreads();
    if (s_stop) return;

    const int src = k & 1;
    const int nx = a.nx, ny = a.ny;
    const size_t gbase = (size_t)b * ny * nx;
    const float* __restrict__ pin = (src ? a.phi1 : a.phi0) + gbase;
    float* __restrict__ pout = (src ? a.phi0 : a.phi1) + gbase;
    const bool vec = (nx & 3) == 0;
    const int x0 = blockIdx.x * kS1Cols + 4 * lane;
    const int y = blockIdx.y * kS1Rows + wid;
    float acc = 0.0f;
    if (y < ny) {
        float c[4], up[4] = {0.f, 0.f, 0.f, 0.f}, dn[4] = {0.f, 0.f, 0.f, 0.f}, dd[4];
        const float* row = pin + (size_t)y * nx;
        load_row4(row, x0, nx, vec, c);
        if (y > 0) load_row4(row - nx, x0, nx, vec, up);
        if (y < ny - 1) load_row4(row + nx, x0, nx, vec, dn);
        load_row4(a.div + gbase + (size_t)y * nx, x0, nx, vec, dd);
        const uint32_t m4 = load_mask4(a.mask + gbase + (size_t)y * nx, x0, nx, vec);
        float left = __shfl_up_sync(0xffffffffu, c[3], 1);
        float right = __shfl_down_sync(0xffffffffu, c[0], 1);
        if (lane == 0) left = (x0 > 0 && x0 - 1 < nx) ? row[x0 - 1] : 0.0f;
        if (lane == 31) right = (x0 + 4 < nx) ? row[x0 + 4] : 0.0f;
        float nv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float pw = q > 0 ? c[q - 1] : left;
            const float pe = q < 3 ? c[q + 1] : right;
            float res;
            nv[q] = cell_update(c[q], pw, pe, up[q], dn[q],
                                make_const(dd[q], (m4 >> (8 * q)) & 0xffu), res);
            acc = __fadd_rn(acc, fabsf(res));
        }
        float* orow = pout + (size_t)y * nx;
        if (vec && x0 + 3 < nx) {
            *reinterpret_cast<float4*>(orow + x0) = make_float4(nv[0], nv[1], nv[2], nv[3]);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (x0 + q < nx) orow[x0 + q] = nv[q];
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc = __fadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, off));
    if (lane == 0) s_w[wid] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0.0;
#pragma unroll
        for (int w = 0; w < kS1Rows; ++w) sum += (double)s_w[w];
        a.partial[((size_t)b * 2 + (k & 1)) * nct + cta] = sum;
    }
}

// ----------------------------------------------------- correction (Eq. 2)

// One thread per cell: corrects its west (u[j][i]) and north (v[j][i]) faces,
// zeroes the closed domain faces u[j][nx] and v[ny][i], writes p = phi*scale.
// u = u* - grad phi on open faces, 0 on closed faces (Eq. 2); with an open
// top its faces take the exterior value phi = 0, and prescribed inflow faces
// keep their velocity.
__global__ void correct_kernel(float* __restrict__ u, float* __restrict__ v,
                               const uint8_t* __restrict__ mask,
                               const uint8_t* __restrict__ flags, const float* __restrict__ phi0,
                               const float* __restrict__ phi1, const GridState* __restrict__ gs,
                               float* __restrict__ p_out, float* __restrict__ phi_out,
                               float scale, int ny, int nx, Boundary bc)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    const int b = blockIdx.z;
    if (i >= nx) return;
    const size_t gb = (size_t)b * ny * nx;
    const float* ph = (gs[b].final_buf ? phi1 : phi0) + gb;
    const size_t c = (size_t)j * nx + i;
    const uint32_t m = mask[gb + c];
    const float pc = ph[c];
    if (u) {
        float* ub = u + (size_t)b * ny * (nx + 1) + (size_t)j * (nx + 1);
        float* vb = v + (size_t)b * (ny + 1) * nx;
        float uw = 0.0f, vn = 0.0f;
        if (m & 1u) uw = __fsub_rn(ub[i], __fsub_rn(pc, ph[c - 1]));
        if (m & 4u)
            vn = __fsub_rn(vb[(size_t)j * nx + i], __fsub_rn(pc, j > 0 ? ph[c - nx] : 0.0f));
        ub[i] = uw;
        vb[(size_t)j * nx + i] = vn;
        if (i == nx - 1) ub[nx] = 0.0f;
        if (j == ny - 1 &&
            !(i >= bc.x0 && i < bc.x1 && flags[(size_t)b * ny * nx + c] == 0))
            vb[(size_t)ny * nx + i] = 0.0f;
    }
    if (p_out) p_out[gb + c] = __fmul_rn(pc, scale);
    if (phi_out) phi_out[gb + c] = pc;
}

// correct_kernel over quads of cells in column strips (rows a multiple of 4
// cells, 16-byte aligned v, flags, p and phi copy): grid (row quads /
// kQuadThreads, blocks of kDivRows rows, B); each thread walks down kDivRows
// rows of its quad column and keeps phi of the row above (its cells' north
// neighbours) in registers from the row before instead of reading it again
// through L2; phi west of the quad from the previous lane; rows in pairs,
// both rows' loads issued before either is used.  (A grid-stride kernel over
// single quads took 335 us for 16 x 2048^2.)
__global__ void __launch_bounds__(kQuadThreads)
    correct_col_kernel(float* __restrict__ u, float* __restrict__ v,
                       const uint8_t* __restrict__ mask, const uint8_t* __restrict__ flags,
                       const float* __restrict__ phi0, const float* __restrict__ phi1,
                       const GridState* __restrict__ gs, float* __restrict__ p_out,
                       float* __restrict__ phi_out, float scale, int ny, int nx, Boundary bc)
{
    const int i0 = 4 * (blockIdx.x * kQuadThreads + threadIdx.x);
    const int rb = blockIdx.y, b = blockIdx.z, lane = threadIdx.x & 31;
    const bool act = i0 < nx;
    // phi west of cell i0: the previous lane's last cell in the same row
    const bool from_left = lane > 0 && i0 > 0;
    const int j0 = rb * kDivRows;
    const int j1 = min(ny, j0 + kDivRows);  // the same for the whole block
    const size_t gb = (size_t)b * ny * nx;
    const float* ph = (gs[b].final_buf ? phi1 : phi0) + gb;
    float* ug = u ? u + (size_t)b * ny * (nx + 1) : nullptr;
    float* vg = u ? v + (size_t)b * (ny + 1) * nx : nullptr;
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    // phi north of row j0 (the exterior above row 0 reads as 0)
    float4 pn = (act && j0 > 0) ? *reinterpret_cast<const float4*>(ph + (size_t)(j0 - 1) * nx + i0) : z;
    struct RowIn {
        float4 p4, vn4;
        float pwm, uw[4];
        uint32_t m4;
    };
    auto load_row = [&](int j, RowIn& in) {
        const size_t c = (size_t)j * nx + i0;
        in.p4 = act ? *reinterpret_cast<const float4*>(ph + c) : z;
        in.pwm = (!from_left && act && i0 > 0) ? ph[c - 1] : 0.0f;
        if (u) {
            in.m4 = act ? ld_u32(mask + gb + c) : 0u;
            in.vn4 = act ? *reinterpret_cast<const float4*>(vg + c) : z;
            const float* ub = ug + (size_t)j * (nx + 1);
#pragma unroll
            for (int q = 0; q < 4; ++q) in.uw[q] = act ? ub[i0 + q] : 0.0f;
        }
    };
    auto row_out = [&](int j, const RowIn& in) {
        const float sh = __shfl_up_sync(0xffffffffu, in.p4.w, 1);
        const float pw = from_left ? sh : in.pwm;
        if (act) {
            const size_t c = (size_t)j * nx + i0;
            const float pc[4] = {in.p4.x, in.p4.y, in.p4.z, in.p4.w};
            if (u) {
                const float pu[4] = {pn.x, pn.y, pn.z, pn.w};
                const float vn[4] = {in.vn4.x, in.vn4.y, in.vn4.z, in.vn4.w};
                float* ub = ug + (size_t)j * (nx + 1);
                float uo[4], vo[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t m = byte_of(in.m4, q);
                    const float west = q == 0 ? pw : pc[q - 1];
                    uo[q] = (m & 1u) ? __fsub_rn(in.uw[q], __fsub_rn(pc[q], west)) : 0.0f;
                    vo[q] = (m & 4u) ? __fsub_rn(vn[q], __fsub_rn(pc[q], pu[q])) : 0.0f;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) ub[i0 + q] = uo[q];
                *reinterpret_cast<float4*>(vg + c) = make_float4(vo[0], vo[1], vo[2], vo[3]);
                if (i0 + 4 == nx) ub[nx] = 0.0f;
                if (j == ny - 1) {
                    const uint32_t f4 = ld_u32(flags + gb + c);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int i = i0 + q;
                        if (!(i >= bc.x0 && i < bc.x1 && byte_of(f4, q) == 0))
                            vg[(size_t)ny * nx + i] = 0.0f;
                    }
                }
            }
            if (p_out)
                *reinterpret_cast<float4*>(p_out + gb + c) =
                    make_float4(__fmul_rn(pc[0], scale), __fmul_rn(pc[1], scale),
                                __fmul_rn(pc[2], scale), __fmul_rn(pc[3], scale));
            if (phi_out) *reinterpret_cast<float4*>(phi_out + gb + c) = in.p4;
        }
        pn = in.p4;
    };
#pragma unroll
    for (int r = 0; r < kDivRows; r += 2) {
        const int j = j0 + r;
        if (j >= j1) break;
        const bool two = j + 1 < j1;
        RowIn in0, in1;
        load_row(j, in0);
        if (two) load_row(j + 1, in1);
        row_out(j, in0);
        if (two) row_out(j + 1, in1);
    }
}

// --------------------------------------------------------- divergence norms
//
// E_1 = mean |div u| and E_inf = max |div u| (Sec. 4.1) of a velocity: one
// 8-byte partial per 256-cell segment of a row (one cell per thread) or of a
// block of kNormRows rows (column strips), in (grid, row or row block,
// segment) order, holding the FP32 sum and max of |div| (float2), then per
// grid the FP64 sum of the sums in a fixed order and the max of the maxima.
// No atomics: every partial has one writer, and E_1 is the same on every call.

// One thread per cell, a block per segment: |div u| over open faces, FP32
// sums per warp and of the warps in order.  (flags is always given; mask may
// be null, the closed box's open faces are then taken from the flags)
__global__ void div_norms_kernel(const float* __restrict__ u, const float* __restrict__ v,
                                 const uint8_t* __restrict__ flags,
                                 const uint8_t* __restrict__ mask, float2* __restrict__ partial,
                                 int ny, int nx, Boundary bc)
{
    __shared__ float s_w[8], s_m[8];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    const int b = blockIdx.z;
    float a = 0.0f;
    if (i < nx) {
        const size_t c = (size_t)j * nx + i;
        uint32_t m;
        if (mask) {
            m = mask[(size_t)b * ny * nx + c];
        } else {
            const uint8_t* fl = flags + (size_t)b * ny * nx;
            m = 0;
            if (fl[c] == 0) {
                if (i > 0 && fl[c - 1] == 0) m |= 1u;
                if (i < nx - 1 && fl[c + 1] == 0) m |= 2u;
                if (j > 0 && fl[c - nx] == 0) m |= 4u;
                if (j < ny - 1 && fl[c + nx] == 0) m |= 8u;
            }
        }
        const float* ub = u + (size_t)b * ny * (nx + 1) + (size_t)j * (nx + 1);
        const float* vb = v + (size_t)b * (ny + 1) * nx;
        const float ue = (m & 2u) ? ub[i + 1] : 0.0f;
        const float uw = (m & 1u) ? ub[i] : 0.0f;
        const bool inflow =
            j == ny - 1 && i >= bc.x0 && i < bc.x1 && flags[(size_t)b * ny * nx + c] == 0;
        const float vs = ((m & 8u) || inflow) ? vb[(size_t)(j + 1) * nx + i] : 0.0f;
        const float vn = (m & 4u) ? vb[(size_t)j * nx + i] : 0.0f;
        a = fabsf(__fadd_rn(__fsub_rn(ue, uw), __fsub_rn(vs, vn)));
    }
    float mx = a;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        a = __fadd_rn(a, __shfl_xor_sync(0xffffffffu, a, off));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        s_w[wid] = a;
        s_m[wid] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float sum = 0.0f, m = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            sum = __fadd_rn(sum, s_w[w]);
            m = fmaxf(m, s_m[w]);
        }
        partial[(size_t)b * gridDim.x * gridDim.y + (size_t)j * gridDim.x + blockIdx.x] =
            make_float2(sum, m);
    }
}

// The partials over column strips (rows a multiple of 4 cells, 16-byte
// aligned v, flags and mask): grid (segment pairs, blocks of kNormRows rows,
// B); a block of 4 warps takes two consecutive 256-cell segments of
// kNormRows rows, warp 2 s + h the quads at 128 h + 4 lane of its segment s,
// and each thread walks down its quad column.  The flags of the row above and
// of its own row and the v faces north of the row stay in registers from the
// row before, so a thread loads each byte it needs once (one flag word, one
// float4 of v and the row's u faces per row) instead of reading the shared
// rows again through L2.  Partial (row block, segment): the FP32 sums of the
// thread's rows in order, over the warp's lanes, of the segment's two warps.
constexpr int kSegCells = 256;
constexpr int kNormThreads = 128;
constexpr int kNormRows = 8;

template <bool MASK>
__global__ void __launch_bounds__(kNormThreads)
    div_norms_col_kernel(const float* __restrict__ u, const float* __restrict__ v,
                         const uint8_t* __restrict__ flags, const uint8_t* __restrict__ mask,
                         float2* __restrict__ partial, int ny, int nx, int nseg, int nrb,
                         Boundary bc)
{
    constexpr uint32_t kSolid = 0x01010101u;
    __shared__ float s_w[4], s_m[4];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int rb = blockIdx.y, b = blockIdx.z;
    const int sx = 2 * blockIdx.x + (wid >> 1);
    const int i0 = sx * kSegCells + 128 * (wid & 1) + 4 * lane;
    const bool act = i0 < nx;
    // the neighbouring quads of the half segment sit in the neighbouring lanes
    const bool from_left = lane > 0;
    const bool from_right = lane < 31 && i0 + 4 < nx;
    const int j0 = rb * kNormRows;
    const int j1 = min(ny, j0 + kNormRows);  // the same for the whole block
    const size_t gb = (size_t)b * ny * nx;
    const uint8_t* fl = flags + gb;
    const float* ug = u + (size_t)b * ny * (nx + 1);
    const float* vg = v + (size_t)b * (ny + 1) * nx;
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    // flags of the row above j0 and of row j0 (closed box: no open top)
    uint32_t fu = kSolid, fc = kSolid;
    if (!MASK && act) {
        if (j0 > 0) fu = ld_u32(fl + (size_t)(j0 - 1) * nx + i0);
        fc = ld_u32(fl + (size_t)j0 * nx + i0);
    }
    float4 vn = act ? *reinterpret_cast<const float4*>(vg + (size_t)j0 * nx + i0) : z;
    float a = 0.0f, mx = 0.0f;
    // one row's loads: the v faces south of it, its u faces, its open-face
    // bits (mask) or the flags of the row below and the bytes beside the quad
    struct RowIn {
        float4 vs;
        float uf[4], ue;
        uint32_t w, fcw, lb, rbt;
    };
    auto load_row = [&](int j, RowIn& in) {
        const size_t row = (size_t)j * nx;
        const float* ub = ug + (size_t)j * (nx + 1);
        in.vs = act ? *reinterpret_cast<const float4*>(vg + row + nx + i0) : z;
#pragma unroll
        for (int q = 0; q < 4; ++q) in.uf[q] = act ? ub[i0 + q] : 0.0f;
        in.ue = (act && !from_right) ? ub[i0 + 4] : 0.0f;
        if (MASK) {
            in.w = act ? ld_u32(mask + gb + row + i0) : 0u;
            in.fcw = (act && j == ny - 1) ? ld_u32(fl + row + i0) : kSolid;
        } else {
            in.w = (act && j < ny - 1) ? ld_u32(fl + row + nx + i0) : kSolid;
            in.lb = (!from_left && act && i0 > 0) ? (uint32_t)fl[row + i0 - 1] : 1u;
            in.rbt = (!from_right && act && i0 + 4 < nx) ? (uint32_t)fl[row + i0 + 4] : 1u;
        }
    };
    // |div| of the row from its loads and the carried state (every lane of
    // the warp takes part in the shuffles)
    auto row_div = [&](int j, const RowIn& in) {
        uint32_t m4, fcw;
        if (MASK) {
            m4 = in.w;
            fcw = in.fcw;
        } else {
            // open-face bits of the four cells (as mask_div_col_kernel)
            const uint32_t fd = in.w;
            const uint32_t sl = __shfl_up_sync(0xffffffffu, fc, 1);
            const uint32_t sr = __shfl_down_sync(0xffffffffu, fc, 1);
            const uint32_t left = from_left ? byte_of(sl, 3) : in.lb;
            const uint32_t right = from_right ? byte_of(sr, 0) : in.rbt;
            const uint32_t west = (fc << 8) | left;
            const uint32_t east = (fc >> 8) | (right << 24);
            const uint32_t open = (__vcmpeq4(west, 0u) & 0x01010101u) |
                                  (__vcmpeq4(east, 0u) & 0x02020202u) |
                                  (__vcmpeq4(fu, 0u) & 0x04040404u) |
                                  (__vcmpeq4(fd, 0u) & 0x08080808u);
            m4 = __vcmpeq4(fc, 0u) & open;
            fcw = fc;
            fu = fc;
            fc = fd;
        }
        const float ush = __shfl_down_sync(0xffffffffu, in.uf[0], 1);
        const float uf4 = (act && !from_right) ? in.ue : ush;
        if (act) {
            const float ufq[5] = {in.uf[0], in.uf[1], in.uf[2], in.uf[3], uf4};
            const float vnq[4] = {vn.x, vn.y, vn.z, vn.w};
            const float vsq[4] = {in.vs.x, in.vs.y, in.vs.z, in.vs.w};
            float d[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = i0 + q;
                const bool inflow = j == ny - 1 && i >= bc.x0 && i < bc.x1 && byte_of(fcw, q) == 0;
                d[q] = fabsf(face_div(byte_of(m4, q), inflow, ufq[q], ufq[q + 1], vnq[q], vsq[q]));
                mx = fmaxf(mx, d[q]);
            }
            a = __fadd_rn(a, __fadd_rn(__fadd_rn(d[0], d[1]), __fadd_rn(d[2], d[3])));
        }
        vn = in.vs;
    };
    // rows in pairs: both rows' loads are issued before either is used (four
    // rows' loads in flight measured slower: 0.136 against 0.132 ms for the
    // norms of 16 x 2048^2, 76 registers)
#pragma unroll
    for (int r = 0; r < kNormRows; r += 2) {
        const int j = j0 + r;
        if (j >= j1) break;
        const bool two = j + 1 < j1;
        RowIn in0, in1;
        load_row(j, in0);
        if (two) load_row(j + 1, in1);
        row_div(j, in0);
        if (two) row_div(j + 1, in1);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        a = __fadd_rn(a, __shfl_xor_sync(0xffffffffu, a, off));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    }
    if (lane == 0) {
        s_w[wid] = a;
        s_m[wid] = mx;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        const int sq = 2 * blockIdx.x + threadIdx.x;
        if (sq < nseg)
            partial[((size_t)b * nrb + rb) * nseg + sq] =
                make_float2(__fadd_rn(s_w[2 * threadIdx.x], s_w[2 * threadIdx.x + 1]),
                            fmaxf(s_m[2 * threadIdx.x], s_m[2 * threadIdx.x + 1]));
    }
}

// The norms kernel for one shape: the column-strip kernel where rows allow
// vector access, else one cell per thread; returns the partials per grid.
static int norms_kernel(const float* u, const float* v, const uint8_t* flags,
                        const uint8_t* mask, float2* partial, hp_shape s, Boundary bc,
                        cudaStream_t st)
{
    const int nseg = (s.nx + kSegCells - 1) / kSegCells;
    if (s.nx % 4 == 0 && aligned16(v) && aligned16(flags) && aligned16(mask)) {
        const int nrb = (s.ny + kNormRows - 1) / kNormRows;
        dim3 grd((nseg + 1) / 2, nrb, s.batch);
        if (mask)
            div_norms_col_kernel<true><<<grd, kNormThreads, 0, st>>>(u, v, flags, mask, partial,
                                                                     s.ny, s.nx, nseg, nrb, bc);
        else
            div_norms_col_kernel<false><<<grd, kNormThreads, 0, st>>>(u, v, flags, mask, partial,
                                                                      s.ny, s.nx, nseg, nrb, bc);
        return nrb * nseg;
    }
    dim3 grd(nseg, s.ny, s.batch);
    div_norms_kernel<<<grd, kSegCells, 0, st>>>(u, v, flags, mask, partial, s.ny, s.nx, bc);
    return s.ny * nseg;
}

// One block of kFinishWarps warps per grid: warp w adds its contiguous share
// of the grid's partial sums (lane order, FP64) and takes their max, then
// thread 0 the warps' results in order; a fixed order, so E_1 is the same on
// every call.
constexpr int kFinishWarps = 8;

__global__ void norms_finish_kernel(const float2* __restrict__ partial, int nblk, double* e1,
                                    double* einf, const GridState* gs, int32_t* iters,
                                    uint8_t* conv, int B, double inv_cells)
{
    __shared__ double s_w[kFinishWarps];
    __shared__ float s_m[kFinishWarps];
    const int b = blockIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int share = (nblk + kFinishWarps - 1) / kFinishWarps;
    const int q0 = wid * share, q1 = min(nblk, q0 + share);
    const float2* p = partial + (size_t)b * nblk;
    double s = 0.0;
    float m = 0.0f;
    int i = q0 + lane;
    for (; i + 7 * 32 < q1; i += 8 * 32) {
        float2 t[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) t[k] = __ldcg(p + i + 32 * k);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            s += (double)t[k].x;
            m = fmaxf(m, t[k].y);
        }
    }
    for (; i < q1; i += 32) {
        const float2 t = __ldcg(p + i);
        s += (double)t.x;
        m = fmaxf(m, t.y);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, off);
        m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, off));
    }
    if (lane == 0) {
        s_w[wid] = s;
        s_m[wid] = m;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        s = 0.0;
        m = 0.0f;
        for (int w = 0; w < kFinishWarps; ++w) {
            s += s_w[w];
            m = fmaxf(m, s_m[w]);
        }
        if (e1) e1[b] = s * inv_cells;
        if (einf) einf[b] = (double)m;
        if (gs) {
            if (iters) iters[b] = gs[b].kstar;
            if (conv) conv[b] = (uint8_t)gs[b].converged;
        }
    }
}

hp_status launch_div_norms(const float* u, const float* v, const uint8_t* flags, double* partial,
                           int nblk_cap, double* e1, double* einf, hp_shape s, cudaStream_t st)
{
    if (((s.nx + kSegCells - 1) / kSegCells) * s.ny > nblk_cap) return HP_ERR_INVALID_ARG;
    return launch_div_norms_scratch(u, v, flags, partial, e1, einf, s, st);
}

// Same reduction as launch_div_norms with caller-given scratch: partial
// holds >= batch * ny * ceil(nx / 256) slots of 8 bytes (the column-strip
// kernel uses fewer).
hp_status launch_div_norms_scratch(const float* u, const float* v, const uint8_t* flags,
                                   double* partial, double* e1, double* einf, hp_shape s,
                                   cudaStream_t st)
{
    float2* p2 = reinterpret_cast<float2*>(partial);
    const int nblk = norms_kernel(u, v, flags, nullptr, p2, s, Boundary{}, st);
    hp_status rc = check_launch();
    if (rc != HP_OK) return rc;
    norms_finish_kernel<<<s.batch, kFinishWarps * 32, 0, st>>>(
        p2, nblk, e1, einf, nullptr, nullptr, nullptr, s.batch, 1.0 / ((double)s.nx * (double)s.ny));
    return check_launch();
}

// ------------------------------------------------------------- sweep loop

// rows per thread of the blocked kernel: 4 (16 warps) or 2 (32 warps)
static void* sweep_kernel_ptr(int H, int R)
{
    if (R == 2) return H == 4 ? (void*)sweep_tb_kernel<4, 2> : (void*)sweep_tb_kernel<8, 2>;
    return H == 4 ? (void*)sweep_tb_kernel<4, 4> : (void*)sweep_tb_kernel<8, 4>;
}

static int sweep_threads(int R) { return (kTileRows / R) * 32; }
static size_t sweep_smem(int R) { return (size_t)4 * (kTileRows / R) * 32 * sizeof(float4); }

static hp_status prepare_sweep_kernel(int H, int R)
{
    static bool done[2][2] = {{false, false}, {false, false}};
    bool& d = done[H == 8][R == 2];
    if (d) return HP_OK;
    cudaError_t e = cudaFuncSetAttribute(sweep_kernel_ptr(H, R),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sweep_smem(R));
    if (e != cudaSuccess) { set_cuda_error(e); return HP_ERR_CUDA; }
    d = true;
    return HP_OK;
}

static hp_status launch_sweep(const SweepArgs& a, int H, int R, cudaStream_t st)
{
    hp_status rc = prepare_sweep_kernel(H, R);
    if (rc != HP_OK) return rc;
    dim3 grd(ctas_x(a.nx, H), ctas_y(a.ny, H), a.B), blk(sweep_threads(R));
    const size_t sm = sweep_smem(R);
    if (R == 2) {
        if (H == 4) sweep_tb_kernel<4, 2><<<grd, blk, sm, st>>>(a);
        else sweep_tb_kernel<8, 2><<<grd, blk, sm, st>>>(a);
    } else {
        if (H == 4) sweep_tb_kernel<4, 4><<<grd, blk, sm, st>>>(a);
        else sweep_tb_kernel<8, 4><<<grd, blk, sm, st>>>(a);
    }
    return check_launch();
}

// Sweep launches per iteration of the graph loop with the streaming kernel
// (grids that stopped skip the remaining launches of the iteration).
constexpr int kStreamUnroll = 8;

static hp_status build_loop_graph(hp_ctx* ctx, SweepArgs a, int H, int R, bool stream)
{
    if (!stream) {
        hp_status prc = prepare_sweep_kernel(H, R);
        if (prc != HP_OK) return prc;
    }
    if (ctx->graph_exec) {
        cudaGraphExecDestroy(ctx->graph_exec);
        ctx->graph_exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaGraphCreate(&graph, 0);
    if (e != cudaSuccess) { set_cuda_error(e); return HP_ERR_CUDA; }
    cudaGraphConditionalHandle handle;
    e = cudaGraphConditionalHandleCreate(&handle, graph, 1u, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) {
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = handle;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t cnode;
        e = cudaGraphAddNode(&cnode, graph, nullptr, nullptr, 0, &cp);
        if (e == cudaSuccess) {
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            a.cond = (unsigned long long)handle;
            void* args[] = {&a};
            cudaKernelNodeParams kp = {};
            if (stream) {
                kp.func = (void*)sweep1_kernel;
                kp.gridDim = dim3(s1_blocks_x(a.nx), s1_blocks_y(a.ny), a.B + 1);
                kp.blockDim = dim3(kS1Rows * 32);
                kp.sharedMemBytes = 0;
            } else {
                kp.func = sweep_kernel_ptr(H, R);
                kp.gridDim = dim3(ctas_x(a.nx, H), ctas_y(a.ny, H), a.B);
                kp.blockDim = dim3(sweep_threads(R));
                kp.sharedMemBytes = (unsigned)sweep_smem(R);
            }
            kp.kernelParams = args;
            cudaGraphNode_t prev = nullptr, knode = nullptr;
            const int nodes = stream ? kStreamUnroll : 1;
            for (int i = 0; i < nodes && e == cudaSuccess; ++i) {
                e = cudaGraphAddKernelNode(&knode, body, prev ? &prev : nullptr, prev ? 1 : 0, &kp);
                prev = knode;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&ctx->graph_exec, graph, 0);
        }
    }
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        ctx->graph_exec = nullptr;
        set_cuda_error(e);
        return HP_ERR_CUDA;
    }
    return HP_OK;
}

// Runs blocks of T sweeps until every grid has stopped, then replays each grid
// to its exact stop index.  Expects ctx->mask, ctx->div and ctx->phi[0] ready.
static hp_status launch_sweep1(const SweepArgs& a, cudaStream_t st)
{
    dim3 grd(s1_blocks_x(a.nx), s1_blocks_y(a.ny), a.B + 1), blk(kS1Rows * 32);
    sweep1_kernel<<<grd, blk, 0, st>>>(a);
    return check_launch();
}

static hp_status run_sweep_loop(hp_ctx* ctx, hp_shape s, int T, int R, bool stream,
                                double threshold, int max_iters, double* e_hist, int hist_len,
                                bool use_graph, cudaStream_t st)
{
    const int H = halo_for(T);
    const int nct = ctas_x(s.nx, H) * ctas_y(s.ny, H);
    if ((size_t)s.batch * kMaxBlock * nct > ctx->partial_len) return HP_ERR_INVALID_ARG;
    if ((size_t)s.batch * 2 * s1_blocks_x(s.nx) * s1_blocks_y(s.ny) > ctx->partial_len)
        return HP_ERR_INVALID_ARG;
    SweepArgs a = {};
    a.phi0 = ctx->phi[0];
    a.phi1 = ctx->phi[1];
    a.div = ctx->div;
    a.mask = ctx->mask;
    a.gs = ctx->gs;
    a.ls = ctx->ls;
    a.partial = ctx->partial;
    a.e_hist = e_hist;
    a.hist_len = hist_len;
    a.B = s.batch;
    a.ny = s.ny;
    a.nx = s.nx;
    a.T = T;
    a.max_iters = max_iters;
    a.threshold = threshold;
    a.mode = 0;
    a.cond = 0;

    reset_state_kernel<<<(s.batch + 255) / 256, 256, 0, st>>>(ctx->gs, ctx->ls, s.batch);
    hp_status rc = check_launch();
    if (rc != HP_OK) return rc;

    if (use_graph) {
        const bool same = ctx->graph_exec && ctx->graph_shape.batch == s.batch &&
                          ctx->graph_shape.ny == s.ny && ctx->graph_shape.nx == s.nx &&
                          ctx->graph_T == T && ctx->graph_hist == hist_len &&
                          ctx->graph_hist_ptr == e_hist && ctx->graph_threshold == threshold &&
                          ctx->graph_max_iters == max_iters &&
                          ctx->graph_kernel == (stream ? 1 : 10 + R);
        if (!same) {
            rc = build_loop_graph(ctx, a, H, R, stream);
            if (rc != HP_OK) return rc;
            ctx->graph_kernel = stream ? 1 : 10 + R;
            ctx->graph_shape = s;
            ctx->graph_T = T;
            ctx->graph_hist = hist_len;
            ctx->graph_hist_ptr = e_hist;
            ctx->graph_threshold = threshold;
            ctx->graph_max_iters = max_iters;
        }
        cudaError_t e = cudaGraphLaunch(ctx->graph_exec, st);
        if (e != cudaSuccess) { set_cuda_error(e); return HP_ERR_CUDA; }
    } else {
        // host-polled: launch a few blocks, read the flag, repeat; bounded by
        // the cap (every grid stops at k = max_iters at the latest)
        const int max_blocks = stream ? max_iters + 3 : max_iters / T + 2;
        int launched = 0;
        const int chunk = stream ? kStreamUnroll : 4;
        while (launched < max_blocks) {
            for (int c = 0; c < chunk && launched < max_blocks; ++c, ++launched) {
                rc = stream ? launch_sweep1(a, st) : launch_sweep(a, H, R, st);
                if (rc != HP_OK) return rc;
            }
            cudaError_t e = cudaMemcpyAsync(ctx->host_flag, &ctx->ls->any_active, sizeof(int32_t),
                                            cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) { set_cuda_error(e); return HP_ERR_CUDA; }
            if (*ctx->host_flag == 0) break;
        }
    }
    if (stream) return HP_OK;  // the streaming kernel stops exactly, nothing to replay
    a.mode = 1;
    return launch_sweep(a, H, R, st);
}

static int pick_T(const hp_project_params* prm)
{
    int T = prm->temporal_block;
    if (T <= 0) T = kMaxBlock;
    if (T > kMaxBlock) T = kMaxBlock;
    return T;
}

hp_status project_impl(hp_ctx* ctx, float* u, float* v, const uint8_t* flags, hp_shape s,
                       const hp_project_params* prm, const float* phi0, float* p_out,
                       int32_t* iters_out, double* e1_out, double* einf_out, uint8_t* conv_out,
                       double* e_hist, int32_t hist_len, cudaStream_t st, float* phi_copy_out,
                       bool have_div)
{
    const size_t cells = (size_t)s.batch * s.ny * s.nx;
    hp_status rc = HP_OK;
    if (u && !have_div) {
        // without a velocity the caller has prepared ctx->mask and ctx->div
        rc = launch_mask_div(u, v, flags, ctx->mask, ctx->div, s, st, boundary_of(*prm));
        if (rc != HP_OK) return rc;
    }
    init_phi_kernel<<<(unsigned)((cells + 255) / 256), 256, 0, st>>>(phi0, ctx->mask, ctx->phi[0],
                                                                     cells);
    if ((rc = check_launch()) != HP_OK) return rc;

    const bool fixed = prm->fixed_iters > 0;
    const int cap = fixed ? prm->fixed_iters : prm->max_iters;
    const double thr = fixed ? -1.0 : prm->threshold;
    // otherwise the temporally blocked kernel (measured faster than the
    // streaming one at 16 x 512^2 and above)
    const bool stream = prm->sweep_kernel == 1;
    const int R = prm->sweep_kernel == 3 ? 2 : 4;
    bool resident = false;
    if (prm->sweep_kernel == 4 || prm->sweep_kernel == 0) {
        // library choice: the whole grid on chip, one cluster per grid
        // (measured 1.85x faster than the blocked kernel at 16 x 512^2); the
        // blocked loop when the grid is larger or the cluster does not fit
        reset_state_kernel<<<(s.batch + 255) / 256, 256, 0, st>>>(ctx->gs, ctx->ls, s.batch);
        if ((rc = check_launch()) != HP_OK) return rc;
        rc = launch_resident(ctx, s, thr, cap, e_hist, hist_len, st, &resident);
        if (rc != HP_OK) return rc;
    }
    if (!resident) {
        rc = run_sweep_loop(ctx, s, pick_T(prm), R, stream, thr, cap, e_hist, hist_len,
                            prm->use_graph != 0, st);
        if (rc != HP_OK) return rc;
    }

    dim3 blk(256), grd((s.nx + 255) / 256, s.ny, s.batch);
    const float scale = prm->rho0 / prm->dt;
    const Boundary bc = boundary_of(*prm);
    if (s.nx % 4 == 0 && (!u || aligned16(v)) && aligned16(flags) && aligned16(p_out) &&
        aligned16(phi_copy_out)) {
        dim3 g4((s.nx / 4 + kQuadThreads - 1) / kQuadThreads, (s.ny + kDivRows - 1) / kDivRows,
                s.batch);
        correct_col_kernel<<<g4, kQuadThreads, 0, st>>>(u, v, ctx->mask, flags, ctx->phi[0],
                                                        ctx->phi[1], ctx->gs, p_out, phi_copy_out,
                                                        scale, s.ny, s.nx, bc);
    } else {
        correct_kernel<<<grd, blk, 0, st>>>(u, v, ctx->mask, flags, ctx->phi[0], ctx->phi[1],
                                            ctx->gs, p_out, phi_copy_out, scale, s.ny, s.nx, bc);
    }
    if ((rc = check_launch()) != HP_OK) return rc;

    // norms of the corrected velocity
    if ((size_t)s.batch * ((s.nx + kSegCells - 1) / kSegCells) * s.ny > ctx->partial2_len)
        return HP_ERR_INVALID_ARG;
    float2* p2 = reinterpret_cast<float2*>(ctx->partial2);
    int nblk = 1;
    if (u) {
        nblk = norms_kernel(u, v, flags, ctx->mask, p2, s, bc, st);
        if ((rc = check_launch()) != HP_OK) return rc;
    }
    norms_finish_kernel<<<s.batch, kFinishWarps * 32, 0, st>>>(
        p2, nblk, u ? e1_out : nullptr, u ? einf_out : nullptr, ctx->gs, iters_out,
        fixed ? nullptr : conv_out, s.batch, 1.0 / ((double)s.nx * (double)s.ny));
    if ((rc = check_launch()) != HP_OK) return rc;
    if (fixed && conv_out) {
        cudaError_t e = cudaMemsetAsync(conv_out, 1, (size_t)s.batch, st);
        if (e != cudaSuccess) { set_cuda_error(e); return HP_ERR_CUDA; }
    }
    return HP_OK;
}

}  // namespace hp
