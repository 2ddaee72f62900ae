// Internal declarations of the GB300 projection library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/hproj.h"

namespace hp {

// Maximum sweeps fused into one launch of the temporally blocked sweep kernel;
// it is also the halo width of a tile (a multiple of 4 so that tiles stay
// 16-byte aligned).
constexpr int kMaxBlock = 8;

// Sweep tile: 16 warps, each thread holds 4 rows x 4 columns in registers, so
// one CTA covers 64 rows x 128 columns including the halo.
constexpr int kTileWarps = 16;
constexpr int kTileRows = 4 * kTileWarps;  // 64
constexpr int kTileCols = 128;

// Boundary of the box beyond the closed walls: an open top (exterior at
// phi = 0) and the bottom-boundary v faces of columns [x0, x1) under fluid
// cells with a prescribed (inflow) velocity.  All zero: a closed box.
struct Boundary {
    int32_t open_top;
    int32_t x0, x1;
};

__host__ __device__ inline Boundary boundary_of(const hp_project_params& p)
{
    return Boundary{p.open_top, p.inflow_x0, p.inflow_x1};
}

// Per-grid state of one projection, device resident.
struct GridState {
    int32_t active;      // 1 while the grid still sweeps
    int32_t kstar;       // stop index k*
    int32_t k0_stop;     // first sweep index of the block in which k* fell
    int32_t replay;      // sweeps to replay from buffer `src` to reach k*
    int32_t src;         // buffer holding phi_{k0_stop}
    int32_t final_buf;   // buffer holding phi_{k*}
    int32_t converged;   // 1 when E(phi_{k*}) <= threshold
    int32_t pad_;
    double e_stop;       // E(phi_{k*})
    uint32_t arrivals;   // CTA arrival counter of the current launch
    uint32_t pad2_;
};

// Loop state shared by all grids.
struct LoopState {
    int32_t k0;          // first sweep index of the current block
    int32_t blk;         // block counter; parity selects the phi buffers
    uint32_t arrivals;   // CTA (blocked kernel) or grid (streaming kernel) arrivals
    int32_t any_active;  // 1 while some grid still sweeps
    int32_t n_active;    // grids still sweeping when the current launch started
    int32_t pad_;
};

struct SweepArgs {
    float* phi0;                 // ping-pong buffers [B][ny][nx]
    float* phi1;
    const float* div;            // [B][ny][nx]
    const uint8_t* mask;         // open-face bits [B][ny][nx]
    GridState* gs;               // [B]
    LoopState* ls;
    double* partial;             // [B][kMaxBlock][ctas per grid]
    double* e_hist;              // [B][hist_len] or null
    int32_t hist_len;
    int32_t B, ny, nx;
    int32_t T;                   // sweeps per launch (<= kMaxBlock)
    int32_t max_iters;
    double threshold;            // < 0 never stops before the cap
    int32_t mode;                // 0 = loop block, 1 = replay
    unsigned long long cond;     // CUDA-graph conditional handle (0 = none)
};

// Guard zones (a substitute for a memory checker): every device workspace
// of a context, a network and a trainer is allocated kGuardBytes longer and
// the extra bytes are filled with kGuardByte; the check calls compare them,
// so a kernel that writes past the end of a workspace is reported.
constexpr size_t kGuardBytes = 256;
constexpr int kGuardByte = 0xA5;
struct Guards {
    std::vector<unsigned char*> zones;  // device address of each guard zone
};
// cudaMalloc(bytes + kGuardBytes), zero the buffer, fill its guard zone
cudaError_t guarded_malloc(void** p, size_t bytes, Guards* g);
// synchronous: HP_ERR_GUARD if a guard byte changed, HP_ERR_CUDA on a CUDA error
hp_status check_guards(const Guards& g);

// Contents of a network checkpoint file (checkpoint.cu).
struct CkptData {
    int32_t arch = -1;
    int64_t step = 0;
    bool has_moments = false;
    std::vector<float> w, m, v;
};
hp_status ckpt_write(const char* path, const CkptData& d);
// HP_ERR_IO for a missing, short, foreign or corrupted file
hp_status ckpt_read(const char* path, CkptData* d);

}  // namespace hp

struct hp_ctx {
    hp::Guards guards;
    int device;
    int num_sms;
    hp_shape max_shape;
    size_t max_cells;
    uint8_t* mask;
    float* div;
    float* phi[2];
    double* partial;
    size_t partial_len;
    double* partial2;
    size_t partial2_len;
    hp::GridState* gs;
    hp::LoopState* ls;
    float* ckpt;         // [max_cells] checkpoint buffer of the resident sweep kernel
    int res_clusters[17];  // per cluster size: 0 unknown, else 1 + clusters that fit
    int32_t* host_flag;  // pinned
    // cached conditional-graph loop
    cudaGraphExec_t graph_exec;
    hp_shape graph_shape;
    int graph_T;
    int graph_hist;
    double* graph_hist_ptr;
    double graph_threshold;
    int graph_max_iters;
    int graph_kernel;
};

namespace hp {

// ------------------------------------------------------------ cell update

// Per-cell constants derived from the open-face bits m:
//   inv = 1/n (0 when n = 0), c = 4 - n, w = (n > 0).
struct CellConst {
    float d, inv, c, w;
};

__device__ __forceinline__ CellConst make_const(float d, uint32_t m)
{
    const int n = __popc(m & 15u);
    CellConst k;
    k.d = d;
    k.inv = n == 4 ? 0.25f : n == 3 ? (1.0f / 3.0f) : n == 2 ? 0.5f : n == 1 ? 1.0f : 0.0f;
    k.c = (float)(4 - n);
    k.w = n > 0 ? 1.0f : 0.0f;
    return k;
}

// One Jacobi update of one cell; returns phi' and writes the residual of phi.
// Every operation is an explicitly rounded intrinsic so that all kernels that
// use it produce bit-identical iterates.
__device__ __forceinline__ float cell_update(float pc, float pw, float pe, float pn, float ps,
                                             const CellConst& k, float& res)
{
    const float dw = __fsub_rn(pw, pc);
    const float de = __fsub_rn(pe, pc);
    const float dn = __fsub_rn(pn, pc);
    const float ds = __fsub_rn(ps, pc);
    const float lapd = __fadd_rn(__fadd_rn(dw, de), __fadd_rn(dn, ds));
    const float lap = __fmaf_rn(k.c, pc, lapd);
    const float r = __fmaf_rn(-k.w, lap, k.d);
    res = r;
    return __fmaf_rn(-r, k.inv, pc);
}

// The same update from the four neighbour differences dw = pw - pc, ...;
// a caller that forms each difference between two cells once and negates it
// for the other cell (x - y == -(y - x) exactly) gets identical results.
__device__ __forceinline__ float cell_update_diff(float pc, float dw, float de, float dn,
                                                  float ds, const CellConst& k, float& res)
{
    const float lapd = __fadd_rn(__fadd_rn(dw, de), __fadd_rn(dn, ds));
    const float lap = __fmaf_rn(k.c, pc, lapd);
    const float r = __fmaf_rn(-k.w, lap, k.d);
    res = r;
    return __fmaf_rn(-r, k.inv, pc);
}

// Loads four consecutive cells of a row (float), zero outside [0, nx).
__device__ __forceinline__ void load_row4(const float* __restrict__ row, int x0, int nx, bool vec,
                                          float out[4])
{
    if (vec && x0 >= 0 && x0 + 3 < nx) {
        const float4 t = *reinterpret_cast<const float4*>(row + x0);
        out[0] = t.x; out[1] = t.y; out[2] = t.z; out[3] = t.w;
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int x = x0 + q;
            out[q] = (x >= 0 && x < nx) ? row[x] : 0.0f;
        }
    }
}

__device__ __forceinline__ uint32_t load_mask4(const uint8_t* __restrict__ row, int x0, int nx,
                                               bool vec)
{
    if (vec && x0 >= 0 && x0 + 3 < nx) return *reinterpret_cast<const uint32_t*>(row + x0);
    uint32_t m = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int x = x0 + q;
        if (x >= 0 && x < nx) m |= (uint32_t)row[x] << (8 * q);
    }
    return m;
}

void set_cuda_error(cudaError_t e);
int resident_tiles(hp_shape s);
int resident_capacity(hp_ctx* ctx, hp_shape s);
hp_status launch_resident(hp_ctx* ctx, hp_shape s, double threshold, int max_iters,
                          double* e_hist, int hist_len, cudaStream_t st, bool* launched);
hp_status check_launch();
bool shape_ok(hp_shape s);

// kernels launched from the API layer
hp_status launch_mask_div(const float* u, const float* v, const uint8_t* flags, uint8_t* mask,
                          float* div, hp_shape s, cudaStream_t st, Boundary bc = Boundary{});
hp_status launch_mask(const uint8_t* flags, uint8_t* mask, hp_shape s, cudaStream_t st);
// out = (phi + J(phi)) / 2, J one masked Jacobi sweep on the right-hand side div
hp_status launch_mean_sweep(const float* phi, const float* div, const uint8_t* mask, float* out,
                            hp_shape s, cudaStream_t st);
// E_1, E_inf of a velocity (closed box); partial: >= nblk_cap 8-byte slots
// per grid, one per 256-cell segment of a row
hp_status launch_div_norms(const float* u, const float* v, const uint8_t* flags,
                           double* partial, int nblk_cap, double* e1, double* einf, hp_shape s,
                           cudaStream_t st);
hp_status launch_div_norms_scratch(const float* u, const float* v, const uint8_t* flags,
                                   double* partial, double* e1, double* einf, hp_shape s,
                                   cudaStream_t st);
// have_div: ctx->mask and ctx->div already hold this velocity's open faces
// and divergence (no second pass over u, v)
hp_status project_impl(hp_ctx* ctx, float* u, float* v, const uint8_t* flags, hp_shape s,
                       const hp_project_params* prm, const float* phi0, float* p_out,
                       int32_t* iters_out, double* e1_out, double* einf_out,
                       uint8_t* conv_out, double* e_hist, int32_t hist_len, cudaStream_t st,
                       float* phi_copy_out, bool have_div = false);
// the argument checks of hp_project
bool project_args_ok(const hp_ctx* c, const float* u, const float* v, const uint8_t* flags,
                     hp_shape s, const hp_project_params* prm, const int32_t* iters_out,
                     const double* e_hist, int32_t hist_len);

int ctas_per_grid(int ny, int nx, int T);
// wait_limit: polls of each bounded pipeline wait of the tensor-core kernels
// before it gives up and raises bit 0 of *err (0 = the compiled limit); pdl:
// launched as a programmatic dependent of the kernel before it in the stream
// (its prologue overlaps that kernel's end; it reads and writes activations
// only after that kernel has completed)
hp_status launch_conv3x3_tc(const void* x, const void* w, const float* bias, void* y, int B,
                            int H, int W, int cin, int cout, int relu, int* err, int nsm,
                            cudaStream_t st, uint32_t wait_limit = 0, bool pdl = false);
// narrowest image the warp-specialised convolution (and the tensor-core first
// and last layers of a branch) serves
int conv_tc_min_width();
hp_status launch_conv3x3_tc_out1(const void* x, const void* w, const float* bias, float* y,
                                 int B, int H, int W, int* err, int nsm, cudaStream_t st,
                                 uint32_t wait_limit = 0, bool pdl = false);
// backward of a tensor-core layer cin -> cout (32 or 64 channels each):
// input gradient (BF16, zero-padded transposed convolution with the flipped
// weights wdg BF16 [9][cin][cout], ReLU derivative of act applied; the
// replicated-border terms are added separately) and per-CTA weight- and
// bias-gradient partial sums part[g][9][cout][cin], partb[g][cout],
// g < *grid_out
hp_status launch_conv3x3_tc_dgrad(const void* gy, const void* wdg, const float* zero_bias,
                                  const void* act, void* gx, int B, int H, int W, int cin,
                                  int cout, int* err, int nsm, cudaStream_t st,
                                  uint32_t wait_limit = 0);
hp_status launch_conv3x3_tc_wgrad(const void* x, const void* gy, float* part, size_t part_len,
                                  float* partb, size_t partb_len, int B, int H, int W, int cin,
                                  int cout, int* err, int nsm, int* grid_out, cudaStream_t st,
                                  uint32_t wait_limit = 0);
hp_status launch_advect(const float* u, const float* v, const float* rho, const uint8_t* flags,
                        float* u_out, float* v_out, float* rho_out, hp_shape s,
                        const hp_plume_params& p, cudaStream_t st);

}  // namespace hp
