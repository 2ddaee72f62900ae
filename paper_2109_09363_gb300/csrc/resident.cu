// Grid-resident masked Jacobi sweeps for sm_103a (Sec. 2.2 Jacobi iteration,
// stop rule of Sec. 3.3 / 4.1).
//
// One thread-block cluster holds one whole grid on chip for all of its sweeps:
// each CTA owns a 128 x 128 tile (16 warps; thread (w, l) holds rows 8w..8w+7,
// columns 4l..4l+3), phi lives in registers, div, 1/n and 4 - n (as BF16,
// exact for 0..4) in shared memory; the open-face flag n > 0 follows from
// 1/n.  A cluster has up to 16 CTAs (a 512 x 512 grid), a grid of at most
// 128 x 128 runs as a single CTA.  Per sweep k:
//   1. the boundary values of phi_k are out: every warp's top and bottom rows
//      in shared memory, the tile's boundary rows / columns in the
//      neighbouring CTAs' halo buffers (distributed shared memory); sweep k-1
//      stored each of them as soon as it had computed it;
//   2. one cluster barrier (release / acquire), split in arrive and wait;
//   3. every kBatch-th sweep, between arrive and wait and on data that a
//      barrier already made visible, warp 0 runs one round of the E
//      book-keeping for kBatch sweeps at once (8 lanes per sweep): the CTA
//      partials (sums of the 16 warp sums of |r|) of sweeps k-6..k-3, stored
//      into every CTA of the cluster, and E of sweeps k-10..k-7 from the
//      cluster's partials (FP64, fixed shuffle trees, identical in every
//      CTA), with the stop decisions in sweep order (E <= E_t, cap, or
//      non-finite E); a round costs about one sweep's FP64 latency, paid
//      once per kBatch sweeps;
//   4. all threads read the decision for sweep k - kResLag and leave together;
//   5. the update phi_{k+1} = phi_k - r(phi_k) / n (the shared cell_update,
//      so the iterates are bit-identical to the other sweep kernels) and the
//      warp sums of |r(phi_k)|.
// Buffers rotate with the sweep parity (halos) or in rings indexed by sweep
// (warp sums, CTA partials, decisions), sized so that the one barrier per
// sweep keeps them race-free.  The decision arrives kResLag sweeps late; phi
// is checkpointed to global memory every kCkptEvery sweeps, and after the
// stop the cluster reloads the checkpoint at or below k* and replays the
// sweeps up to k* exactly.  All CTAs of a cluster execute the same number of
// barriers: the decision is computed from the same values in the same order
// everywhere.
#include <cuda_runtime.h>
#include <math.h>

#include <type_traits>

#include "hproj_internal.cuh"

namespace hp {

namespace {

constexpr int kResWarps = 16;
constexpr int kResRows = 8;  // rows per thread
constexpr int kResThreads = kResWarps * 32;
constexpr int kResTile = 128;  // tile side per CTA
constexpr int kCkptEvery = 32;  // > kResLag: the two latest checkpoints cover k*
// E book-keeping in rounds of kBatch sweeps (every kBatch-th sweep, 8 lanes
// of warp 0 per sweep); the stop decision of sweep j is read at sweep j + kResLag.
// The warp sums of sweep j are stored during sweep j + 1, after its arrive,
// so a barrier orders them before a read only from sweep j + 3 on: a round
// at sweep k takes the warp sums of sweeps k - kBatch - 2 .. k - 3.
constexpr int kBatch = 4;
constexpr int kResLag = 2 * kBatch + 3;
constexpr int kWsumRing = 8;   // warp sums, by sweep
constexpr int kEpartRing = 8;  // CTA partials, by sweep
constexpr int kDecRing = 16;   // decisions, by sweep
constexpr int kResMaxCluster = 16;

// dynamic shared memory (bytes)
constexpr int kOffInv = 0;                                            // [128][128] float
constexpr int kOffD = kOffInv + kResTile * kResTile * 4;              // [128][128] float
constexpr int kOffC = kOffD + kResTile * kResTile * 4;                // [128][128] bf16 (exact)
constexpr int kOffXch = kOffC + kResTile * kResTile * 2;              // [2][2][16][32] float4
constexpr int kOffHRow = kOffXch + 2 * 2 * kResWarps * 32 * 16;       // [2][2][32] float4
constexpr int kOffHCol = kOffHRow + 2 * 2 * 32 * 16;                  // [2][2][16][8] float
constexpr int kOffWsum = kOffHCol + 2 * 2 * kResWarps * kResRows * 4; // [8][16] float
constexpr int kOffEpart = kOffWsum + 8 * kResWarps * 4;               // [8][16] double
constexpr int kResSmem = kOffEpart + 8 * kResMaxCluster * 8;

struct ResArgs {
    float* phi;        // [B][ny][nx]: phi_0 in, phi_{k*} out
    float* ck[2];      // checkpoint buffers [B][ny][nx]
    const float* div;  // [B][ny][nx]
    const uint8_t* mask;
    GridState* gs;
    double* e_hist;    // [B][hist_len] or null
    int32_t hist_len;
    int32_t ny, nx;
    int32_t cx, cy;    // tiles (CTAs) per grid
    int32_t max_iters;
    double threshold;  // < 0: never stops before the cap
};

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// address of the same shared-memory location in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t remote(const void* local, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_addr(local)), "r"(rank));
    return r;
}

__device__ __forceinline__ void st_cluster(uint32_t addr, float4 v)
{
    asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(v.x),
                 "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}

__device__ __forceinline__ void st_cluster(uint32_t addr, float v)
{
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}

__device__ __forceinline__ void st_cluster(uint32_t addr, double v)
{
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}

template <bool CLUSTER>
__device__ __forceinline__ void sweep_barrier()
{
    if (CLUSTER) {
        asm volatile(
            "barrier.cluster.arrive.release.aligned;\n\t"
            "barrier.cluster.wait.acquire.aligned;" ::: "memory");
    } else {
        __syncthreads();
    }
}

// The same barrier in two halves (cluster only): work between arrive and wait
// overlaps the barrier latency; for a single CTA the wait is __syncthreads.
template <bool CLUSTER>
__device__ __forceinline__ void sweep_arrive()
{
    if (CLUSTER) asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}

template <bool CLUSTER>
__device__ __forceinline__ void sweep_wait()
{
    if (CLUSTER) {
        asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
    } else {
        __syncthreads();
    }
}

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

struct ResGeom {
    int lane, wid;
    uint32_t rank;
    bool up, down, left, right;  // neighbouring tiles exist in the cluster
    int cx;
    // cluster addresses of this thread's halo slots (parity 0) in the
    // neighbouring CTAs, computed once: up / down row slot of this lane,
    // left / right column slots of this warp (row 0); parity p adds
    // p * kParityBytes, row r of a column adds 4 r
    uint32_t r_up, r_down, r_left, r_right;
};

// byte offset between the parity-0 and parity-1 halo buffers (rows and columns)
constexpr uint32_t kParityBytes = 2 * 32 * 16;
static_assert(2 * kResWarps * kResRows * 4 == (int)kParityBytes,
              "row and column halo buffers share the parity stride");

// Step 1: this thread's boundary values of phi into the parity-p buffers.
template <bool CLUSTER>
__device__ __forceinline__ void res_publish(const ResGeom& g, const float (&phi)[kResRows][4],
                                            int p, float4* s_xch, float4* s_hrow, float* s_hcol)
{
    const float4 top = make_float4(phi[0][0], phi[0][1], phi[0][2], phi[0][3]);
    const float4 bot = make_float4(phi[kResRows - 1][0], phi[kResRows - 1][1],
                                   phi[kResRows - 1][2], phi[kResRows - 1][3]);
    s_xch[((p * 2 + 0) * kResWarps + g.wid) * 32 + g.lane] = top;
    s_xch[((p * 2 + 1) * kResWarps + g.wid) * 32 + g.lane] = bot;
    if (CLUSTER) {
        // the tile above receives our top row as its row "from below" (slot 1),
        // the tile below our bottom row as "from above" (slot 0)
        if (g.wid == 0 && g.up) st_cluster(g.r_up + p * kParityBytes, top);
        if (g.wid == kResWarps - 1 && g.down) st_cluster(g.r_down + p * kParityBytes, bot);
        // the tile to the left receives our left column as "from right" (slot
        // 1), the tile to the right our right column as "from left" (slot 0)
        if (g.lane == 0 && g.left) {
#pragma unroll
            for (int r = 0; r < kResRows; ++r)
                st_cluster(g.r_left + p * kParityBytes + 4 * r, phi[r][0]);
        }
        if (g.lane == 31 && g.right) {
#pragma unroll
            for (int r = 0; r < kResRows; ++r)
                st_cluster(g.r_right + p * kParityBytes + 4 * r, phi[r][3]);
        }
    }
}

// Step 5: phi_{k+1} from phi_k (parity-p neighbour buffers); returns this
// thread's FP32 sum of |r(phi_k)| when WITH_E.  With BOOK (warp 0), the two
// FP64 reduction trees t0, t1 over lanes 0..15 advance one level after each
// of the first four rows.
template <bool CLUSTER, bool WITH_E, bool BOOK, int p>
__device__ __forceinline__ float res_update(const ResGeom& g, float (&phi)[kResRows][4],
                                            float4* s_xch,
                                            float4* s_hrow, float* s_hcol,
                                            const float4* s_inv4, const float4* s_d4,
                                            const uint2* s_c2, double& t0, double& t1)
{
    // boundary values of phi_{k+1} go out (parity p ^ 1) as soon as they are
    // computed, so that the stores have landed by the next barrier; those
    // buffers were last read in the previous sweep, before the barrier this
    // thread has passed
    constexpr int q1 = p ^ 1;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 nb = g.wid > 0 ? s_xch[((p * 2 + 1) * kResWarps + g.wid - 1) * 32 + g.lane]
                      : g.up    ? s_hrow[(p * 2 + 0) * 32 + g.lane]
                                : zero;
    const float4 sb = g.wid < kResWarps - 1
                          ? s_xch[((p * 2 + 0) * kResWarps + g.wid + 1) * 32 + g.lane]
                      : g.down ? s_hrow[(p * 2 + 1) * 32 + g.lane]
                               : zero;
    const float* hl = s_hcol + ((p * 2 + 0) * kResWarps + g.wid) * kResRows;
    const float* hr = s_hcol + ((p * 2 + 1) * kResWarps + g.wid) * kResRows;
    const float north[4] = {nb.x, nb.y, nb.z, nb.w};
    const float south[4] = {sb.x, sb.y, sb.z, sb.w};
    // each difference between two cells is formed once: the south difference
    // of row r is minus the north difference of row r + 1, the east
    // difference of a cell minus the west difference of the next
    float dn[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) dn[q] = __fsub_rn(north[q], phi[0][q]);
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};  // one |r| sum per column: short chains
#pragma unroll
    for (int r = 0; r < kResRows; ++r) {
        float left = __shfl_up_sync(0xffffffffu, phi[r][3], 1);
        float right = __shfl_down_sync(0xffffffffu, phi[r][0], 1);
        if (g.lane == 0) left = g.left ? hl[r] : 0.0f;
        if (g.lane == 31) right = g.right ? hr[r] : 0.0f;
        const int slot = (g.wid * kResRows + r) * 32 + g.lane;
        const float4 iv = s_inv4[slot];
        const float4 dv = s_d4[slot];
        const uint2 cb = s_c2[slot];
        const float inv[4] = {iv.x, iv.y, iv.z, iv.w};
        const float dd[4] = {dv.x, dv.y, dv.z, dv.w};
        const float cc[4] = {__uint_as_float(cb.x << 16), __uint_as_float(cb.x & 0xffff0000u),
                             __uint_as_float(cb.y << 16), __uint_as_float(cb.y & 0xffff0000u)};
        // east differences: ex[0] = phi[0] - left, ex[q + 1] = east of cell q
        float ex[5];
        ex[0] = __fsub_rn(phi[r][0], left);
#pragma unroll
        for (int q = 0; q < 3; ++q) ex[q + 1] = __fsub_rn(phi[r][q + 1], phi[r][q]);
        ex[4] = __fsub_rn(right, phi[r][3]);
        float nw[4], ds[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float ps = r < kResRows - 1 ? phi[r + 1][q] : south[q];
            ds[q] = __fsub_rn(ps, phi[r][q]);
            CellConst kc;
            kc.d = dd[q];
            kc.inv = inv[q];
            kc.c = cc[q];
            // [n > 0] from 1/n in {0, 1/4, 1/3, 1/2, 1}: saturate(4/n) is exactly 0 or 1
            kc.w = __saturatef(inv[q] * 4.0f);
            float res;
            nw[q] = cell_update_diff(phi[r][q], -ex[q], ex[q + 1], dn[q], ds[q], kc, res);
            if (WITH_E) acc[q] = __fadd_rn(acc[q], fabsf(res));
        }
        if (r == 0 || r == kResRows - 1) {
            const float4 v4 = make_float4(nw[0], nw[1], nw[2], nw[3]);
            s_xch[((q1 * 2 + (r == 0 ? 0 : 1)) * kResWarps + g.wid) * 32 + g.lane] = v4;
            if (CLUSTER) {
                if (r == 0 && g.wid == 0 && g.up) st_cluster(g.r_up + q1 * kParityBytes, v4);
                if (r == kResRows - 1 && g.wid == kResWarps - 1 && g.down)
                    st_cluster(g.r_down + q1 * kParityBytes, v4);
            }
        }
        if (CLUSTER) {
            if (g.lane == 0 && g.left) st_cluster(g.r_left + q1 * kParityBytes + 4 * r, nw[0]);
            if (g.lane == 31 && g.right) st_cluster(g.r_right + q1 * kParityBytes + 4 * r, nw[3]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            dn[q] = -ds[q];
            phi[r][q] = nw[q];
        }
        if (BOOK && r < 4) {
            t0 += __shfl_down_sync(0xffffffffu, t0, 8 >> r);
            t1 += __shfl_down_sync(0xffffffffu, t1, 8 >> r);
        }
    }
    return __fadd_rn(__fadd_rn(acc[0], acc[1]), __fadd_rn(acc[2], acc[3]));
}

__device__ __forceinline__ float* ckpt_buf(const ResArgs& a, int m)
{
    // checkpoint m holds phi_{m * kCkptEvery}; m = 0 is the input phi_0
    return m == 0 ? a.phi : (m & 1) ? a.ck[1] : a.ck[0];
}

template <bool CLUSTER>
__global__ void __launch_bounds__(kResThreads, 1) sweep_resident_kernel(ResArgs a)
{
    extern __shared__ __align__(16) uint8_t sm[];
    float4* s_inv4 = reinterpret_cast<float4*>(sm + kOffInv);
    float4* s_d4 = reinterpret_cast<float4*>(sm + kOffD);
    uint2* s_c2 = reinterpret_cast<uint2*>(sm + kOffC);
    float4* s_xch = reinterpret_cast<float4*>(sm + kOffXch);
    float4* s_hrow = reinterpret_cast<float4*>(sm + kOffHRow);
    float* s_hcol = reinterpret_cast<float*>(sm + kOffHCol);
    float* s_wsum = reinterpret_cast<float*>(sm + kOffWsum);
    double* s_epart = reinterpret_cast<double*>(sm + kOffEpart);
    __shared__ int s_dec[kDecRing];      // decision of sweep j: 0 go on, 1 converged, 2 stop
    __shared__ double s_edec[kDecRing];  // E_j

    ResGeom g;
    g.lane = threadIdx.x & 31;
    g.wid = threadIdx.x >> 5;
    g.cx = a.cx;
    const int tx = blockIdx.x, ty = blockIdx.y, b = blockIdx.z;
    g.rank = CLUSTER ? cluster_rank() : 0u;
    g.up = ty > 0;
    g.down = ty < a.cy - 1;
    g.left = tx > 0;
    g.right = tx < a.cx - 1;
    g.r_up = g.r_down = g.r_left = g.r_right = 0u;
    if (CLUSTER) {
        if (g.up) g.r_up = remote(&s_hrow[1 * 32 + g.lane], g.rank - g.cx);
        if (g.down) g.r_down = remote(&s_hrow[0 * 32 + g.lane], g.rank + g.cx);
        if (g.left) g.r_left = remote(&s_hcol[(1 * kResWarps + g.wid) * kResRows], g.rank - 1);
        if (g.right) g.r_right = remote(&s_hcol[(0 * kResWarps + g.wid) * kResRows], g.rank + 1);
    }
    const int nranks = a.cx * a.cy;
    const int nx = a.nx, ny = a.ny;
    const size_t gbase = (size_t)b * ny * nx;
    const int x0 = tx * kResTile + 4 * g.lane;
    const int y0 = ty * kResTile + kResRows * g.wid;
    const bool vec = (nx & 3) == 0;

    // ---- load phi_0, div and the per-cell constants
    float phi[kResRows][4];
#pragma unroll
    for (int r = 0; r < kResRows; ++r) {
        const int y = y0 + r;
        uint32_t m4 = 0;
        float dr[4];
        if (y < ny) {
            load_row4(a.phi + gbase + (size_t)y * nx, x0, nx, vec, phi[r]);
            load_row4(a.div + gbase + (size_t)y * nx, x0, nx, vec, dr);
            m4 = load_mask4(a.mask + gbase + (size_t)y * nx, x0, nx, vec);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) phi[r][q] = dr[q] = 0.0f;
        }
        float iv[4], dv[4];
        uint32_t cb[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const CellConst k = make_const(dr[q], (m4 >> (8 * q)) & 0xffu);
            dv[q] = k.d;
            iv[q] = k.inv;
            cb[q] = __float_as_uint(k.c) >> 16;  // 0..4: exact in the upper half
        }
        const int slot = (g.wid * kResRows + r) * 32 + g.lane;
        s_inv4[slot] = make_float4(iv[0], iv[1], iv[2], iv[3]);
        s_d4[slot] = make_float4(dv[0], dv[1], dv[2], dv[3]);
        s_c2[slot] = make_uint2(cb[0] | (cb[1] << 16), cb[2] | (cb[3] << 16));
    }
    if (threadIdx.x < kDecRing) s_dec[threadIdx.x] = 0;
    // every CTA of the cluster is running before any CTA stores into
    // another's shared memory
    sweep_barrier<CLUSTER>();

    auto store_cells = [&](float* dst) {
#pragma unroll
        for (int r = 0; r < kResRows; ++r) {
            const int y = y0 + r;
            if (y >= ny) continue;
            float* row = dst + gbase + (size_t)y * nx;
            if (vec && x0 + 3 < nx) {
                *reinterpret_cast<float4*>(row + x0) =
                    make_float4(phi[r][0], phi[r][1], phi[r][2], phi[r][3]);
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (x0 + q < nx) row[x0 + q] = phi[r][q];
            }
        }
    };

    const double inv_cells = 1.0 / ((double)nx * (double)ny);
    bool decided = false;  // thread 0: a stop was decided (no more history writes)
    int kstar = 0, dec = 0;
    double estar = 0.0;
    // ---- main loop; registers hold phi_k at the top of sweep k, its
    // boundary values are in the parity-(k & 1) buffers (sweep k - 1 wrote
    // them during its update; phi_0's go out here)
    res_publish<CLUSTER>(g, phi, 0, s_xch, s_hrow, s_hcol);
    float pending = 0.0f;  // this thread's sum of |r| of the previous sweep
    // one sweep k of parity P (the loop below runs them in pairs so that the
    // halo buffers' parity is a compile-time constant); true: stop
    auto sweep = [&](auto parity, int k) -> bool {
        constexpr int P = decltype(parity)::value;
        // checkpoints (every 32nd sweep) and E rounds (every 4th) fall on even k
        if (P == 0 && k > 0 && k % kCkptEvery == 0) store_cells(ckpt_buf(a, k / kCkptEvery));
        sweep_arrive<CLUSTER>();
        if (k > 0) {
            // warp sum of sweep k - 1, reduced while the barrier completes; the
            // book-keeping reads warp sums two or more sweeps old
            float t = pending;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1)
                t = __fadd_rn(t, __shfl_xor_sync(0xffffffffu, t, off));
            if (g.lane == 0) s_wsum[((k - 1) % kWsumRing) * kResWarps + g.wid] = t;
        }
        if (P == 0 && g.wid == 0 && k % kBatch == 0) {
            // one round, between arrive and wait, on data that an earlier
            // barrier made visible (the warp sums of sweep jc were stored in
            // sweep jc + 1 and passed the barrier of sweep jc + 2 <= k - 1,
            // the CTA partials of je in the round before and the barrier of
            // sweep k - 3); lane group gi (8 lanes) takes sweep
            // jc = k - kBatch - 2 + gi for the CTA partial (its 16 warp sums)
            // and sweep je = jc - kBatch for E (the cluster's CTA partials);
            // fixed FP64 trees, the same in every CTA
            const int gi = g.lane >> 3, li = g.lane & 7;
            const int jc = k - kBatch - 2 + gi, je = jc - kBatch;
            double t0 = 0.0, t1 = 0.0;
            if (jc >= 0) {
                const float* ws = s_wsum + (jc % kWsumRing) * kResWarps;
                t0 = (double)ws[2 * li] + (double)ws[2 * li + 1];
            }
            if (je >= 0) {
                const double* ep = s_epart + (je % kEpartRing) * kResMaxCluster;
                t1 = (2 * li < nranks ? ep[2 * li] : 0.0) + (2 * li + 1 < nranks ? ep[2 * li + 1] : 0.0);
            }
#pragma unroll
            for (int off = 4; off > 0; off >>= 1) {
                t0 += __shfl_down_sync(0xffffffffu, t0, off, 8);
                t1 += __shfl_down_sync(0xffffffffu, t1, off, 8);
            }
            const double cp = __shfl_sync(0xffffffffu, t0, 0, 8);
            if (jc >= 0) {
                // CTA partial of E_jc into slot [rank] of every CTA (this
                // lane: ranks 2 li and 2 li + 1)
                double* slot = &s_epart[(jc % kEpartRing) * kResMaxCluster + g.rank];
                if (CLUSTER) {
                    if (2 * li < nranks) st_cluster(remote(slot, (uint32_t)(2 * li)), cp);
                    if (2 * li + 1 < nranks) st_cluster(remote(slot, (uint32_t)(2 * li + 1)), cp);
                } else if (li == 0) {
                    *slot = cp;
                }
            }
            double ev[kBatch];
#pragma unroll
            for (int q = 0; q < kBatch; ++q) ev[q] = __shfl_sync(0xffffffffu, t1, 8 * q);
            if (g.lane == 0) {
                // the round's decisions in sweep order; the first stop counts
#pragma unroll
                for (int q = 0; q < kBatch; ++q) {
                    const int j = k - 2 * kBatch - 2 + q;
                    if (j < 0) continue;
                    const double e = ev[q] * inv_cells;
                    int dj = 0;
                    if (!decided) {
                        if (g.rank == 0 && a.e_hist && j < a.hist_len)
                            a.e_hist[(size_t)b * a.hist_len + j] = e;
                        if (e <= a.threshold) dj = 1;
                        else if (j >= a.max_iters || !isfinite(e)) dj = 2;
                        decided = dj != 0;
                    }
                    s_dec[j % kDecRing] = dj;
                    s_edec[j % kDecRing] = e;
                }
            }
        }
        sweep_wait<CLUSTER>();
        if (k >= kResLag) {
            const int j = k - kResLag;
            const int dj = s_dec[j % kDecRing];
            if (dj != 0) {
                kstar = j;
                dec = dj;
                estar = s_edec[j % kDecRing];
                return true;
            }
        }
        double t0 = 0.0, t1 = 0.0;
        pending = res_update<CLUSTER, true, false, P>(g, phi, s_xch, s_hrow, s_hcol, s_inv4,
                                                      s_d4, s_c2, t0, t1);
        return false;
    };
    for (int k = 0;; k += 2) {
        if (sweep(std::integral_constant<int, 0>{}, k)) break;
        if (sweep(std::integral_constant<int, 1>{}, k + 1)) break;
    }

    // ---- replay from the checkpoint at or below k* to phi_{k*}
    const int m = kstar / kCkptEvery;
    {
        const float* src = ckpt_buf(a, m);
#pragma unroll
        for (int r = 0; r < kResRows; ++r) {
            const int y = y0 + r;
            if (y < ny) load_row4(src + gbase + (size_t)y * nx, x0, nx, vec, phi[r]);
            else {
#pragma unroll
                for (int q = 0; q < 4; ++q) phi[r][q] = 0.0f;
            }
        }
    }
    // nobody reads a halo buffer after the main loop's last barrier, so the
    // checkpoint's boundary values can go out at once
    res_publish<CLUSTER>(g, phi, (m * kCkptEvery) & 1, s_xch, s_hrow, s_hcol);
    for (int j = m * kCkptEvery; j < kstar; ++j) {
        sweep_barrier<CLUSTER>();
        double t0 = 0.0, t1 = 0.0;
        if (j & 1)
            res_update<CLUSTER, false, false, 1>(g, phi, s_xch, s_hrow, s_hcol, s_inv4, s_d4,
                                                 s_c2, t0, t1);
        else
            res_update<CLUSTER, false, false, 0>(g, phi, s_xch, s_hrow, s_hcol, s_inv4, s_d4,
                                                 s_c2, t0, t1);
    }
    store_cells(a.phi);
    if (threadIdx.x == 0 && g.rank == 0) {
        GridState* gs = a.gs + b;
        gs->active = 0;
        gs->kstar = kstar;
        gs->k0_stop = kstar;
        gs->replay = 0;
        gs->src = 0;
        gs->final_buf = 0;
        gs->converged = dec == 1 ? 1 : 0;
        gs->e_stop = estar;
    }
    // no CTA may leave while another can still store into its shared memory
    sweep_barrier<CLUSTER>();
}

}  // namespace

// Tiles per grid for the resident kernel, 0 when the grid is too large.
int resident_tiles(hp_shape s)
{
    const int cx = (s.nx + kResTile - 1) / kResTile, cy = (s.ny + kResTile - 1) / kResTile;
    return cx * cy <= kResMaxCluster ? cx * cy : 0;
}

static cudaLaunchConfig_t resident_config(hp_shape s, cudaStream_t st, cudaLaunchAttribute* at)
{
    const int cx = (s.nx + kResTile - 1) / kResTile, cy = (s.ny + kResTile - 1) / kResTile;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cx, cy, s.batch);
    cfg.blockDim = dim3(kResThreads, 1, 1);
    cfg.dynamicSmemBytes = kResSmem;
    cfg.stream = st;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cx;
    at[0].val.clusterDim.y = cy;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cfg;
}

static hp_status resident_attrs(bool cluster)
{
    static bool done[2] = {false, false};
    if (done[cluster]) return HP_OK;
    const void* fn = cluster ? (const void*)sweep_resident_kernel<true>
                             : (const void*)sweep_resident_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kResSmem);
    if (e == cudaSuccess && cluster)
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) { set_cuda_error(e); return HP_ERR_CUDA; }
    done[cluster] = true;
    return HP_OK;
}

// Clusters (grids) of shape s that can be resident at once; 0 when the
// resident kernel cannot run this shape (cached per cluster size).
int resident_capacity(hp_ctx* ctx, hp_shape s)
{
    const int n = resident_tiles(s);
    if (n == 0) return 0;
    if (ctx->res_clusters[n] == 0) {
        int ncl = 0;
        if (resident_attrs(n > 1) == HP_OK) {
            cudaLaunchAttribute at[1];
            hp_shape one = s;
            one.batch = 1;
            cudaLaunchConfig_t cfg = resident_config(one, nullptr, at);
            cudaError_t e = n > 1
                ? cudaOccupancyMaxActiveClusters(&ncl, sweep_resident_kernel<true>, &cfg)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ncl, sweep_resident_kernel<false>,
                                                                kResThreads, kResSmem);
            if (e != cudaSuccess) {
                cudaGetLastError();
                ncl = 0;
            }
            if (n == 1) ncl *= ctx->num_sms;
        }
        ctx->res_clusters[n] = ncl + 1;
    }
    return ctx->res_clusters[n] - 1;
}

// Launches the resident sweep loop when one cluster per grid fits on the
// device; *launched = false (and nothing queued) otherwise.
hp_status launch_resident(hp_ctx* ctx, hp_shape s, double threshold, int max_iters,
                          double* e_hist, int hist_len, cudaStream_t st, bool* launched)
{
    *launched = false;
    if (resident_capacity(ctx, s) < 1) return HP_OK;
    const int n = resident_tiles(s);
    ResArgs a;
    a.phi = ctx->phi[0];
    a.ck[0] = ctx->ckpt;
    a.ck[1] = ctx->phi[1];
    a.div = ctx->div;
    a.mask = ctx->mask;
    a.gs = ctx->gs;
    a.e_hist = e_hist;
    a.hist_len = hist_len;
    a.ny = s.ny;
    a.nx = s.nx;
    a.cx = (s.nx + kResTile - 1) / kResTile;
    a.cy = (s.ny + kResTile - 1) / kResTile;
    a.max_iters = max_iters;
    a.threshold = threshold;
    hp_status rc = resident_attrs(n > 1);
    if (rc != HP_OK) return rc;
    if (n == 1) {
        sweep_resident_kernel<false><<<dim3(1, 1, s.batch), kResThreads, kResSmem, st>>>(a);
    } else {
        cudaLaunchAttribute at[1];
        cudaLaunchConfig_t cfg = resident_config(s, st, at);
        cudaError_t e = cudaLaunchKernelEx(&cfg, sweep_resident_kernel<true>, a);
        if (e != cudaSuccess) { set_cuda_error(e); return HP_ERR_CUDA; }
    }
    *launched = true;
    return check_launch();
}

}  // namespace hp

extern "C" int32_t hp_resident_clusters(hp_ctx* ctx, hp_shape s)
{
    if (!ctx || !hp::shape_ok(s)) return 0;
    return hp::resident_capacity(ctx, s);
}
