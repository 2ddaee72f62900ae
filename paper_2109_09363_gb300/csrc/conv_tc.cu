// 3x3 convolution with replicated borders as an implicit GEMM on the sm_103a
// tensor cores (tcgen05): the dense contraction of the MultiScale CNN
// (Sec. 3.1).  BF16 activations and weights, FP32 accumulation in tensor
// memory, bias + optional ReLU + BF16 rounding in the epilogue.
//
// GEMM view of one tile: M = 128 output pixels (flattened over batch, rows
// and columns), N = Cout, K = 9 taps x Cin.  For every tap the A operand is
// the gathered neighbour pixel of each output pixel (replicated borders
// handled by clamping the coordinates), written to shared memory in the
// canonical no-swizzle K-major layout: core matrices of 8 rows x 16 bytes,
// [tap][channel chunk of 8][row][8 channels].  The weights are packed the
// same way once per CTA: [tap][chunk][cout][8 channels].  One thread issues
// the 9 x Cin/16 MMAs (M = 128, N = Cout, K = 16) into one TMEM accumulator,
// commits them to an mbarrier, and the 128 threads read their row back with
// tcgen05.ld.  This gather form serves widths below 32; wider images use the
// warp-specialised row walk further down.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "hproj_internal.cuh"

namespace hp {

namespace {

constexpr int kConvThreads = 128;  // one thread per GEMM row (output pixel)
constexpr int kTileM = 128;
constexpr uint32_t kSpinLimit = 1u << 26;  // bounded mbarrier wait

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor (tcgen05): start address, leading-dimension
// byte offset (between core matrices along K), stride-dimension byte offset
// (between core matrices along M or N), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N = n, M = m.
__host__ __device__ constexpr uint32_t mma_idesc(int m, int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase)
{
    for (uint32_t it = 0; it < kSpinLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 32 consecutive FP32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v)
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
        "%28, %29, %30, %31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

template <int CIN, int COUT>
struct ConvSmem {
    static constexpr int kChunks = CIN / 8;
    static constexpr int kABytes = 9 * kChunks * kTileM * 16;  // all taps of one tile
    static constexpr int kBBytes = 9 * kChunks * COUT * 16;    // all weights
    static constexpr int kBytes = kABytes + kBBytes;
    static constexpr int kTmemCols = COUT < 32 ? 32 : COUT;
};

// x: [P][CIN] bf16 with P = B*H*W pixels (NHWC); w: [9][COUT][CIN] bf16 (tap
// = 3*dy + dx, dy, dx in 0..2 for offsets -1..1); y: [P][COUT] bf16.
template <int CIN, int COUT>
__global__ void __launch_bounds__(kConvThreads, 1)
    conv3x3_tc_kernel(const uint4* __restrict__ x, const uint4* __restrict__ w,
                      const float* __restrict__ bias, __nv_bfloat16* __restrict__ y, int B,
                      int H, int W, int relu, int ntiles, int* err)
{
    using S = ConvSmem<CIN, COUT>;
    constexpr int NCH = S::kChunks;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* sA = smem;
    uint8_t* sB = smem + S::kABytes;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ float s_bias[COUT];

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const uint32_t mbar_a = smem_u32(&mbar);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"((uint32_t)S::kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar_a), "r"(1u));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    for (int i = tid; i < COUT; i += kConvThreads) s_bias[i] = bias[i];
    // weights -> [tap][chunk][cout][8]
    for (int i = tid; i < 9 * COUT * NCH; i += kConvThreads) {
        const int ch = i % NCH;
        const int n = (i / NCH) % COUT;
        const int tap = i / (NCH * COUT);
        const uint4 v = w[(size_t)(tap * COUT + n) * NCH + ch];
        *reinterpret_cast<uint4*>(sB + ((tap * NCH + ch) * COUT + n) * 16) = v;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    // a programmatic dependent of the layer before it: inputs read and outputs
    // written once that layer has completed
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    const long P = (long)B * H * W;
    const uint32_t idesc = mma_idesc(kTileM, COUT);
    const uint32_t a_base = smem_u32(sA), b_base = smem_u32(sB);
    uint32_t phase = 0;
    bool ok = true;

    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        // gather the 9 tap rows of this thread's output pixel
        const long p = (long)tile * kTileM + tid;
        const bool valid = p < P;
        int b = 0, yy = 0, xx = 0;
        if (valid) {
            b = (int)(p / ((long)H * W));
            const int r = (int)(p - (long)b * H * W);
            yy = r / W;
            xx = r - yy * W;
        }
#pragma unroll 1
        for (int dy = 0; dy < 3; ++dy) {
            const int sy = min(max(yy + dy - 1, 0), H - 1);
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
                const int sx = min(max(xx + dx - 1, 0), W - 1);
                const uint4* src = x + (((size_t)b * H + sy) * W + sx) * NCH;
                const int tap = dy * 3 + dx;
#pragma unroll
                for (int ch = 0; ch < NCH; ++ch) {
                    const uint4 v = valid ? src[ch] : make_uint4(0u, 0u, 0u, 0u);
                    *reinterpret_cast<uint4*>(sA + ((tap * NCH + ch) * kTileM + tid) * 16) = v;
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int tap = 0; tap < 9; ++tap) {
#pragma unroll
                for (int ks = 0; ks < NCH / 2; ++ks) {
                    const uint64_t ad = smem_desc(a_base + (tap * NCH + 2 * ks) * kTileM * 16,
                                                  kTileM * 16, 128);
                    const uint64_t bd =
                        smem_desc(b_base + (tap * NCH + 2 * ks) * COUT * 16, COUT * 16, 128);
                    mma_bf16(tmem, ad, bd, idesc, (tap | ks) != 0);
                }
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    mbar_a)
                : "memory");
        }
        // a timed-out wait (never expected) ends the kernel on every thread
        ok = __syncthreads_and(mbar_wait(mbar_a, phase) ? 1 : 0) != 0;
        if (!ok) {
            // the MMAs must land before their accumulator is freed: wait once
            // more (bounded) before leaving
            mbar_wait(mbar_a, phase);
            __syncthreads();
            break;
        }
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // epilogue: this thread's row = TMEM lane tid
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
        for (int c0 = 0; c0 < COUT; c0 += 32) {
            float acc[32];
            tmem_ld32(lane_addr + c0, acc);
            if (valid) {
                __nv_bfloat16* out = y + (size_t)p * COUT + c0;
#pragma unroll
                for (int j = 0; j < 32; j += 8) {
                    __align__(16) __nv_bfloat16 o[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        float vq = acc[j + q] + s_bias[c0 + j + q];
                        if (relu) vq = fmaxf(vq, 0.0f);
                        o[q] = __float2bfloat16_rn(vq);
                    }
                    *reinterpret_cast<uint4*>(out + j) = *reinterpret_cast<const uint4*>(o);
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    if (!ok && err) atomicOr(err, 1);
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"((uint32_t)S::kTmemCols));
    }
}

// Row-walking layout for width >= 128: a CTA walks a 128-pixel column strip
// down a band of rows.  Input rows live once in a ring in shared memory,
// [slot][chunk][130 pixels][8 channels] (pixels x0-1 .. x0+128, replicated at
// the borders), so the A operand of tap (dy, dx) is a descriptor view of the
// slot holding row y + dy - 1, shifted by dx pixels (16 bytes): LBO = 130 * 16
// bytes between channel chunks, SBO = 128 bytes between groups of 8 pixels.
constexpr int kHaloPx = kTileM + 2;

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src));
}

// 16 bytes from global memory, or 16 zero bytes when !valid (src is not read)
__device__ __forceinline__ void cp_async16_zfill(uint32_t dst, const void* src, bool valid)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
                 "r"(valid ? 16u : 0u));
}

// Warp-specialised persistent row walk (width >= 128).  Each CTA loops over
// work items (grid, 128-pixel column strip, band of rows); the input rows of
// all its items form one stream through a kWsSlots-deep ring of halo rows in
// shared memory (the layout and descriptor views above).
//
// One input row r feeds three output rows: r + 1 through the kernel row
// dy = 0, r through dy = 1 and r - 1 through dy = 2.  The weights are staged
// as [dx][chunk][dy][cout][8 channels], so for each (dx, K step) the three
// dy blocks are adjacent along N, and the accumulators of consecutive output
// rows sit in adjacent TMEM column blocks of a ring of kAccSlots (output o of
// the CTA's stream at columns Cout * (kAccSlots - 1 - o % kAccSlots)).  One
// MMA with N = 3 Cout then adds row r's contribution to all three outputs:
// the A operand (the 4 KB input view) is read once for three output rows,
// and each input row needs 3 x Cin/16 MMAs.  At the first and last rows of a
// band only the dy blocks whose output lies in the band are issued, and an
// MMA whose column range would wrap around the ring is split in two; this
// plan is made once per input row, so the unrolled issue loop costs two
// descriptor additions per MMA.  Accumulator slots are pre-filled with the
// bias, so every MMA accumulates.
//
// Roles, overlapping through mbarriers:
//   warp 5 (producer): cp.async of input row j into slot j % kWsSlots once the
//     MMAs that read the slot's previous row have completed (empty[slot],
//     arrived by tcgen05.commit); completion signalled with
//     cp.async.mbarrier.arrive on full[slot];
//   warp 4, one thread (MMA): per input row waits for the row and, when it
//     starts a new output row, for that accumulator slot to be refilled;
//     issues the MMAs, commits to empty[] of the row and, when an output row
//     is complete, to out_full[] of its slot;
//   warps 0-3 (epilogue): wait out_full, tcgen05.ld their 32 TMEM lanes,
//     refill the slot with the bias (tcgen05.st) and release it (slot_free),
//     then ReLU + BF16 rounding in one conversion and a store staged through
//     shared memory so that each warp writes contiguous 512-byte runs.
// The weights are staged once per CTA.  Every wait is bounded; on a timeout
// the CTA raises the error flag and all roles leave their loops.
constexpr int kWsSlots = 6;
// Narrower images use the gather kernel.  Measured on 256 images, 64 -> 64:
// width 64 0.171 ms (gather 0.434 ms), width 32 0.088 ms (gather 0.119 ms).
constexpr int kWsMinWidth = 32;
constexpr int kAccSlots = 8;
constexpr int kWsThreads = 192;
constexpr uint32_t kWsSpinLimit = 1u << 22;

// CTAs per SM: the edge layers of a branch (16 -> 32 and the 32 -> 1 layer
// as 32 -> 16) and 32 -> 32 leave room in shared memory, registers and tensor
// memory for two or three CTAs, whose pipelines then hide each other's
// latency; the 64-channel layers take one.
template <int CIN, int COUT, bool OUT1>
constexpr int ws_ctas_per_sm()
{
    return OUT1 ? 3 : (CIN == 16 || (CIN == 32 && COUT == 32)) ? 2 : 1;
}

// OUT1: the layer has one output channel (the last convolution of a
// branch), computed as channel 0 of COUT = 16 (the other weights are zero)
// and stored as FP32 [P] without rounding.
template <int CIN, int COUT, bool OUT1 = false>
struct WsSmem {
    static constexpr int kChunks = CIN / 8;
    static constexpr int kSlotBytes = kChunks * kHaloPx * 16;
    static constexpr int kRingBytes = kWsSlots * kSlotBytes;
    static constexpr int kBBytes = 9 * kChunks * COUT * 16;
    // per epilogue warp: its 32 output pixels in BF16, 16-byte chunks XOR-swizzled
    static constexpr int kStageBytes = OUT1 ? 0 : 4 * 32 * COUT * 2;
    static constexpr int kBytes = kRingBytes + kBBytes + kStageBytes;
    static constexpr int kTmemCols = kAccSlots * COUT;  // 128, 256 or 512
    static constexpr int kCtas = ws_ctas_per_sm<CIN, COUT, OUT1>();
    // shared memory requested per CTA: enough that no more than kCtas CTAs
    // share an SM (228 KB, 1 KB reserved per CTA), so their tensor memory
    // (kCtas x kTmemCols <= 512 columns) always fits
    static constexpr int kSmemRequest =
        kCtas == 1 || kBytes > 228 * 1024 / (kCtas + 1) ? kBytes : 228 * 1024 / (kCtas + 1) + 1;
    static_assert(COUT == 32 || COUT == 64 || (COUT == 16 && OUT1),
                  "accumulator ring sized for 32 or 64 channels (16 for one output)");
    static_assert(CIN % 16 == 0, "K steps of 16 channels");
    static_assert(kCtas * kTmemCols <= 512, "tensor memory of the CTAs that share an SM");
    static_assert(kCtas * (kSmemRequest + 1024) <= 228 * 1024, "shared memory per SM");
};

// A bounded wait on an mbarrier phase: gives up after `limit` polls, or
// earlier once another role of the CTA has raised abort_flag.
__device__ __forceinline__ bool mbar_wait_ws(uint32_t mbar, uint32_t parity,
                                             const volatile int* abort_flag,
                                             uint32_t limit = kWsSpinLimit)
{
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 1023u) == 1023u && *abort_flag) return false;
    }
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
        : "memory");
}

// 32 consecutive 32-bit TMEM columns of this thread's lane, without the wait.
__device__ __forceinline__ void tmem_ld32_raw(uint32_t taddr, uint32_t* r)
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
        "%28, %29, %30, %31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
}

// Write 32 consecutive 32-bit TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t* r)
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, "
        "%10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, "
        "%27, %28, %29, %30, %31, %32};\n" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
        "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]),
        "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]),
        "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
}

// 16 consecutive 32-bit TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t* r)
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, "
        "%10, %11, %12, %13, %14, %15, %16};\n" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
        "r"(r[15])
        : "memory");
}

// One 32-bit TMEM column of this thread's lane, without the wait.
__device__ __forceinline__ uint32_t tmem_ld1_raw(uint32_t taddr)
{
    uint32_t r;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];\n" : "=r"(r) : "r"(taddr));
    return r;
}

// An accumulator slot (COUT columns) set to the given 32-bit values.
template <int COUT>
__device__ __forceinline__ void tmem_fill(uint32_t taddr, const uint32_t* bits)
{
    if (COUT % 32 == 0) {
#pragma unroll
        for (int c0 = 0; c0 < COUT; c0 += 32) tmem_st32(taddr + c0, bits + c0);
    } else {
        tmem_st16(taddr, bits);
    }
}

// Two FP32 values to packed BF16 (lo in the low half), round to nearest even,
// optionally with ReLU in the same conversion.
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi, bool relu)
{
    uint32_t d;
    if (relu)
        asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    else
        asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

// Two packed BF16 values v kept where the matching BF16 value of a is
// positive, zeroed elsewhere.
__device__ __forceinline__ uint32_t relu_mask2(uint32_t v, uint32_t a)
{
    uint32_t m = 0;
    if ((a & 0xFFFFu) != 0u && !(a & 0x8000u)) m |= 0xFFFFu;
    if ((a >> 16) != 0u && !(a & 0x80000000u)) m |= 0xFFFF0000u;
    return v & m;
}

struct WsItem {
    int b, x0, y0, y1;
};

__device__ __forceinline__ WsItem ws_item(int w, int segs, int nbands, int band, int H)
{
    WsItem it;
    const int seg = w % segs;
    const int t = w / segs;
    const int bi = t % nbands;
    it.b = t / nbands;
    it.x0 = seg * kTileM;
    it.y0 = bi * band;
    it.y1 = min(H, it.y0 + band);
    return it;
}

__device__ __forceinline__ uint32_t idesc_for_rows(int n_out, int cout)
{
    return n_out == 1 ? mma_idesc(kTileM, cout)
           : n_out == 2 ? mma_idesc(kTileM, 2 * cout)
                        : mma_idesc(kTileM, 3 * cout);
}

// DGRAD: the input gradient of a convolution as the convolution of the output
// gradient x with the flipped, transposed weights w: zero padding instead of
// replicated borders (the border terms of the replicated padding are added
// by a separate pass), and in the epilogue every value whose activation in
// act (same layout as the output) is not positive is zeroed (the ReLU
// derivative of the layer that produced act; act may be null).
template <int CIN, int COUT, bool OUT1, bool DGRAD = false>
__global__ void __launch_bounds__(kWsThreads, (ws_ctas_per_sm<CIN, COUT, OUT1>()))
    conv3x3_tc_ws_kernel(const uint4* __restrict__ x, const uint4* __restrict__ w,
                         const float* __restrict__ bias, void* __restrict__ yout, int H, int W,
                         int segs, int nbands, int band, int items, int relu, int* err,
                         uint32_t wait_limit, const uint4* __restrict__ act = nullptr)
{
    using S = WsSmem<CIN, COUT, OUT1>;
    // polls of each pipeline wait before it gives up (0: the compiled limit);
    // the final waits for issued MMAs always use the compiled limit
    const uint32_t lim = wait_limit ? wait_limit : kWsSpinLimit;
    __nv_bfloat16* __restrict__ y = reinterpret_cast<__nv_bfloat16*>(yout);
    constexpr int NCH = S::kChunks;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* ring = smem;
    uint8_t* sB = smem + S::kRingBytes;
    __shared__ __align__(8) uint64_t full_bar[kWsSlots];
    __shared__ __align__(8) uint64_t empty_bar[kWsSlots];
    __shared__ __align__(8) uint64_t outf_bar[kAccSlots];
    __shared__ __align__(8) uint64_t free_bar[kAccSlots];
    __shared__ uint32_t tmem_base;
    __shared__ float s_bias[COUT];
    __shared__ volatile int s_abort;

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"((uint32_t)S::kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int s = 0; s < kWsSlots; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full_bar[s])),
                         "r"(32u));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty_bar[s])),
                         "r"(1u));
        }
        for (int k = 0; k < kAccSlots; ++k) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&outf_bar[k])),
                         "r"(1u));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&free_bar[k])),
                         "r"(4u));
        }
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    for (int i = tid; i < COUT; i += kWsThreads) s_bias[i] = bias[i];
    // weights [tap = 3 dy + dx][cout][chunk] -> [dx][chunk][dy][cout] (16 B each)
    for (int i = tid; i < 9 * COUT * NCH; i += kWsThreads) {
        const int ch = i % NCH;
        const int n = (i / NCH) % COUT;
        const int tap = i / (NCH * COUT);
        const int dy = tap / 3, dx = tap - 3 * (tap / 3);
        const uint4 v = w[(size_t)(tap * COUT + n) * NCH + ch];
        *reinterpret_cast<uint4*>(sB + (((dx * NCH + ch) * 3 + dy) * COUT + n) * 16) = v;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
    // the bias as raw bits, the value every accumulator slot starts from
    uint32_t bias_bits[COUT];
#pragma unroll
    for (int c = 0; c < COUT; ++c) bias_bits[c] = __float_as_uint(s_bias[c]);
    if (warp < 4) {
#pragma unroll
        for (int sl = 0; sl < kAccSlots; ++sl)
            tmem_fill<COUT>(tmem + lane_off + (uint32_t)(sl * COUT), bias_bits);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // Launched as a programmatic dependent of the layer before it, the
    // prologue above (tensor memory, barriers, weights, bias) overlaps that
    // layer's end; the inputs are read, and the outputs written, only once it
    // has completed.  The next layer may then start its own prologue.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    bool ok = true;

    if (warp == 5) {
        // ---------------------------------------------------------- producer
        // lane: channel chunk ch of pixels p0, p0 + kPass, ...; a warp copies
        // kPass whole pixels (512 contiguous bytes) per instruction
        constexpr int kPass = 32 / NCH;
        const int ch = lane % NCH, p0 = lane / NCH;
        uint32_t jg = 0;
        for (int wi = blockIdx.x; wi < items && ok; wi += gridDim.x) {
            const WsItem it = ws_item(wi, segs, nbands, band, H);
            const bool interior = it.x0 >= 1 && it.x0 + kHaloPx - 1 <= W;
            for (int r = it.y0 - 1; r <= it.y1 && ok; ++r, ++jg) {
                const uint32_t s = jg % kWsSlots, u = jg / kWsSlots;
                // the lanes take one decision (no lane runs ahead of the others)
                if (u > 0)
                    ok = __all_sync(0xffffffffu,
                                    mbar_wait_ws(smem_u32(&empty_bar[s]), (u - 1) & 1u, &s_abort,
                                                 lim));
                if (!ok) break;
                const int sr = min(max(r, 0), H - 1);
                const uint32_t dst = smem_u32(ring + s * S::kSlotBytes) + (uint32_t)(ch * kHaloPx * 16);
                const uint4* src_row = x + ((size_t)it.b * H + sr) * W * NCH + ch;
                if constexpr (DGRAD) {
                    // zero outside the image
                    const bool row_in = r >= 0 && r < H;
                    for (int px = p0; px < kHaloPx; px += kPass) {
                        const int gx = it.x0 - 1 + px;
                        const int sx = min(max(gx, 0), W - 1);
                        cp_async16_zfill(dst + (uint32_t)(px * 16), src_row + (size_t)sx * NCH,
                                         row_in && gx >= 0 && gx < W);
                    }
                } else if (interior) {
                    const uint4* src = src_row + (size_t)(it.x0 - 1 + p0) * NCH;
#pragma unroll 4
                    for (int px = p0; px < kHaloPx; px += kPass, src += kPass * NCH)
                        cp_async16(dst + (uint32_t)(px * 16), src);
                } else {
                    for (int px = p0; px < kHaloPx; px += kPass) {
                        const int sx = min(max(it.x0 - 1 + px, 0), W - 1);
                        cp_async16(dst + (uint32_t)(px * 16), src_row + (size_t)sx * NCH);
                    }
                }
                asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(
                                 smem_u32(&full_bar[s]))
                             : "memory");
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else if (warp == 4) {
        // --------------------------------------------------------------- MMA
        if (lane == 0) {
            const uint64_t a_hi = smem_desc(0, kHaloPx * 16, 128);
            const uint64_t bd_base = smem_desc(smem_u32(sB), 3 * COUT * 16, 128);
            const uint32_t ring_a = smem_u32(ring);
            uint32_t jg = 0, og = 0;
            int last_row = -1, last_out = -1;
            for (int wi = blockIdx.x; wi < items && ok; wi += gridDim.x) {
                const WsItem it = ws_item(wi, segs, nbands, band, H);
                for (int r = it.y0 - 1; r <= it.y1 && ok; ++r, ++jg) {
                    ok = mbar_wait_ws(smem_u32(&full_bar[jg % kWsSlots]),
                                      (jg / kWsSlots) & 1u, &s_abort, lim);
                    // dy blocks whose output row r + 1 - dy lies in [y0, y1)
                    const int dlo = max(0, r + 2 - it.y1), dhi = min(2, r + 1 - it.y0);
                    const int nd = dhi - dlo + 1;
                    const uint32_t o_first = og + (uint32_t)(r + 1 - dlo - it.y0);
                    if (ok && dlo == 0 && o_first >= (uint32_t)kAccSlots)
                        ok = mbar_wait_ws(smem_u32(&free_bar[o_first % kAccSlots]),
                                          ((o_first / kAccSlots) - 1) & 1u, &s_abort, lim);
                    if (!ok) break;
                    // plan: outputs o_first, o_first - 1, ... in at most two
                    // runs of adjacent TMEM column blocks (split at the wrap)
                    const int m = (int)(o_first % kAccSlots);
                    const int len0 = nd < m + 1 ? nd : m + 1;
                    const int len1 = nd - len0;
                    const uint32_t d0 = tmem + (uint32_t)(COUT * (kAccSlots - 1 - m));
                    const uint32_t d1 = tmem;  // the run after the wrap starts at slot 0
                    const uint32_t id0 = idesc_for_rows(len0, COUT);
                    const uint32_t id1 = idesc_for_rows(len1 > 0 ? len1 : 1, COUT);
                    // B row offsets (16-byte units) of the first dy block of each run
                    const uint64_t b0 = bd_base + (uint64_t)(dlo * COUT);
                    const uint64_t b1 = bd_base + (uint64_t)((dlo + len0) * COUT);
                    const uint64_t ad_row =
                        a_hi | (uint64_t)((ring_a + (jg % kWsSlots) * S::kSlotBytes) >> 4);
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx) {
#pragma unroll
                        for (int ks = 0; ks < NCH / 2; ++ks) {
                            // A: input view shifted by dx pixels, channel chunk 2 ks;
                            // B: weights of (dx, chunk 2 ks)
                            const uint64_t ad = ad_row + (uint64_t)(2 * ks * kHaloPx + dx);
                            const uint64_t boff = (uint64_t)((dx * NCH + 2 * ks) * 3 * COUT);
                            mma_bf16(d0, ad, b0 + boff, id0, 1u);
                            if (len1 > 0) mma_bf16(d1, ad, b1 + boff, id1, 1u);
                        }
                    }
                    if constexpr (DGRAD) {
                        // ghost output rows -1 and H of the zero-padded
                        // transpose, folded into rows 0 and H - 1 (the
                        // replicated border); both are still accumulating
                        // while input rows 0 and H - 1 are issued
                        for (int f = 0; f < 2; ++f) {
                            const bool fold = f == 0 ? (r == 0 && it.y0 == 0)
                                                     : (r == H - 1 && it.y1 == H);
                            if (!fold) continue;
                            const int o = f == 0 ? 0 : H - 1;
                            const int dsrc = f == 0 ? 2 : 0;  // block of output row -1 / H
                            const uint32_t sl =
                                (og + (uint32_t)(o - it.y0)) % (uint32_t)kAccSlots;
                            const uint32_t dd = tmem + (uint32_t)(COUT * (kAccSlots - 1 - (int)sl));
                            const uint32_t idf = idesc_for_rows(1, COUT);
#pragma unroll
                            for (int dx = 0; dx < 3; ++dx)
#pragma unroll
                                for (int ks = 0; ks < NCH / 2; ++ks) {
                                    const uint64_t ad = ad_row + (uint64_t)(2 * ks * kHaloPx + dx);
                                    const uint64_t boff =
                                        (uint64_t)((dx * NCH + 2 * ks) * 3 * COUT + dsrc * COUT);
                                    mma_bf16(dd, ad, bd_base + boff, idf, 1u);
                                }
                        }
                    }
                    mma_commit(smem_u32(&empty_bar[jg % kWsSlots]));
                    last_row = (int)jg;
                    if (dhi == 2) {
                        // output row r - 1 has all three contributions
                        const uint32_t o_done = og + (uint32_t)(r - 1 - it.y0);
                        mma_commit(smem_u32(&outf_bar[o_done % kAccSlots]));
                        last_out = (int)o_done;
                    }
                }
                og += (uint32_t)(it.y1 - it.y0);
            }
            // the MMAs and the arrivals of the last commits must have landed
            // before the accumulators are freed and the CTA exits (also on
            // the error path)
            const volatile int no_abort = 0;
            bool drained = true;
            if (last_row >= 0)
                drained = mbar_wait_ws(smem_u32(&empty_bar[last_row % kWsSlots]),
                                       ((uint32_t)last_row / kWsSlots) & 1u, &no_abort);
            if (last_out >= 0 && drained)
                drained = mbar_wait_ws(smem_u32(&outf_bar[last_out % kAccSlots]),
                                       ((uint32_t)last_out / kAccSlots) & 1u, &no_abort);
            ok = ok && drained;
        }
    } else {
        // ---------------------------------------------------------- epilogue
        constexpr int CPP = COUT / 8;  // 16-byte chunks per pixel
        auto stage_swz = [](int p) { return (p / (8 / CPP)) & (CPP - 1); };
        uint8_t* stage = sB + S::kBBytes + warp * 32 * COUT * 2;
        const bool do_relu = relu != 0;
        uint32_t og = 0;
        for (int wi = blockIdx.x; wi < items && ok; wi += gridDim.x) {
            const WsItem it = ws_item(wi, segs, nbands, band, H);
            for (int yy = it.y0; yy < it.y1; ++yy, ++og) {
                const uint32_t sl = og % kAccSlots;
                // DGRAD: this lane's activation chunks of the row, loaded while
                // the MMAs of the row are still running
                uint4 act_r[DGRAD ? CPP : 1];
                if constexpr (DGRAD) {
                    if (act) {
#pragma unroll
                        for (int i = 0; i < CPP; ++i) {
                            const int k = lane + 32 * i;
                            const int p = k / CPP, c = k % CPP;
                            const int xo = it.x0 + warp * 32 + p;
                            act_r[i] = xo < W ? act[(((size_t)it.b * H + yy) * W + xo) * CPP + c]
                                              : make_uint4(0u, 0u, 0u, 0u);
                        }
                    }
                }
                // one decision per warp: the tcgen05.ld below is warp-collective
                ok = __all_sync(0xffffffffu, mbar_wait_ws(smem_u32(&outf_bar[sl]),
                                                          (og / kAccSlots) & 1u, &s_abort, lim));
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t taddr =
                    tmem + lane_off + (uint32_t)(COUT * (kAccSlots - 1 - (int)sl));
                if constexpr (OUT1) {
                    // channel 0 only, FP32 (bias included by the slot's fill)
                    const uint32_t v = tmem_ld1_raw(taddr);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    tmem_fill<COUT>(taddr, bias_bits);
                    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&free_bar[sl]));
                    const int xo = it.x0 + warp * 32 + lane;
                    if (xo < W)
                        reinterpret_cast<float*>(yout)[((size_t)it.b * H + yy) * W + xo] =
                            __uint_as_float(v);
                    continue;
                } else {
                uint32_t acc[COUT];
#pragma unroll
                for (int c0 = 0; c0 < COUT; c0 += 32) tmem_ld32_raw(taddr + c0, acc + c0);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                // refill the slot with the bias for the output row that reuses it
                tmem_fill<COUT>(taddr, bias_bits);
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&free_bar[sl]));
                // the warp's 32 pixels go through shared memory so that the
                // global stores are contiguous: chunk c of pixel p (16 bytes,
                // 8 channels) sits at position c ^ swz(p), conflict-free on
                // both sides
#pragma unroll
                for (int c = 0; c < CPP; ++c) {
                    uint4 o;
                    o.x = pack_bf16x2(__uint_as_float(acc[8 * c + 0]),
                                      __uint_as_float(acc[8 * c + 1]), do_relu);
                    o.y = pack_bf16x2(__uint_as_float(acc[8 * c + 2]),
                                      __uint_as_float(acc[8 * c + 3]), do_relu);
                    o.z = pack_bf16x2(__uint_as_float(acc[8 * c + 4]),
                                      __uint_as_float(acc[8 * c + 5]), do_relu);
                    o.w = pack_bf16x2(__uint_as_float(acc[8 * c + 6]),
                                      __uint_as_float(acc[8 * c + 7]), do_relu);
                    *reinterpret_cast<uint4*>(stage + lane * (COUT * 2) +
                                              ((c ^ stage_swz(lane)) * 16)) = o;
                }
                __syncwarp();
                __nv_bfloat16* row = y + (((size_t)it.b * H + yy) * W + it.x0 + warp * 32) * COUT;
#pragma unroll
                for (int i = 0; i < CPP; ++i) {
                    const int k = lane + 32 * i;
                    const int p = k / CPP, c = k % CPP;
                    uint4 v = *reinterpret_cast<const uint4*>(
                        stage + p * (COUT * 2) + ((c ^ stage_swz(p)) * 16));
                    if (it.x0 + warp * 32 + p < W) {
                        if constexpr (DGRAD) {
                            if (act) {
                                const uint4 a = act_r[i];
                                v.x = relu_mask2(v.x, a.x);
                                v.y = relu_mask2(v.y, a.y);
                                v.z = relu_mask2(v.z, a.z);
                                v.w = relu_mask2(v.w, a.w);
                            }
                        }
                        *reinterpret_cast<uint4*>(row + (size_t)p * COUT + 8 * c) = v;
                    }
                }
                __syncwarp();
                }
            }
        }
    }
    if (!ok) {
        s_abort = 1;
        if (err) atomicOr(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"((uint32_t)S::kTmemCols));
    }
}

// warp-specialised row walk, one persistent CTA per SM; bands sized for about
// eight work items per CTA (an image narrower than 128 pixels is one strip
// whose pixels past its width are clamped on load and not stored)
template <int CIN, int COUT, bool OUT1, bool DGRAD = false>
hp_status launch_ws(const void* x, const void* w, const float* bias, void* y, int B, int H,
                    int W, int relu, int* err, int nsm, cudaStream_t st,
                    const void* act = nullptr, uint32_t wait_limit = 0, bool pdl = false)
{
    using R = WsSmem<CIN, COUT, OUT1>;
    static bool rattr = false;
    if (!rattr) {
        cudaError_t e = cudaFuncSetAttribute(conv3x3_tc_ws_kernel<CIN, COUT, OUT1, DGRAD>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             R::kSmemRequest);
        if (e != cudaSuccess) { set_cuda_error(e); return HP_ERR_CUDA; }
        rattr = true;
    }
    const int segs = (W + kTileM - 1) / kTileM;
    const long rows = (long)B * H * segs;
    const long ctas = (long)R::kCtas * nsm;
    int band = (int)((rows + 8L * ctas - 1) / (8L * ctas));
    band = band < 4 ? 4 : band > H ? H : band;
    const int nbands = (H + band - 1) / band;
    const long items = (long)B * segs * nbands;
    if (items > 0x7fffffffL) return HP_ERR_INVALID_ARG;
    const int grid = items < ctas ? (int)items : (int)ctas;
    // pdl: a programmatic dependent of the kernel before it in the stream
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kWsThreads);
    cfg.dynamicSmemBytes = R::kSmemRequest;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    cudaError_t e = cudaLaunchKernelEx(&cfg, conv3x3_tc_ws_kernel<CIN, COUT, OUT1, DGRAD>,
                                       (const uint4*)x, (const uint4*)w, bias, y, H, W, segs,
                                       nbands, band, (int)items, relu, err, wait_limit,
                                       (const uint4*)act);
    if (e != cudaSuccess) { set_cuda_error(e); return HP_ERR_CUDA; }
    return check_launch();
}

// ---------------------------------------------------------------------------
// Weight gradient of a 3 x 3 convolution with replicated borders on the
// tensor cores:
//     gW[dy][dx][co][ci] = sum over pixels p of gy[p][co] * x[clamp(p + (dy, dx))][ci]
// Per 128-pixel row segment of an output-gradient row r this is a GEMM over
// K = the 130 input pixels x0 - 1 .. x0 + 128 (padded to 144, 9 steps of 16):
//   A = input rows (M = 128 = kRows rows x CI channels), taken MN-major straight
//       from an input-row ring laid out [row][channel chunk][pixel][8 channels]
//       with replicated halo pixels; consecutive rows are adjacent in shared
//       memory (the first kRows - 1 ring slots are mirrored after the last),
//       so one descriptor spans kRows rows;
//   B = the gradient row in three copies shifted by dx (pixel q of copy dx
//       holds gy[q - dx], zero outside the segment), N = 3 CO, MN-major;
//   D = TMEM, lane (row i of the tile, ci), column (dx, co), accumulating over
//       every row and segment the CTA visits.
// CI = 64: two tiles per gradient row, input rows (r-1, r) and (r, r+1) (the
// second tile's r half repeats the first and is not read out); CI = 32: one
// tile of rows r-1 .. r+2 (the r+2 quarter is not read out and may hold any
// row).  Warps 0-3 load (cp.async) and finally read the accumulators out to
// per-CTA partial sums part[cta][3 dy + dx][co][ci]; warp 4 issues the MMAs.
constexpr int kWgPx = 144;
constexpr int kWgThreads = 160;

template <int CI, int CO>
struct WgSmem {
    static constexpr int kChunksX = CI / 8, kChunksG = CO / 8;
    // bytes per channel chunk of a row: 144 pixels plus 16 bytes, so that the
    // chunks of one pixel fall in different shared-memory banks (the
    // producers write them together)
    static constexpr int kStride = kWgPx * 16 + 16;
    static constexpr int kSlotBytes = kChunksX * kStride;
    static constexpr int kRows = 128 / CI;
    static constexpr int kSlots = kRows == 2 ? 4 : 5;
    static constexpr int kMirror = kRows - 1;
    static constexpr int kRingBytes = (kSlots + kMirror) * kSlotBytes;
    static constexpr int kGBytes = 3 * kChunksG * kStride;
    static constexpr int kTiles = kRows == 2 ? 2 : 1;
    static constexpr int kN = 3 * CO;
    static constexpr int kBytes = kRingBytes + 2 * kGBytes;
    static constexpr int kTmemCols = kTiles * kN <= 128 ? 128 : kTiles * kN <= 256 ? 256 : 512;
    static_assert(CI == 32 || CI == 64, "input channels 32 or 64");
    static_assert(CO == 32 || CO == 64, "output channels 32 or 64");
    static_assert(kBytes <= 227 * 1024, "shared memory");
};

template <int CI, int CO>
__global__ void __launch_bounds__(kWgThreads, 1)
    conv3x3_wgrad_tc_kernel(const uint4* __restrict__ x, const uint4* __restrict__ gy,
                            float* __restrict__ part, float* __restrict__ partb, int H, int W,
                            int segs, int nbands, int band, int items, int* err,
                            uint32_t wait_limit)
{
    using S = WgSmem<CI, CO>;
    // polls of each pipeline wait before it gives up (0: the compiled limit);
    // the waits for the issued MMAs (done_bar) always use the compiled limit
    const uint32_t lim = wait_limit ? wait_limit : kWsSpinLimit;
    constexpr int NX = S::kChunksX, NG = S::kChunksG;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* ring = smem;
    uint8_t* gbuf = smem + S::kRingBytes;
    __shared__ __align__(8) uint64_t xfull[S::kSlots];
    __shared__ __align__(8) uint64_t xempty[S::kSlots];
    __shared__ __align__(8) uint64_t gfull[2];
    __shared__ __align__(8) uint64_t gempty[2];
    __shared__ __align__(8) uint64_t done_bar;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int s_abort;
    __shared__ float s_bias[128][8];

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    // bias-gradient partial sums of the producer threads: channels 8 (tid % NG)
    // .. + 7 over the pixels of every gradient row this CTA loads
    float bacc[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"((uint32_t)S::kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int i = 0; i < S::kSlots; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&xfull[i])),
                         "r"(128u));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&xempty[i])),
                         "r"(1u));
        }
        for (int i = 0; i < 2; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&gfull[i])),
                         "r"(128u));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&gempty[i])),
                         "r"(1u));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&done_bar)),
                     "r"(1u));
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    // pixels 130..143 of every input row are never loaded: zero them once so
    // that the MMAs read finite values there (the gradient copies are zero
    // at those pixels)
    for (int i = tid; i < (S::kSlots + S::kMirror) * NX * (kWgPx - kHaloPx); i += kWgThreads) {
        const int px = kHaloPx + i % (kWgPx - kHaloPx);
        const int ch = (i / (kWgPx - kHaloPx)) % NX;
        const int sl = i / ((kWgPx - kHaloPx) * NX);
        *reinterpret_cast<uint4*>(ring + sl * S::kSlotBytes + ch * S::kStride + px * 16) =
            make_uint4(0u, 0u, 0u, 0u);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    bool ok = true;

    if (warp < 4) {
        // ---------------------------------------------------------- producer
        uint32_t xpos = 0, gcnt = 0;
        uint4 pend[NG];
#pragma unroll
        for (int i = 0; i < NG; ++i) pend[i] = make_uint4(0u, 0u, 0u, 0u);
        auto add_pend = [&]() {
#pragma unroll
            for (int i = 0; i < NG; ++i) {
                const uint32_t e[4] = {pend[i].x, pend[i].y, pend[i].z, pend[i].w};
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    bacc[2 * h] += __uint_as_float(e[h] << 16);
                    bacc[2 * h + 1] += __uint_as_float(e[h] & 0xFFFF0000u);
                }
                pend[i] = make_uint4(0u, 0u, 0u, 0u);
            }
        };
        auto load_x = [&](int b, int x0, int r, uint32_t pos) -> bool {
            const uint32_t sl = pos % S::kSlots, u = pos / S::kSlots;
            if (u > 0 && !mbar_wait_ws(smem_u32(&xempty[sl]), (u - 1) & 1u, &s_abort, lim))
                return false;
            const int sr = min(max(r, 0), H - 1);
            const uint4* src_row = x + ((size_t)b * H + sr) * W * NX;
            const uint32_t dst = smem_u32(ring + sl * S::kSlotBytes);
            const uint32_t dst2 = smem_u32(ring + (S::kSlots + sl) * S::kSlotBytes);
            for (int q = tid; q < kHaloPx * NX; q += 128) {
                const int ch = q % NX, px = q / NX;
                const int sx = min(max(x0 - 1 + px, 0), W - 1);
                const uint4* src = src_row + (size_t)sx * NX + ch;
                const uint32_t off = (uint32_t)(ch * S::kStride + px * 16);
                cp_async16(dst + off, src);
                if (sl < (uint32_t)S::kMirror) cp_async16(dst2 + off, src);
            }
            asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(
                             smem_u32(&xfull[sl]))
                         : "memory");
            return true;
        };
        auto load_g = [&](int b, int x0, int r, uint32_t cnt) -> bool {
            const uint32_t bb = cnt & 1u, u = cnt >> 1;
            if (u > 0 && !mbar_wait_ws(smem_u32(&gempty[bb]), (u - 1) & 1u, &s_abort, lim))
                return false;
            const uint4* src_row = gy + ((size_t)b * H + r) * W * NG;
            const uint32_t dst = smem_u32(gbuf + bb * S::kGBytes);
            const int xend = min(x0 + kTileM, W);
            for (int q = tid; q < 3 * kWgPx * NG; q += 128) {
                const int ch = q % NG, k = (q / NG) % kWgPx, dx = q / (NG * kWgPx);
                const int col = x0 + k - dx;  // gradient pixel at input pixel x0 - 1 + k
                const bool valid = col >= x0 && col < xend;
                const uint4* src = src_row + (size_t)(valid ? col : x0) * NG + ch;
                cp_async16_zfill(dst + (uint32_t)((dx * NG + ch) * S::kStride + k * 16), src, valid);
            }
            asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(
                             smem_u32(&gfull[bb]))
                         : "memory");
            // bias sums: the previous row's values (loaded one row earlier, so
            // that their latency overlaps) are added, this row's are loaded
            add_pend();
            const int chb = tid % NG;
#pragma unroll
            for (int i = 0; i < NG; ++i) {
                const int j = tid / NG + i * (128 / NG);
                pend[i] = x0 + j < xend ? src_row[(size_t)(x0 + j) * NG + chb]
                                        : make_uint4(0u, 0u, 0u, 0u);
            }
            return true;
        };
        for (int wi = blockIdx.x; wi < items && ok; wi += gridDim.x) {
            const WsItem it = ws_item(wi, segs, nbands, band, H);
            ok = load_x(it.b, it.x0, it.y0 - 1, xpos++) && load_x(it.b, it.x0, it.y0, xpos++);
            for (int r = it.y0; r < it.y1 && ok; ++r) {
                ok = load_x(it.b, it.x0, r + 1, xpos++) && load_g(it.b, it.x0, r, gcnt++);
            }
        }
        add_pend();
        if (!ok) s_abort = 1;  // the MMA thread stops waiting for rows
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else if (lane == 0) {
        // --------------------------------------------------------------- MMA
        constexpr uint32_t idesc = mma_idesc(128, S::kN) | (1u << 15) | (1u << 16);
        const uint32_t ring_a = smem_u32(ring), g_a = smem_u32(gbuf);
        uint32_t xpos = 0, gcnt = 0;
        bool first = true;
        for (int wi = blockIdx.x; wi < items && ok; wi += gridDim.x) {
            const WsItem it = ws_item(wi, segs, nbands, band, H);
            const uint32_t p0 = xpos;
            const int nb = it.y1 - it.y0;
            for (int i = 0; i < nb && ok; ++i) {
                // input rows at positions p0 + i .. p0 + i + 2 (the first two
                // were waited for by the previous row unless i == 0)
                for (uint32_t pos = p0 + (i == 0 ? 0u : (uint32_t)i + 2u);
                     pos <= p0 + (uint32_t)i + 2u && ok; ++pos)
                    ok = mbar_wait_ws(smem_u32(&xfull[pos % S::kSlots]),
                                      (pos / S::kSlots) & 1u, &s_abort, lim);
                if (ok)
                    ok = mbar_wait_ws(smem_u32(&gfull[gcnt & 1u]), (gcnt >> 1) & 1u, &s_abort,
                                      lim);
                if (!ok) break;
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t gb_a = g_a + (gcnt & 1u) * S::kGBytes;
#pragma unroll
                for (int t = 0; t < S::kTiles; ++t) {
                    const uint32_t a0 = ring_a + ((p0 + (uint32_t)(i + t)) % S::kSlots) * S::kSlotBytes;
#pragma unroll
                    for (int ks = 0; ks < kWgPx / 16; ++ks) {
                        const uint64_t ad = smem_desc(a0 + ks * 256, 128, S::kStride);
                        const uint64_t bd = smem_desc(gb_a + ks * 256, 128, S::kStride);
                        mma_bf16(tmem + (uint32_t)(t * S::kN), ad, bd, idesc,
                                 (first && ks == 0) ? 0u : 1u);
                    }
                }
                first = false;
                mma_commit(smem_u32(&gempty[gcnt & 1u]));
                ++gcnt;
                // input row p0 + i is not read again; after the last row of the
                // item neither are the two after it
                mma_commit(smem_u32(&xempty[(p0 + (uint32_t)i) % S::kSlots]));
                if (i == nb - 1) {
                    mma_commit(smem_u32(&xempty[(p0 + (uint32_t)i + 1u) % S::kSlots]));
                    mma_commit(smem_u32(&xempty[(p0 + (uint32_t)i + 2u) % S::kSlots]));
                }
            }
            xpos = p0 + (uint32_t)nb + 2u;
        }
        if (!ok) s_abort = 1;
        // every MMA issued must have landed before the accumulators are read
        // or freed, also on the error path
        mma_commit(smem_u32(&done_bar));
        const volatile int no_abort = 0;
        if (!mbar_wait_ws(smem_u32(&done_bar), 0u, &no_abort)) ok = false;
    }
    // ------------------------------------------------------------- epilogue
    if (warp < 4) {
        // the MMA thread commits done_bar on every path, so this wait ends
        // once its MMAs have landed (abort only shortens the error path)
        const volatile int no_abort = 0;
        const bool landed = mbar_wait_ws(smem_u32(&done_bar), 0u, &no_abort);
        if (!landed) ok = false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int L = warp * 32 + lane;  // TMEM lane = GEMM row
        const int ci = L % CI, ri = L / CI;
        const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
        float* dst = part + (size_t)blockIdx.x * 9 * CO * CI;
#pragma unroll
        for (int t = 0; t < S::kTiles; ++t) {
            // tile t row ri is input row r - 1 + t + ri, i.e. dy index t + ri
            const int dyi = t + ri;
            const bool keep = landed && (S::kTiles == 2 ? (t == 0 || ri == 1) : ri < 3);
#pragma unroll
            for (int c0 = 0; c0 < S::kN; c0 += 32) {
                uint32_t v[32];
                tmem_ld32_raw(tmem + lane_off + (uint32_t)(t * S::kN + c0), v);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (keep) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int n = c0 + j, dxi = n / CO, co = n % CO;
                        dst[((size_t)(3 * dyi + dxi) * CO + co) * CI + ci] = __uint_as_float(v[j]);
                    }
                }
            }
        }
    }
    if (!ok) {
        s_abort = 1;
        if (err) atomicOr(err, 1);
    }
    if (warp < 4) {
#pragma unroll
        for (int k = 0; k < 8; ++k) s_bias[tid][k] = bacc[k];
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"((uint32_t)S::kTmemCols));
    }
    // bias partial of the CTA: the producer threads of each channel chunk,
    // in a fixed order
    if (tid < CO) {
        const int chb = tid / 8, k = tid % 8;
        float t = 0.0f;
        for (int q = chb; q < 128; q += NG) t += s_bias[q][k];
        partb[(size_t)blockIdx.x * CO + tid] = t;
    }
}

template <int CI, int CO>
hp_status launch_wgrad_t(const void* x, const void* gy, float* part, size_t part_len,
                         float* partb, size_t partb_len, int B, int H, int W, int* err, int nsm,
                         int* grid_out, cudaStream_t st, uint32_t wait_limit)
{
    using S = WgSmem<CI, CO>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(conv3x3_wgrad_tc_kernel<CI, CO>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, S::kBytes);
        if (e != cudaSuccess) { set_cuda_error(e); return HP_ERR_CUDA; }
        attr = true;
    }
    const int segs = (W + kTileM - 1) / kTileM;
    const long rows = (long)B * H * segs;
    int band = (int)((rows + 4L * nsm - 1) / (4L * nsm));
    band = band < 2 ? 2 : band > H ? H : band;
    const int nbands = (H + band - 1) / band;
    const long items = (long)B * segs * nbands;
    if (items > 0x7fffffffL) return HP_ERR_INVALID_ARG;
    const int grid = items < nsm ? (int)items : nsm;
    if ((size_t)grid * 9 * CO * CI > part_len || (size_t)grid * CO > partb_len)
        return HP_ERR_INVALID_ARG;
    conv3x3_wgrad_tc_kernel<CI, CO><<<grid, kWgThreads, S::kBytes, st>>>(
        (const uint4*)x, (const uint4*)gy, part, partb, H, W, segs, nbands, band, (int)items, err,
        wait_limit);
    *grid_out = grid;
    return check_launch();
}

template <int CIN, int COUT>
hp_status launch_conv_t(const void* x, const void* w, const float* bias, void* y, int B, int H,
                        int W, int relu, int* err, int nsm, cudaStream_t st, uint32_t wait_limit,
                        bool pdl)
{
    if (W >= kWsMinWidth) return launch_ws<CIN, COUT, false>(x, w, bias, y, B, H, W, relu, err,
                                                            nsm, st, nullptr, wait_limit, pdl);
    using S = ConvSmem<CIN, COUT>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(conv3x3_tc_kernel<CIN, COUT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, S::kBytes);
        if (e != cudaSuccess) { set_cuda_error(e); return HP_ERR_CUDA; }
        attr = true;
    }
    const long P = (long)B * H * W;
    const int ntiles = (int)((P + kTileM - 1) / kTileM);
    const int grid = ntiles < nsm ? ntiles : nsm;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kConvThreads);
    cfg.dynamicSmemBytes = S::kBytes;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    cudaError_t e = cudaLaunchKernelEx(&cfg, conv3x3_tc_kernel<CIN, COUT>, (const uint4*)x,
                                       (const uint4*)w, bias, (__nv_bfloat16*)y, B, H, W, relu,
                                       ntiles, err);
    if (e != cudaSuccess) { set_cuda_error(e); return HP_ERR_CUDA; }
    return check_launch();
}

}  // namespace

hp_status launch_conv3x3_tc(const void* x, const void* w, const float* bias, void* y, int B,
                            int H, int W, int cin, int cout, int relu, int* err, int nsm,
                            cudaStream_t st, uint32_t wait_limit, bool pdl)
{
    if (cin == 32 && cout == 32)
        return launch_conv_t<32, 32>(x, w, bias, y, B, H, W, relu, err, nsm, st, wait_limit, pdl);
    if (cin == 32 && cout == 64)
        return launch_conv_t<32, 64>(x, w, bias, y, B, H, W, relu, err, nsm, st, wait_limit, pdl);
    if (cin == 64 && cout == 32)
        return launch_conv_t<64, 32>(x, w, bias, y, B, H, W, relu, err, nsm, st, wait_limit, pdl);
    if (cin == 64 && cout == 64)
        return launch_conv_t<64, 64>(x, w, bias, y, B, H, W, relu, err, nsm, st, wait_limit, pdl);
    // first layer of a branch, input padded to 16 channels (warp-specialised
    // kernel only; narrower images take the CUDA-core layer)
    if (cin == 16 && cout == 32 && W >= kWsMinWidth)
        return launch_ws<16, 32, false>(x, w, bias, y, B, H, W, relu, err, nsm, st, nullptr,
                                        wait_limit, pdl);
    return HP_ERR_UNSUPPORTED;
}

int conv_tc_min_width() { return kWsMinWidth; }

// Input gradient of a tensor-core layer (cin -> cout): the convolution of the
// output gradient gy (BF16 [P][cout]) with wdg = the flipped, transposed
// weights (BF16 [9][cin][cout], tap 8 - t of the forward's tap t), zero
// padding, zero bias (cout floats), the ReLU derivative of act (BF16
// [P][cin], may be null) applied; gx BF16 [P][cin].  Widths from
// conv_tc_min_width() up.
hp_status launch_conv3x3_tc_dgrad(const void* gy, const void* wdg, const float* zero_bias,
                                  const void* act, void* gx, int B, int H, int W, int cin,
                                  int cout, int* err, int nsm, cudaStream_t st,
                                  uint32_t wait_limit)
{
    if (W < kWsMinWidth) return HP_ERR_UNSUPPORTED;
    if (cin == 64 && cout == 64)
        return launch_ws<64, 64, false, true>(gy, wdg, zero_bias, gx, B, H, W, 0, err, nsm, st, act,
                                               wait_limit);
    if (cin == 32 && cout == 64)
        return launch_ws<64, 32, false, true>(gy, wdg, zero_bias, gx, B, H, W, 0, err, nsm, st, act,
                                               wait_limit);
    if (cin == 64 && cout == 32)
        return launch_ws<32, 64, false, true>(gy, wdg, zero_bias, gx, B, H, W, 0, err, nsm, st, act,
                                               wait_limit);
    if (cin == 32 && cout == 32)
        return launch_ws<32, 32, false, true>(gy, wdg, zero_bias, gx, B, H, W, 0, err, nsm, st, act,
                                               wait_limit);
    return HP_ERR_UNSUPPORTED;
}

// Weight- and bias-gradient partial sums of a tensor-core layer (cin ->
// cout) into part[g][9][cout][cin] and partb[g][cout] for g < *grid_out (one
// per CTA); x BF16 [P][cin], gy BF16 [P][cout].
hp_status launch_conv3x3_tc_wgrad(const void* x, const void* gy, float* part, size_t part_len,
                                  float* partb, size_t partb_len, int B, int H, int W, int cin,
                                  int cout, int* err, int nsm, int* grid_out, cudaStream_t st,
                                  uint32_t wait_limit)
{
    if (cin == 64 && cout == 64)
        return launch_wgrad_t<64, 64>(x, gy, part, part_len, partb, partb_len, B, H, W, err, nsm,
                                      grid_out, st, wait_limit);
    if (cin == 32 && cout == 64)
        return launch_wgrad_t<32, 64>(x, gy, part, part_len, partb, partb_len, B, H, W, err, nsm,
                                      grid_out, st, wait_limit);
    if (cin == 64 && cout == 32)
        return launch_wgrad_t<64, 32>(x, gy, part, part_len, partb, partb_len, B, H, W, err, nsm,
                                      grid_out, st, wait_limit);
    if (cin == 32 && cout == 32)
        return launch_wgrad_t<32, 32>(x, gy, part, part_len, partb, partb_len, B, H, W, err, nsm,
                                      grid_out, st, wait_limit);
    return HP_ERR_UNSUPPORTED;
}

// Last layer of a branch, 32 -> 1, as channel 0 of a 32 -> 16 convolution
// (w: BF16 [9][16][32], rows 1..15 zero; bias: 16 floats) written as FP32
// [B][H][W] without rounding; HP_ERR_UNSUPPORTED below the width the
// warp-specialised kernel serves.
hp_status launch_conv3x3_tc_out1(const void* x, const void* w, const float* bias, float* y,
                                 int B, int H, int W, int* err, int nsm, cudaStream_t st,
                                 uint32_t wait_limit, bool pdl)
{
    if (W < kWsMinWidth) return HP_ERR_UNSUPPORTED;
    return launch_ws<32, 16, true>(x, w, bias, y, B, H, W, 0, err, nsm, st, nullptr, wait_limit,
                                   pdl);
}

}  // namespace hp

extern "C" hp_status hp_conv3x3_bf16(const uint16_t* x, const uint16_t* w, const float* bias,
                                     uint16_t* y, int32_t batch, int32_t height, int32_t width,
                                     int32_t cin, int32_t cout, int32_t relu, int32_t* err,
                                     void* stream)
{
    if (!x || !w || !bias || !y || batch <= 0 || height <= 0 || width <= 0) return HP_ERR_INVALID_ARG;
    if ((uintptr_t)x % 16 || (uintptr_t)w % 16 || (uintptr_t)y % 16) return HP_ERR_INVALID_ARG;
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) { hp::set_cuda_error(e); return HP_ERR_CUDA; }
    return hp::launch_conv3x3_tc(x, w, bias, y, batch, height, width, cin, cout, relu, err, nsm,
                                 (cudaStream_t)stream);
}
