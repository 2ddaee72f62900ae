// The CNNs of Sec. 3.1 on sm_103a and the hybrid projection (Sec. 3.3): the
// network predicts the scaled pressure from [div/s, flags] and hands it to
// the Jacobi sweeps as the initial guess.
//
// MultiScale (3 x 3 convolutions, replicated borders; ReLU after every
// convolution of a branch except its last two):
//   scale 1/4: [pool4(div/s), pool4(flags)]          2 -> 32 -> 64 -> 64 -> 32 -> 1
//   scale 1/2: [pool2(div/s), pool2(flags), up(o4)]  3 -> 32 -> 64 -> 64 -> 64 -> 64 -> 32 -> 1
//   scale 1  : [div/s, flags, up(o2)]                3 -> 32 -> 64 -> 64 -> 64 -> 64 -> 32 -> 1
// SmallScale: the same with every 64-channel layer at 32 channels.
// MonoScale: one branch, [div/s, flags] 2 -> 32 -> 64 x 6 -> 32 -> 1 at full
// resolution.  A network is its layer table; its branches are the runs of
// layers that end in one output channel.
// pool = average pooling (2 x 2 / 4 x 4), up = bilinear x 2 at half-pixel
// centres with the edge repeated.  s = mean |div| over the fluid cells (1 if
// zero); phi_0 = s * output on cells with an open face (the Poisson equation
// is linear in div).  BF16 activations and weights, FP32 accumulation; the
// 1-channel branch outputs are kept in FP32.
//
// Kernels: cnn_scale_partial/finish_kernel (s per grid), branch_input_kernel
// (pooling, up-sampling and scaling into the branch input), conv_first_kernel
// (2/3 -> 32 on CUDA cores), the tensor-core conv3x3 (conv_tc.cu) for the
// 32/64-channel layers, conv_last_kernel (32 -> 1 on CUDA cores), phi0_kernel.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "hproj_internal.cuh"

namespace hp {

namespace {

struct LayerSpec {
    int scale, cin, cout, relu;
    int ks = 3;  // kernel size: 3, or 1 (run as a 3 x 3 with only the centre tap)
};

// network order: scale 1/4, then 1/2, then 1
constexpr int kLayers = 19;      // MultiScale and SmallScale
constexpr int kMaxLayers = 20;   // the most of any architecture (the Unet)
constexpr int kMaxBranches = 3;
const LayerSpec kSpecMulti[kLayers] = {
    {4, 2, 32, 1},  {4, 32, 64, 1}, {4, 64, 64, 1}, {4, 64, 32, 0}, {4, 32, 1, 0},
    {2, 3, 32, 1},  {2, 32, 64, 1}, {2, 64, 64, 1}, {2, 64, 64, 1}, {2, 64, 64, 1},
    {2, 64, 32, 0}, {2, 32, 1, 0},  {1, 3, 32, 1},  {1, 32, 64, 1}, {1, 64, 64, 1},
    {1, 64, 64, 1}, {1, 64, 64, 1}, {1, 64, 32, 0}, {1, 32, 1, 0}};
// SmallScale (Sec. 3.1): the same graph with fewer filters, every 64-channel
// layer at 32 channels (123,491 parameters, about three times fewer)
const LayerSpec kSpecSmall[kLayers] = {
    {4, 2, 32, 1},  {4, 32, 32, 1}, {4, 32, 32, 1}, {4, 32, 32, 0}, {4, 32, 1, 0},
    {2, 3, 32, 1},  {2, 32, 32, 1}, {2, 32, 32, 1}, {2, 32, 32, 1}, {2, 32, 32, 1},
    {2, 32, 32, 0}, {2, 32, 1, 0},  {1, 3, 32, 1},  {1, 32, 32, 1}, {1, 32, 32, 1},
    {1, 32, 32, 1}, {1, 32, 32, 1}, {1, 32, 32, 0}, {1, 32, 1, 0}};

// MonoScale (Sec. 3.1): one feed-forward branch of 9 convolutions at full
// resolution on [div/s, flags]
constexpr int kLayersMono = 9;
const LayerSpec kSpecMono[kLayersMono] = {
    {1, 2, 32, 1},  {1, 32, 64, 1}, {1, 64, 64, 1}, {1, 64, 64, 1}, {1, 64, 64, 1},
    {1, 64, 64, 1}, {1, 64, 64, 1}, {1, 64, 32, 0}, {1, 32, 1, 0}};

// Unet (Sec. 3.1): encoder levels n, n/2, n/4, n/8 ending in 32-channel skip
// features (2 -> 32 -> 32, then 2 x 2 max pooling and 32 -> 64 -> 32), the
// bottom n/16 32 -> 64 -> 64 -> 32, decoder levels on [up(coarser), skip]
// (64 channels) 64 -> 64 -> 32, the last 64 -> 32 -> 32 and a 1 x 1 32 -> 1
constexpr int kLayersUnet = 20;
const LayerSpec kSpecUnet[kLayersUnet] = {
    {1, 2, 32, 1},   {1, 32, 32, 1},  {2, 32, 64, 1},  {2, 64, 32, 1},  {4, 32, 64, 1},
    {4, 64, 32, 1},  {8, 32, 64, 1},  {8, 64, 32, 1},  {16, 32, 64, 1}, {16, 64, 64, 1},
    {16, 64, 32, 1}, {8, 64, 64, 1},  {8, 64, 32, 1},  {4, 64, 64, 1},  {4, 64, 32, 1},
    {2, 64, 64, 1},  {2, 64, 32, 1},  {1, 64, 32, 1},  {1, 32, 32, 0},  {1, 32, 1, 0, 1}};

const LayerSpec* spec_for(int arch)
{
    return arch == HP_CNN_MULTISCALE   ? kSpecMulti
           : arch == HP_CNN_SMALLSCALE ? kSpecSmall
           : arch == HP_CNN_MONOSCALE  ? kSpecMono
           : arch == HP_CNN_UNET       ? kSpecUnet
                                       : nullptr;
}

int layers_for(int arch)
{
    return arch == HP_CNN_MONOSCALE ? kLayersMono : arch == HP_CNN_UNET ? kLayersUnet : kLayers;
}

// grid sizes a network accepts: multiples of 4 (16 for the Unet's five scales)
int size_multiple(int arch) { return arch == HP_CNN_UNET ? 16 : 4; }

// The branches of a network in order: consecutive layers up to a 1-channel
// output.  A branch after the first takes the up-sampled output of the one
// before it as its third input channel.
struct Branches {
    int n;
    int first[kMaxBranches], last[kMaxBranches], scale[kMaxBranches];
};

Branches branches_of(const LayerSpec* sp, int nl)
{
    Branches br = {};
    int start = 0;
    for (int l = 0; l < nl && br.n < kMaxBranches; ++l)
        if (sp[l].cout == 1) {
            br.first[br.n] = start;
            br.last[br.n] = l;
            br.scale[br.n] = sp[l].scale;
            ++br.n;
            start = l + 1;
        }
    return br;
}

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// s[b] = mean |div| over fluid cells, 1 when there is none or it is zero.
// s[b] = mean |div| over fluid cells, 1 when there is none or it is zero.
// Pass 1: kScaleCtas CTAs per grid, each a contiguous slice of the cells;
// FP32 sums per thread (at most a few dozen terms), FP64 across the warp and
// the CTA.  Pass 2: one warp per grid adds the CTA partials in a fixed order.
constexpr int kScaleCtas = 32;
constexpr int kScaleThreads = 256;

__global__ void cnn_scale_partial_kernel(const float* __restrict__ div,
                                         const uint8_t* __restrict__ flags,
                                         double* __restrict__ part_sum,
                                         unsigned long long* __restrict__ part_cnt, size_t cells)
{
    __shared__ double sh_sum[kScaleThreads / 32];
    __shared__ unsigned long long sh_cnt[kScaleThreads / 32];
    const int b = blockIdx.y;
    const size_t per = (cells + kScaleCtas - 1) / kScaleCtas;
    const size_t q0 = (size_t)blockIdx.x * per;
    const size_t q1 = q0 + per < cells ? q0 + per : cells;
    const float* d = div + (size_t)b * cells;
    const uint8_t* f = flags + (size_t)b * cells;
    float sum = 0.0f;
    unsigned cnt = 0;
    for (size_t q = q0 + threadIdx.x; q < q1; q += kScaleThreads) {
        if (f[q] == 0) {
            sum += fabsf(d[q]);
            ++cnt;
        }
    }
    double ds = (double)sum;
    unsigned long long dc = cnt;
    for (int off = 16; off > 0; off >>= 1) {
        ds += __shfl_down_sync(0xffffffffu, ds, off);
        dc += __shfl_down_sync(0xffffffffu, dc, off);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { sh_sum[wid] = ds; sh_cnt[wid] = dc; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        unsigned long long c = 0;
        for (int w = 0; w < kScaleThreads / 32; ++w) { t += sh_sum[w]; c += sh_cnt[w]; }
        part_sum[(size_t)b * kScaleCtas + blockIdx.x] = t;
        part_cnt[(size_t)b * kScaleCtas + blockIdx.x] = c;
    }
}

__global__ void cnn_scale_finish_kernel(const double* __restrict__ part_sum,
                                        const unsigned long long* __restrict__ part_cnt,
                                        float* __restrict__ s)
{
    // a programmatic dependent of the partial sums
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int b = blockIdx.x, lane = threadIdx.x;
    double t = lane < kScaleCtas ? part_sum[(size_t)b * kScaleCtas + lane] : 0.0;
    unsigned long long c = lane < kScaleCtas ? part_cnt[(size_t)b * kScaleCtas + lane] : 0ull;
    for (int off = 16; off > 0; off >>= 1) {
        t += __shfl_down_sync(0xffffffffu, t, off);
        c += __shfl_down_sync(0xffffffffu, c, off);
    }
    if (lane == 0) {
        const double m = c ? t / (double)c : 0.0;
        s[b] = m > 0.0 ? (float)m : 1.0f;
    }
}

// Input channel values of the branch at `scale` for pixel (i, j) of that
// scale: [pool(div/s), pool(flags), up(prev)] (BF16-rounded).
struct BranchIn {
    const float* div;       // [B][H][W] full resolution
    const uint8_t* flags;
    const float* s;
    const float* prev;      // [B][H/2s? ] coarser branch output (FP32) or null
    int H, W;               // full resolution
    int scale;              // 1, 2, 4
    __device__ void at(int b, int i, int j, float out[3]) const
    {
        const int hs = H / scale, ws = W / scale;
        if (scale == 1) {
            // one pixel: the FP64 mean of one FP32 value is that value, so
            // this is the pooled form below without the FP64 arithmetic
            const size_t q = ((size_t)b * H + j) * W + i;
            out[0] = bf16r(div[q] / s[b]);
            out[1] = flags[q] != 0 ? 1.0f : 0.0f;
        } else {
            double sd = 0.0, sf = 0.0;
            for (int dy = 0; dy < scale; ++dy)
                for (int dx = 0; dx < scale; ++dx) {
                    const size_t q = ((size_t)b * H + (size_t)j * scale + dy) * W +
                                     (size_t)i * scale + dx;
                    sd += div[q];
                    sf += flags[q] != 0 ? 1.0 : 0.0;
                }
            const double inv = 1.0 / (scale * scale);
            out[0] = bf16r((float)(sd * inv) / s[b]);
            out[1] = bf16r((float)(sf * inv));
        }
        out[2] = 0.0f;
        if (prev) {
            // bilinear x 2 from the coarser (hs/2 x ws/2) output
            const int hc = hs / 2, wc = ws / 2;
            const float* pc = prev + (size_t)b * hc * wc;
            const int ci = i >> 1, cj = j >> 1;
            const int ni = (i & 1) ? min(ci + 1, wc - 1) : max(ci - 1, 0);
            const int nj = (j & 1) ? min(cj + 1, hc - 1) : max(cj - 1, 0);
            const float rx0 = 0.75f * pc[(size_t)cj * wc + ci] + 0.25f * pc[(size_t)cj * wc + ni];
            const float rx1 = 0.75f * pc[(size_t)nj * wc + ci] + 0.25f * pc[(size_t)nj * wc + ni];
            out[2] = bf16r(0.75f * rx0 + 0.25f * rx1);
        }
    }
};

// Branch input, once per pixel of the branch: xin [P][cin] FP32 holding the
// BF16-rounded values [pool(div)/s, pool(flags)(, up(coarser output))].
// Block (x, y) covers blockDim.x pixels of the rows y, y + gridDim.y, ... of
// the B x hs rows of the branch.
__global__ void branch_input_kernel(BranchIn in, int cin, float* __restrict__ xin,
                                    __nv_bfloat16* __restrict__ x16, int B)
{
    // a programmatic dependent of the kernel before it (s, the coarser output)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int hs = in.H / in.scale, ws = in.W / in.scale;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ws) return;
    for (int row = blockIdx.y; row < B * hs; row += gridDim.y) {
        const int b = row / hs, j = row - b * hs;
        const size_t p = (size_t)row * ws + i;
        float xc[3];
        in.at(b, i, j, xc);
        if (xin)
            for (int c = 0; c < cin; ++c) xin[p * cin + c] = xc[c];
        if (x16) {
            // the tensor-core first layer: 16 channels, the inputs then zeros
            // (the values are BF16-rounded already, so this is exact)
            __align__(16) __nv_bfloat16 v[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) v[c] = __float2bfloat16_rn(c < cin ? xc[c] : 0.0f);
            uint4* dst = reinterpret_cast<uint4*>(x16 + p * 16);
            dst[0] = reinterpret_cast<const uint4*>(v)[0];
            dst[1] = reinterpret_cast<const uint4*>(v)[1];
        }
    }
}

// The same inputs for four consecutive pixels i0..i0+3 of a row of the branch
// (i0 a multiple of 4, W a multiple of 4 * scale): vector loads of the rows
// the four pixels pool, issued before any arithmetic.  The pooled mean is
// taken in FP32 as the mean of 2 x 2 means (for scale 4, of the four 2 x 2
// means), the flag count as an exact integer.
__device__ __forceinline__ void branch_at4(const BranchIn& in, int b, int i0, int j,
                                           float out[4][3])
{
    const float sb = in.s[b];
    const int W = in.W;
    if (in.scale == 1) {
        const size_t q = ((size_t)b * in.H + j) * W + i0;
        const float4 d = *reinterpret_cast<const float4*>(in.div + q);
        const uint32_t f = *reinterpret_cast<const uint32_t*>(in.flags + q);
        const float dv[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            out[k][0] = bf16r(dv[k] / sb);
            out[k][1] = ((f >> (8 * k)) & 0xffu) != 0u ? 1.0f : 0.0f;
        }
    } else if (in.scale == 2) {
        const size_t q = ((size_t)b * in.H + 2 * j) * W + 2 * i0;
        float v[2][8];
        uint2 f[2];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const float4 a = *reinterpret_cast<const float4*>(in.div + q + (size_t)r * W);
            const float4 c = *reinterpret_cast<const float4*>(in.div + q + (size_t)r * W + 4);
            v[r][0] = a.x; v[r][1] = a.y; v[r][2] = a.z; v[r][3] = a.w;
            v[r][4] = c.x; v[r][5] = c.y; v[r][6] = c.z; v[r][7] = c.w;
            f[r] = *reinterpret_cast<const uint2*>(in.flags + q + (size_t)r * W);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float m = ((v[0][2 * k] + v[0][2 * k + 1]) + (v[1][2 * k] + v[1][2 * k + 1])) * 0.25f;
            int cnt = 0;
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const uint32_t w2 = ((k < 2 ? f[r].x : f[r].y) >> (16 * (k & 1))) & 0xffffu;
                cnt += ((w2 & 0xffu) != 0u) + ((w2 >> 8) != 0u);
            }
            out[k][0] = bf16r(m / sb);
            out[k][1] = (float)cnt * 0.25f;
        }
    } else {
        const size_t q = ((size_t)b * in.H + 4 * j) * W + 4 * i0;
        float m2[2][8];  // 2 x 2 means of the two row pairs, 8 per pair
        int cnt[4] = {0, 0, 0, 0};
#pragma unroll
        for (int rp = 0; rp < 2; ++rp) {
            float v[2][16];
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const float* src = in.div + q + (size_t)(2 * rp + r) * W;
#pragma unroll
                for (int c4 = 0; c4 < 4; ++c4) {
                    const float4 a = *reinterpret_cast<const float4*>(src + 4 * c4);
                    v[r][4 * c4] = a.x; v[r][4 * c4 + 1] = a.y;
                    v[r][4 * c4 + 2] = a.z; v[r][4 * c4 + 3] = a.w;
                }
                const uint4 f = *reinterpret_cast<const uint4*>(in.flags + q + (size_t)(2 * rp + r) * W);
                const uint32_t fw[4] = {f.x, f.y, f.z, f.w};
#pragma unroll
                for (int k = 0; k < 4; ++k) cnt[k] += __popc(__vcmpne4(fw[k], 0u)) >> 3;
            }
#pragma unroll
            for (int c = 0; c < 8; ++c)
                m2[rp][c] = ((v[0][2 * c] + v[0][2 * c + 1]) + (v[1][2 * c] + v[1][2 * c + 1])) * 0.25f;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float m = ((m2[0][2 * k] + m2[0][2 * k + 1]) + (m2[1][2 * k] + m2[1][2 * k + 1])) * 0.25f;
            out[k][0] = bf16r(m / sb);
            out[k][1] = (float)cnt[k] * 0.0625f;
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) out[k][2] = 0.0f;
    if (in.prev) {
        // bilinear x 2 from the coarser output: coarse columns i0/2 - 1 ..
        // i0/2 + 2 (clamped) of coarse rows cj and nj
        const int hs = in.H / in.scale, ws = W / in.scale;
        const int hc = hs / 2, wc = ws / 2;
        const float* pc = in.prev + (size_t)b * hc * wc;
        const int cj = j >> 1;
        const int nj = (j & 1) ? min(cj + 1, hc - 1) : max(cj - 1, 0);
        const int c0 = i0 >> 1;
        float r0[4], r1[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int cc = min(max(c0 - 1 + t, 0), wc - 1);
            r0[t] = pc[(size_t)cj * wc + cc];
            r1[t] = pc[(size_t)nj * wc + cc];
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            // pixel i0 + k: coarse column c0 + k / 2 (index 1 + k / 2), its
            // neighbour one to the left (even k) or right (odd k)
            const int ci = 1 + (k >> 1), ni = (k & 1) ? ci + 1 : ci - 1;
            const float rx0 = 0.75f * r0[ci] + 0.25f * r0[ni];
            const float rx1 = 0.75f * r1[ci] + 0.25f * r1[ni];
            out[k][2] = bf16r(0.75f * rx0 + 0.25f * rx1);
        }
    }
}

// Branch input, four pixels per thread (rows of the branch a multiple of 4
// wide); the same outputs as branch_input_kernel.
__global__ void branch_input4_kernel(BranchIn in, int cin, float* __restrict__ xin,
                                     __nv_bfloat16* __restrict__ x16, int B)
{
    // a programmatic dependent of the kernel before it (s, the coarser output)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int hs = in.H / in.scale, ws = in.W / in.scale;
    const size_t quads = (size_t)B * hs * ws / 4;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < quads;
         t += (size_t)gridDim.x * blockDim.x) {
        const size_t p = 4 * t;
        const size_t row = p / (size_t)ws;
        const int i0 = (int)(p - row * ws);
        const int b = (int)(row / (size_t)hs), j = (int)(row - (size_t)b * hs);
        float xc[4][3];
        branch_at4(in, b, i0, j, xc);
        if (xin) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    if (c < cin) xin[(p + k) * cin + c] = xc[k][c];
            }
        }
        if (x16) {
            uint4* dst = reinterpret_cast<uint4*>(x16 + p * 16);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                // 16 channels: the inputs, then zeros (exact: already BF16)
                const uint32_t w0 = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(xc[k][0])) |
                                    ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(xc[k][1])) << 16);
                const uint32_t w1 = cin > 2 ? (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(xc[k][2])) : 0u;
                dst[2 * k] = make_uint4(w0, w1, 0u, 0u);
                dst[2 * k + 1] = make_uint4(0u, 0u, 0u, 0u);
            }
        }
    }
}

// 2 x 2 max pooling of BF16 [B][H][W][C] (H, W even) into [B][H/2][W/2][C].
// Block x = one output row (b, i); its threads cover the row's (pixel,
// 8-channel chunk) items, c8 chunks per pixel.  The maximum of BF16 values is
// exact.
__global__ void maxpool2_kernel(const uint4* __restrict__ x, uint4* __restrict__ y, int H, int W,
                                int c8)
{
    // a programmatic dependent of the layer before it
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    const int Ho = H / 2, Wo = W / 2;
    const int xi = blockIdx.y * blockDim.x + threadIdx.x;
    if (xi >= Wo * c8) return;
    const int c = xi % c8, j = xi / c8;
    const int row = blockIdx.x;
    const int i = row % Ho, b = row / Ho;
    const size_t q = ((size_t)row * Wo + j) * c8 + c;
    const size_t r0 = (((size_t)b * H + 2 * i) * W + 2 * j) * c8 + c;
    const size_t r1 = r0 + (size_t)W * c8;
    uint4 v[4] = {x[r0], x[r0 + c8], x[r1], x[r1 + c8]};
    uint4 m = v[0];
    uint32_t* mw = reinterpret_cast<uint32_t*>(&m);
    for (int k = 1; k < 4; ++k) {
        const uint32_t* vw = reinterpret_cast<const uint32_t*>(&v[k]);
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            __nv_bfloat162 a, bb;
            memcpy(&a, &mw[h], 4);
            memcpy(&bb, &vw[h], 4);
            a = __hmax2(a, bb);
            memcpy(&mw[h], &a, 4);
        }
    }
    y[q] = m;
}

// Decoder input of the Unet, BF16 [B][H][W][64]: channels 0-31 the bilinear
// x 2 up-sampling (half-pixel centres, edge sample repeated, FP32 then
// rounded to BF16) of coarse [B][H/2][W/2][32], channels 32-63 the skip
// features [B][H][W][32].  Block x = one output row (b, j); its threads cover
// first the row's interpolated (pixel, 8-channel chunk) items, then its copied
// ones, so that a warp takes one kind only.
__global__ void up_concat_kernel(const uint4* __restrict__ coarse, const uint4* __restrict__ skip,
                                 uint4* __restrict__ y, int H, int W)
{
    // a programmatic dependent of the layer before it
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    const int Hc = H / 2, Wc = W / 2;
    const int xi = blockIdx.y * blockDim.x + threadIdx.x;
    if (xi >= W * 8) return;
    const int row = blockIdx.x;
    const bool copy = xi >= W * 4;
    const int k = copy ? xi - W * 4 : xi;
    const int c = (k & 3) + (copy ? 4 : 0);  // chunk of the 64-channel output pixel
    const int i = k >> 2;                      // column
    const size_t p = (size_t)row * W + i;
    const size_t q = p * 8 + c;
    if (copy) {
        y[q] = skip[p * 4 + (c - 4)];
        return;
    }
    const int j = row % H;  // row within the grid
    const int b = row / H;
    const int ci = i >> 1, cj = j >> 1;
    const int ni = (i & 1) ? min(ci + 1, Wc - 1) : max(ci - 1, 0);
    const int nj = (j & 1) ? min(cj + 1, Hc - 1) : max(cj - 1, 0);
    const uint4* base = coarse + (size_t)b * Hc * Wc * 4 + c;
    const uint4 q00 = base[((size_t)cj * Wc + ci) * 4], q01 = base[((size_t)cj * Wc + ni) * 4];
    const uint4 q10 = base[((size_t)nj * Wc + ci) * 4], q11 = base[((size_t)nj * Wc + ni) * 4];
    const __nv_bfloat16* a00 = reinterpret_cast<const __nv_bfloat16*>(&q00);
    const __nv_bfloat16* a01 = reinterpret_cast<const __nv_bfloat16*>(&q01);
    const __nv_bfloat16* a10 = reinterpret_cast<const __nv_bfloat16*>(&q10);
    const __nv_bfloat16* a11 = reinterpret_cast<const __nv_bfloat16*>(&q11);
    __align__(16) __nv_bfloat16 o[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const float rx0 = 0.75f * __bfloat162float(a00[e]) + 0.25f * __bfloat162float(a01[e]);
        const float rx1 = 0.75f * __bfloat162float(a10[e]) + 0.25f * __bfloat162float(a11[e]);
        o[e] = __float2bfloat16_rn(0.75f * rx0 + 0.25f * rx1);
    }
    y[q] = *reinterpret_cast<const uint4*>(o);
}

// BF16 tensor-core copies of a branch's first and last layer from their
// CUDA-core (FP32, BF16-rounded) weights: first [tap][cin][32] ->
// [tap][32][16] with zero channels cin..15; last [tap][32] -> [tap][16][32]
// with zero output channels 1..15, bias -> 16 floats.
__global__ void pack_edge_layers_kernel(const float* __restrict__ wf, int cin,
                                        __nv_bfloat16* __restrict__ wf16,
                                        const float* __restrict__ wl,
                                        const float* __restrict__ bl,
                                        __nv_bfloat16* __restrict__ wl16, float* __restrict__ bl16)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 9 * 32 * 16) {
        const int c = i % 16, o = (i / 16) % 32, t = i / (16 * 32);
        wf16[i] = __float2bfloat16_rn(c < cin ? wf[(t * cin + c) * 32 + o] : 0.0f);
        const int c2 = i % 32, o2 = (i / 32) % 16, t2 = i / (32 * 16);
        wl16[i] = __float2bfloat16_rn(o2 == 0 ? wl[t2 * 32 + c2] : 0.0f);
    }
    if (i < 16) bl16[i] = i == 0 ? bl[0] : 0.0f;
}

// First convolution of a branch: cin (2 or 3) -> 32, bias, ReLU, BF16 NHWC,
// from the branch input xin [P][cin].  Each thread computes two horizontally
// adjacent pixels, so every weight read from shared memory (a broadcast) feeds
// two FMAs.  w: float [9][cin][32] (BF16-rounded values), bias float [32].
template <int CIN>
__global__ void __launch_bounds__(128)
    conv_first_kernel(const float* __restrict__ xin, const float* __restrict__ w,
                      const float* __restrict__ bias, __nv_bfloat16* __restrict__ y, int B,
                      int H, int W)
{
    __shared__ __align__(16) float sw[9 * CIN * 32];
    __shared__ __align__(16) float sb[32];
    for (int q = threadIdx.x; q < 9 * CIN * 32; q += blockDim.x) sw[q] = w[q];
    if (threadIdx.x < 32) sb[threadIdx.x] = bias[threadIdx.x];
    __syncthreads();
    // weights staged; the input is the branch input kernel's output
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    const int W2 = (W + 1) / 2;
    const long P2 = (long)B * H * W2;
    for (long p2 = (long)blockIdx.x * blockDim.x + threadIdx.x; p2 < P2;
         p2 += (long)gridDim.x * blockDim.x) {
        const int b = (int)(p2 / ((long)H * W2));
        const int r = (int)(p2 - (long)b * H * W2);
        const int j = r / W2, i0 = 2 * (r - j * W2);
        const bool two = i0 + 1 < W;
        float acc0[32], acc1[32];
#pragma unroll
        for (int o = 0; o < 32; ++o) { acc0[o] = sb[o]; acc1[o] = sb[o]; }
#pragma unroll 1
        for (int dy = 0; dy < 3; ++dy) {
            const int sy = min(max(j + dy - 1, 0), H - 1);
            const float* xr = xin + ((size_t)b * H + sy) * W * CIN;
#pragma unroll 1
            for (int dx = 0; dx < 3; ++dx) {
                // input columns of the two outputs for this tap (clamped)
                const int sx0 = min(max(i0 - 1 + dx, 0), W - 1);
                const int sx1 = min(max(i0 + dx, 0), W - 1);
                const float* wt = sw + (dy * 3 + dx) * CIN * 32;
#pragma unroll
                for (int c = 0; c < CIN; ++c) {
                    const float a0 = xr[(size_t)sx0 * CIN + c], a1 = xr[(size_t)sx1 * CIN + c];
                    const float4* w4 = reinterpret_cast<const float4*>(wt + c * 32);
#pragma unroll
                    for (int o4 = 0; o4 < 8; ++o4) {
                        const float4 wv = w4[o4];
                        acc0[4 * o4 + 0] = fmaf(wv.x, a0, acc0[4 * o4 + 0]);
                        acc0[4 * o4 + 1] = fmaf(wv.y, a0, acc0[4 * o4 + 1]);
                        acc0[4 * o4 + 2] = fmaf(wv.z, a0, acc0[4 * o4 + 2]);
                        acc0[4 * o4 + 3] = fmaf(wv.w, a0, acc0[4 * o4 + 3]);
                        acc1[4 * o4 + 0] = fmaf(wv.x, a1, acc1[4 * o4 + 0]);
                        acc1[4 * o4 + 1] = fmaf(wv.y, a1, acc1[4 * o4 + 1]);
                        acc1[4 * o4 + 2] = fmaf(wv.z, a1, acc1[4 * o4 + 2]);
                        acc1[4 * o4 + 3] = fmaf(wv.w, a1, acc1[4 * o4 + 3]);
                    }
                }
            }
        }
        __align__(16) __nv_bfloat16 ob[32];
        const size_t p = ((size_t)b * H + j) * W + i0;
#pragma unroll
        for (int o = 0; o < 32; ++o) ob[o] = __float2bfloat16_rn(fmaxf(acc0[o], 0.0f));
        uint4* dst = reinterpret_cast<uint4*>(y + p * 32);
#pragma unroll
        for (int q = 0; q < 4; ++q) dst[q] = reinterpret_cast<const uint4*>(ob)[q];
        if (two) {
#pragma unroll
            for (int o = 0; o < 32; ++o) ob[o] = __float2bfloat16_rn(fmaxf(acc1[o], 0.0f));
            dst += 4;
#pragma unroll
            for (int q = 0; q < 4; ++q) dst[q] = reinterpret_cast<const uint4*>(ob)[q];
        }
    }
}

// Last convolution of a branch: 32 -> 1, bias, no ReLU, FP32 output.  A
// thread walks kLastRows output rows of one column: every input row (its
// three clamped neighbours in that row) is loaded once and dotted with the
// three kernel rows, adding to the outputs above, at and below it.  Lanes of
// a warp take consecutive columns, so the loads are contiguous.
// w: float [9][32] (BF16-rounded), bias float [1].
constexpr int kLastRows = 8;

__global__ void __launch_bounds__(128)
    conv_last_kernel(const __nv_bfloat16* __restrict__ x, const float* __restrict__ w,
                     const float* __restrict__ bias, float* __restrict__ y, int B, int H, int W)
{
    __shared__ __align__(16) float sw[9 * 32];
    for (int q = threadIdx.x; q < 9 * 32; q += blockDim.x) sw[q] = w[q];
    __syncthreads();
    // weights staged; the input is the layer before's output
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const float b0 = bias[0];
    const int strips = (H + kLastRows - 1) / kLastRows;
    const long T = (long)B * strips * W;
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < T;
         t += (long)gridDim.x * blockDim.x) {
        const int i = (int)(t % W);
        const long bs = t / W;
        const int b = (int)(bs / strips);
        const int j0 = (int)(bs - (long)b * strips) * kLastRows;
        const int j1 = min(H, j0 + kLastRows);
        // a0: partial sum of output row r - 1, a1: of output row r
        float a0 = 0.0f, a1 = 0.0f;
#pragma unroll 1
        for (int r = j0 - 1; r <= j1; ++r) {  // input rows
            const int sr = min(max(r, 0), H - 1);
            float d[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll 1
            for (int dx = 0; dx < 3; ++dx) {
                const int sx = min(max(i + dx - 1, 0), W - 1);
                const uint4* src =
                    reinterpret_cast<const uint4*>(x + (((size_t)b * H + sr) * W + sx) * 32);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint4 v = src[q];
                    const __nv_bfloat162* e = reinterpret_cast<const __nv_bfloat162*>(&v);
                    float f[8];
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        const float2 t2 = __bfloat1622float2(e[h]);
                        f[2 * h] = t2.x;
                        f[2 * h + 1] = t2.y;
                    }
#pragma unroll
                    for (int dy = 0; dy < 3; ++dy) {
                        const float4* wq = reinterpret_cast<const float4*>(
                            sw + (dy * 3 + dx) * 32 + q * 8);
                        const float4 wa = wq[0], wb = wq[1];
                        d[dy] = fmaf(wa.x, f[0], d[dy]);
                        d[dy] = fmaf(wa.y, f[1], d[dy]);
                        d[dy] = fmaf(wa.z, f[2], d[dy]);
                        d[dy] = fmaf(wa.w, f[3], d[dy]);
                        d[dy] = fmaf(wb.x, f[4], d[dy]);
                        d[dy] = fmaf(wb.y, f[5], d[dy]);
                        d[dy] = fmaf(wb.z, f[6], d[dy]);
                        d[dy] = fmaf(wb.w, f[7], d[dy]);
                    }
                }
            }
            // input row r is tap dy = 2 of output r - 1 (now complete), dy = 1
            // of output r and dy = 0 of output r + 1
            if (r - 1 >= j0) y[((size_t)b * H + (r - 1)) * W + i] = (a0 + d[2]) + b0;
            a0 = a1 + d[1];
            a1 = d[0];
        }
    }
}

// bad[b] = 1 when the guess s * out of grid b is not finite on some cell
// with an open face (bad cleared beforehand; every writer stores 1).
__global__ void guess_check_kernel(const float* __restrict__ out, const float* __restrict__ s,
                                   const uint8_t* __restrict__ mask, int32_t* __restrict__ bad,
                                   int B, size_t cells)
{
    const size_t n = (size_t)B * cells;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(q / cells);
        if ((mask[q] & 15u) && !isfinite(s[b] * out[q])) bad[b] = 1;
    }
}

// phi_0 = s * out on cells with an open face, 0 elsewhere; the whole grid 0
// when its guess is not finite (the Jacobi sweeps then start from zero, the
// plain method).  The first cell of such a grid raises bit 1 of *err.
__global__ void phi0_kernel(const float* __restrict__ out, const float* __restrict__ s,
                            const uint8_t* __restrict__ mask, const int32_t* __restrict__ bad,
                            float* __restrict__ phi, int* err, int B, size_t cells)
{
    const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (size_t)B * cells) return;
    const int b = (int)(q / cells);
    const bool fallback = bad[b] != 0;
    phi[q] = ((mask[q] & 15u) && !fallback) ? s[b] * out[q] : 0.0f;
    if (fallback && q == (size_t)b * cells) atomicOr(err, 2);
}

}  // namespace

}  // namespace hp

using namespace hp;

struct hp_cnn {
    Guards guards;          // guard zones of the workspaces
    int arch;               // hp_cnn_arch
    const LayerSpec* spec;  // its layer table
    int nlayers;
    Branches br;
    int device;
    int num_sms;
    hp_shape max_shape;
    // per layer: weights in the layout of its kernel, FP32 bias
    void* w[kMaxLayers];
    float* bias[kMaxLayers];
    std::vector<float> master;  // FP32 parameters, oracle order
    // workspace
    __nv_bfloat16* act[2];
    float* out[kMaxBranches];  // branch outputs (FP32, one channel at the branch's scale)
    float* xin;     // branch input [P][cin] FP32 (largest branch)
    __nv_bfloat16* x16;  // branch input [P][16] BF16 for the tensor-core first layer
    // tensor-core copies of the first / last layer of each branch
    __nv_bfloat16* wtc_first[kMaxBranches];  // [9][32][16]
    __nv_bfloat16* wtc_last[kMaxBranches];   // [9][16][32]
    float* btc_last[kMaxBranches];           // [16]
    __nv_bfloat16* skip[4];  // Unet: the encoder's skip features per level, BF16 [P_level][32]
    float* s;
    double* s_part;                // [B][kScaleCtas] partial sums of |div|
    unsigned long long* s_cnt;     // [B][kScaleCtas] fluid-cell counts
    // device status word: bit 0 a tensor-core wait gave up, bit 1 a grid's
    // guess was not finite and the hybrid projection started it from zero
    int* err;
    uint32_t wait_limit;  // polls per bounded pipeline wait (0 = compiled limit)
    int32_t* guess_bad;   // [max batch] per grid: the network's guess is not finite
};

// a batch this network's workspace holds, with sides its architecture takes
static bool cnn_shape_ok(const hp_cnn* c, hp_shape s)
{
    return shape_ok(s) && s.ny % size_multiple(c->arch) == 0 &&
           s.nx % size_multiple(c->arch) == 0 && s.batch <= c->max_shape.batch &&
           (size_t)s.batch * s.ny * s.nx <=
               (size_t)c->max_shape.batch * c->max_shape.ny * c->max_shape.nx;
}

// A launch as a programmatic dependent of the kernel before it in the stream:
// the kernel waits (griddepcontrol.wait) before it reads what that kernel
// wrote, and may start while that kernel ends.
template <typename... KArgs, typename... Args>
static cudaError_t launch_dependent(void (*kernel)(KArgs...), dim3 grid, dim3 block,
                                    cudaStream_t st, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

static hp_status launch_scale(hp_cnn* c, const float* div, const uint8_t* flags, int B,
                              size_t cells, cudaStream_t st)
{
    cnn_scale_partial_kernel<<<dim3(kScaleCtas, B), kScaleThreads, 0, st>>>(div, flags, c->s_part,
                                                                          c->s_cnt, cells);
    hp_status rc = check_launch();
    if (rc != HP_OK) return rc;
    cudaError_t e = launch_dependent(cnn_scale_finish_kernel, dim3(B), dim3(32), st,
                                     (const double*)c->s_part,
                                     (const unsigned long long*)c->s_cnt, c->s);
    if (e != cudaSuccess) { set_cuda_error(e); return HP_ERR_CUDA; }
    return check_launch();
}

// branch input (pooling / up-sampling) and the cin -> 32 convolution: on the
// tensor cores (input padded to 16 BF16 channels) from the width the
// warp-specialised kernel serves, else on CUDA cores from the FP32 input.
// xin_keep (may be null) receives the FP32 branch input for the weight
// gradient of training.
static hp_status launch_first(hp_cnn* c, int k, const BranchIn& in, int cin, float* xin_keep,
                              const float* w, const float* bias, __nv_bfloat16* y, int B, int H,
                              int W, cudaStream_t st)
{
    const bool tc = W >= conv_tc_min_width();
    float* xin = xin_keep ? xin_keep : (tc ? nullptr : c->xin);
    const long cap = 16L * c->num_sms;
    // the four-pixel kernel's vector loads need 16-byte aligned rows
    if (W % 4 == 0 && in.W % (4 * in.scale) == 0 && (reinterpret_cast<uintptr_t>(in.div) & 15) == 0 &&
        (reinterpret_cast<uintptr_t>(in.flags) & 15) == 0) {
        const long quads = (long)B * H * W / 4;
        const int blocks = (int)((quads + 255) / 256 < cap ? (quads + 255) / 256 : cap);
        cudaError_t e = launch_dependent(branch_input4_kernel, dim3(blocks), dim3(256), st, in, cin,
                                         xin, tc ? c->x16 : nullptr, B);
        if (e != cudaSuccess) { set_cuda_error(e); return HP_ERR_CUDA; }
    } else {
        const int rows = B * H;
        const dim3 grid((W + 127) / 128, rows < 65535 ? rows : 65535);
        cudaError_t e = launch_dependent(branch_input_kernel, grid, dim3(128), st, in, cin, xin,
                                         tc ? c->x16 : nullptr, B);
        if (e != cudaSuccess) { set_cuda_error(e); return HP_ERR_CUDA; }
    }
    hp_status rc = check_launch();
    if (rc != HP_OK) return rc;
    if (tc)
        return launch_conv3x3_tc(c->x16, c->wtc_first[k], bias, y, B, H, W, 16, 32, 1, c->err,
                                 c->num_sms, st, c->wait_limit, true);
    const long P2 = (long)B * H * ((W + 1) / 2);
    const int blocks2 = (int)((P2 + 127) / 128 < cap ? (P2 + 127) / 128 : cap);
    cudaError_t e;
    if (cin == 2)
        e = launch_dependent(conv_first_kernel<2>, dim3(blocks2), dim3(128), st,
                             (const float*)xin, w, bias, y, B, H, W);
    else if (cin == 3)
        e = launch_dependent(conv_first_kernel<3>, dim3(blocks2), dim3(128), st,
                             (const float*)xin, w, bias, y, B, H, W);
    else
        return HP_ERR_UNSUPPORTED;
    if (e != cudaSuccess) { set_cuda_error(e); return HP_ERR_CUDA; }
    return check_launch();
}

// the 32 -> 1 convolution: tensor cores from the width the warp-specialised
// kernel serves, else CUDA cores
static hp_status launch_last(hp_cnn* c, int k, const __nv_bfloat16* x, const float* w,
                             const float* bias, float* y, int B, int H, int W, cudaStream_t st)
{
    if (W >= conv_tc_min_width())
        return launch_conv3x3_tc_out1(x, c->wtc_last[k], c->btc_last[k], y, B, H, W, c->err,
                                      c->num_sms, st, c->wait_limit, true);
    const long T = (long)B * ((H + kLastRows - 1) / kLastRows) * W;
    const long cap = 16L * c->num_sms;
    const int blocks = (int)((T + 127) / 128 < cap ? (T + 127) / 128 : cap);
    cudaError_t e = launch_dependent(conv_last_kernel, dim3(blocks), dim3(128), st, x, w, bias, y,
                                     B, H, W);
    if (e != cudaSuccess) { set_cuda_error(e); return HP_ERR_CUDA; }
    return check_launch();
}

// What a trainer keeps of a Unet forward: every layer's output, the inputs
// that are not a layer output (the max-pooled skip features of levels 1-4,
// the concatenated decoder inputs of levels 0-3) and the FP32 first-layer
// input.
struct UnetKeep {
    void* act[kLayersUnet];
    __nv_bfloat16* pooled[5];  // [lev], lev = 1..4: input of layer 2 lev
    __nv_bfloat16* cat[4];     // [lev]: input of the first decoder layer of level lev
    float* xin0;
};

// The Unet's forward: its 20 layers in order on the stream (tensor-core
// convolutions from a width of 32 pixels, the gather kernel or CUDA cores
// below), skip features kept per level, decoder inputs built by
// up_concat_kernel.  Activations ping-pong between act[0] and act[1], or with
// `keep` go to the trainer's buffers.
static hp_status unet_forward(hp_cnn* c, const float* div, const uint8_t* flags, float* phi_hat,
                              hp_shape s, cudaStream_t st, const UnetKeep* keep = nullptr)
{
    const LayerSpec* sp = c->spec;
    const int B = s.batch;
    int l = 0;
    hp_status rc = HP_OK;
    auto conv = [&](const void* x, void* y, int H, int W) {
        if (rc == HP_OK)
            rc = launch_conv3x3_tc(x, c->w[l], c->bias[l], y, B, H, W, sp[l].cin, sp[l].cout,
                                   sp[l].relu, c->err, c->num_sms, st, c->wait_limit, true);
        ++l;
    };
    // one block row per output row, the row's items across blockIdx.y
    auto pool = [&](const __nv_bfloat16* x, __nv_bfloat16* y, int H, int W) {
        if (rc != HP_OK) return;
        const dim3 grid((unsigned)(B * (H / 2)), (unsigned)((W / 2 * 4 + 255) / 256));
        cudaError_t e = launch_dependent(maxpool2_kernel, grid, dim3(256), st, (const uint4*)x,
                                         (uint4*)y, H, W, 4);
        if (e != cudaSuccess) { set_cuda_error(e); rc = HP_ERR_CUDA; return; }
        rc = check_launch();
    };
    auto up_concat = [&](const __nv_bfloat16* coarse, const __nv_bfloat16* sk, __nv_bfloat16* y,
                         int H, int W) {
        if (rc != HP_OK) return;
        const dim3 grid((unsigned)(B * H), (unsigned)((W * 8 + 255) / 256));
        cudaError_t e = launch_dependent(up_concat_kernel, grid, dim3(256), st,
                                         (const uint4*)coarse, (const uint4*)sk, (uint4*)y, H, W);
        if (e != cudaSuccess) { set_cuda_error(e); rc = HP_ERR_CUDA; return; }
        rc = check_launch();
    };
    __nv_bfloat16* a = c->act[0];
    __nv_bfloat16* b = c->act[1];
    // the output buffer of layer `layer`: the trainer's, else the given one
    auto out = [&](int layer, __nv_bfloat16* pp) {
        return keep ? (__nv_bfloat16*)keep->act[layer] : pp;
    };
    __nv_bfloat16* skip[4];
    // encoder level 0: [div/s, flags] -> 32 -> 32
    BranchIn in = {div, flags, c->s, nullptr, s.ny, s.nx, 1};
    __nv_bfloat16* x = out(0, a);
    rc = launch_first(c, 0, in, sp[0].cin, keep ? keep->xin0 : nullptr, (const float*)c->w[0],
                      c->bias[0], x, B, s.ny, s.nx, st);
    l = 1;
    skip[0] = out(1, c->skip[0]);
    conv(x, skip[0], s.ny, s.nx);
    // levels 1-3: max pooling, 32 -> 64 -> 32
    for (int lev = 1; lev < 4; ++lev) {
        const int H = s.ny >> lev, W = s.nx >> lev;
        __nv_bfloat16* pin = keep ? keep->pooled[lev] : a;
        pool(skip[lev - 1], pin, 2 * H, 2 * W);
        __nv_bfloat16* y = out(l, b);
        conv(pin, y, H, W);
        skip[lev] = out(l, c->skip[lev]);
        conv(y, skip[lev], H, W);
    }
    // bottom: 32 -> 64 -> 64 -> 32
    __nv_bfloat16* cur;
    {
        const int H = s.ny >> 4, W = s.nx >> 4;
        __nv_bfloat16* pin = keep ? keep->pooled[4] : a;
        pool(skip[3], pin, 2 * H, 2 * W);
        __nv_bfloat16* y1 = out(l, b);
        conv(pin, y1, H, W);
        __nv_bfloat16* y2 = out(l, a);
        conv(y1, y2, H, W);
        cur = out(l, b);
        conv(y2, cur, H, W);
    }
    // decoder: [up(coarser), skip] -> two convolutions
    __nv_bfloat16* other = a;
    for (int lev = 3; lev >= 0; --lev) {
        const int H = s.ny >> lev, W = s.nx >> lev;
        __nv_bfloat16* catb = keep ? keep->cat[lev] : other;
        up_concat(cur, skip[lev], catb, H, W);
        __nv_bfloat16* y1 = out(l, cur);
        conv(catb, y1, H, W);
        __nv_bfloat16* y2 = out(l, other);
        conv(y1, y2, H, W);
        other = y1;
        cur = y2;
    }
    if (rc != HP_OK) return rc;
    // the 1 x 1 output convolution 32 -> 1 (FP32)
    float* o = keep ? (float*)keep->act[l] : phi_hat;
    return launch_last(c, 0, cur, (const float*)c->w[l], c->bias[l], o, B, s.ny, s.nx, st);
}

// tensor-core copies of the first and last layer of every branch
static hp_status pack_edge_layers(hp_cnn* c, cudaStream_t st)
{
    for (int k = 0; k < c->br.n; ++k) {
        const int lf = c->br.first[k], ll = c->br.last[k];
        pack_edge_layers_kernel<<<(9 * 32 * 16 + 255) / 256, 256, 0, st>>>(
            (const float*)c->w[lf], c->spec[lf].cin, c->wtc_first[k], (const float*)c->w[ll],
            c->bias[ll], c->wtc_last[k], c->btc_last[k]);
        hp_status rc = check_launch();
        if (rc != HP_OK) return rc;
    }
    return HP_OK;
}

// weights of layer l in the parameter vector (ks x ks taps) and on the device
// (always 9 taps; a 1 x 1 layer has only the centre tap non-zero)
static size_t layer_wcount(const LayerSpec* sp, int l)
{
    return (size_t)sp[l].ks * sp[l].ks * sp[l].cin * sp[l].cout;
}

static size_t dev_wcount(const LayerSpec* sp, int l) { return (size_t)9 * sp[l].cin * sp[l].cout; }

extern "C" {

int64_t hp_cnn_arch_param_count(int32_t arch)
{
    const LayerSpec* sp = spec_for(arch);
    if (!sp) return -1;
    int64_t n = 0;
    for (int l = 0; l < layers_for(arch); ++l) n += (int64_t)layer_wcount(sp, l) + sp[l].cout;
    return n;
}

int64_t hp_cnn_param_count(void) { return hp_cnn_arch_param_count(HP_CNN_MULTISCALE); }

int32_t hp_cnn_get_arch(const hp_cnn* c) { return c ? c->arch : -1; }

void hp_cnn_destroy(hp_cnn* c)
{
    if (!c) return;
    for (int l = 0; l < kMaxLayers; ++l) {
        cudaFree(c->w[l]);
        cudaFree(c->bias[l]);
    }
    cudaFree(c->act[0]);
    cudaFree(c->act[1]);
    for (int k = 0; k < kMaxBranches; ++k) cudaFree(c->out[k]);
    cudaFree(c->xin);
    cudaFree(c->x16);
    for (int k = 0; k < kMaxBranches; ++k) {
        cudaFree(c->wtc_first[k]);
        cudaFree(c->wtc_last[k]);
        cudaFree(c->btc_last[k]);
    }
    for (int k = 0; k < 4; ++k) cudaFree(c->skip[k]);
    cudaFree(c->s_part);
    cudaFree(c->s_cnt);
    cudaFree(c->s);
    cudaFree(c->err);
    cudaFree(c->guess_bad);
    delete c;
}

hp_status hp_cnn_create_arch(hp_cnn** out, int32_t arch, hp_shape mx, int device)
{
    if (!out) return HP_ERR_INVALID_ARG;
    *out = nullptr;
    if (!spec_for(arch) || !shape_ok(mx) || mx.ny % size_multiple(arch) ||
        mx.nx % size_multiple(arch))
        return HP_ERR_INVALID_ARG;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) { set_cuda_error(e); return HP_ERR_CUDA; }
    hp_cnn* c = new hp_cnn();
    c->arch = arch;
    c->spec = spec_for(arch);
    c->nlayers = layers_for(arch);
    c->br = branches_of(c->spec, c->nlayers);
    memset(c->w, 0, sizeof(c->w));
    memset(c->out, 0, sizeof(c->out));
    memset(c->skip, 0, sizeof(c->skip));
    memset(c->bias, 0, sizeof(c->bias));
    c->device = device;
    c->max_shape = mx;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    c->master.assign((size_t)hp_cnn_arch_param_count(arch), 0.0f);
    const size_t px = (size_t)mx.batch * mx.ny * mx.nx;
    bool okm = true;
    // every buffer with a guard zone (checked by hp_cnn_check)
    auto ga = [&](auto pp, size_t bytes) {
        return guarded_malloc((void**)pp, bytes, &c->guards);
    };
    for (int l = 0; l < c->nlayers && okm; ++l) {
        const LayerSpec& ls = c->spec[l];
        const size_t wb = dev_wcount(c->spec, l) * (ls.cin >= 32 && ls.cout >= 32 ? 2 : 4);
        okm = ga(&c->w[l], wb) == cudaSuccess &&
              ga((void**)&c->bias[l], c->spec[l].cout * sizeof(float)) == cudaSuccess;
        if (okm) {
            cudaMemset(c->w[l], 0, wb);
            cudaMemset(c->bias[l], 0, c->spec[l].cout * sizeof(float));
        }
    }
    okm = okm && ga((void**)&c->act[0], px * 64 * 2) == cudaSuccess &&
          ga((void**)&c->act[1], px * 64 * 2) == cudaSuccess &&
          ga((void**)&c->xin, px * 3 * sizeof(float)) == cudaSuccess &&
          ga((void**)&c->x16, px * 16 * 2) == cudaSuccess &&
          ga((void**)&c->s_part, (size_t)mx.batch * kScaleCtas * sizeof(double)) ==
              cudaSuccess &&
          ga((void**)&c->s_cnt, (size_t)mx.batch * kScaleCtas * sizeof(unsigned long long)) ==
              cudaSuccess &&
          ga((void**)&c->s, mx.batch * sizeof(float)) == cudaSuccess &&
          ga((void**)&c->err, sizeof(int)) == cudaSuccess &&
          ga((void**)&c->guess_bad, mx.batch * sizeof(int32_t)) == cudaSuccess;
    for (int k = 0; k < c->br.n && okm; ++k)
        okm = ga((void**)&c->out[k], px / ((size_t)c->br.scale[k] * c->br.scale[k]) * 4) ==
                  cudaSuccess &&
              ga((void**)&c->wtc_first[k], 9 * 32 * 16 * 2) == cudaSuccess &&
              ga((void**)&c->wtc_last[k], 9 * 16 * 32 * 2) == cudaSuccess &&
              ga((void**)&c->btc_last[k], 16 * sizeof(float)) == cudaSuccess;
    if (arch == HP_CNN_UNET)
        for (int k = 0; k < 4 && okm; ++k)
            okm = ga((void**)&c->skip[k], (px >> (2 * k)) * 32 * 2) == cudaSuccess;
    if (!okm) {
        set_cuda_error(cudaGetLastError());
        hp_cnn_destroy(c);
        return HP_ERR_OOM;
    }
    cudaMemset(c->err, 0, sizeof(int));
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { set_cuda_error(e); hp_cnn_destroy(c); return HP_ERR_CUDA; }
    *out = c;
    return HP_OK;
}

hp_status hp_cnn_create(hp_cnn** out, hp_shape mx, int device)
{
    return hp_cnn_create_arch(out, HP_CNN_MULTISCALE, mx, device);
}

// params: host FP32 in the order of the network, each layer weights
// [cout][cin][ks][ks] then bias [cout].  Weights are rounded to BF16 on
// upload; a 1 x 1 layer is stored as a 3 x 3 with zero outer taps.
hp_status hp_cnn_set_params(hp_cnn* c, const float* params, int64_t n)
{
    if (!c || !params || n != hp_cnn_arch_param_count(c->arch)) return HP_ERR_INVALID_ARG;
    memcpy(c->master.data(), params, (size_t)n * sizeof(float));
    const float* p = params;
    for (int l = 0; l < c->nlayers; ++l) {
        const int ci = c->spec[l].cin, co = c->spec[l].cout;
        const bool tc = ci >= 32 && co >= 32;
        std::vector<uint16_t> wb;
        std::vector<float> wf;
        const size_t nw = dev_wcount(c->spec, l);
        const bool k1 = c->spec[l].ks == 1;
        if (tc) wb.assign(nw, 0); else wf.assign(nw, 0.0f);
        for (int o = 0; o < co; ++o)
            for (int i = 0; i < ci; ++i)
                for (int t = 0; t < 9; ++t) {
                    const float v = k1 ? (t == 4 ? p[(size_t)o * ci + i] : 0.0f)
                                       : p[((size_t)o * ci + i) * 9 + t];
                    const __nv_bfloat16 h = __float2bfloat16_rn(v);
                    if (tc) {
                        uint16_t bits;
                        memcpy(&bits, &h, 2);
                        wb[((size_t)t * co + o) * ci + i] = bits;  // [tap][cout][cin]
                    } else if (co == 1) {
                        wf[(size_t)t * ci + i] = __bfloat162float(h);  // [tap][cin]
                    } else {
                        wf[((size_t)t * ci + i) * co + o] = __bfloat162float(h);  // [tap][cin][cout]
                    }
                }
        p += layer_wcount(c->spec, l);
        cudaError_t e = tc ? cudaMemcpy(c->w[l], wb.data(), wb.size() * 2, cudaMemcpyHostToDevice)
                           : cudaMemcpy(c->w[l], wf.data(), wf.size() * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(c->bias[l], p, co * sizeof(float), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { set_cuda_error(e); return HP_ERR_CUDA; }
        p += co;
    }
    // the tensor-core copies of the first and last layers
    hp_status rc = pack_edge_layers(c, nullptr);
    if (rc != HP_OK) return rc;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { set_cuda_error(e); return HP_ERR_CUDA; }
    return HP_OK;
}

hp_status hp_cnn_get_params(const hp_cnn* c, float* params, int64_t n)
{
    if (!c || !params || n != hp_cnn_arch_param_count(c->arch)) return HP_ERR_INVALID_ARG;
    memcpy(params, c->master.data(), (size_t)n * sizeof(float));
    return HP_OK;
}

// phi_hat (FP32 [B][H][W], unscaled network output) and s (FP32 [B]).
hp_status hp_cnn_forward(hp_cnn* c, const float* div, const uint8_t* flags, float* phi_hat,
                         float* s_out, hp_shape s, void* stream)
{
    if (!c || !div || !flags || !cnn_shape_ok(c, s)) return HP_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t cells = (size_t)s.ny * s.nx;
    hp_status rc = launch_scale(c, div, flags, s.batch, cells, st);
    if (rc != HP_OK) return rc;
    if (c->arch == HP_CNN_UNET) {
        rc = unet_forward(c, div, flags, phi_hat ? phi_hat : c->out[0], s, st);
        if (rc != HP_OK) return rc;
        if (s_out) {
            cudaError_t e = cudaMemcpyAsync(s_out, c->s, s.batch * sizeof(float),
                                            cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) { set_cuda_error(e); return HP_ERR_CUDA; }
        }
        return HP_OK;
    }
    int l = 0;
    const float* prev = nullptr;
    for (int k = 0; k < c->br.n; ++k) {
        const int scale = c->br.scale[k];
        const int H = s.ny / scale, W = s.nx / scale;
        BranchIn in = {div, flags, c->s, prev, s.ny, s.nx, scale};
        int cur = 0;
        rc = launch_first(c, k, in, c->spec[l].cin, nullptr, (const float*)c->w[l], c->bias[l],
                          c->act[cur], s.batch, H, W, st);
        if (rc != HP_OK) return rc;
        ++l;
        while (c->spec[l].cout != 1) {
            rc = launch_conv3x3_tc(c->act[cur], c->w[l], c->bias[l], c->act[cur ^ 1], s.batch, H,
                                   W, c->spec[l].cin, c->spec[l].cout, c->spec[l].relu, c->err,
                                   c->num_sms, st, c->wait_limit, true);
            if (rc != HP_OK) return rc;
            cur ^= 1;
            ++l;
        }
        float* o = (k == c->br.n - 1 && phi_hat) ? phi_hat : c->out[k];
        rc = launch_last(c, k, c->act[cur], (const float*)c->w[l], c->bias[l], o, s.batch, H, W,
                         st);
        if (rc != HP_OK) return rc;
        ++l;
        prev = o;
    }
    if (s_out) {
        cudaError_t e = cudaMemcpyAsync(s_out, c->s, s.batch * sizeof(float),
                                        cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) { set_cuda_error(e); return HP_ERR_CUDA; }
    }
    return HP_OK;
}

hp_status hp_project_hybrid(hp_ctx* ctx, hp_cnn* cnn, float* u, float* v, const uint8_t* flags,
                            hp_shape s, const hp_project_params* prm, float* p_out,
                            int32_t* iters_out, double* e1_out, double* einf_out,
                            uint8_t* conv_out, double* e_hist, int32_t hist_len, void* stream)
{
    // every argument of both halves is checked before anything is launched
    if (!cnn || !project_args_ok(ctx, u, v, flags, s, prm, iters_out, e_hist, hist_len) ||
        !cnn_shape_ok(cnn, s))
        return HP_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    // divergence into the context, CNN guess into the second phi buffer
    hp_status rc = launch_mask_div(u, v, flags, ctx->mask, ctx->div, s, st, boundary_of(*prm));
    if (rc != HP_OK) return rc;
    float* phi_hat = cnn->out[cnn->br.n - 1];
    rc = hp_cnn_forward(cnn, ctx->div, flags, phi_hat, nullptr, s, stream);
    if (rc != HP_OK) return rc;
    // a grid whose guess is not finite starts from zero (the network's guess
    // is always followed and judged by the Jacobi sweeps, Sec. 3.3)
    const size_t cells = (size_t)s.ny * s.nx;
    cudaError_t e = cudaMemsetAsync(cnn->guess_bad, 0, s.batch * sizeof(int32_t), st);
    if (e != cudaSuccess) { set_cuda_error(e); return HP_ERR_CUDA; }
    const size_t n = (size_t)s.batch * cells;
    const size_t cap = (size_t)8 * cnn->num_sms;
    guess_check_kernel<<<(unsigned)((n + 255) / 256 < cap ? (n + 255) / 256 : cap), 256, 0, st>>>(
        phi_hat, cnn->s, ctx->mask, cnn->guess_bad, s.batch, cells);
    if ((rc = check_launch()) != HP_OK) return rc;
    phi0_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(phi_hat, cnn->s, ctx->mask,
                                                             cnn->guess_bad, ctx->phi[1],
                                                             cnn->err, s.batch, cells);
    if ((rc = check_launch()) != HP_OK) return rc;
    // the mask and divergence of the context are those of this velocity
    return project_impl(ctx, u, v, flags, s, prm, ctx->phi[1], p_out, iters_out, e1_out,
                        einf_out, conv_out, e_hist, hist_len, st, nullptr, true);
}

hp_status hp_cnn_set_wait_limit(hp_cnn* c, uint32_t polls)
{
    if (!c) return HP_ERR_INVALID_ARG;
    c->wait_limit = polls;
    return HP_OK;
}

}  // extern "C"

// ======================================================================
// Training of the MultiScale CNN (Sec. 3.2: the networks are trained with a
// gradient-descent algorithm; here the pairs come from the plain solver).
// FP32 master weights, Adam, BF16 weights refreshed after every step; the
// backward convolutions run on CUDA cores in FP32.
//
// Loss per grid (readings in the design notes), averaged over the batch; both
// terms are relative (t = phi*/s, d = div/s, e = phi_hat - t):
//   sup = sum_fluid (e - mean e)^2 / sum_fluid (t - mean t)^2
//   div = lambda * sum r^2 / sum d^2,  r = d - L phi_hat on cells with an open
//         face (the divergence of the corrected field of the scaled problem)
// ======================================================================

namespace hp {

namespace {

__global__ void relu_mask_kernel(float* __restrict__ g, const __nv_bfloat16* __restrict__ y,
                                 size_t n)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && !(__bfloat162float(y[i]) > 0.0f)) g[i] = 0.0f;
}

// Input pixel i receives, through tap offset o in {-1, 0, 1}, from the output
// rows y with clamp(y + o) == i: among {i-o-1, i-o, i-o+1}.
__device__ __forceinline__ bool reads(int y, int o, int i, int n)
{
    return y >= 0 && y < n && min(max(y + o, 0), n - 1) == i;
}

__device__ __forceinline__ float ld_act(const __nv_bfloat16* x, size_t i) { return __bfloat162float(x[i]); }
__device__ __forceinline__ float ld_act(const float* x, size_t i) { return x[i]; }
__device__ __forceinline__ void st_val(float* y, size_t i, float v) { y[i] = v; }
__device__ __forceinline__ void st_val(__nv_bfloat16* y, size_t i, float v) { y[i] = __float2bfloat16_rn(v); }

// dL/dx of a 3 x 3 convolution with replicated borders: gx[p][ci] = sum over
// taps and the output pixels that read p through that tap of
// w[t][co][ci] * gy[o][co].  w: FP32 [9][CO][CI] (the BF16-rounded weights).
// With act (BF16 [P][CI]) the result is zeroed where act is not positive
// (the ReLU derivative of the layer that produced the input).
template <int CI, int CO, typename GT = float, typename OT = float>
__global__ void conv_dgrad_kernel(const GT* __restrict__ gy, const float* __restrict__ w,
                                  OT* __restrict__ gx, int B, int H, int W,
                                  const __nv_bfloat16* __restrict__ act = nullptr)
{
    extern __shared__ float sw[];
    for (int q = threadIdx.x; q < 9 * CO * CI; q += blockDim.x) sw[q] = w[q];
    __syncthreads();
    // a thread computes 16 input channels of one pixel (more threads than
    // one per pixel: the narrow images this kernel serves have few pixels)
    constexpr int CG = 16, NG = CI / CG;
    const long P = (long)B * H * W;
    for (long item = (long)blockIdx.x * blockDim.x + threadIdx.x; item < P * NG;
         item += (long)gridDim.x * blockDim.x) {
        const long p = item / NG;
        const int c0 = (int)(item - p * NG) * CG;
        const int b = (int)(p / ((long)H * W));
        const int r = (int)(p - (long)b * H * W);
        const int i = r / W, j = r - i * W;
        float acc[CG];
#pragma unroll
        for (int c = 0; c < CG; ++c) acc[c] = 0.0f;
        for (int t = 0; t < 9; ++t) {
            const int oy = t / 3 - 1, ox = t % 3 - 1;
            for (int yy = i - oy - 1; yy <= i - oy + 1; ++yy) {
                if (!reads(yy, oy, i, H)) continue;
                for (int xx = j - ox - 1; xx <= j - ox + 1; ++xx) {
                    if (!reads(xx, ox, j, W)) continue;
                    const size_t g = (((size_t)b * H + yy) * W + xx) * CO;
                    const float* wt = sw + t * CO * CI + c0;
                    for (int co = 0; co < CO; ++co) {
                        const float gv = ld_act(gy, g + co);
#pragma unroll
                        for (int c = 0; c < CG; ++c) acc[c] = fmaf(wt[co * CI + c], gv, acc[c]);
                    }
                }
            }
        }
#pragma unroll
        for (int c = 0; c < CG; ++c) {
            const size_t q = (size_t)p * CI + c0 + c;
            const bool keep = !act || __bfloat162float(act[q]) > 0.0f;
            st_val(gx, q, keep ? acc[c] : 0.0f);
        }
    }
}

// Weight gradient partial sums over a chunk of pixels for one tap:
// part[(chunk * 9 + t)][co][ci] = sum_p gy[p][co] * x[clamp(p + offset_t)][ci];
// the centre tap also writes the bias partials partb[chunk][co] = sum_p gy.
// Each thread owns a BCO x BCI block of (co, ci).
template <int CI, int CO, int BCI, int BCO, typename XT, typename GT = float>
__global__ void conv_wgrad_kernel(const GT* __restrict__ gy, const XT* __restrict__ x,
                                  float* __restrict__ part, float* __restrict__ partb, int B,
                                  int H, int W, int chunk)
{
    constexpr int TP = 32;  // pixels per shared-memory tile
    __shared__ float sg[TP][CO];
    __shared__ float sx[TP][CI];
    const int t = blockIdx.y;
    const int oy = t / 3 - 1, ox = t % 3 - 1;
    const long P = (long)B * H * W;
    const long p0 = (long)blockIdx.x * chunk;
    const long p1 = min(P, p0 + chunk);
    const int ncb = CI / BCI;
    const int tco = (threadIdx.x / ncb) * BCO, tci = (threadIdx.x % ncb) * BCI;
    float acc[BCO][BCI];
    float accb[BCO];
#pragma unroll
    for (int a = 0; a < BCO; ++a) {
        accb[a] = 0.0f;
#pragma unroll
        for (int c = 0; c < BCI; ++c) acc[a][c] = 0.0f;
    }
    for (long pt = p0; pt < p1; pt += TP) {
        for (int q = threadIdx.x; q < TP * CO; q += blockDim.x) {
            const long p = pt + q / CO;
            sg[q / CO][q % CO] = p < p1 ? ld_act(gy, (size_t)p * CO + q % CO) : 0.0f;
        }
        for (int q = threadIdx.x; q < TP * CI; q += blockDim.x) {
            const long p = pt + q / CI;
            float v = 0.0f;
            if (p < p1) {
                const int b = (int)(p / ((long)H * W));
                const int r = (int)(p - (long)b * H * W);
                const int i = r / W, j = r - i * W;
                const int si = min(max(i + oy, 0), H - 1), sj = min(max(j + ox, 0), W - 1);
                v = ld_act(x, (((size_t)b * H + si) * W + sj) * CI + q % CI);
            }
            sx[q / CI][q % CI] = v;
        }
        __syncthreads();
        if (threadIdx.x < (CO / BCO) * ncb) {
            for (int k = 0; k < TP; ++k) {
#pragma unroll
                for (int a = 0; a < BCO; ++a) {
                    const float g = sg[k][tco + a];
                    accb[a] += g;
#pragma unroll
                    for (int c = 0; c < BCI; ++c) acc[a][c] = fmaf(g, sx[k][tci + c], acc[a][c]);
                }
            }
        }
        __syncthreads();
    }
    if (threadIdx.x < (CO / BCO) * ncb) {
        float* dst = part + ((size_t)blockIdx.x * 9 + t) * CO * CI;
#pragma unroll
        for (int a = 0; a < BCO; ++a)
#pragma unroll
            for (int c = 0; c < BCI; ++c) dst[(tco + a) * CI + tci + c] = acc[a][c];
        if (t == 4 && tci == 0)
#pragma unroll
            for (int a = 0; a < BCO; ++a) partb[(size_t)blockIdx.x * CO + tco + a] = accb[a];
    }
}

// grad[co][ci][t] (oracle order) = sum over chunks of part[k][t][co][ci];
// bias likewise.  A block of 256 threads serves 32 outputs; thread group j
// (of 8) sums the chunks k = j (mod 8) in FP64, and the 8 group sums are
// added in a fixed order.
// Launch with ceil((9 CO CI + CO) / 32) blocks of 256 threads.
__global__ void __launch_bounds__(256) wgrad_reduce_kernel(const float* __restrict__ part,
                                                           const float* __restrict__ partb,
                                                           int nchunks, int CI, int CO,
                                                           float* __restrict__ gw,
                                                           float* __restrict__ gb)
{
    __shared__ double sh[8][32];
    const int o = threadIdx.x & 31, j = threadIdx.x >> 5;
    // q walks the partials' own layout [t][co][ci], so that the 32 lanes of a
    // group read 32 consecutive floats of every partial; the result goes to
    // the oracle order [co][ci][t]
    const int q = blockIdx.x * 32 + o;
    const int nw = 9 * CO * CI;
    double s = 0.0;
    if (q < nw) {
        const size_t step = (size_t)9 * CO * CI;
        for (int k = j; k < nchunks; k += 8) s += part[(size_t)k * step + q];
    } else if (q < nw + CO) {
        const int co = q - nw;
        for (int k = j; k < nchunks; k += 8) s += partb[(size_t)k * CO + co];
    }
    sh[j][o] = s;
    __syncthreads();
    if (j == 0) {
        double t = 0.0;
        for (int g = 0; g < 8; ++g) t += sh[g][o];
        if (q < nw) {
            const int tap = q / (CO * CI), co = (q / CI) % CO, ci = q % CI;
            gw[((size_t)co * CI + ci) * 9 + tap] = (float)t;
        } else if (q < nw + CO) {
            gb[q - nw] = (float)t;
        }
    }
}

static unsigned reduce_blocks(int ci, int co) { return (unsigned)((9 * co * ci + co + 31) / 32); }

// The three (position p, tap offset d) pairs through which a 3-tap
// convolution with replicated borders along an axis of length n reads
// position j: clamp(p + d) == j (interior: p = j - d; at an end one tap is
// clamped onto j; n == 1: every tap).
struct AxisPairs {
    int p[3], d[3];
};

__device__ __forceinline__ AxisPairs axis_pairs(int j, int n)
{
    AxisPairs a;
    if (n == 1) {
        a.p[0] = 0; a.d[0] = -1; a.p[1] = 0; a.d[1] = 0; a.p[2] = 0; a.d[2] = 1;
    } else if (j == 0) {
        a.p[0] = 1; a.d[0] = -1; a.p[1] = 0; a.d[1] = 0; a.p[2] = 0; a.d[2] = -1;
    } else if (j == n - 1) {
        a.p[0] = n - 1; a.d[0] = 1; a.p[1] = n - 1; a.d[1] = 0; a.p[2] = n - 2; a.d[2] = 1;
    } else {
        a.p[0] = j + 1; a.d[0] = -1; a.p[1] = j; a.d[1] = 0; a.p[2] = j - 1; a.d[2] = 1;
    }
    return a;
}

// Input gradient of the last layer of a branch (32 -> 1): gx[j][ci] = sum
// over the 9 pairs of w[tap][ci] * gy[p], optionally zeroed where act (BF16
// [P][32]) is not positive.  Thread = (pixel, chunk of 8 channels), so that
// a warp stores 8 whole pixels.  w: FP32 [9][32].
template <typename OT>
__global__ void dgrad_last_kernel(const float* __restrict__ gy, const float* __restrict__ w,
                                  OT* __restrict__ gx, int B, int H, int W,
                                  const __nv_bfloat16* __restrict__ act)
{
    __shared__ float sw[9 * 32];
    for (int i = threadIdx.x; i < 9 * 32; i += blockDim.x) sw[i] = w[i];
    __syncthreads();
    const long P = (long)B * H * W;
    const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= P * 4) return;
    const long pix = q >> 2;
    const int c = (int)(q & 3);
    const int b = (int)(pix / ((long)H * W));
    const int rem = (int)(pix - (long)b * H * W);
    const int jy = rem / W, jx = rem - jy * W;
    const AxisPairs ay = axis_pairs(jy, H), ax = axis_pairs(jx, W);
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const float* g = gy + (size_t)b * H * W;
#pragma unroll
    for (int u = 0; u < 3; ++u)
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            const float gv = g[(size_t)ay.p[u] * W + ax.p[v]];
            const float* wt = sw + (3 * (ay.d[u] + 1) + ax.d[v] + 1) * 32 + 8 * c;
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[k] = fmaf(wt[k], gv, acc[k]);
        }
    const size_t o = (size_t)pix * 32 + 8 * c;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const bool keep = !act || __bfloat162float(act[o + k]) > 0.0f;
        st_val(gx, o + k, keep ? acc[k] : 0.0f);
    }
}

// Gradient of input channel 2 (the up-sampled coarser output) of the first
// layer of a branch (3 -> 32): gx2[j] = sum over the 9 pairs of
// sum_co w[tap][co][2] * gy[p][co].  w: FP32 [9][32][3]; gx2 FP32 [P].
template <typename GT>
__global__ void dgrad_first_ch2_kernel(const GT* __restrict__ gy, const float* __restrict__ w,
                                       float* __restrict__ gx2, int B, int H, int W)
{
    __shared__ float sw[9 * 32];
    for (int i = threadIdx.x; i < 9 * 32; i += blockDim.x) sw[i] = w[i * 3 + 2];
    __syncthreads();
    const long P = (long)B * H * W;
    const long pix = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= P) return;
    const int b = (int)(pix / ((long)H * W));
    const int rem = (int)(pix - (long)b * H * W);
    const int jy = rem / W, jx = rem - jy * W;
    const AxisPairs ay = axis_pairs(jy, H), ax = axis_pairs(jx, W);
    float acc = 0.0f;
#pragma unroll
    for (int u = 0; u < 3; ++u)
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            const size_t src = (((size_t)b * H + ay.p[u]) * W + ax.p[v]) * 32;
            const float* wt = sw + (3 * (ay.d[u] + 1) + ax.d[v] + 1) * 32;
            if constexpr (sizeof(GT) == 2) {
                const uint4* g4 = reinterpret_cast<const uint4*>(gy + src);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint4 t = g4[k];
                    const uint32_t e[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        acc = fmaf(wt[8 * k + 2 * h], __uint_as_float(e[h] << 16), acc);
                        acc = fmaf(wt[8 * k + 2 * h + 1], __uint_as_float(e[h] & 0xFFFF0000u), acc);
                    }
                }
            } else {
#pragma unroll 8
                for (int co = 0; co < 32; ++co) acc = fmaf(wt[co], ld_act(gy, src + co), acc);
            }
        }
    gx2[pix] = acc;
}

// Row groups per block of the sliding-window weight gradients.
constexpr int kRowGroups = 4;

// Weight and bias gradient of the last layer of a branch (32 -> 1) over the
// g-th of G equal ranges of image rows: part[g][tap][ci], partb[g].  Block =
// kRowGroups x 3 warps: row group rg takes every kRowGroups-th row of the
// range, warp = row offset dy, lane = input channel; every input pixel is
// read once per warp and feeds the three column taps through a sliding
// window of the output gradient (with the replicated-border terms at both row
// ends); the row groups are added in a fixed order.
__global__ void __launch_bounds__(96 * kRowGroups) wgrad_last_kernel(
    const float* __restrict__ gy, const __nv_bfloat16* __restrict__ x, float* __restrict__ part,
    float* __restrict__ partb, int B, int H, int W)
{
    __shared__ float sh[kRowGroups][4][96];
    const int rg = threadIdx.x / 96, tw = threadIdx.x % 96;
    const int dyo = tw / 32 - 1, ci = tw & 31;
    const long R = (long)B * H;
    const long r0 = R * blockIdx.x / gridDim.x, r1 = R * (blockIdx.x + 1) / gridDim.x;
    float am = 0.0f, a0 = 0.0f, ap = 0.0f, bsum = 0.0f;
    for (long r = r0 + rg; r < r1; r += kRowGroups) {
        const int b = (int)(r / H), y = (int)(r - (long)b * H);
        const int ys = min(max(y + dyo, 0), H - 1);
        const float* g = gy + (size_t)r * W;
        const __nv_bfloat16* xr = x + ((size_t)b * H + ys) * W * 32 + ci;
        float gl = 0.0f, gc = g[0];
#pragma unroll 4
        for (int xs = 0; xs < W; ++xs) {
            const float gr = xs + 1 < W ? g[xs + 1] : 0.0f;
            const float X = __bfloat162float(xr[(size_t)xs * 32]);
            am = fmaf(gr + (xs == 0 ? gc : 0.0f), X, am);
            a0 = fmaf(gc, X, a0);
            ap = fmaf(gl + (xs == W - 1 ? gc : 0.0f), X, ap);
            bsum += gc;
            gl = gc;
            gc = gr;
        }
    }
    sh[rg][0][tw] = am;
    sh[rg][1][tw] = a0;
    sh[rg][2][tw] = ap;
    sh[rg][3][tw] = bsum;
    __syncthreads();
    if (rg == 0) {
        float v[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        for (int k = 0; k < kRowGroups; ++k)
#pragma unroll
            for (int c = 0; c < 4; ++c) v[c] += sh[k][c][tw];
        float* dst = part + (size_t)blockIdx.x * 9 * 32;
        const int t0 = 3 * (dyo + 1);
        dst[(t0 + 0) * 32 + ci] = v[0];
        dst[(t0 + 1) * 32 + ci] = v[1];
        dst[(t0 + 2) * 32 + ci] = v[2];
        if (dyo == 0 && ci == 0) partb[blockIdx.x] = v[3];
    }
}

// Weight and bias gradient of the first layer of a branch (CX -> 32, input
// FP32 [P][CX]) over the g-th of G row ranges: part[g][tap][co][ci],
// partb[g][co].  Same organisation as wgrad_last_kernel with lane = output
// channel.
template <int CX, typename GT>
__global__ void __launch_bounds__(96 * kRowGroups) wgrad_first_kernel(
    const GT* __restrict__ gy, const float* __restrict__ x, float* __restrict__ part,
    float* __restrict__ partb, int B, int H, int W)
{
    constexpr int NV = 3 * CX + 1;
    __shared__ float sh[kRowGroups][NV][96];
    const int rg = threadIdx.x / 96, tw = threadIdx.x % 96;
    const int dyo = tw / 32 - 1, co = tw & 31;
    const long R = (long)B * H;
    const long r0 = R * blockIdx.x / gridDim.x, r1 = R * (blockIdx.x + 1) / gridDim.x;
    float am[CX], a0[CX], ap[CX];
#pragma unroll
    for (int c = 0; c < CX; ++c) am[c] = a0[c] = ap[c] = 0.0f;
    float bsum = 0.0f;
    for (long r = r0 + rg; r < r1; r += kRowGroups) {
        const int b = (int)(r / H), y = (int)(r - (long)b * H);
        const int ys = min(max(y + dyo, 0), H - 1);
        const size_t g0 = (size_t)r * W * 32 + co;
        const float* xr = x + ((size_t)b * H + ys) * W * CX;
        float gl = 0.0f, gc = ld_act(gy, g0);
#pragma unroll 4
        for (int xs = 0; xs < W; ++xs) {
            const float gr = xs + 1 < W ? ld_act(gy, g0 + (size_t)(xs + 1) * 32) : 0.0f;
            const float gm = gr + (xs == 0 ? gc : 0.0f);
            const float gq = gl + (xs == W - 1 ? gc : 0.0f);
#pragma unroll
            for (int c = 0; c < CX; ++c) {
                const float X = xr[(size_t)xs * CX + c];
                am[c] = fmaf(gm, X, am[c]);
                a0[c] = fmaf(gc, X, a0[c]);
                ap[c] = fmaf(gq, X, ap[c]);
            }
            bsum += gc;
            gl = gc;
            gc = gr;
        }
    }
#pragma unroll
    for (int c = 0; c < CX; ++c) {
        sh[rg][3 * c + 0][tw] = am[c];
        sh[rg][3 * c + 1][tw] = a0[c];
        sh[rg][3 * c + 2][tw] = ap[c];
    }
    sh[rg][3 * CX][tw] = bsum;
    __syncthreads();
    if (rg == 0) {
        float v[NV];
#pragma unroll
        for (int c = 0; c < NV; ++c) v[c] = 0.0f;
        for (int k = 0; k < kRowGroups; ++k)
#pragma unroll
            for (int c = 0; c < NV; ++c) v[c] += sh[k][c][tw];
        float* dst = part + (size_t)blockIdx.x * 9 * 32 * CX;
        const int t0 = 3 * (dyo + 1);
#pragma unroll
        for (int c = 0; c < CX; ++c) {
            dst[((t0 + 0) * 32 + co) * CX + c] = v[3 * c + 0];
            dst[((t0 + 1) * 32 + co) * CX + c] = v[3 * c + 1];
            dst[((t0 + 2) * 32 + co) * CX + c] = v[3 * c + 2];
        }
        if (dyo == 0) partb[(size_t)blockIdx.x * 32 + co] = v[3 * CX];
    }
}

// Border terms of the input gradient of a 3 x 3 convolution with replicated
// borders.  The forward reads x at clamp(p + d); extended by a ring of ghost
// pixels holding the replicated values, it is a plain convolution, whose
// transpose puts w[d]^T gy[q - d] on every extended pixel q, and an input
// pixel j collects the ghost pixels q with clamp(q) = j.  The tensor-core
// pass computes the transpose with zero padding on the image and folds the
// ghost rows -1 and H into rows 0 and H - 1; this kernel adds the ghost
// pixels in columns -1 and W (corner ghosts included) to the first and last
// column.  One warp per pixel, lanes over the input channels; the terms get
// the ReLU derivative of act (may be null) and are added to gx (BF16 [P][CI],
// rounded again).  w: FP32 [9][CO][CI].
template <int CI, int CO>
__global__ void dgrad_border_kernel(const __nv_bfloat16* __restrict__ gy,
                                    const float* __restrict__ w,
                                    const __nv_bfloat16* __restrict__ act,
                                    __nv_bfloat16* __restrict__ gx, int B, int H, int W)
{
    constexpr int PER = CI / 32;
    const int ncol = W > 1 ? 2 : 1;
    const long per_img = (long)H * ncol;
    const long e_all = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (e_all >= (long)B * per_img) return;
    const int b = (int)(e_all / per_img);
    const int e = (int)(e_all - (long)b * per_img);
    const int jy = e / ncol, jx = (e % ncol) ? W - 1 : 0;
    float acc[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) acc[k] = 0.0f;
    const int gys[3] = {jy, jy == 0 ? -1 : jy, jy == H - 1 ? H : jy};
    const int gxs[3] = {jx, jx == 0 ? -1 : jx, jx == W - 1 ? W : jx};
    for (int a = 0; a < 3; ++a) {
        const int qy = gys[a];
        if (a > 0 && qy == jy) continue;
        for (int c = 1; c < 3; ++c) {
            const int qx = gxs[c];
            if (qx == jx) continue;  // only ghost columns; the rest is the tensor-core pass
            for (int dy = -1; dy <= 1; ++dy) {
                const int py = qy - dy;
                if (py < 0 || py >= H) continue;
                for (int dx = -1; dx <= 1; ++dx) {
                    const int px = qx - dx;
                    if (px < 0 || px >= W) continue;
                    const __nv_bfloat16* g = gy + (((size_t)b * H + py) * W + px) * CO;
                    const float* wt = w + (size_t)(3 * (dy + 1) + dx + 1) * CO * CI;
                    for (int co = 0; co < CO; ++co) {
                        const float gv = __bfloat162float(g[co]);
#pragma unroll
                        for (int k = 0; k < PER; ++k)
                            acc[k] = fmaf(wt[co * CI + lane + 32 * k], gv, acc[k]);
                    }
                }
            }
        }
    }
    const size_t q = (((size_t)b * H + jy) * W + jx) * CI;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int ci = lane + 32 * k;
        if (act && !(__bfloat162float(act[q + ci]) > 0.0f)) continue;
        gx[q + ci] = __float2bfloat16_rn(__bfloat162float(gx[q + ci]) + acc[k]);
    }
}

// transpose of the bilinear x 2 up-sampling (gradient of the coarse output)
// from channel `ch` of a fine-grid gradient with `stride` channels
__device__ __forceinline__ float up_w(int f, int I, int n)
{
    const int c = f >> 1, a = f & 1;
    const int nb = a ? min(c + 1, n - 1) : max(c - 1, 0);
    return (c == I ? 0.75f : 0.0f) + (nb == I ? 0.25f : 0.0f);
}

__global__ void upsample_adjoint_kernel(const float* __restrict__ gfine, int stride, int ch,
                                        float* __restrict__ gcoarse, int B, int hc, int wc)
{
    const long P = (long)B * hc * wc;
    const long p = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int b = (int)(p / ((long)hc * wc));
    const int r = (int)(p - (long)b * hc * wc);
    const int J = r / wc, I = r - J * wc;
    const int hf = 2 * hc, wf = 2 * wc;
    float s = 0.0f;
    for (int fy = 2 * J - 1; fy <= 2 * J + 2; ++fy) {
        if (fy < 0 || fy >= hf) continue;
        const float wy = up_w(fy, J, hc);
        if (wy == 0.0f) continue;
        for (int fx = 2 * I - 1; fx <= 2 * I + 2; ++fx) {
            if (fx < 0 || fx >= wf) continue;
            const float wx = up_w(fx, I, wc);
            if (wx == 0.0f) continue;
            s += wy * wx * gfine[(((size_t)b * hf + fy) * wf + fx) * stride + ch];
        }
    }
    gcoarse[p] = s;
}

// residual of the scaled problem and per-grid loss sums (one CTA per grid):
// stats[b] = {sum_f e, sum_f e^2, N_f, sum r^2, sum_f t, sum_f t^2, sum d^2}
// with t = target/s, d = div/s, e = phi - t
constexpr int kStats = 7;

__global__ void loss_stats_kernel(const float* __restrict__ phi, const float* __restrict__ target,
                                  const float* __restrict__ div, const uint8_t* __restrict__ mask,
                                  const uint8_t* __restrict__ flags, const float* __restrict__ s,
                                  float* __restrict__ rbuf, double* __restrict__ stats, int ny,
                                  int nx)
{
    __shared__ double sh[kStats][32];
    const int b = blockIdx.x;
    const size_t cells = (size_t)ny * nx, base = (size_t)b * cells;
    const float inv_s = 1.0f / s[b];
    double v[kStats] = {0, 0, 0, 0, 0, 0, 0};
    for (size_t c = threadIdx.x; c < cells; c += blockDim.x) {
        const uint32_t m = mask[base + c];
        const float pc = phi[base + c];
        const float dc = div[base + c] * inv_s;
        float r = 0.0f;
        if (m & 15u) {
            float lap = 0.0f;
            if (m & 1u) lap += phi[base + c - 1] - pc;
            if (m & 2u) lap += phi[base + c + 1] - pc;
            if (m & 4u) lap += phi[base + c - nx] - pc;
            if (m & 8u) lap += phi[base + c + nx] - pc;
            r = dc - lap;
        }
        rbuf[base + c] = r;
        v[3] += (double)r * r;
        v[6] += (double)dc * dc;
        if (flags[base + c] == 0) {
            const double t = (double)target[base + c] * inv_s;
            const double e = (double)pc - t;
            v[0] += e;
            v[1] += e * e;
            v[2] += 1.0;
            v[4] += t;
            v[5] += t * t;
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < kStats; ++k) {
        for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
        if (lane == 0) sh[k][wid] = v[k];
    }
    __syncthreads();
    if (threadIdx.x < kStats) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[threadIdx.x][w];
        stats[(size_t)b * kStats + threadIdx.x] = t;
    }
}

__device__ __forceinline__ double target_var(const double* st)
{
    return st[2] > 0.0 ? st[5] - st[4] * st[4] / st[2] : 0.0;
}

// dL/dphi_hat per cell
__global__ void loss_grad_kernel(const float* __restrict__ phi, const float* __restrict__ target,
                                 const float* __restrict__ rbuf, const uint8_t* __restrict__ mask,
                                 const uint8_t* __restrict__ flags, const float* __restrict__ s,
                                 const double* __restrict__ stats, float lambda,
                                 float* __restrict__ g, int B, int ny, int nx)
{
    const size_t cells = (size_t)ny * nx;
    const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (size_t)B * cells) return;
    const int b = (int)(q / cells);
    const double* st = stats + (size_t)b * kStats;
    const double nf = st[2], vt = target_var(st), d2 = st[6];
    float gv = 0.0f;
    if (flags[q] == 0 && nf > 0.0 && vt > 0.0) {
        const double e = (double)phi[q] - (double)target[q] / s[b];
        gv = (float)(2.0 * (e - st[0] / nf) / (vt * B));
    }
    const uint32_t m = mask[q];
    if ((m & 15u) && d2 > 0.0) {
        const float rc = rbuf[q];
        float lr = 0.0f;
        if (m & 1u) lr += rbuf[q - 1] - rc;
        if (m & 2u) lr += rbuf[q + 1] - rc;
        if (m & 4u) lr += rbuf[q - nx] - rc;
        if (m & 8u) lr += rbuf[q + nx] - rc;
        gv -= (float)(2.0 * lambda / (d2 * B)) * lr;
    }
    g[q] = gv;
}

// sum of 32 lanes' values in a fixed order (lane 0 gets the result)
__device__ __forceinline__ double warp_sum_fixed(double v)
{
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    return v;
}

// one warp: lane l takes the grids b = l (mod 32) in order
__global__ void loss_finish_kernel(const double* __restrict__ stats, int B, size_t cells,
                                   float lambda, double* __restrict__ loss)
{
    double L = 0.0;
    for (int b = threadIdx.x; b < B; b += 32) {
        const double* st = stats + (size_t)b * kStats;
        const double vt = target_var(st);
        if (st[2] > 0.0 && vt > 0.0) L += (st[1] - st[0] * st[0] / st[2]) / vt;
        if (st[6] > 0.0) L += lambda * st[3] / st[6];
    }
    (void)cells;
    L = warp_sum_fixed(L);
    if (threadIdx.x == 0) *loss = L / B;
}

// physics-driven loss (Sec. 3.2, Eq. 4) of the network-corrected field: the
// guess s * phi_hat removes the divergence s * r with r = d - L phi_hat, the
// residual of the scaled problem (0 on cells without an open face).  One CTA
// per grid: rbuf <- dloss/dr = weight * norm * s^norm * |r|^(norm-1) sign(r)
// / cells, stats[b] <- sum |s r|^norm
__global__ void pdnn_stats_kernel(const float* __restrict__ phi, const float* __restrict__ div,
                                  const uint8_t* __restrict__ mask, const float* __restrict__ s,
                                  const float* __restrict__ weight, int norm,
                                  float* __restrict__ rbuf, double* __restrict__ stats, int ny,
                                  int nx)
{
    __shared__ double sh[32];
    const int b = blockIdx.x;
    const size_t cells = (size_t)ny * nx, base = (size_t)b * cells;
    const float sb = s[b], inv_s = 1.0f / sb;
    const float coef = norm == 1 ? weight[b] * sb / (float)cells
                                 : 2.0f * weight[b] * sb * sb / (float)cells;
    double acc = 0.0;
    for (size_t c = threadIdx.x; c < cells; c += blockDim.x) {
        const uint32_t m = mask[base + c];
        float r = 0.0f;
        if (m & 15u) {
            const float pc = phi[base + c];
            float lap = 0.0f;
            if (m & 1u) lap += phi[base + c - 1] - pc;
            if (m & 2u) lap += phi[base + c + 1] - pc;
            if (m & 4u) lap += phi[base + c - nx] - pc;
            if (m & 8u) lap += phi[base + c + nx] - pc;
            r = div[base + c] * inv_s - lap;
        }
        const double sr = (double)sb * (double)r;
        float g;
        if (norm == 1) {
            acc += fabs(sr);
            g = r > 0.0f ? coef : r < 0.0f ? -coef : 0.0f;
        } else {
            acc += sr * sr;
            g = coef * r;
        }
        rbuf[base + c] = g;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if (lane == 0) sh[wid] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        stats[b] = t;
    }
}

// dL/dphi_hat = -L^T dL/dr = -L (dL/dr): the masked Laplacian is symmetric
__global__ void pdnn_grad_kernel(const float* __restrict__ rbuf, const uint8_t* __restrict__ mask,
                                 float* __restrict__ g, int B, int ny, int nx)
{
    const size_t cells = (size_t)ny * nx;
    const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (size_t)B * cells) return;
    const uint32_t m = mask[q];
    float lr = 0.0f;
    if (m & 15u) {
        const float rc = rbuf[q];
        if (m & 1u) lr += rbuf[q - 1] - rc;
        if (m & 2u) lr += rbuf[q + 1] - rc;
        if (m & 4u) lr += rbuf[q - nx] - rc;
        if (m & 8u) lr += rbuf[q + nx] - rc;
    }
    g[q] = -lr;
}

// one warp, as loss_finish_kernel
__global__ void pdnn_finish_kernel(const double* __restrict__ stats,
                                   const float* __restrict__ weight, int B, size_t cells,
                                   double* __restrict__ loss)
{
    double L = 0.0;
    for (int b = threadIdx.x; b < B; b += 32) L += (double)weight[b] * stats[b] / (double)cells;
    L = warp_sum_fixed(L);
    if (threadIdx.x == 0) *loss = L;
}

__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, long n, float lr, float b1, float b2, float eps,
                            float c1, float c2)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// masters (oracle order [co][ci][3][3] + bias) of one layer -> the layouts of
// the forward kernels (BF16-rounded) and the FP32 [9][co][ci] copy for dgrad
// and, for the tensor-core layers, the BF16 weights of the input-gradient
// convolution: flipped taps, input and output swapped, wdg[8 - t][ci][co]
// A 1 x 1 layer (ks = 1, masters [co][ci] + bias) is packed as a 3 x 3 whose
// outer taps are zero.
__global__ void pack_layer_kernel(const float* __restrict__ master, int ci, int co, int kind,
                                  int ks, void* __restrict__ wfwd, float* __restrict__ bias,
                                  float* __restrict__ wt, __nv_bfloat16* __restrict__ wdg)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int nw = 9 * ci * co;
    if (q < nw) {
        const int t = q % 9, i = (q / 9) % ci, o = q / (9 * ci);
        const float mv = ks == 3 ? master[q] : (t == 4 ? master[o * ci + i] : 0.0f);
        const __nv_bfloat16 h = __float2bfloat16_rn(mv);
        const float f = __bfloat162float(h);
        if (kind == 0) reinterpret_cast<__nv_bfloat16*>(wfwd)[((size_t)t * co + o) * ci + i] = h;
        else if (kind == 1) reinterpret_cast<float*>(wfwd)[((size_t)t * ci + i) * co + o] = f;
        else reinterpret_cast<float*>(wfwd)[(size_t)t * ci + i] = f;
        wt[((size_t)t * co + o) * ci + i] = f;
        if (wdg) wdg[((size_t)(8 - t) * ci + i) * co + o] = h;
    } else if (q < nw + co) {
        bias[q - nw] = master[(ks == 3 ? nw : ci * co) + (q - nw)];
    }
}

// ------------------------------------------------------ Unet backward

// Transpose of up_concat_kernel at decoder level L (H x W): channels 32-63 of
// gcat ([P][64]) are the gradient of the skip features (copied to FP32
// gskip [P][32]); channels 0-31 go back through the bilinear x 2 up-sampling
// (each coarse pixel gathers its fine pixels with the up-sampling's weights,
// in a fixed order) to the coarse features gcoarse [Pc][32], times the ReLU
// derivative of the coarse activation act (BF16 [Pc][32]).  One warp per
// coarse pixel and one per fine pixel (the copy); lane = channel.
template <typename GT, typename OT>
__global__ void cat_backward_kernel(const GT* __restrict__ gcat, float* __restrict__ gskip,
                                    OT* __restrict__ gcoarse, const __nv_bfloat16* __restrict__ act,
                                    int B, int H, int W)
{
    const int Hc = H / 2, Wc = W / 2;
    const long Pc = (long)B * Hc * Wc, Pf = (long)B * H * W;
    const long wid = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid < Pc) {
        const int b = (int)(wid / ((long)Hc * Wc));
        const int r = (int)(wid - (long)b * Hc * Wc);
        const int J = r / Wc, I = r - J * Wc;
        float sum = 0.0f;
        for (int fy = 2 * J - 1; fy <= 2 * J + 2; ++fy) {
            if (fy < 0 || fy >= H) continue;
            const float wy = up_w(fy, J, Hc);
            if (wy == 0.0f) continue;
            for (int fx = 2 * I - 1; fx <= 2 * I + 2; ++fx) {
                if (fx < 0 || fx >= W) continue;
                const float wx = up_w(fx, I, Wc);
                if (wx == 0.0f) continue;
                sum += wy * wx * ld_act(gcat, (((size_t)b * H + fy) * W + fx) * 64 + lane);
            }
        }
        const size_t q = (size_t)wid * 32 + lane;
        st_val(gcoarse, q, __bfloat162float(act[q]) > 0.0f ? sum : 0.0f);
    } else if (wid < Pc + Pf) {
        const size_t p = (size_t)(wid - Pc);
        gskip[p * 32 + lane] = ld_act(gcat, p * 64 + 32 + lane);
    }
}

// Gradient of the skip features x (BF16 [P][32], encoder level L, H x W) into
// the pre-activation gradient of the layer that produced them: the decoder's
// share gskip (FP32 [P][32]) plus the max-pooling transpose of gpool
// ([P/4][32]: each pooled gradient goes to the first maximum of its 2 x 2
// window in the order (0, 0), (0, 1), (1, 0), (1, 1)), times the ReLU
// derivative of x.  One thread per (pixel, channel).
template <typename GT, typename OT>
__global__ void pool_backward_kernel(const GT* __restrict__ gpool,
                                     const __nv_bfloat16* __restrict__ x,
                                     const float* __restrict__ gskip, OT* __restrict__ gout,
                                     int B, int H, int W)
{
    const size_t n = (size_t)B * H * W * 32;
    const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int c = (int)(q & 31);
    const size_t p = q >> 5;
    const int b = (int)(p / ((size_t)H * W));
    const int r = (int)(p - (size_t)b * H * W);
    const int j = r / W, i = r - j * W;
    const int j0 = j & ~1, i0 = i & ~1;
    const size_t base = (size_t)b * H * W;
    float v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
        v[k] = __bfloat162float(x[((base + (size_t)(j0 + (k >> 1)) * W + i0 + (k & 1)) << 5) + c]);
    const float m = fmaxf(fmaxf(v[0], v[1]), fmaxf(v[2], v[3]));
    const int first = v[0] == m ? 0 : v[1] == m ? 1 : v[2] == m ? 2 : 3;
    const int mine = ((j & 1) << 1) | (i & 1);
    float g = gskip[q];
    if (mine == first) {
        const size_t pc = ((size_t)b * (H / 2) + (j >> 1)) * (W / 2) + (i >> 1);
        g += ld_act(gpool, pc * 32 + c);
    }
    st_val(gout, q, v[mine] > 0.0f ? g : 0.0f);
}

// weight and bias gradient of a 1 x 1 layer from the 3 x 3 gradient of the
// same layer (g9 [co = 1][ci][9] + bias): its centre tap
__global__ void center_tap_kernel(const float* __restrict__ g9, int ci, float* __restrict__ gw,
                                  float* __restrict__ gb)
{
    const int i = threadIdx.x;
    if (i < ci) gw[i] = g9[i * 9 + 4];
    if (i == 0) gb[0] = g9[9 * ci];
}

}  // namespace

}  // namespace hp

struct hp_trainer {
    hp_cnn* cnn;
    hp_shape max;
    long param_count;
    float *master, *grad, *m, *v;
    float* wt[kMaxLayers];
    void* act[kMaxLayers];   // layer outputs: bf16 [P][cout] or float [P] (cout == 1)
    float* xin[kMaxBranches];  // first-layer inputs per branch, FP32 [P][cin]
    float* g[2];          // gradient ping-pong, FP32 [P][64]
    float* gsmall;        // first-layer input gradient, FP32 [P][3]
    __nv_bfloat16* wdg[kMaxLayers];  // input-gradient weights of the tensor-core layers
    float* zero_bias;     // 64 zeros: the bias of an input-gradient convolution
    float *part, *partb;
    size_t part_len, partb_len;
    float* rbuf;
    double* stats;
    double* loss;
    uint8_t* mask;
    int step;
    Guards guards;  // guard zones of the workspaces
    // Unet: the max-pooled and concatenated layer inputs, the skip features'
    // gradients from the decoder, the 3 x 3 gradient of the 1 x 1 layer
    __nv_bfloat16* upool[5];
    __nv_bfloat16* ucat[4];
    float* gskip[4];
    float* g9;
};

static long layer_offset(const LayerSpec* sp, int l)
{
    long off = 0;
    for (int k = 0; k < l; ++k) off += (long)layer_wcount(sp, k) + sp[k].cout;
    return off;
}

// layers whose backward runs on the tensor cores (at widths from
// conv_tc_min_width() up): 32 or 64 channels on both sides
static bool tc_layer(const LayerSpec* sp, int l) { return sp[l].cin >= 32 && sp[l].cout >= 32; }

static hp_status trainer_pack(hp_trainer* t, cudaStream_t st);

extern "C" {

void hp_trainer_destroy(hp_trainer* t)
{
    if (!t) return;
    cudaFree(t->master); cudaFree(t->grad); cudaFree(t->m); cudaFree(t->v);
    for (int l = 0; l < kMaxLayers; ++l) {
        cudaFree(t->wt[l]); cudaFree(t->act[l]); cudaFree(t->wdg[l]);
    }
    cudaFree(t->zero_bias);
    for (int k = 0; k < kMaxBranches; ++k) cudaFree(t->xin[k]);
    cudaFree(t->g[0]); cudaFree(t->g[1]); cudaFree(t->gsmall);
    cudaFree(t->part); cudaFree(t->partb); cudaFree(t->rbuf); cudaFree(t->stats);
    cudaFree(t->loss); cudaFree(t->mask);
    for (int k = 0; k < 5; ++k) cudaFree(t->upool[k]);
    for (int k = 0; k < 4; ++k) { cudaFree(t->ucat[k]); cudaFree(t->gskip[k]); }
    cudaFree(t->g9);
    delete t;
}

static constexpr int kWgradChunk = 2048;

hp_status hp_trainer_create(hp_trainer** out, hp_cnn* cnn, hp_shape mx)
{
    if (out) *out = nullptr;
    if (!out || !cnn || !shape_ok(mx) || mx.ny % size_multiple(cnn->arch) ||
        mx.nx % size_multiple(cnn->arch))
        return HP_ERR_INVALID_ARG;
    // the forward pass of training runs in the network's own input workspace
    // (scale, BF16 branch input), sized for its max_shape
    if (mx.batch > cnn->max_shape.batch || mx.ny > cnn->max_shape.ny ||
        mx.nx > cnn->max_shape.nx)
        return HP_ERR_INVALID_ARG;
    *out = nullptr;
    hp_trainer* t = new hp_trainer();
    t->cnn = cnn;
    t->max = mx;
    t->param_count = hp_cnn_arch_param_count(cnn->arch);
    const LayerSpec* sp = cnn->spec;
    const size_t P = (size_t)mx.batch * mx.ny * mx.nx;
    bool ok = true;
    auto al = [&](void** p, size_t bytes) {
        if (ok && guarded_malloc(p, bytes, &t->guards) != cudaSuccess) ok = false;
    };
    al((void**)&t->master, t->param_count * 4);
    al((void**)&t->grad, t->param_count * 4);
    al((void**)&t->m, t->param_count * 4);
    al((void**)&t->v, t->param_count * 4);
    for (int l = 0; l < cnn->nlayers; ++l) {
        const int sc = sp[l].scale;
        const size_t Pl = P / (sc * sc);
        al(&t->act[l], sp[l].cout == 1 ? Pl * 4 : Pl * sp[l].cout * 2);
        al((void**)&t->wt[l], dev_wcount(sp, l) * 4);
        if (tc_layer(sp, l)) al((void**)&t->wdg[l], layer_wcount(sp, l) * 2);
    }
    al((void**)&t->zero_bias, 64 * 4);
    for (int k = 0; k < cnn->br.n; ++k) {
        const int sc = cnn->br.scale[k];
        al((void**)&t->xin[k], P / (sc * sc) * 3 * 4);
    }
    al((void**)&t->g[0], P * 64 * 4);
    al((void**)&t->g[1], P * 64 * 4);
    al((void**)&t->gsmall, P * 3 * 4);
    // partial sums: one per pixel chunk (CUDA-core weight gradient) or per
    // CTA (tensor-core weight gradient, at most one CTA per SM)
    size_t nchunks = (P + kWgradChunk - 1) / kWgradChunk;
    if (nchunks < (size_t)cnn->num_sms) nchunks = (size_t)cnn->num_sms;
    t->part_len = nchunks * 9 * 64 * 64;
    // bias partials of up to 16 row blocks per SM (sliding-window kernels)
    t->partb_len = (nchunks > 16 * (size_t)cnn->num_sms ? nchunks : 16 * (size_t)cnn->num_sms) * 64;
    al((void**)&t->part, t->part_len * 4);
    al((void**)&t->partb, t->partb_len * 4);
    al((void**)&t->rbuf, P * 4);
    al((void**)&t->stats, (size_t)mx.batch * kStats * 8);
    al((void**)&t->loss, 8);
    al((void**)&t->mask, P);
    if (cnn->arch == HP_CNN_UNET) {
        for (int lev = 0; lev < 5; ++lev) {
            const size_t Pl = P >> (2 * lev);
            if (lev >= 1) al((void**)&t->upool[lev], Pl * 32 * 2);
            if (lev <= 3) {
                al((void**)&t->ucat[lev], Pl * 64 * 2);
                al((void**)&t->gskip[lev], Pl * 32 * 4);
            }
        }
        al((void**)&t->g9, (9 * 32 + 1) * 4);
    }
    if (!ok) { set_cuda_error(cudaGetLastError()); hp_trainer_destroy(t); return HP_ERR_OOM; }
    // masters from the network's current parameters
    cudaError_t e = cudaMemcpy(t->master, cnn->master.data(), t->param_count * 4,
                               cudaMemcpyHostToDevice);
    if (e == cudaSuccess && trainer_pack(t, 0) != HP_OK) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { set_cuda_error(e); hp_trainer_destroy(t); return HP_ERR_CUDA; }
    *out = t;
    return HP_OK;
}

}  // extern "C"

static hp_status trainer_pack(hp_trainer* t, cudaStream_t st)
{
    const LayerSpec* sp = t->cnn->spec;
    for (int l = 0; l < t->cnn->nlayers; ++l) {
        const int ci = sp[l].cin, co = sp[l].cout;
        const int kind = (ci >= 32 && co >= 32) ? 0 : (co == 1 ? 2 : 1);
        const int n = 9 * ci * co + co;
        pack_layer_kernel<<<(n + 255) / 256, 256, 0, st>>>(t->master + layer_offset(sp, l), ci, co,
                                                          kind, sp[l].ks, t->cnn->w[l],
                                                          t->cnn->bias[l], t->wt[l], t->wdg[l]);
    }
    hp_status rc = check_launch();
    if (rc != HP_OK) return rc;
    return pack_edge_layers(t->cnn, st);
}

// forward keeping every layer output
static hp_status trainer_forward(hp_trainer* t, const float* div, const uint8_t* flags,
                                 hp_shape s, cudaStream_t st)
{
    const LayerSpec* sp = t->cnn->spec;
    hp_cnn* c = t->cnn;
    const size_t cells = (size_t)s.ny * s.nx;
    hp_status rc = launch_scale(c, div, flags, s.batch, cells, st);
    if (rc != HP_OK) return rc;
    if (c->arch == HP_CNN_UNET) {
        UnetKeep keep;
        for (int l = 0; l < kLayersUnet; ++l) keep.act[l] = t->act[l];
        for (int k = 0; k < 5; ++k) keep.pooled[k] = t->upool[k];
        for (int k = 0; k < 4; ++k) keep.cat[k] = t->ucat[k];
        keep.xin0 = t->xin[0];
        return unet_forward(c, div, flags, nullptr, s, st, &keep);
    }
    const float* prev = nullptr;
    for (int k = 0, l = 0; k < c->br.n; ++k) {
        const int scale = c->br.scale[k];
        const int H = s.ny / scale, W = s.nx / scale;
        BranchIn in = {div, flags, c->s, prev, s.ny, s.nx, scale};
        rc = launch_first(c, k, in, sp[l].cin, t->xin[k], (const float*)c->w[l], c->bias[l],
                          (__nv_bfloat16*)t->act[l], s.batch, H, W, st);
        if (rc != HP_OK) return rc;
        ++l;
        while (sp[l].cout != 1) {
            rc = launch_conv3x3_tc(t->act[l - 1], c->w[l], c->bias[l], t->act[l], s.batch, H, W,
                                   sp[l].cin, sp[l].cout, sp[l].relu, c->err, c->num_sms,
                                   st, c->wait_limit, true);
            if (rc != HP_OK) return rc;
            ++l;
        }
        rc = launch_last(c, k, (const __nv_bfloat16*)t->act[l - 1], (const float*)c->w[l],
                         c->bias[l], (float*)t->act[l], s.batch, H, W, st);
        if (rc != HP_OK) return rc;
        prev = (const float*)t->act[l];
        ++l;
    }
    return HP_OK;
}

template <int CI, int CO, typename GT = float, typename OT = float>
static hp_status dgrad(const GT* gy, const float* w, OT* gx, int B, int H, int W, int nsm,
                       cudaStream_t st, const __nv_bfloat16* act = nullptr)
{
    const size_t smem = (size_t)9 * CI * CO * 4;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(conv_dgrad_kernel<CI, CO, GT, OT>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    const long items = (long)B * H * W * (CI / 16);
    const int blocks = (int)((items + 127) / 128 < 4L * nsm ? (items + 127) / 128 : 4L * nsm);
    conv_dgrad_kernel<CI, CO, GT, OT><<<blocks, 128, smem, st>>>(gy, w, gx, B, H, W, act);
    return check_launch();
}

static hp_status dgrad_dispatch(int ci, int co, const float* gy, const float* w, float* gx, int B,
                                int H, int W, int nsm, cudaStream_t st)
{
    if (ci == 64 && co == 64) return dgrad<64, 64>(gy, w, gx, B, H, W, nsm, st);
    if (ci == 32 && co == 64) return dgrad<32, 64>(gy, w, gx, B, H, W, nsm, st);
    if (ci == 64 && co == 32) return dgrad<64, 32>(gy, w, gx, B, H, W, nsm, st);
    if (ci == 32 && co == 32) return dgrad<32, 32>(gy, w, gx, B, H, W, nsm, st);
    return HP_ERR_UNSUPPORTED;
}

template <int CI, int CO, int BCI, int BCO, typename XT, typename GT = float>
static hp_status wgrad_t(hp_trainer* t, const GT* gy, const XT* x, float* gw, float* gb, int B,
                         int H, int W, cudaStream_t st)
{
    const long P = (long)B * H * W;
    // pixels per chunk: enough CTAs (9 taps x chunks) to fill the GPU about
    // four times over, whole 32-pixel tiles, at most kWgradChunk, and no more
    // chunks than the partial-sum buffer holds
    const long cap = (long)(t->part_len / ((size_t)9 * CO * CI));
    const long target = (4L * t->cnn->num_sms + 8) / 9;
    long chunk = (P + target - 1) / target;
    chunk = (chunk + 31) / 32 * 32;
    if (chunk > kWgradChunk) chunk = kWgradChunk;
    if ((P + chunk - 1) / chunk > cap) chunk = ((P + cap - 1) / cap + 31) / 32 * 32;
    const int nchunks = (int)((P + chunk - 1) / chunk);
    if ((size_t)nchunks * 9 * CO * CI > t->part_len || (size_t)nchunks * CO > t->partb_len)
        return HP_ERR_INVALID_ARG;
    const int threads = ((CO / BCO) * (CI / BCI) + 31) / 32 * 32;
    conv_wgrad_kernel<CI, CO, BCI, BCO, XT, GT><<<dim3(nchunks, 9), threads, 0, st>>>(
        gy, x, t->part, t->partb, B, H, W, (int)chunk);
    hp_status rc = check_launch();
    if (rc != HP_OK) return rc;
    wgrad_reduce_kernel<<<reduce_blocks(CI, CO), 256, 0, st>>>(t->part, t->partb, nchunks, CI, CO,
                                                             gw, gb);
    return check_launch();
}

// row ranges of the sliding-window weight gradients: four blocks of
// kRowGroups x 3 warps per SM (each warp scans its rows serially; the
// latency of one scan is hidden by the others)
static int row_blocks(hp_trainer* t, long rows)
{
    const long g = 4L * t->cnn->num_sms;
    return (int)(rows < g ? rows : g);
}

// weight and bias gradient of the last layer of a branch (32 -> 1)
static hp_status wgrad_last(hp_trainer* t, int l, const float* gy, float* gw, float* gb, int B,
                            int H, int W, cudaStream_t st)
{
    const int G = row_blocks(t, (long)B * H);
    if ((size_t)G * 9 * 32 > t->part_len || (size_t)G > t->partb_len) return HP_ERR_INVALID_ARG;
    wgrad_last_kernel<<<G, 96 * kRowGroups, 0, st>>>(gy, (const __nv_bfloat16*)t->act[l - 1],
                                                     t->part, t->partb, B, H, W);
    wgrad_reduce_kernel<<<reduce_blocks(32, 1), 256, 0, st>>>(t->part, t->partb, G, 32, 1, gw, gb);
    return check_launch();
}

// weight and bias gradient of the first layer of a branch (2 or 3 -> 32)
template <typename GT>
static hp_status wgrad_first(hp_trainer* t, int k, int l, const GT* gy, float* gw, float* gb,
                             int B, int H, int W, cudaStream_t st)
{
    const LayerSpec* sp = t->cnn->spec;
    const int cx = sp[l].cin;
    const int G = row_blocks(t, (long)B * H);
    if ((size_t)G * 9 * 32 * cx > t->part_len || (size_t)G * 32 > t->partb_len)
        return HP_ERR_INVALID_ARG;
    if (cx == 3)
        wgrad_first_kernel<3, GT><<<G, 96 * kRowGroups, 0, st>>>(gy, t->xin[k], t->part,
                                                                 t->partb, B, H, W);
    else
        wgrad_first_kernel<2, GT><<<G, 96 * kRowGroups, 0, st>>>(gy, t->xin[k], t->part,
                                                                 t->partb, B, H, W);
    wgrad_reduce_kernel<<<reduce_blocks(cx, 32), 256, 0, st>>>(t->part, t->partb, G, cx, 32, gw,
                                                              gb);
    return check_launch();
}

// gradient of input channel 2 of a first layer into t->gsmall (FP32 [P])
template <typename GT>
static hp_status dgrad_first_ch2(hp_trainer* t, int l, const GT* gy, int B, int H, int W,
                                 cudaStream_t st)
{
    const long P = (long)B * H * W;
    dgrad_first_ch2_kernel<GT><<<(unsigned)((P + 255) / 256), 256, 0, st>>>(gy, t->wt[l],
                                                                          t->gsmall, B, H, W);
    return check_launch();
}

template <typename OT>
static hp_status dgrad_last(hp_trainer* t, int l, const float* gy, OT* gx, int B, int H, int W,
                            const __nv_bfloat16* act, cudaStream_t st)
{
    const long n = (long)B * H * W * 4;
    dgrad_last_kernel<OT><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(gy, t->wt[l], gx, B, H, W,
                                                                      act);
    return check_launch();
}

static hp_status wgrad_dispatch(hp_trainer* t, int k, int l, const float* gy, const void* x,
                                float* gw, float* gb, int B, int H, int W, cudaStream_t st)
{
    const LayerSpec* sp = t->cnn->spec;
    const int ci = sp[l].cin, co = sp[l].cout;
    const __nv_bfloat16* xb = (const __nv_bfloat16*)x;
    if (ci == 64 && co == 64) return wgrad_t<64, 64, 4, 4>(t, gy, xb, gw, gb, B, H, W, st);
    if (ci == 32 && co == 64) return wgrad_t<32, 64, 4, 4>(t, gy, xb, gw, gb, B, H, W, st);
    if (ci == 64 && co == 32) return wgrad_t<64, 32, 4, 4>(t, gy, xb, gw, gb, B, H, W, st);
    if (ci == 32 && co == 32) return wgrad_t<32, 32, 4, 4>(t, gy, xb, gw, gb, B, H, W, st);
    if (ci == 32 && co == 1) return wgrad_last(t, l, gy, gw, gb, B, H, W, st);
    if (co == 32 && (ci == 3 || ci == 2)) return wgrad_first(t, k, l, gy, gw, gb, B, H, W, st);
    return HP_ERR_UNSUPPORTED;
}

// replicated-border terms of a tensor-core input gradient in the first and
// last column (the ghost rows are folded in by the tensor-core pass)
template <int CI, int CO>
static hp_status border_terms(const __nv_bfloat16* gy, const float* w, const __nv_bfloat16* act,
                              __nv_bfloat16* gx, int B, int H, int W, cudaStream_t st)
{
    const long nb = (long)B * H * (W > 1 ? 2 : 1);
    dgrad_border_kernel<CI, CO><<<(unsigned)((nb * 32 + 255) / 256), 256, 0, st>>>(gy, w, act, gx,
                                                                                  B, H, W);
    return check_launch();
}

// first layer of a branch (2 or 3 -> 32) from a BF16 gradient: weight
// gradient, and for the finer branches the gradient of the up-sampled coarser
// output (input channel 2) into gsmall
static hp_status first_layer_bf16(hp_trainer* t, int k, int l, const __nv_bfloat16* gy, int B,
                                  int H, int W, cudaStream_t st)
{
    const LayerSpec* sp = t->cnn->spec;
    float* gw = t->grad + layer_offset(sp, l);
    hp_status rc = wgrad_first(t, k, l, gy, gw, gw + layer_wcount(sp, l), B, H, W, st);
    if (rc != HP_OK || k == 0) return rc;
    return dgrad_first_ch2(t, l, gy, B, H, W, st);
}

// One branch on the tensor cores (width >= conv_tc_min_width()): gradients
// in BF16 [P][C], the ReLU derivative applied by the layer that produces each
// gradient.  gout: FP32 [P] gradient of the branch's 1-channel output.
static hp_status branch_backward_tc(hp_trainer* t, int k, int lfirst, int llast, float* gout,
                                    __nv_bfloat16* gbuf[2], int B, int H, int W, cudaStream_t st)
{
    const LayerSpec* sp = t->cnn->spec;
    hp_cnn* c = t->cnn;
    // last layer (32 -> 1, CUDA cores): weight gradient from the FP32 output
    // gradient, input gradient into BF16
    float* gw = t->grad + layer_offset(sp, llast);
    hp_status rc = wgrad_last(t, llast, gout, gw, gw + layer_wcount(sp, llast), B, H, W, st);
    if (rc != HP_OK) return rc;
    const __nv_bfloat16* mask_last =
        sp[llast - 1].relu ? (const __nv_bfloat16*)t->act[llast - 1] : nullptr;
    rc = dgrad_last(t, llast, gout, gbuf[0], B, H, W, mask_last, st);
    if (rc != HP_OK) return rc;
    int cur = 0;
    for (int l = llast - 1; l > lfirst; --l) {
        const int ci = sp[l].cin, co = sp[l].cout;
        const __nv_bfloat16* gy = gbuf[cur];
        const __nv_bfloat16* x = (const __nv_bfloat16*)t->act[l - 1];
        int grid = 0;
        rc = launch_conv3x3_tc_wgrad(x, gy, t->part, t->part_len, t->partb, t->partb_len, B, H, W,
                                     ci, co, c->err, c->num_sms, &grid, st, c->wait_limit);
        if (rc != HP_OK) return rc;
        gw = t->grad + layer_offset(sp, l);
        wgrad_reduce_kernel<<<reduce_blocks(ci, co), 256, 0, st>>>(t->part, t->partb, grid, ci, co,
                                                                   gw, gw + layer_wcount(sp, l));
        if ((rc = check_launch()) != HP_OK) return rc;
        // input gradient with the ReLU derivative of layer l - 1
        const __nv_bfloat16* act = sp[l - 1].relu ? x : nullptr;
        __nv_bfloat16* gx = gbuf[cur ^ 1];
        rc = launch_conv3x3_tc_dgrad(gy, t->wdg[l], t->zero_bias, act, gx, B, H, W, ci, co,
                                     c->err, c->num_sms, st, c->wait_limit);
        if (rc != HP_OK) return rc;
        if (ci == 64 && co == 64)
            rc = border_terms<64, 64>(gy, t->wt[l], act, gx, B, H, W, st);
        else if (ci == 32 && co == 64)
            rc = border_terms<32, 64>(gy, t->wt[l], act, gx, B, H, W, st);
        else if (ci == 64 && co == 32)
            rc = border_terms<64, 32>(gy, t->wt[l], act, gx, B, H, W, st);
        else
            rc = border_terms<32, 32>(gy, t->wt[l], act, gx, B, H, W, st);
        if (rc != HP_OK) return rc;
        cur ^= 1;
    }
    return first_layer_bf16(t, k, lfirst, gbuf[cur], B, H, W, st);
}

// Backward of one 3 x 3 layer l (32/64 channels) of an image H x W from the
// gradient gy of its pre-activation: weight and bias gradients into t->grad;
// with gx, the gradient of its input x with the ReLU derivative of mask_act
// (the activation x, when the layer that made it has a ReLU; may be null)
// applied.  From the width the tensor-core kernels serve, gy and gx are BF16
// and the contractions run on the tensor cores; below it they are FP32 on
// CUDA cores.
static hp_status layer_backward(hp_trainer* t, int l, const __nv_bfloat16* x, const void* gy,
                                void* gx, const __nv_bfloat16* mask_act, int B, int H, int W,
                                cudaStream_t st)
{
    const LayerSpec* sp = t->cnn->spec;
    hp_cnn* c = t->cnn;
    const int ci = sp[l].cin, co = sp[l].cout;
    float* gw = t->grad + layer_offset(sp, l);
    float* gb = gw + layer_wcount(sp, l);
    hp_status rc;
    if (W >= conv_tc_min_width()) {
        int grid = 0;
        rc = launch_conv3x3_tc_wgrad(x, gy, t->part, t->part_len, t->partb, t->partb_len, B, H, W,
                                     ci, co, c->err, c->num_sms, &grid, st, c->wait_limit);
        if (rc != HP_OK) return rc;
        wgrad_reduce_kernel<<<reduce_blocks(ci, co), 256, 0, st>>>(t->part, t->partb, grid, ci, co,
                                                                   gw, gb);
        if ((rc = check_launch()) != HP_OK || !gx) return rc;
        const __nv_bfloat16* g16 = (const __nv_bfloat16*)gy;
        __nv_bfloat16* gx16 = (__nv_bfloat16*)gx;
        rc = launch_conv3x3_tc_dgrad(g16, t->wdg[l], t->zero_bias, mask_act, gx16, B, H, W, ci, co,
                                     c->err, c->num_sms, st, c->wait_limit);
        if (rc != HP_OK) return rc;
        const float* wl = t->wt[l];
        if (ci == 64 && co == 64) return border_terms<64, 64>(g16, wl, mask_act, gx16, B, H, W, st);
        if (ci == 32 && co == 64) return border_terms<32, 64>(g16, wl, mask_act, gx16, B, H, W, st);
        if (ci == 64 && co == 32) return border_terms<64, 32>(g16, wl, mask_act, gx16, B, H, W, st);
        return border_terms<32, 32>(g16, wl, mask_act, gx16, B, H, W, st);
    }
    const float* g32 = (const float*)gy;
    rc = wgrad_dispatch(t, 0, l, g32, x, gw, gb, B, H, W, st);
    if (rc != HP_OK || !gx) return rc;
    float* gx32 = (float*)gx;
    const int nsm = c->num_sms;
    if (ci == 64 && co == 64) return dgrad<64, 64>(g32, t->wt[l], gx32, B, H, W, nsm, st, mask_act);
    if (ci == 32 && co == 64) return dgrad<32, 64>(g32, t->wt[l], gx32, B, H, W, nsm, st, mask_act);
    if (ci == 64 && co == 32) return dgrad<64, 32>(g32, t->wt[l], gx32, B, H, W, nsm, st, mask_act);
    return dgrad<32, 32>(g32, t->wt[l], gx32, B, H, W, nsm, st, mask_act);
}

template <typename GT, typename OT>
static hp_status cat_backward(const void* gcat, float* gskip, void* gcoarse,
                              const __nv_bfloat16* act, int B, int H, int W, cudaStream_t st)
{
    const long warps = (long)B * H * W + (long)B * (H / 2) * (W / 2);
    cat_backward_kernel<GT, OT><<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(
        (const GT*)gcat, gskip, (OT*)gcoarse, act, B, H, W);
    return check_launch();
}

template <typename GT, typename OT>
static hp_status pool_backward(const void* gpool, const __nv_bfloat16* x, const float* gskip,
                               void* gout, int B, int H, int W, cudaStream_t st)
{
    const size_t n = (size_t)B * H * W * 32;
    pool_backward_kernel<GT, OT><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
        (const GT*)gpool, x, gskip, (OT*)gout, B, H, W);
    return check_launch();
}

// The Unet's backward (the reading of the network is in the forward above):
// from dL/dphi_hat in t->g[0] down the decoder, through the bottom and back
// up the encoder, where each level's skip features collect the decoder's
// share and the max-pooling transpose.  Gradients ping-pong between g[0] and
// g[1] (BF16 at levels the tensor-core kernels serve, FP32 below).
static hp_status unet_backward(hp_trainer* t, hp_shape s, cudaStream_t st)
{
    hp_cnn* c = t->cnn;
    const LayerSpec* sp = c->spec;
    const int B = s.batch;
    auto Hl = [&](int lev) { return s.ny >> lev; };
    auto Wl = [&](int lev) { return s.nx >> lev; };
    auto bf = [&](int lev) { return Wl(lev) >= conv_tc_min_width(); };
    auto act = [&](int l) { return (const __nv_bfloat16*)t->act[l]; };
    // the activation of layer l when that layer has a ReLU (its derivative
    // is then applied), else null
    auto relu_of = [&](int l) { return sp[l].relu ? act(l) : nullptr; };
    void* g[2] = {t->g[0], t->g[1]};
    hp_status rc;
    // layer 19, the 1 x 1 output convolution 32 -> 1 (run as a 3 x 3 with
    // zero outer taps): its weight gradient is the centre tap
    const int L1 = kLayersUnet - 1;
    const float* gout = t->g[0];
    rc = wgrad_last(t, L1, gout, t->g9, t->g9 + 9 * 32, B, Hl(0), Wl(0), st);
    if (rc != HP_OK) return rc;
    {
        float* gw = t->grad + layer_offset(sp, L1);
        center_tap_kernel<<<1, 32, 0, st>>>(t->g9, 32, gw, gw + 32);
        if ((rc = check_launch()) != HP_OK) return rc;
    }
    if (bf(0))
        rc = dgrad_last(t, L1, gout, (__nv_bfloat16*)g[1], B, Hl(0), Wl(0), relu_of(L1 - 1), st);
    else
        rc = dgrad_last(t, L1, gout, (float*)g[1], B, Hl(0), Wl(0), relu_of(L1 - 1), st);
    if (rc != HP_OK) return rc;
    int cur = 1;  // g[cur] holds the pre-activation gradient of the next layer
    int l = L1 - 1;
    // decoder, level 0 up to 3: two convolutions, then the concatenation's
    // transpose into the skip gradient and the coarser level
    for (int lev = 0; lev < 4; ++lev) {
        const int H = Hl(lev), W = Wl(lev);
        // second convolution: input = output of the first (ReLU)
        rc = layer_backward(t, l, act(l - 1), g[cur], g[cur ^ 1], relu_of(l - 1), B, H, W, st);
        if (rc != HP_OK) return rc;
        cur ^= 1;
        --l;
        // first convolution: input = [up(coarser), skip], no ReLU of its own
        rc = layer_backward(t, l, t->ucat[lev], g[cur], g[cur ^ 1], nullptr, B, H, W, st);
        if (rc != HP_OK) return rc;
        cur ^= 1;
        --l;
        // l is now the layer whose output was up-sampled (the coarser level)
        const void* gc = g[cur];
        void* gn = g[cur ^ 1];
        float* gs = t->gskip[lev];
        if (bf(lev) && bf(lev + 1))
            rc = cat_backward<__nv_bfloat16, __nv_bfloat16>(gc, gs, gn, act(l), B, H, W, st);
        else if (bf(lev))
            rc = cat_backward<__nv_bfloat16, float>(gc, gs, gn, act(l), B, H, W, st);
        else
            rc = cat_backward<float, float>(gc, gs, gn, act(l), B, H, W, st);
        if (rc != HP_OK) return rc;
        cur ^= 1;
    }
    // bottom (level 4): 64 -> 32, 64 -> 64, 32 -> 64 on the pooled skip 3
    {
        const int H = Hl(4), W = Wl(4);
        rc = layer_backward(t, l, act(l - 1), g[cur], g[cur ^ 1], relu_of(l - 1), B, H, W, st);
        if (rc != HP_OK) return rc;
        cur ^= 1; --l;
        rc = layer_backward(t, l, act(l - 1), g[cur], g[cur ^ 1], relu_of(l - 1), B, H, W, st);
        if (rc != HP_OK) return rc;
        cur ^= 1; --l;
        rc = layer_backward(t, l, t->upool[4], g[cur], g[cur ^ 1], nullptr, B, H, W, st);
        if (rc != HP_OK) return rc;
        cur ^= 1; --l;
    }
    // encoder, level 3 down to 0: the skip features' gradient (decoder share
    // plus the pooling transpose), then the level's two convolutions
    for (int lev = 3; lev >= 0; --lev) {
        const int H = Hl(lev), W = Wl(lev);
        // l is the layer that produced the skip features of this level
        const void* gc = g[cur];
        void* gn = g[cur ^ 1];
        const float* gs = t->gskip[lev];
        if (bf(lev + 1) && bf(lev))
            rc = pool_backward<__nv_bfloat16, __nv_bfloat16>(gc, act(l), gs, gn, B, H, W, st);
        else if (bf(lev))
            rc = pool_backward<float, __nv_bfloat16>(gc, act(l), gs, gn, B, H, W, st);
        else
            rc = pool_backward<float, float>(gc, act(l), gs, gn, B, H, W, st);
        if (rc != HP_OK) return rc;
        cur ^= 1;
        rc = layer_backward(t, l, act(l - 1), g[cur], g[cur ^ 1], relu_of(l - 1), B, H, W, st);
        if (rc != HP_OK) return rc;
        cur ^= 1; --l;
        if (lev == 0) break;  // l = 0: the first layer, below
        // the level's first convolution reads the pooled skip features of
        // the level above; its input gradient feeds that level's pooling
        rc = layer_backward(t, l, t->upool[lev], g[cur], g[cur ^ 1], nullptr, B, H, W, st);
        if (rc != HP_OK) return rc;
        cur ^= 1; --l;
    }
    // layer 0, [div/s, flags] -> 32: weight gradient only
    float* gw = t->grad + layer_offset(sp, 0);
    if (bf(0))
        return wgrad_first(t, 0, 0, (const __nv_bfloat16*)g[cur], gw, gw + layer_wcount(sp, 0), B,
                           Hl(0), Wl(0), st);
    return wgrad_first(t, 0, 0, (const float*)g[cur], gw, gw + layer_wcount(sp, 0), B, Hl(0),
                       Wl(0), st);
}

// dL/dparams into t->grad from dL/dphi_hat in t->g[0] (the activations of
// the last trainer_forward)
static hp_status trainer_backward(hp_trainer* t, hp_shape s, cudaStream_t st)
{
    const LayerSpec* sp = t->cnn->spec;
    hp_cnn* c = t->cnn;
    hp_status rc = HP_OK;
    if (c->arch == HP_CNN_UNET) return unet_backward(t, s, st);
    // backward, branch by branch from full resolution
    int cur = 0;
    for (int k = c->br.n - 1, l = c->nlayers - 1; k >= 0; --k) {
        const int scale = c->br.scale[k];
        const int H = s.ny / scale, W = s.nx / scale;
        const long P = (long)s.batch * H * W;
        const int lfirst = c->br.first[k];
        if (W >= conv_tc_min_width()) {
            // the FP32 gradient of the branch output stays in g[cur]; the
            // BF16 gradients use g[cur ^ 1] and the unused half of g[cur]
            __nv_bfloat16* gbuf[2] = {(__nv_bfloat16*)t->g[cur ^ 1],
                                      (__nv_bfloat16*)(t->g[cur ^ 1]) + (size_t)P * 64};
            rc = branch_backward_tc(t, k, lfirst, l, t->g[cur], gbuf, s.batch, H, W, st);
            if (rc != HP_OK) return rc;
            if (k > 0) {
                const long Pc = P / 4;
                upsample_adjoint_kernel<<<(unsigned)((Pc + 255) / 256), 256, 0, st>>>(
                    t->gsmall, 1, 0, t->g[cur ^ 1], s.batch, H / 2, W / 2);
                if ((rc = check_launch()) != HP_OK) return rc;
                cur ^= 1;
            }
            l = lfirst - 1;
            continue;
        }
        for (; l >= lfirst; --l) {
            const int ci = sp[l].cin, co = sp[l].cout;
            float* gy = t->g[cur];
            if (sp[l].relu) {
                const size_t n = (size_t)P * co;
                relu_mask_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
                    gy, (const __nv_bfloat16*)t->act[l], n);
            }
            const void* x = l == lfirst ? (const void*)t->xin[k] : t->act[l - 1];
            float* gw = t->grad + layer_offset(sp, l);
            rc = wgrad_dispatch(t, k, l, gy, x, gw, gw + layer_wcount(sp, l), s.batch, H, W, st);
            if (rc != HP_OK) return rc;
            if (l > lfirst) {
                rc = co == 1 ? dgrad_last(t, l, gy, t->g[cur ^ 1], s.batch, H, W, nullptr, st)
                             : dgrad_dispatch(ci, co, gy, t->wt[l], t->g[cur ^ 1], s.batch, H, W,
                                              c->num_sms, st);
                if (rc != HP_OK) return rc;
                cur ^= 1;
            } else if (k > 0) {
                // gradient of the up-sampled coarser output (input channel 2)
                rc = dgrad_first_ch2(t, l, gy, s.batch, H, W, st);
                if (rc != HP_OK) return rc;
                const long Pc = P / 4;
                upsample_adjoint_kernel<<<(unsigned)((Pc + 255) / 256), 256, 0, st>>>(
                    t->gsmall, 1, 0, t->g[cur ^ 1], s.batch, H / 2, W / 2);
                if ((rc = check_launch()) != HP_OK) return rc;
                cur ^= 1;
            }
        }
    }
    return HP_OK;
}

// dL/dparams for one batch into t->grad; loss (mean over the batch) into t->loss
static hp_status trainer_grad(hp_trainer* t, const float* div, const uint8_t* flags,
                              const float* target, hp_shape s, float lambda, cudaStream_t st)
{
    hp_cnn* c = t->cnn;
    hp_status rc = trainer_forward(t, div, flags, s, st);
    if (rc != HP_OK) return rc;
    // loss and its gradient w.r.t. the full-resolution output
    if ((rc = launch_mask(flags, t->mask, s, st)) != HP_OK) return rc;
    const size_t cells = (size_t)s.ny * s.nx;
    const float* phi = (const float*)t->act[c->nlayers - 1];
    loss_stats_kernel<<<s.batch, 512, 0, st>>>(phi, target, div, t->mask, flags, c->s, t->rbuf,
                                               t->stats, s.ny, s.nx);
    loss_grad_kernel<<<(unsigned)(((size_t)s.batch * cells + 255) / 256), 256, 0, st>>>(
        phi, target, t->rbuf, t->mask, flags, c->s, t->stats, lambda, t->g[0], s.batch, s.ny,
        s.nx);
    loss_finish_kernel<<<1, 32, 0, st>>>(t->stats, s.batch, cells, lambda, t->loss);
    if ((rc = check_launch()) != HP_OK) return rc;
    return trainer_backward(t, s, st);
}

// the same for the physics-driven loss: sum over grids of weight_b * mean
// |div u_b|^norm, u_b the input velocity corrected by s_b * phi_hat_b
static hp_status trainer_pdnn_grad(hp_trainer* t, const float* div, const uint8_t* flags,
                                   const float* weight, hp_shape s, int norm, cudaStream_t st)
{
    hp_cnn* c = t->cnn;
    hp_status rc = trainer_forward(t, div, flags, s, st);
    if (rc != HP_OK) return rc;
    if ((rc = launch_mask(flags, t->mask, s, st)) != HP_OK) return rc;
    const size_t cells = (size_t)s.ny * s.nx;
    const float* phi = (const float*)t->act[c->nlayers - 1];
    pdnn_stats_kernel<<<s.batch, 512, 0, st>>>(phi, div, t->mask, c->s, weight, norm, t->rbuf,
                                               t->stats, s.ny, s.nx);
    pdnn_grad_kernel<<<(unsigned)(((size_t)s.batch * cells + 255) / 256), 256, 0, st>>>(
        t->rbuf, t->mask, t->g[0], s.batch, s.ny, s.nx);
    pdnn_finish_kernel<<<1, 32, 0, st>>>(t->stats, weight, s.batch, cells, t->loss);
    if ((rc = check_launch()) != HP_OK) return rc;
    return trainer_backward(t, s, st);
}

static hp_status trainer_copy_out(hp_trainer* t, float* grad_out, double* loss_out,
                                  cudaStream_t st)
{
    cudaError_t e = cudaSuccess;
    if (grad_out)
        e = cudaMemcpyAsync(grad_out, t->grad, t->param_count * 4, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && loss_out)
        e = cudaMemcpyAsync(loss_out, t->loss, 8, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) { set_cuda_error(e); return HP_ERR_CUDA; }
    return HP_OK;
}

// Adam on the masters from t->grad, then the BF16 / FP32 copies of the network
static hp_status trainer_adam(hp_trainer* t, const hp_train_params* p, cudaStream_t st)
{
    t->step += 1;
    const float c1 = 1.0f - powf(p->beta1, (float)t->step);
    const float c2 = 1.0f - powf(p->beta2, (float)t->step);
    adam_kernel<<<(unsigned)((t->param_count + 255) / 256), 256, 0, st>>>(
        t->master, t->grad, t->m, t->v, t->param_count, p->lr, p->beta1, p->beta2, p->eps, c1, c2);
    hp_status rc = check_launch();
    if (rc != HP_OK) return rc;
    return trainer_pack(t, st);
}

static bool trainer_shape_ok(const hp_trainer* t, hp_shape s)
{
    const int m = size_multiple(t->cnn->arch);
    return shape_ok(s) && s.batch <= t->max.batch && s.ny <= t->max.ny && s.nx <= t->max.nx &&
           s.ny % m == 0 && s.nx % m == 0;
}

extern "C" {

hp_status hp_trainer_gradient(hp_trainer* t, const float* div, const uint8_t* flags,
                              const float* target, hp_shape s, float lambda, float* grad_out,
                              double* loss_out, void* stream)
{
    if (!t || !div || !flags || !target || !trainer_shape_ok(t, s)) return HP_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    hp_status rc = trainer_grad(t, div, flags, target, s, lambda, st);
    if (rc != HP_OK) return rc;
    return trainer_copy_out(t, grad_out, loss_out, st);
}

hp_status hp_trainer_step(hp_trainer* t, const float* div, const uint8_t* flags,
                          const float* target, hp_shape s, const hp_train_params* p,
                          double* loss_out, void* stream)
{
    if (!p || !(p->lr > 0.0f)) return HP_ERR_INVALID_ARG;
    hp_status rc = hp_trainer_gradient(t, div, flags, target, s, p->lambda_div, nullptr, loss_out,
                                       stream);
    if (rc != HP_OK) return rc;
    return trainer_adam(t, p, (cudaStream_t)stream);
}

hp_status hp_trainer_pdnn_gradient(hp_trainer* t, const float* div, const uint8_t* flags,
                                   const float* weight, hp_shape s, int32_t norm,
                                   float* grad_out, double* loss_out, void* stream)
{
    if (!t || !div || !flags || !weight || !trainer_shape_ok(t, s) || (norm != 1 && norm != 2))
        return HP_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    hp_status rc = trainer_pdnn_grad(t, div, flags, weight, s, norm, st);
    if (rc != HP_OK) return rc;
    return trainer_copy_out(t, grad_out, loss_out, st);
}

hp_status hp_trainer_pdnn_step(hp_trainer* t, const float* div, const uint8_t* flags,
                               const float* weight, hp_shape s, int32_t norm,
                               const hp_train_params* p, double* loss_out, void* stream)
{
    if (!p || !(p->lr > 0.0f)) return HP_ERR_INVALID_ARG;
    hp_status rc = hp_trainer_pdnn_gradient(t, div, flags, weight, s, norm, nullptr, loss_out,
                                            stream);
    if (rc != HP_OK) return rc;
    return trainer_adam(t, p, (cudaStream_t)stream);
}

// copy the FP32 masters back into the network object (host copy, synchronous)
hp_status hp_trainer_sync_params(hp_trainer* t)
{
    if (!t) return HP_ERR_INVALID_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess)
        e = cudaMemcpy(t->cnn->master.data(), t->master, t->param_count * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) { set_cuda_error(e); return HP_ERR_CUDA; }
    return hp_cnn_check(t->cnn);
}

hp_status hp_trainer_get_state(hp_trainer* t, float* master, float* m, float* v, int64_t* step)
{
    if (!t) return HP_ERR_INVALID_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    const size_t bytes = (size_t)t->param_count * 4;
    if (e == cudaSuccess && master)
        e = cudaMemcpy(master, t->master, bytes, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && m) e = cudaMemcpy(m, t->m, bytes, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && v) e = cudaMemcpy(v, t->v, bytes, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) { set_cuda_error(e); return HP_ERR_CUDA; }
    if (step) *step = t->step;
    return HP_OK;
}

hp_status hp_cnn_save(const hp_cnn* c, const char* path)
{
    if (!c || !path) return HP_ERR_INVALID_ARG;
    CkptData d;
    d.arch = c->arch;
    d.w = c->master;
    return ckpt_write(path, d);
}

hp_status hp_cnn_load(hp_cnn** out, const char* path, hp_shape mx, int device)
{
    if (!out || !path) return HP_ERR_INVALID_ARG;
    *out = nullptr;
    CkptData d;
    hp_status rc = ckpt_read(path, &d);
    if (rc != HP_OK) return rc;
    if (!spec_for(d.arch) || (int64_t)d.w.size() != hp_cnn_arch_param_count(d.arch))
        return HP_ERR_IO;
    hp_cnn* c = nullptr;
    if ((rc = hp_cnn_create_arch(&c, d.arch, mx, device)) != HP_OK) return rc;
    if ((rc = hp_cnn_set_params(c, d.w.data(), (int64_t)d.w.size())) != HP_OK) {
        hp_cnn_destroy(c);
        return rc;
    }
    *out = c;
    return HP_OK;
}

hp_status hp_trainer_save(hp_trainer* t, const char* path)
{
    if (!t || !path) return HP_ERR_INVALID_ARG;
    CkptData d;
    d.arch = t->cnn->arch;
    d.has_moments = true;
    d.w.assign((size_t)t->param_count, 0.0f);
    d.m.assign((size_t)t->param_count, 0.0f);
    d.v.assign((size_t)t->param_count, 0.0f);
    int64_t step = 0;
    hp_status rc = hp_trainer_get_state(t, d.w.data(), d.m.data(), d.v.data(), &step);
    if (rc != HP_OK) return rc;
    d.step = step;
    return ckpt_write(path, d);
}

hp_status hp_trainer_load(hp_trainer* t, const char* path)
{
    if (!t || !path) return HP_ERR_INVALID_ARG;
    CkptData d;
    hp_status rc = ckpt_read(path, &d);
    if (rc != HP_OK) return rc;
    if (d.arch != t->cnn->arch || (int64_t)d.w.size() != t->param_count) return HP_ERR_IO;
    const size_t bytes = (size_t)t->param_count * 4;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(t->master, d.w.data(), bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        if (d.has_moments) {
            e = cudaMemcpy(t->m, d.m.data(), bytes, cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMemcpy(t->v, d.v.data(), bytes, cudaMemcpyHostToDevice);
        } else {
            e = cudaMemset(t->m, 0, bytes);
            if (e == cudaSuccess) e = cudaMemset(t->v, 0, bytes);
        }
    }
    if (e != cudaSuccess) { set_cuda_error(e); return HP_ERR_CUDA; }
    t->step = d.has_moments ? (int)d.step : 0;
    memcpy(t->cnn->master.data(), d.w.data(), bytes);
    // the network's BF16 weights from the restored masters, as after a step
    if ((rc = trainer_pack(t, nullptr)) != HP_OK) return rc;
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { set_cuda_error(e); return HP_ERR_CUDA; }
    return HP_OK;
}

hp_status hp_cnn_check(hp_cnn* c)
{
    if (!c) return HP_ERR_INVALID_ARG;
    int flag = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&flag, c->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && flag) e = cudaMemset(c->err, 0, sizeof(int));
    if (e != cudaSuccess) { set_cuda_error(e); return HP_ERR_CUDA; }
    if (flag & 1) return HP_ERR_TIMEOUT;
    e = cudaSetDevice(c->device);
    if (e != cudaSuccess) { set_cuda_error(e); return HP_ERR_CUDA; }
    const hp_status g = check_guards(c->guards);
    if (g != HP_OK) return g;
    return (flag & 2) ? HP_WARN_CNN_NONFINITE : HP_OK;
}

hp_status hp_trainer_check(hp_trainer* t)
{
    if (!t) return HP_ERR_INVALID_ARG;
    const hp_status g = check_guards(t->guards);
    if (g != HP_OK) return g;
    return hp_cnn_check(t->cnn);
}

}  // extern "C"
