// MultiScale CNN (Sec. 3.1) on sm_103a and the hybrid projection (Sec. 3.3):
// the network predicts the scaled pressure from [div/s, flags] and hands it to
// the Jacobi sweeps as the initial guess.
//
// Network (3 x 3 convolutions, replicated borders; ReLU after every
// convolution of a branch except its last two):
//   scale 1/4: [pool4(div/s), pool4(flags)]          2 -> 32 -> 64 -> 64 -> 32 -> 1
//   scale 1/2: [pool2(div/s), pool2(flags), up(o4)]  3 -> 32 -> 64 -> 64 -> 64 -> 64 -> 32 -> 1
//   scale 1  : [div/s, flags, up(o2)]                3 -> 32 -> 64 -> 64 -> 64 -> 64 -> 32 -> 1
// pool = average pooling (2 x 2 / 4 x 4), up = bilinear x 2 at half-pixel
// centres with the edge repeated.  s = mean |div| over the fluid cells (1 if
// zero); phi_0 = s * output on cells with an open face (the Poisson equation
// is linear in div).  BF16 activations and weights, FP32 accumulation; the
// 1-channel branch outputs are kept in FP32.
//
// Kernels: cnn_scale_kernel (s per grid), conv_first_kernel (2/3 -> 32 on
// CUDA cores, pooling and up-sampling fused into its input read), the
// tensor-core conv3x3 (conv_tc.cu) for the 32/64-channel layers,
// conv_last_kernel (32 -> 1 on CUDA cores), phi0_kernel.
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
};

// network order: scale 1/4, then 1/2, then 1
constexpr int kLayers = 19;
const LayerSpec kSpec[kLayers] = {
    {4, 2, 32, 1},  {4, 32, 64, 1}, {4, 64, 64, 1}, {4, 64, 32, 0}, {4, 32, 1, 0},
    {2, 3, 32, 1},  {2, 32, 64, 1}, {2, 64, 64, 1}, {2, 64, 64, 1}, {2, 64, 64, 1},
    {2, 64, 32, 0}, {2, 32, 1, 0},  {1, 3, 32, 1},  {1, 32, 64, 1}, {1, 64, 64, 1},
    {1, 64, 64, 1}, {1, 64, 64, 1}, {1, 64, 32, 0}, {1, 32, 1, 0}};

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// s[b] = mean |div| over fluid cells, 1 when there is none or it is zero.
__global__ void cnn_scale_kernel(const float* __restrict__ div, const uint8_t* __restrict__ flags,
                                 float* __restrict__ s, size_t cells)
{
    __shared__ double sh_sum[32];
    __shared__ unsigned long long sh_cnt[32];
    const int b = blockIdx.x;
    double sum = 0.0;
    unsigned long long cnt = 0;
    for (size_t q = threadIdx.x; q < cells; q += blockDim.x) {
        if (flags[b * cells + q] == 0) {
            sum += fabs((double)div[b * cells + q]);
            ++cnt;
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        sum += __shfl_down_sync(0xffffffffu, sum, off);
        cnt += __shfl_down_sync(0xffffffffu, cnt, off);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { sh_sum[wid] = sum; sh_cnt[wid] = cnt; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        unsigned long long c = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { t += sh_sum[w]; c += sh_cnt[w]; }
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
        double sd = 0.0, sf = 0.0;
        for (int dy = 0; dy < scale; ++dy)
            for (int dx = 0; dx < scale; ++dx) {
                const size_t q = ((size_t)b * H + (size_t)j * scale + dy) * W + (size_t)i * scale + dx;
                sd += div[q];
                sf += flags[q] != 0 ? 1.0 : 0.0;
            }
        const double inv = 1.0 / (scale * scale);
        out[0] = bf16r((float)(sd * inv) / s[b]);
        out[1] = bf16r((float)(sf * inv));
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

// First convolution of a branch: cin (2 or 3) -> 32, bias, ReLU, BF16 NHWC.
// w: float [9][cin][32] (BF16-rounded values), bias float [32].
__global__ void conv_first_kernel(BranchIn in, int cin, const float* __restrict__ w,
                                  const float* __restrict__ bias, __nv_bfloat16* __restrict__ y,
                                  int B)
{
    __shared__ float sw[9 * 3 * 32];
    __shared__ float sb[32];
    for (int q = threadIdx.x; q < 9 * cin * 32; q += blockDim.x) sw[q] = w[q];
    if (threadIdx.x < 32) sb[threadIdx.x] = bias[threadIdx.x];
    __syncthreads();
    const int hs = in.H / in.scale, ws = in.W / in.scale;
    const long P = (long)B * hs * ws;
    for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < P;
         p += (long)gridDim.x * blockDim.x) {
        const int b = (int)(p / ((long)hs * ws));
        const int r = (int)(p - (long)b * hs * ws);
        const int j = r / ws, i = r - j * ws;
        float acc[32];
#pragma unroll
        for (int o = 0; o < 32; ++o) acc[o] = 0.0f;
        for (int dy = 0; dy < 3; ++dy)
            for (int dx = 0; dx < 3; ++dx) {
                float xv[3];
                in.at(b, min(max(i + dx - 1, 0), ws - 1), min(max(j + dy - 1, 0), hs - 1), xv);
                const float* wt = sw + (dy * 3 + dx) * cin * 32;
                for (int c = 0; c < cin; ++c)
#pragma unroll
                    for (int o = 0; o < 32; ++o) acc[o] = fmaf(wt[c * 32 + o], xv[c], acc[o]);
            }
        __align__(16) __nv_bfloat16 ob[32];
#pragma unroll
        for (int o = 0; o < 32; ++o) ob[o] = __float2bfloat16_rn(fmaxf(acc[o] + sb[o], 0.0f));
        uint4* dst = reinterpret_cast<uint4*>(y + (size_t)p * 32);
#pragma unroll
        for (int q = 0; q < 4; ++q) dst[q] = reinterpret_cast<const uint4*>(ob)[q];
    }
}

// Last convolution of a branch: 32 -> 1, bias, no ReLU, FP32 output.
// w: float [9][32] (BF16-rounded), bias float [1].
__global__ void conv_last_kernel(const __nv_bfloat16* __restrict__ x, const float* __restrict__ w,
                                 const float* __restrict__ bias, float* __restrict__ y, int B, int H,
                                 int W)
{
    __shared__ float sw[9 * 32];
    for (int q = threadIdx.x; q < 9 * 32; q += blockDim.x) sw[q] = w[q];
    __syncthreads();
    const long P = (long)B * H * W;
    for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < P;
         p += (long)gridDim.x * blockDim.x) {
        const int b = (int)(p / ((long)H * W));
        const int r = (int)(p - (long)b * H * W);
        const int j = r / W, i = r - j * W;
        float acc = 0.0f;
        for (int dy = 0; dy < 3; ++dy)
            for (int dx = 0; dx < 3; ++dx) {
                const int sy = min(max(j + dy - 1, 0), H - 1), sx = min(max(i + dx - 1, 0), W - 1);
                const uint4* src = reinterpret_cast<const uint4*>(x + (((size_t)b * H + sy) * W + sx) * 32);
                const float* wt = sw + (dy * 3 + dx) * 32;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint4 v = src[q];
                    const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&v);
#pragma unroll
                    for (int k = 0; k < 8; ++k) acc = fmaf(wt[q * 8 + k], __bfloat162float(e[k]), acc);
                }
            }
        y[p] = acc + bias[0];
    }
}

// phi_0 = s * out on cells with an open face, 0 elsewhere.
__global__ void phi0_kernel(const float* __restrict__ out, const float* __restrict__ s,
                            const uint8_t* __restrict__ mask, float* __restrict__ phi, int B,
                            size_t cells)
{
    const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (size_t)B * cells) return;
    const int b = (int)(q / cells);
    phi[q] = (mask[q] & 15u) ? s[b] * out[q] : 0.0f;
}

}  // namespace

}  // namespace hp

using namespace hp;

struct hp_cnn {
    int device;
    int num_sms;
    hp_shape max_shape;
    // per layer: weights in the layout of its kernel, FP32 bias
    void* w[kLayers];
    float* bias[kLayers];
    std::vector<float> master;  // FP32 parameters, oracle order
    // workspace
    __nv_bfloat16* act[2];
    float* out[3];  // branch outputs at 1/4, 1/2, 1
    float* s;
    int* err;
};

static size_t layer_wcount(int l) { return (size_t)9 * kSpec[l].cin * kSpec[l].cout; }

extern "C" {

int64_t hp_cnn_param_count(void)
{
    int64_t n = 0;
    for (int l = 0; l < kLayers; ++l) n += (int64_t)layer_wcount(l) + kSpec[l].cout;
    return n;
}

void hp_cnn_destroy(hp_cnn* c)
{
    if (!c) return;
    for (int l = 0; l < kLayers; ++l) {
        cudaFree(c->w[l]);
        cudaFree(c->bias[l]);
    }
    cudaFree(c->act[0]);
    cudaFree(c->act[1]);
    for (int k = 0; k < 3; ++k) cudaFree(c->out[k]);
    cudaFree(c->s);
    cudaFree(c->err);
    delete c;
}

hp_status hp_cnn_create(hp_cnn** out, hp_shape mx, int device)
{
    if (!out || !shape_ok(mx) || mx.ny % 4 || mx.nx % 4) return HP_ERR_INVALID_ARG;
    *out = nullptr;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) { set_cuda_error(e); return HP_ERR_CUDA; }
    hp_cnn* c = new hp_cnn();
    memset(c->w, 0, sizeof(c->w));
    memset(c->bias, 0, sizeof(c->bias));
    c->device = device;
    c->max_shape = mx;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    c->master.assign((size_t)hp_cnn_param_count(), 0.0f);
    const size_t px = (size_t)mx.batch * mx.ny * mx.nx;
    bool okm = true;
    for (int l = 0; l < kLayers && okm; ++l) {
        const size_t wb = layer_wcount(l) * (kSpec[l].cin >= 32 && kSpec[l].cout >= 32 ? 2 : 4);
        okm = cudaMalloc(&c->w[l], wb) == cudaSuccess &&
              cudaMalloc((void**)&c->bias[l], kSpec[l].cout * sizeof(float)) == cudaSuccess;
        if (okm) {
            cudaMemset(c->w[l], 0, wb);
            cudaMemset(c->bias[l], 0, kSpec[l].cout * sizeof(float));
        }
    }
    okm = okm && cudaMalloc((void**)&c->act[0], px * 64 * 2) == cudaSuccess &&
          cudaMalloc((void**)&c->act[1], px * 64 * 2) == cudaSuccess &&
          cudaMalloc((void**)&c->out[0], px / 16 * 4 + 16) == cudaSuccess &&
          cudaMalloc((void**)&c->out[1], px / 4 * 4 + 16) == cudaSuccess &&
          cudaMalloc((void**)&c->out[2], px * 4) == cudaSuccess &&
          cudaMalloc((void**)&c->s, mx.batch * sizeof(float)) == cudaSuccess &&
          cudaMalloc((void**)&c->err, sizeof(int)) == cudaSuccess;
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

// params: host FP32 in the order of the network (scale 1/4, 1/2, 1), each
// layer weights [cout][cin][3][3] then bias [cout].  Weights are rounded to
// BF16 on upload.
hp_status hp_cnn_set_params(hp_cnn* c, const float* params, int64_t n)
{
    if (!c || !params || n != hp_cnn_param_count()) return HP_ERR_INVALID_ARG;
    memcpy(c->master.data(), params, (size_t)n * sizeof(float));
    const float* p = params;
    for (int l = 0; l < kLayers; ++l) {
        const int ci = kSpec[l].cin, co = kSpec[l].cout;
        const bool tc = ci >= 32 && co >= 32;
        std::vector<uint16_t> wb;
        std::vector<float> wf;
        if (tc) wb.assign(layer_wcount(l), 0); else wf.assign(layer_wcount(l), 0.0f);
        for (int o = 0; o < co; ++o)
            for (int i = 0; i < ci; ++i)
                for (int t = 0; t < 9; ++t) {
                    const float v = p[((size_t)o * ci + i) * 9 + t];
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
        p += layer_wcount(l);
        cudaError_t e = tc ? cudaMemcpy(c->w[l], wb.data(), wb.size() * 2, cudaMemcpyHostToDevice)
                           : cudaMemcpy(c->w[l], wf.data(), wf.size() * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(c->bias[l], p, co * sizeof(float), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { set_cuda_error(e); return HP_ERR_CUDA; }
        p += co;
    }
    return HP_OK;
}

hp_status hp_cnn_get_params(const hp_cnn* c, float* params, int64_t n)
{
    if (!c || !params || n != hp_cnn_param_count()) return HP_ERR_INVALID_ARG;
    memcpy(params, c->master.data(), (size_t)n * sizeof(float));
    return HP_OK;
}

// phi_hat (FP32 [B][H][W], unscaled network output) and s (FP32 [B]).
hp_status hp_cnn_forward(hp_cnn* c, const float* div, const uint8_t* flags, float* phi_hat,
                         float* s_out, hp_shape s, void* stream)
{
    if (!c || !div || !flags || !shape_ok(s) || s.ny % 4 || s.nx % 4 ||
        s.batch > c->max_shape.batch || (size_t)s.batch * s.ny * s.nx >
                                            (size_t)c->max_shape.batch * c->max_shape.ny *
                                                c->max_shape.nx)
        return HP_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t cells = (size_t)s.ny * s.nx;
    cnn_scale_kernel<<<s.batch, 1024, 0, st>>>(div, flags, c->s, cells);
    hp_status rc = check_launch();
    if (rc != HP_OK) return rc;
    int l = 0;
    const float* prev = nullptr;
    for (int k = 0; k < 3; ++k) {
        const int scale = k == 0 ? 4 : k == 1 ? 2 : 1;
        const int H = s.ny / scale, W = s.nx / scale;
        const long P = (long)s.batch * H * W;
        BranchIn in = {div, flags, c->s, prev, s.ny, s.nx, scale};
        int cur = 0;
        const int blocks = (int)((P + 255) / 256 < 8L * c->num_sms ? (P + 255) / 256 : 8L * c->num_sms);
        conv_first_kernel<<<blocks, 256, 0, st>>>(in, kSpec[l].cin, (const float*)c->w[l],
                                                  c->bias[l], c->act[cur], s.batch);
        if ((rc = check_launch()) != HP_OK) return rc;
        ++l;
        while (kSpec[l].cout != 1) {
            rc = launch_conv3x3_tc(c->act[cur], c->w[l], c->bias[l], c->act[cur ^ 1], s.batch, H,
                                   W, kSpec[l].cin, kSpec[l].cout, kSpec[l].relu, c->err,
                                   c->num_sms, st);
            if (rc != HP_OK) return rc;
            cur ^= 1;
            ++l;
        }
        float* o = (k == 2 && phi_hat) ? phi_hat : c->out[k];
        conv_last_kernel<<<blocks, 256, 0, st>>>(c->act[cur], (const float*)c->w[l], c->bias[l],
                                                 o, s.batch, H, W);
        if ((rc = check_launch()) != HP_OK) return rc;
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
    if (!ctx || !cnn || !u || !v || !flags || !prm || !iters_out) return HP_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    // divergence into the context, CNN guess into the second phi buffer
    hp_status rc = launch_mask_div(u, v, flags, ctx->mask, ctx->div, s, st);
    if (rc != HP_OK) return rc;
    rc = hp_cnn_forward(cnn, ctx->div, flags, cnn->out[2], nullptr, s, stream);
    if (rc != HP_OK) return rc;
    const size_t cells = (size_t)s.ny * s.nx;
    phi0_kernel<<<(unsigned)(((size_t)s.batch * cells + 255) / 256), 256, 0, st>>>(
        cnn->out[2], cnn->s, ctx->mask, ctx->phi[1], s.batch, cells);
    if ((rc = check_launch()) != HP_OK) return rc;
    return hp_project(ctx, u, v, flags, s, prm, ctx->phi[1], p_out, iters_out, e1_out, einf_out,
                      conv_out, e_hist, hist_len, stream);
}

}  // extern "C"
