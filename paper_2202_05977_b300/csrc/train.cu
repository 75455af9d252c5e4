// Training step (Eq. 1): forward with the network output kept, L1 loss,
// backward through the reconstruction (Eq. 3-5) and the convolutions with
// the activations recomputed from the inputs (not stored between forward
// and backward), and one Adam update of the weights.
#include <algorithm>
#include <cmath>
#include <vector>

#include <cuda_bf16.h>

#include "ctx.h"

namespace wskpn {

wskpn_status launch_prep(const wskpn_frame* frames, int B, int H, int W, float gamma, float dnear, float dfar,
                         void* const* out, int layout, cudaStream_t st, std::string& err);
wskpn_status launch_conv_simt(const float* const* in, float* const* out, int B, int H, int W, int Cin, int Cout,
                              int KS, const float* w_packed, const float* bias_padded, int relu, cudaStream_t st,
                              std::string& err);
wskpn_status launch_conv_simt_masked(const float* const* in, float* const* out, const float* const* mask, int B,
                                     int H, int W, int Cin, int Cout, int KS, const float* w_packed,
                                     const float* bias_padded, int relu, cudaStream_t st, std::string& err);
wskpn_status launch_pack_simt_transposed(const float* w, int Cin, int Cout, int KS, float* wp, float* bp,
                                         cudaStream_t st, std::string& err);
int simt_coutp(int cout);
size_t wgrad_part_floats(int Cin, int KS, int G);
wskpn_status launch_wgrad(const float* const* x, const float* const* gy, int B, int H, int W, int Cin, int Cout,
                          int KS, int G, float* part, float* dw, float* db, cudaStream_t st, std::string& err);
bool wgrad_tc_supported(int KS, int Cin, int Cout, int B, int H, int W, int nsm, size_t* part_floats);
wskpn_status launch_wgrad_tc(const void* x, int xcp, const void* gy_nhwc, int gcp_stride, int B, int H, int W,
                             int Cin, int Cout, int KS, float* part, size_t part_cap, float* dw, unsigned int* status,
                             int device, cudaStream_t st, std::string& err);
wskpn_status launch_decode_fuse_fwd(const float* const* z, const float* const* r, const float* const* a,
                                    float* const* out, int B, int H, int W, int M, const int* ks, float eps,
                                    unsigned int* fallbacks, cudaStream_t st, std::string& err);
wskpn_status launch_decode_fuse_bwd(const float* const* z, const float* const* r, const float* const* a,
                                    const float* const* G, float* const* dz, float* const* scratch, int B, int H,
                                    int W, int M, const int* ks, float eps, unsigned int* fallbacks,
                                    cudaStream_t st, std::string& err);

namespace {
constexpr int kWgradGroups = 256;
constexpr int GP_TILE = 64;  // pixels per block of the gradient pack
constexpr int kLossBlocks = 1024;
}

struct TrainWs {
    size_t px = 0;
    float* acts = nullptr;      // x_0 .. x_{L-1}, planar FP32, layer after layer
    size_t act_off[WSKPN_MAX_LAYERS] = {};
    float* gA = nullptr;        // gradient ping-pong [B][maxw][H][W] (FP32 gradient paths, on first use)
    float* gB = nullptr;
    size_t g_floats = 0;
    float* dz = nullptr;        // [B][2M][H][W]
    float* dscratch = nullptr;  // reconstruction-backward scratch [B][2M+3][H][W]
    float* part = nullptr;      // wgrad partial sums
    float* wT[WSKPN_MAX_LAYERS] = {};  // transposed + flipped packed weights
    float* bT[WSKPN_MAX_LAYERS] = {};
    float* loss_part = nullptr;
    float* m = nullptr;         // Adam moments
    float* v = nullptr;
    // BF16 contexts: input and weight gradients on the tensor cores
    Layer lt[WSKPN_MAX_LAYERS];         // layer l's input-gradient conv (weights transposed, flipped)
    bool lt_ok[WSKPN_MAX_LAYERS] = {};  // a kernel exists for lt[l]'s shape
    bool wg_ok[WSKPN_MAX_LAYERS] = {};  // layer l's weight gradient has a tensor-core kernel
    float* wt = nullptr;                // transposed weights of one layer (packing scratch)
    float* zero_bias = nullptr;         // [64] zeros
    void* gpack = nullptr;              // gradient as NHWC BF16 [B][H][W][cp], two buffers
    void* gpack2 = nullptr;
    void* xnhwc = nullptr;              // layer inputs x_0 .. x_{L-1}, NHWC BF16 hi/lo, layer after layer
    uint32_t* xbits = nullptr;          // their positive-channel bits [L][px][2] (x_1 .. x_{L-1} used)
    size_t x_off[WSKPN_MAX_LAYERS] = {};  // byte offsets in xnhwc
    size_t x_bytes = 0;
    bool all_tc = false;                // every layer has its tensor-core gradient kernels
    float* bias_part = nullptr;         // per-tile bias-gradient sums [tiles][64]
    float* wg_part = nullptr;           // tensor-core weight-gradient partial sums
    size_t wg_part_floats = 0;
    size_t acts_floats = 0;             // planar acts (FP32 gradient paths), allocated on first use
    // xnhwc as written by the last wskpn_forward_train on the tensor-core
    // path: the layer inputs of that forward, reused by a backward over the
    // same frames (buffer pointers), batch and size instead of recomputed
    bool kept = false;
    int kept_batch = 0, kept_h = 0, kept_w = 0;
    wskpn_frame kept_frames[WSKPN_MAX_BATCH] = {};
};

static bool same_frames(const wskpn_frame& x, const wskpn_frame& y) {
    return x.radiance == y.radiance && x.albedo == y.albedo && x.normal == y.normal && x.depth == y.depth;
}

static void free_train(TrainWs* t) {
    if (!t) return;
    cudaFree(t->acts);
    cudaFree(t->gA);
    cudaFree(t->gB);
    cudaFree(t->dz);
    cudaFree(t->dscratch);
    cudaFree(t->part);
    for (int l = 0; l < WSKPN_MAX_LAYERS; ++l) {
        cudaFree(t->wT[l]);
        cudaFree(t->bT[l]);
    }
    cudaFree(t->loss_part);
    cudaFree(t->m);
    cudaFree(t->v);
    for (int l = 0; l < WSKPN_MAX_LAYERS; ++l) tc_layer_free(t->lt[l]);
    cudaFree(t->wt);
    cudaFree(t->zero_bias);
    cudaFree(t->gpack);
    cudaFree(t->xnhwc);
    cudaFree(t->xbits);
    cudaFree(t->gpack2);
    cudaFree(t->bias_part);
    cudaFree(t->wg_part);
    delete t;
}

void ctx_free_train(wskpn_ctx* ctx) {
    free_train(static_cast<TrainWs*>(ctx->train));
    ctx->train = nullptr;
}

#define WSKPN_TRY_ALLOC(ptr, bytes)                                                               \
    do {                                                                                          \
        if (cudaMalloc((void**)&(ptr), (bytes)) != cudaSuccess) {                                 \
            ctx->err = std::string("training workspace allocation failed: ") + #ptr;             \
            return WSKPN_ENOMEM;                                                                  \
        }                                                                                         \
    } while (0)

static wskpn_status ensure_train(wskpn_ctx* ctx) {
    if (ctx->train) return WSKPN_OK;
    const wskpn_config& c = ctx->cfg;
    TrainWs* t = new TrainWs();
    ctx->train = t;
    t->px = ctx->ws_pixels;
    const int L = c.n_layers, M = c.n_kernels, KS = c.conv_ks;
    size_t off = 0;
    int maxw = 0, maxcin = 0;
    for (int l = 0; l < L; ++l) {
        t->act_off[l] = off;
        off += (size_t)c.widths[l] * t->px;
    }
    for (int l = 1; l <= L; ++l) maxw = std::max(maxw, c.widths[l]);
    for (int l = 0; l < L; ++l) maxcin = std::max(maxcin, c.widths[l]);
    t->acts_floats = off;  // allocated by the first backward that needs planar activations
    t->g_floats = (size_t)maxw * t->px;
    WSKPN_TRY_ALLOC(t->dz, (size_t)2 * M * t->px * sizeof(float));
    WSKPN_TRY_ALLOC(t->dscratch, (size_t)(2 * M + 3) * t->px * sizeof(float));
    WSKPN_TRY_ALLOC(t->part, wgrad_part_floats(maxcin, KS, kWgradGroups) * sizeof(float));
    for (int l = 1; l < L; ++l) {  // layer 0 needs no input gradient
        const int cin = c.widths[l], cout = c.widths[l + 1];
        WSKPN_TRY_ALLOC(t->wT[l], (size_t)cout * KS * KS * simt_coutp(cin) * sizeof(float));
        WSKPN_TRY_ALLOC(t->bT[l], (size_t)simt_coutp(cin) * sizeof(float));
    }
    WSKPN_TRY_ALLOC(t->loss_part, kLossBlocks * sizeof(float));
    if (c.prec == WSKPN_BF16) {
        // input gradients of layers 1 .. L-1 as BF16 tensor-core convolutions,
        // weight gradients of every layer as tensor-core GEMMs over the pixels
        int nsm = 148;
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device);
        size_t wmax = 0, gcp = 0;
        t->all_tc = true;
        for (int l = 0; l < L; ++l) {
            const int cin = c.widths[l], cout = c.widths[l + 1];
            size_t pf = 0;
            t->wg_ok[l] = wgrad_tc_supported(KS, cin, cout, c.max_batch, c.max_h, c.max_w, nsm, &pf);
            t->all_tc = t->all_tc && t->wg_ok[l];
            t->wg_part_floats = std::max(t->wg_part_floats, pf);
            gcp = std::max(gcp, (size_t)(cout + 15) / 16 * 16);
            t->x_off[l] = t->x_bytes;
            t->x_bytes += (size_t)(cin + 15) / 16 * 16 * 2 * sizeof(uint16_t) * t->px;
            if (l + 1 < L) t->all_tc = t->all_tc && tc_relu_bits_supported(ctx, l);
            if (l == 0) continue;
            std::string e;
            t->lt_ok[l] = tc_dgrad_layer_alloc(t->lt[l], KS, cin, cout, e) == WSKPN_OK;
            t->all_tc = t->all_tc && t->lt_ok[l];
            wmax = std::max(wmax, (size_t)cin * cout * KS * KS);
        }
        if (t->all_tc) {
            WSKPN_TRY_ALLOC(t->wt, std::max<size_t>(wmax, 1) * sizeof(float));
            WSKPN_TRY_ALLOC(t->zero_bias, 64 * sizeof(float));
            if (cudaMemset(t->zero_bias, 0, 64 * sizeof(float)) != cudaSuccess) {
                ctx->err = "training workspace: cudaMemset failed";
                return WSKPN_ECUDA;
            }
            WSKPN_TRY_ALLOC(t->gpack, gcp * 2 * sizeof(uint16_t) * t->px);
            WSKPN_TRY_ALLOC(t->gpack2, gcp * 2 * sizeof(uint16_t) * t->px);
            WSKPN_TRY_ALLOC(t->wg_part, t->wg_part_floats * sizeof(float));
            // rows of bias sums: tiles of GP_TILE pixels per frame for every
            // frame of a call (gradient packing), 4 per CTA of an
            // input-gradient convolution (at most one CTA per SM)
            const size_t tiles = (size_t)c.max_batch * (((size_t)c.max_h * c.max_w + GP_TILE - 1) / GP_TILE);
            WSKPN_TRY_ALLOC(t->bias_part, std::max(tiles, (size_t)4 * nsm) * 64 * sizeof(float));
        }
    }
    return WSKPN_OK;
}

// Gradient planes g (planar FP32 [C][HW] per frame, C <= CMAX) written
// channels-last as BF16 nhwc [B][HW][cp] (channels C .. cp - 1 zero): the
// input of a tensor-core input-gradient convolution and of the weight
// gradient.
// One block per tile of 4096 / CMAX pixels of one frame, transposed through
// shared memory so that both layouts are read and written in whole runs
// (every thread issues its 16 loads before storing any).  bias_part
// [tiles][64] receives each tile's per-channel sum (pixels in a fixed order),
// from which the bias gradient is added up.
__device__ __forceinline__ void bf16x8_to_float(const uint4& u, float f[8]) {
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float2 t = __bfloat1622float2(h[j]);
        f[2 * j] = t.x;
        f[2 * j + 1] = t.y;
    }
}
template <int CMAX>
__global__ void __launch_bounds__(256) grad_pack_kernel(PtrBatch<const float*> g, int C, int cp, size_t HW,
                                                        uint4* __restrict__ nhwc, float* __restrict__ bias_part) {
    constexpr int TILE = 4096 / CMAX;  // pixels per block
    constexpr int TPC = 256 / CMAX;    // threads per channel in the tile sums
    __shared__ float sg[CMAX][TILE + 1];
    const int b = blockIdx.y, tid = threadIdx.x;
    const size_t p0 = (size_t)blockIdx.x * TILE;
    const float* __restrict__ gb = g.p[b];
    {
        float v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int k = tid + 256 * u, c = k / TILE, i = k % TILE;
            v[u] = c < C && p0 + i < HW ? gb[(size_t)c * HW + p0 + i] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int k = tid + 256 * u;
            sg[k / TILE][k % TILE] = v[u];
        }
    }
    __syncthreads();
    // per (pixel, 8-channel chunk): one 16-byte store of BF16 values
    const int nq = cp / 8;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int k = tid + 256 * u;
        if (k >= TILE * nq) break;
        const int i = k / nq, q = k % nq;
        const size_t p = p0 + i;
        if (p >= HW) continue;
        __nv_bfloat162 h[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) h[j] = __floats2bfloat162_rn(sg[q * 8 + 2 * j][i], sg[q * 8 + 2 * j + 1][i]);
        uint4* dst = nhwc + ((size_t)b * HW + p) * (size_t)(cp / 8);  // cp BF16 = cp / 8 uint4
        dst[q] = *reinterpret_cast<const uint4*>(h);
    }
    // per-channel tile sums: TPC threads per channel, 16 pixels each in order
    {
        const int c = tid / TPC, part = tid % TPC;
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < 16; ++i) s += sg[c][part * 16 + i];
#pragma unroll
        for (int o = 1; o < TPC; o <<= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (part == 0 && c < C) bias_part[((size_t)b * gridDim.x + blockIdx.x) * 64 + c] = s;
    }
}

// db[o] = sum over the tiles (fixed order: thread t adds tiles t, t + 256,
// ..., then a fixed tree) of bias_part[tile][o]; one block per channel.
__global__ void bias_from_tiles_kernel(const float* __restrict__ part, int ntiles, float* __restrict__ db) {
    const int o = blockIdx.x;
    __shared__ float red[256];
    float s = 0.f;
    for (int k = threadIdx.x; k < ntiles; k += 256) s += part[(size_t)k * 64 + o];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) db[o] = red[0];
}


// Packs the gradient of a layer with C output channels (planar FP32) as
// NHWC BF16 with cp channels, then writes its bias gradient db (from the
// FP32 values).
static wskpn_status launch_grad_pack(const float* const* g, int B, int C, int cp, size_t HW, void* nhwc,
                                     float* bias_part, float* db, cudaStream_t st, std::string& err) {
    if (C > cp || cp > 64 || cp % 16 || B > WSKPN_MAX_BATCH) {
        err = "gradient pack: at most 64 channels and 16 frames";
        return WSKPN_EUNSUPPORTED;
    }
    PtrBatch<const float*> gp{};
    for (int b = 0; b < B; ++b) gp.p[b] = g[b];
    const int tile = cp <= 16 ? 256 : 64;
    const unsigned tiles = (unsigned)((HW + tile - 1) / tile);
    if (cp <= 16)
        grad_pack_kernel<16><<<dim3(tiles, B), 256, 0, st>>>(gp, C, cp, HW, static_cast<uint4*>(nhwc), bias_part);
    else
        grad_pack_kernel<64><<<dim3(tiles, B), 256, 0, st>>>(gp, C, cp, HW, static_cast<uint4*>(nhwc), bias_part);
    WSKPN_CUDA_TRY(cudaGetLastError(), err);
    bias_from_tiles_kernel<<<C, 256, 0, st>>>(bias_part, (int)tiles * B, db);
    WSKPN_CUDA_TRY(cudaGetLastError(), err);
    return WSKPN_OK;
}

// ------------------------------------------------------------------ loss
// L1: loss = sum |o - t| / n,  dout = sign(o - t) / n (sign(0) = 0).
__global__ void l1_loss_kernel(const float* __restrict__ o, const float* __restrict__ t, size_t n,
                               float* __restrict__ part, float* __restrict__ grad) {
    float s = 0.f;
    const float inv = 1.f / (float)n;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float d = o[i] - t[i];
        s += fabsf(d);
        if (grad) grad[i] = d > 0.f ? inv : (d < 0.f ? -inv : 0.f);
    }
    __shared__ float red[32];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float b = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += red[w];
        part[blockIdx.x] = b;
    }
}

// One block of 256 threads: thread t adds partials t, t + 256, ... in FP64,
// then a fixed-order tree (deterministic).
__global__ void sum_partials_kernel(const float* __restrict__ part, int n, double scale, float* __restrict__ out) {
    __shared__ double red[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = (float)(red[0] * scale);
}

// ------------------------------------------------------------------ Adam
__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, size_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

}  // namespace wskpn

using namespace wskpn;

extern "C" {

size_t wskpn_decode_fuse_bwd_scratch_floats(int batch, int h, int w, int M) {
    if (batch < 1 || h < 1 || w < 1 || M < 1 || M > WSKPN_MAX_KERNELS) return 0;
    return (size_t)(2 * M + 3) * batch * h * w;
}

wskpn_status wskpn_decode_fuse_bwd(const float* z, const float* radiance, const float* albedo, const float* dout,
                                   int batch, int h, int w, int M, const int* ksizes, float eps, float* dz,
                                   float* scratch, unsigned int* fallbacks, void* stream) {
    if (!z || !radiance || !albedo || !dout || !dz || !scratch || !ksizes || batch < 1 || h < 1 || w < 1 || M < 1 ||
        M > WSKPN_MAX_KERNELS || !(eps > 0.f)) {
        set_thread_error("wskpn_decode_fuse_bwd: invalid argument");
        return WSKPN_EINVAL;
    }
    for (int i = 0; i < M; ++i)
        if (ksizes[i] < 1 || ksizes[i] > 13 || (ksizes[i] & 1) == 0) {
            set_thread_error("wskpn_decode_fuse_bwd: ksizes must be odd and in [1, 13]");
            return WSKPN_EINVAL;
        }
    const size_t HW = (size_t)h * w;
    std::vector<const float*> zz(batch), rr(batch), aa(batch), gg(batch);
    std::vector<float*> dd(batch), ss(batch);
    for (int b = 0; b < batch; ++b) {
        zz[b] = z + (size_t)b * 2 * M * HW;
        rr[b] = radiance + (size_t)b * 3 * HW;
        aa[b] = albedo + (size_t)b * 3 * HW;
        gg[b] = dout + (size_t)b * 3 * HW;
        dd[b] = dz + (size_t)b * 2 * M * HW;
        ss[b] = scratch + (size_t)b * (2 * M + 3) * HW;
    }
    std::string err;
    wskpn_status s = launch_decode_fuse_bwd(zz.data(), rr.data(), aa.data(), gg.data(), dd.data(), ss.data(), batch,
                                            h, w, M, ksizes, eps, fallbacks, (cudaStream_t)stream, err);
    if (s) set_thread_error(err);
    return s;
}

wskpn_status wskpn_forward_train(wskpn_ctx* ctx, const wskpn_frame* frames, int batch, int h, int w, float* out,
                                 float* z_saved, void* stream) {
    if (!ctx) return WSKPN_EINVAL;
    if (!z_saved || !out) {
        ctx->err = "wskpn_forward_train: out or z_saved is NULL";
        return WSKPN_EINVAL;
    }
    const wskpn_config& c = ctx->cfg;
    cudaStream_t st = (cudaStream_t)stream;
    // Kept activations (BF16, tensor-core backward): the layer inputs x_0 ..
    // x_{L-1} go to the training workspace (NHWC hi/lo, where the backward
    // reads them) instead of the inference ping-pong buffers; same kernels,
    // same values.
    const bool keep = ctx->train_keep && c.prec == WSKPN_BF16 && tc_split_all(ctx) &&
                      ctx->train_tc_recompute == 1 && batch >= 1 && batch <= WSKPN_MAX_BATCH;
    wskpn_status s = WSKPN_OK;
    TrainWs* t = nullptr;
    if (keep) {
        s = check_frames(ctx, frames, batch, h, w);
        if (!s) s = ensure_train(ctx);
        if (s) return s;
        t = static_cast<TrainWs*>(ctx->train);
        t->kept = false;
        if (!t->all_tc) t = nullptr;
    } else if (ctx->train) {
        static_cast<TrainWs*>(ctx->train)->kept = false;
    }
    if (t) {
        if (!t->xnhwc) WSKPN_TRY_ALLOC(t->xnhwc, t->x_bytes);
        if (!t->xbits) WSKPN_TRY_ALLOC(t->xbits, (size_t)c.n_layers * t->px * 2 * sizeof(uint32_t));
        const int L = c.n_layers;
        std::vector<void*> xs(L);
        std::vector<uint32_t*> bits(L);
        for (int l = 0; l < L; ++l) {
            xs[l] = static_cast<uint8_t*>(t->xnhwc) + t->x_off[l];
            bits[l] = t->xbits + (size_t)l * t->px * 2;
        }
        s = tc_recompute_nhwc(ctx, frames, batch, h, w, xs, st, &bits);
        if (!s) s = tc_conv_layer(ctx, L - 1, xs[L - 1], z_saved, batch, h, w, st);
        if (s) return s;
        t->kept = true;
        t->kept_batch = batch;
        t->kept_h = h;
        t->kept_w = w;
        for (int b = 0; b < batch; ++b) t->kept_frames[b] = frames[b];
    } else {
        s = wskpn_logits(ctx, frames, batch, h, w, z_saved, stream);
        if (s) return s;
    }
    const size_t HW = (size_t)h * w;
    std::vector<const float*> z(batch), r(batch), a(batch);
    std::vector<float*> o(batch);
    for (int b = 0; b < batch; ++b) {
        z[b] = z_saved + (size_t)b * 2 * c.n_kernels * HW;
        r[b] = frames[b].radiance;
        a[b] = frames[b].albedo;
        o[b] = out + (size_t)b * 3 * HW;
    }
    return launch_decode_fuse_fwd(z.data(), r.data(), a.data(), o.data(), batch, h, w, c.n_kernels, c.ksizes,
                                  c.albedo_eps, ctx->d_fallbacks, st, ctx->err);
}

wskpn_status wskpn_backward(wskpn_ctx* ctx, const wskpn_frame* frames, int batch, int h, int w,
                            const float* z_saved, const float* dout, float* dz_out, float* dweights, void* stream) {
    if (!ctx) return WSKPN_EINVAL;
    if (!frames || !z_saved || !dout || !dweights) {
        ctx->err = "wskpn_backward: NULL argument";
        return WSKPN_EINVAL;
    }
    if (batch < 1 || batch > ctx->cfg.max_batch || batch > WSKPN_MAX_BATCH || h < 1 || w < 1 ||
        h > ctx->cfg.max_h || w > ctx->cfg.max_w || (size_t)batch * h * w > ctx->ws_pixels) {
        ctx->err = "wskpn_backward: batch or size out of range (batch <= 16 and <= max_batch)";
        return WSKPN_EINVAL;
    }
    wskpn_status s = ensure_train(ctx);
    if (s) return s;
    TrainWs* t = static_cast<TrainWs*>(ctx->train);
    const wskpn_config& c = ctx->cfg;
    const int L = c.n_layers, M = c.n_kernels, KS = c.conv_ks;
    const size_t HW = (size_t)h * w;
    cudaStream_t st = (cudaStream_t)stream;
    float* dz = dz_out ? dz_out : t->dz;

    // 1. reconstruction backward
    {
        std::vector<const float*> zz(batch), rr(batch), aa(batch), gg(batch);
        std::vector<float*> dd(batch), ss(batch);
        for (int b = 0; b < batch; ++b) {
            zz[b] = z_saved + (size_t)b * 2 * M * HW;
            rr[b] = frames[b].radiance;
            aa[b] = frames[b].albedo;
            gg[b] = dout + (size_t)b * 3 * HW;
            dd[b] = dz + (size_t)b * 2 * M * HW;
            ss[b] = t->dscratch + (size_t)b * (2 * M + 3) * HW;
        }
        s = launch_decode_fuse_bwd(zz.data(), rr.data(), aa.data(), gg.data(), dd.data(), ss.data(), batch, h, w, M,
                                   c.ksizes, c.albedo_eps, ctx->d_fallbacks, st, ctx->err);
        if (s) return s;
    }
    // 2. the layer inputs x_0 .. x_{L-1}: kept by wskpn_forward_train over the
    //    same frames, or recomputed with the context's own convolutions for
    //    BF16 (tensor cores, hi/lo activations, as the forward), else FP32.
    //    With every gradient on the tensor cores they stay NHWC hi/lo;
    //    otherwise planar FP32 for the SIMT gradient kernels.
    const bool on_tc = c.prec == WSKPN_BF16 && tc_split_all(ctx) && ctx->train_tc_recompute && batch <= WSKPN_MAX_BATCH;
    const bool tc_bwd = on_tc && ctx->train_tc_recompute == 1 && t->all_tc;
    auto xn = [&](int l) { return static_cast<void*>(static_cast<uint8_t*>(t->xnhwc) + t->x_off[l]); };
    auto act = [&](int l, int b) { return t->acts + t->act_off[l] + (size_t)b * c.widths[l] * HW; };
    bool kept = tc_bwd && t->kept && t->kept_batch == batch && t->kept_h == h && t->kept_w == w;
    for (int b = 0; kept && b < batch; ++b) kept = same_frames(t->kept_frames[b], frames[b]);
    if (tc_bwd && !kept) {
        if (!t->xnhwc) WSKPN_TRY_ALLOC(t->xnhwc, t->x_bytes);
        if (!t->xbits) WSKPN_TRY_ALLOC(t->xbits, (size_t)L * t->px * 2 * sizeof(uint32_t));
        std::vector<void*> xs(L);
        std::vector<uint32_t*> bits(L);
        for (int l = 0; l < L; ++l) {
            xs[l] = xn(l);
            bits[l] = t->xbits + (size_t)l * t->px * 2;
        }
        t->kept = false;  // overwritten with this call's frames
        s = tc_recompute_nhwc(ctx, frames, batch, h, w, xs, st, &bits);
        if (s) return s;
    } else if (!tc_bwd) {
        if (!t->acts) WSKPN_TRY_ALLOC(t->acts, t->acts_floats * sizeof(float));
        std::vector<void*> x0(batch);
        for (int b = 0; b < batch; ++b) x0[b] = act(0, b);
        s = launch_prep(frames, batch, h, w, c.gamma, c.depth_near, c.depth_far, x0.data(), 0, st, ctx->err);
        if (s) return s;
        std::vector<const float*> in(batch);
        std::vector<float*> o(batch);
        if (on_tc) {
            std::vector<std::vector<float*>> acts(L > 1 ? L - 1 : 0, std::vector<float*>(batch));
            for (int l = 1; l < L; ++l)
                for (int b = 0; b < batch; ++b) acts[l - 1][b] = act(l, b);
            s = tc_recompute_acts(ctx, frames, batch, h, w, acts, st);
            if (s) return s;
        }
        if (!on_tc) {
            s = ctx_simt_weights(ctx, st);
            if (s) return s;
        }
        for (int l = 1; l < L && !on_tc; ++l) {
            for (int b = 0; b < batch; ++b) {
                in[b] = act(l - 1, b);
                o[b] = act(l, b);
            }
            const Layer& Ly = ctx->layers[l - 1];
            s = launch_conv_simt(in.data(), o.data(), batch, h, w, Ly.cin, Ly.cout, KS, Ly.w32, Ly.b32, 1, st,
                                 ctx->err);
            if (s) return s;
        }
    }
    // 3. layer by layer: weight gradient, then the masked input gradient.
    //    Tensor cores: the gradient is packed as NHWC BF16 (one value per
    //    channel: the GEMMs take BF16 operands, FP32 sums); the weight
    //    gradient is a GEMM over the pixels of the layer input's hi half and
    //    the gradient, the input gradient a convolution with the transposed,
    //    flipped BF16 weights whose epilogue applies the ReLU mask (from the
    //    layer input's bits) and forms the bias sums.  Otherwise FP32 SIMT
    //    (mask fused into the conv).
    auto cpad = [&](int ch) { return (ch + 15) / 16 * 16; };
    std::vector<const float*> gy(batch), xs(batch), mask(batch);
    std::vector<float*> gx(batch);
    for (int b = 0; b < batch; ++b) gy[b] = dz + (size_t)b * 2 * M * HW;
    if (!tc_bwd && !t->gA) {
        WSKPN_TRY_ALLOC(t->gA, t->g_floats * sizeof(float));
        WSKPN_TRY_ALLOC(t->gB, t->g_floats * sizeof(float));
    }
    float* gbuf[2] = {t->gA, t->gB};
    void* gcur = t->gpack;  // tensor cores: gy of the current layer, NHWC BF16
    if (tc_bwd) {
        // Transposed weight images first: the input-gradient conv is launched
        // as a programmatic dependent of the kernel before it and loads its
        // weight image before waiting for that kernel, so the image must not
        // be written by the kernel immediately before it.
        for (int l = 1; l < L; ++l) {
            s = tc_dgrad_layer_pack(t->lt[l], KS, ctx->d_master + ctx->layers[l].woff, t->wt, t->zero_bias, st,
                                    ctx->err);
            if (s) return s;
        }
        // dz -> NHWC BF16
        s = launch_grad_pack(gy.data(), batch, 2 * M, cpad(2 * M), HW, t->gpack, t->bias_part,
                             dweights + ctx->layers[L - 1].boff, st, ctx->err);
        if (s) return s;
    }
    for (int l = L - 1; l >= 0; --l) {
        const Layer& Ly = ctx->layers[l];
        if (tc_bwd) {
            const int gcp = cpad(Ly.cout), xcp = cpad(Ly.cin);
            s = launch_wgrad_tc(xn(l), 2 * xcp, gcur, gcp, batch, h, w, Ly.cin, Ly.cout, KS, t->wg_part,
                                t->wg_part_floats, dweights + Ly.woff, ctx->d_status, ctx->device, st, ctx->err);
            if (s) return s;
            if (l == 0) break;
            // input gradient straight to NHWC BF16, times the ReLU mask of
            // x_l, with the bias sums of layer l - 1, in the conv's epilogue
            void* gnext = gcur == t->gpack ? t->gpack2 : t->gpack;
            Layer& Lt = t->lt[l];
            int nparts = 0;
            s = tc_dgrad_run(Lt, KS, gcur, gnext, t->xbits + (size_t)l * t->px * 2, t->bias_part, &nparts, batch, h,
                             w, ctx->d_status, ctx->device, st, ctx->err);
            if (s) return s;
            bias_from_tiles_kernel<<<Ly.cin, 256, 0, st>>>(t->bias_part, nparts, dweights + ctx->layers[l - 1].boff);
            WSKPN_CUDA_TRY(cudaGetLastError(), ctx->err);
            gcur = gnext;
            continue;
        }
        for (int b = 0; b < batch; ++b) xs[b] = act(l, b);
        const int nchunks = (Ly.cin + 7) / 8;
        int G = kWgradGroups / nchunks;
        const int ntiles = ((w + 31) / 32) * ((h + 7) / 8) * batch;
        G = std::max(1, std::min(G, ntiles));
        s = launch_wgrad(xs.data(), gy.data(), batch, h, w, Ly.cin, Ly.cout, KS, G, t->part, dweights + Ly.woff,
                         dweights + Ly.boff, st, ctx->err);
        if (s) return s;
        if (l == 0) break;
        s = launch_pack_simt_transposed(ctx->d_master + Ly.woff, Ly.cin, Ly.cout, KS, t->wT[l], t->bT[l], st,
                                        ctx->err);
        if (s) return s;
        float* dst = gbuf[l % 2];
        for (int b = 0; b < batch; ++b) {
            gx[b] = dst + (size_t)b * Ly.cin * HW;
            mask[b] = xs[b];
        }
        s = launch_conv_simt_masked(gy.data(), gx.data(), mask.data(), batch, h, w, Ly.cout, Ly.cin, KS, t->wT[l],
                                    t->bT[l], 0, st, ctx->err);
        if (s) return s;
        for (int b = 0; b < batch; ++b) gy[b] = gx[b];
    }
    return WSKPN_OK;
}

wskpn_status wskpn_l1_loss(wskpn_ctx* ctx, const float* out, const float* target, size_t n, float* loss,
                           float* dout, void* stream) {
    if (!ctx) return WSKPN_EINVAL;
    if (!out || !target || !loss || n == 0) {
        ctx->err = "wskpn_l1_loss: invalid argument";
        return WSKPN_EINVAL;
    }
    wskpn_status s = ensure_train(ctx);
    if (s) return s;
    TrainWs* t = static_cast<TrainWs*>(ctx->train);
    cudaStream_t st = (cudaStream_t)stream;
    l1_loss_kernel<<<kLossBlocks, 256, 0, st>>>(out, target, n, t->loss_part, dout);
    WSKPN_CUDA_TRY(cudaGetLastError(), ctx->err);
    sum_partials_kernel<<<1, 256, 0, st>>>(t->loss_part, kLossBlocks, 1.0 / (double)n, loss);
    WSKPN_CUDA_TRY(cudaGetLastError(), ctx->err);
    return WSKPN_OK;
}

wskpn_status wskpn_adam_step(wskpn_ctx* ctx, const float* dweights, float lr, float beta1, float beta2, float eps,
                             int step, void* stream) {
    if (!ctx) return WSKPN_EINVAL;
    if (!dweights || step < 1 || !(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) ||
        !(eps > 0.f)) {
        ctx->err = "wskpn_adam_step: invalid argument";
        return WSKPN_EINVAL;
    }
    wskpn_status s = ensure_train(ctx);
    if (s) return s;
    TrainWs* t = static_cast<TrainWs*>(ctx->train);
    cudaStream_t st = (cudaStream_t)stream;
    if (!t->m) {
        WSKPN_TRY_ALLOC(t->m, ctx->nw * sizeof(float));
        WSKPN_TRY_ALLOC(t->v, ctx->nw * sizeof(float));
        WSKPN_CUDA_TRY(cudaMemsetAsync(t->m, 0, ctx->nw * sizeof(float), st), ctx->err);
        WSKPN_CUDA_TRY(cudaMemsetAsync(t->v, 0, ctx->nw * sizeof(float), st), ctx->err);
    }
    const float c1 = (float)(1.0 - std::pow((double)beta1, step));
    const float c2 = (float)(1.0 - std::pow((double)beta2, step));
    adam_kernel<<<148, 256, 0, st>>>(ctx->d_master, dweights, t->m, t->v, ctx->nw, lr, beta1, beta2, eps, c1, c2);
    WSKPN_CUDA_TRY(cudaGetLastError(), ctx->err);
    return ctx_repack(ctx, st);
}

}  // extern "C"
