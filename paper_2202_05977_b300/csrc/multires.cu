// Multi-resolution variant of the denoiser (the paper's configuration for
// high-spp input, Sec. 5.3 "Implementation", Eq. 7), U-Net in FP32 or BF16.
//
// A U-Net of 3x3 convolutions predicts, at 3 resolutions, importance maps for
// kernel sizes 3 and 5, their fusion logits and (levels 0 and 1) a blending
// logit b, alpha = sigmoid(b):
//   encoder  E0 10->32, E0b 32->32 | D | E1 32->48, E1b 48->48 | D | E2 48->64, E2b 64->64
//   heads    H2 64->4 on E2b;  D1 = conv([U E2b, E1b]) 112->48, H1 48->5;
//            D0 = conv([U D1, E0b]) 80->32, H0 32->5
// (ReLU after every conv except the heads; D = 2x2 box average over the
// in-image pixels of a block, U = nearest-neighbour upsampling).  Each level
// filters the demodulated irradiance y_l = D^l (r / (a + eps)) with its two
// fused kernels (Eq. 3-5, the reconstruction kernel in irradiance mode), and
// the levels combine from the coarsest with Eq. 7:
//   o_l = i_l - alpha_l U D i_l + alpha_l U o_{l+1},   out = (a + eps) o_0.
//
// FP32: planar [C][h][w] per level, SIMT convolutions.  BF16: channels-last
// hi/lo activations [pixel][hi(C) | lo(C)] and tcgen05 convolutions, FP32
// network outputs.  Concatenations cost nothing in either layout: the skip
// activation E0b (E1b) is written straight into its channels (planes) of
// the buffer the upsampling of D1 (E2b) fills, so [U D1, E0b] is one input.
#include <cuda_bf16.h>

#include <vector>

#include "ctx.h"

namespace wskpn {

wskpn_status launch_prep(const wskpn_frame* frames, int B, int H, int W, float gamma, float dnear, float dfar,
                         void* const* out, int layout, cudaStream_t st, std::string& err);
wskpn_status launch_conv_simt(const float* const* in, float* const* out, int B, int H, int W, int Cin, int Cout,
                              int KS, const float* w_packed, const float* bias_padded, int relu, cudaStream_t st,
                              std::string& err);
wskpn_status launch_pack_simt(const float* w, const float* b, int Cin, int Cout, int KS, float* wp, float* bp,
                              cudaStream_t st, std::string& err);
int simt_coutp(int cout);
wskpn_status launch_decode_fuse_fwd(const float* const* z, const float* const* r, const float* const* a,
                                    float* const* out, int B, int H, int W, int M, const int* ks, float eps,
                                    unsigned int* fallbacks, cudaStream_t st, std::string& err);

namespace mr {
struct LayerSpec {
    int cin, cout, relu;
};
// weight-blob order; every layer is W[cout][cin][3][3] then b[cout]
constexpr LayerSpec LAYERS[] = {{10, 32, 1}, {32, 32, 1}, {32, 48, 1}, {48, 48, 1}, {48, 64, 1}, {64, 64, 1},
                                {64, 4, 0},  {112, 48, 1}, {48, 5, 0}, {80, 32, 1}, {32, 5, 0}};
enum { E0, E0B, E1, E1B, E2, E2B, H2, D1, H1, D0, H0, NL };
constexpr int KS = 3, LEVELS = 3, M = 2;
constexpr int KSIZES[M] = {3, 5};

size_t n_weights() {
    size_t n = 0;
    for (const auto& L : LAYERS) n += (size_t)L.cout * L.cin * KS * KS + L.cout;
    return n;
}

// y = r / (a + eps), 3 planes
__global__ void demod_kernel(const float* __restrict__ r, const float* __restrict__ a, float eps, size_t HW,
                             float* __restrict__ y) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < 3 * HW; i += (size_t)gridDim.x * blockDim.x)
        y[i] = r[i] / (a[i] + eps);
}

// D: C planes [h][w] -> [(h+1)/2][(w+1)/2], mean over the in-image pixels of each 2x2 block
__global__ void down_kernel(const float* __restrict__ x, int C, int h, int w, float* __restrict__ y) {
    const int h2 = (h + 1) / 2, w2 = (w + 1) / 2;
    const size_t n = (size_t)C * h2 * w2;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int X = (int)(i % w2), Y = (int)((i / w2) % h2), c = (int)(i / ((size_t)w2 * h2));
        const float* p = x + (size_t)c * h * w;
        const int x0 = 2 * X, y0 = 2 * Y;
        const bool xr = x0 + 1 < w, yr = y0 + 1 < h;
        float s = p[(size_t)y0 * w + x0];
        if (xr) s += p[(size_t)y0 * w + x0 + 1];
        if (yr) s += p[(size_t)(y0 + 1) * w + x0];
        if (xr && yr) s += p[(size_t)(y0 + 1) * w + x0 + 1];
        y[i] = s / (float)((xr ? 2 : 1) * (yr ? 2 : 1));
    }
}

// U: C planes [(h+1)/2][(w+1)/2] -> [h][w], nearest neighbour
__global__ void up_kernel(const float* __restrict__ x, int C, int h, int w, float* __restrict__ y) {
    const int h2 = (h + 1) / 2, w2 = (w + 1) / 2;
    const size_t n = (size_t)C * h * w;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int X = (int)(i % w), Y = (int)((i / w) % h), c = (int)(i / ((size_t)w * h));
        y[i] = x[((size_t)c * h2 + Y / 2) * w2 + X / 2];
    }
}

// Eq. 7 at one level: o = i - alpha [U D i] + alpha [U o_c], alpha = sigmoid(b);
// with albedo, the result is re-modulated: out = (a + eps) o.
__global__ void combine_kernel(const float* __restrict__ i_f, const float* __restrict__ o_c,
                               const float* __restrict__ blend, const float* __restrict__ a, float eps, int h, int w,
                               float* __restrict__ o) {
    const int h2 = (h + 1) / 2, w2 = (w + 1) / 2;
    const size_t HW = (size_t)h * w;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < HW; i += (size_t)gridDim.x * blockDim.x) {
        const int X = (int)(i % w), Y = (int)(i / w);
        const int x0 = X & ~1, y0 = Y & ~1;
        const bool xr = x0 + 1 < w, yr = y0 + 1 < h;
        const float inv = 1.f / (float)((xr ? 2 : 1) * (yr ? 2 : 1));
        const float al = 1.f / (1.f + expf(-blend[i]));
        const size_t ic = (size_t)(Y / 2) * w2 + X / 2;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float* p = i_f + c * HW;
            float s = p[(size_t)y0 * w + x0];
            if (xr) s += p[(size_t)y0 * w + x0 + 1];
            if (yr) s += p[(size_t)(y0 + 1) * w + x0];
            if (xr && yr) s += p[(size_t)(y0 + 1) * w + x0 + 1];
            const float v = p[i] - al * (s * inv) + al * o_c[(size_t)c * h2 * w2 + ic];
            o[c * HW + i] = a ? (a[c * HW + i] + eps) * v : v;
        }
    }
}

// BF16 hi/lo NHWC: D over channels [c0, c0 + C) of pixels [hi(in_cp) | lo(in_cp)]
// -> [hi(C) | lo(C)] at ceil halves; the mean of hi + lo is split again.
__global__ void pool_nhwc_kernel(const __nv_bfloat16* __restrict__ x, int in_cp, int c0, int C, int h, int w,
                                 __nv_bfloat16* __restrict__ y) {
    const int h2 = (h + 1) / 2, w2 = (w + 1) / 2;
    const size_t n = (size_t)C * h2 * w2;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const size_t q = i / C;
        const int X = (int)(q % w2), Y = (int)(q / w2);
        const int x0 = 2 * X, y0 = 2 * Y;
        float s = 0.f;
        int cnt = 0;
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                if (x0 + dx >= w || y0 + dy >= h) continue;
                const __nv_bfloat16* p = x + ((size_t)(y0 + dy) * w + x0 + dx) * 2 * in_cp + c0 + c;
                s += __bfloat162float(p[0]) + __bfloat162float(p[in_cp]);
                ++cnt;
            }
        const float v = s / (float)cnt;
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        y[q * 2 * C + c] = hi;
        y[q * 2 * C + C + c] = __float2bfloat16_rn(v - __bfloat162float(hi));
    }
}

// BF16 hi/lo NHWC: U of [hi(C) | lo(C)] at ceil halves into channels
// [c0, c0 + C) of pixels [hi(out_cp) | lo(out_cp)] at (h, w).
__global__ void up_nhwc_kernel(const __nv_bfloat16* __restrict__ x, int C, int h, int w, int out_cp, int c0,
                               __nv_bfloat16* __restrict__ y) {
    const int w2 = (w + 1) / 2;
    const size_t n = (size_t)C * h * w;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const size_t q = i / C;
        const int X = (int)(q % w), Y = (int)(q / w);
        const size_t src = ((size_t)(Y / 2) * w2 + X / 2) * 2 * C;
        y[q * 2 * out_cp + c0 + c] = x[src + c];
        y[q * 2 * out_cp + out_cp + c0 + c] = x[src + C + c];
    }
}

inline int grid_for(size_t n) {
    const size_t g = (n + 255) / 256;
    return (int)(g < 148 * 16 ? (g > 0 ? g : 1) : 148 * 16);
}
}  // namespace mr
}  // namespace wskpn

using namespace wskpn;

struct wskpn_mr {
    wskpn_mr_config cfg{};
    int device = 0;
    float* d_master = nullptr;  // FP32 weight blob
    float* w32[mr::NL] = {};    // SIMT packing per layer (FP32)
    float* b32[mr::NL] = {};
    wskpn::Layer tcL[mr::NL];   // tensor-core layers (BF16)
    // BF16 activations, hi/lo NHWC: t0 [32], c0 [48 + 32], p1 [32], t1 [48],
    // c1 [64 + 48], p2 [48], t2 [64], e2 [64] (E0 assembles its own input)
    __nv_bfloat16 *bt0 = nullptr, *bc0 = nullptr, *bp1 = nullptr, *bt1 = nullptr,
                  *bc1 = nullptr, *bp2 = nullptr, *bt2 = nullptr, *be2 = nullptr;
    unsigned int* d_status = nullptr;
    // workspaces, sized for max_h x max_w (levels: l1 = ceil halves, l2 = ceil quarters)
    float* x0 = nullptr;   // [10] level 0
    float* t0 = nullptr;   // [32] E0 / D0 scratch, level 0
    float* c0 = nullptr;   // [48 + 32]: U D1 | E0b
    float* z0 = nullptr;   // [5]
    float* p1 = nullptr;   // [32] D E0b
    float* t1 = nullptr;   // [48] E1 / D1
    float* c1 = nullptr;   // [64 + 48]: U E2b | E1b
    float* z1 = nullptr;   // [5]
    float* p2 = nullptr;   // [48] D E1b
    float* t2 = nullptr;   // [64] E2
    float* e2 = nullptr;   // [64] E2b
    float* z2 = nullptr;   // [4]
    float* y[3] = {};      // demodulated irradiance per level [3]
    float* iv[3] = {};     // filtered irradiance per level [3]
    float* o1 = nullptr;   // Eq. 7 result at level 1 [3]
    unsigned int* d_fallbacks = nullptr;
    std::string err;
};

extern "C" void wskpn_mr_config_default(wskpn_mr_config* c) {
    if (!c) return;
    c->max_h = 1080;
    c->max_w = 1920;
    c->albedo_eps = 1e-2f;
    c->gamma = 2.2f;
    c->depth_near = 1.f;
    c->depth_far = 10.f;
    c->prec = WSKPN_FP32;
}

extern "C" size_t wskpn_mr_n_weights(void) { return mr::n_weights(); }

extern "C" void wskpn_mr_destroy(wskpn_mr* m) {
    if (!m) return;
    cudaFree(m->d_master);
    for (int l = 0; l < mr::NL; ++l) {
        cudaFree(m->w32[l]);
        cudaFree(m->b32[l]);
    }
    float* bufs[] = {m->x0, m->t0, m->c0, m->z0, m->p1, m->t1, m->c1, m->z1, m->p2, m->t2, m->e2, m->z2,
                     m->y[0], m->y[1], m->y[2], m->iv[0], m->iv[1], m->iv[2], m->o1};
    for (float* b : bufs) cudaFree(b);
    __nv_bfloat16* hbufs[] = {m->bt0, m->bc0, m->bp1, m->bt1, m->bc1, m->bp2, m->bt2, m->be2};
    for (auto* b : hbufs) cudaFree(b);
    for (auto& L : m->tcL) tc_layer_free(L);
    cudaFree(m->d_fallbacks);
    cudaFree(m->d_status);
    delete m;
}

extern "C" wskpn_status wskpn_mr_create(const wskpn_mr_config* cfg_in, const float* host_weights, size_t n,
                                        wskpn_mr** out) {
    if (!out || !host_weights) {
        set_thread_error("wskpn_mr_create: NULL argument");
        return WSKPN_EINVAL;
    }
    *out = nullptr;
    wskpn_mr_config cfg;
    wskpn_mr_config_default(&cfg);
    if (cfg_in) cfg = *cfg_in;
    if (cfg.max_h < 1 || cfg.max_w < 1 || (long)cfg.max_h * cfg.max_w > (1L << 26) || !(cfg.albedo_eps > 0.f) ||
        !(cfg.gamma > 0.f) || !(cfg.depth_far > cfg.depth_near) ||
        (cfg.prec != WSKPN_FP32 && cfg.prec != WSKPN_BF16)) {
        set_thread_error("wskpn_mr_create: config out of range");
        return WSKPN_EINVAL;
    }
    if (n != mr::n_weights()) {
        set_thread_error("wskpn_mr_create: expected " + std::to_string(mr::n_weights()) + " weights");
        return WSKPN_EINVAL;
    }
    auto* m = new wskpn_mr();
    m->cfg = cfg;
    cudaGetDevice(&m->device);
    const size_t P0 = (size_t)cfg.max_h * cfg.max_w;
    const size_t h1 = (cfg.max_h + 1) / 2, w1 = (cfg.max_w + 1) / 2;
    const size_t P1 = h1 * w1, P2 = ((h1 + 1) / 2) * ((w1 + 1) / 2);
    auto alloc = [&](float** p, size_t floats) { return cudaMalloc(p, floats * sizeof(float)) == cudaSuccess; };
    auto halloc = [&](__nv_bfloat16** p, size_t ch, size_t px) {
        return cudaMalloc(p, ch * 2 * px * sizeof(__nv_bfloat16)) == cudaSuccess;
    };
    const bool bf16 = cfg.prec == WSKPN_BF16;
    bool ok = alloc(&m->d_master, n) && alloc(&m->z0, 5 * P0) && alloc(&m->z1, 5 * P1) && alloc(&m->z2, 4 * P2) &&
              alloc(&m->y[0], 3 * P0) && alloc(&m->y[1], 3 * P1) && alloc(&m->y[2], 3 * P2) &&
              alloc(&m->iv[0], 3 * P0) && alloc(&m->iv[1], 3 * P1) && alloc(&m->iv[2], 3 * P2) &&
              alloc(&m->o1, 3 * P1) && cudaMalloc(&m->d_fallbacks, sizeof(unsigned int)) == cudaSuccess &&
              cudaMalloc(&m->d_status, sizeof(unsigned int)) == cudaSuccess;
    if (ok && !bf16)
        ok = alloc(&m->x0, 10 * P0) && alloc(&m->t0, 32 * P0) && alloc(&m->c0, 80 * P0) && alloc(&m->p1, 32 * P1) &&
             alloc(&m->t1, 48 * P1) && alloc(&m->c1, 112 * P1) && alloc(&m->p2, 48 * P2) && alloc(&m->t2, 64 * P2) &&
             alloc(&m->e2, 64 * P2);
    if (ok && bf16)
        ok = halloc(&m->bt0, 32, P0) && halloc(&m->bc0, 80, P0) &&
             halloc(&m->bp1, 32, P1) && halloc(&m->bt1, 48, P1) && halloc(&m->bc1, 112, P1) &&
             halloc(&m->bp2, 48, P2) && halloc(&m->bt2, 64, P2) && halloc(&m->be2, 64, P2);
    size_t off = 0;
    for (int l = 0; ok && !bf16 && l < mr::NL; ++l) {
        const auto& L = mr::LAYERS[l];
        const int coutp = simt_coutp(L.cout);
        ok = alloc(&m->w32[l], (size_t)L.cin * mr::KS * mr::KS * coutp) && alloc(&m->b32[l], coutp);
    }
    if (!ok) {
        cudaGetLastError();
        wskpn_mr_destroy(m);
        set_thread_error("wskpn_mr_create: device allocation failed");
        return WSKPN_ENOMEM;
    }
    std::string err;
    wskpn_status s = WSKPN_OK;
    if (cudaMemcpy(m->d_master, host_weights, n * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(m->d_fallbacks, 0, sizeof(unsigned int)) != cudaSuccess ||
        cudaMemset(m->d_status, 0, sizeof(unsigned int)) != cudaSuccess)
        s = WSKPN_ECUDA;
    for (int l = 0; !s && l < mr::NL; ++l) {
        const auto& L = mr::LAYERS[l];
        const size_t nw = (size_t)L.cout * L.cin * mr::KS * mr::KS;
        if (bf16) {
            m->tcL[l].cin = L.cin;
            m->tcL[l].cout = L.cout;
            s = tc_layer_create(m->tcL[l], mr::KS, m->d_master + off, m->d_master + off + nw, nullptr, err);
        } else {
            s = launch_pack_simt(m->d_master + off, m->d_master + off + nw, L.cin, L.cout, mr::KS, m->w32[l],
                                 m->b32[l], nullptr, err);
        }
        off += nw + L.cout;
    }
    if (!s && cudaDeviceSynchronize() != cudaSuccess) s = WSKPN_ECUDA;
    if (s) {
        wskpn_mr_destroy(m);
        set_thread_error("wskpn_mr_create: " + (err.empty() ? std::string("CUDA error") : err));
        return s;
    }
    *out = m;
    return WSKPN_OK;
}

namespace {
wskpn_status mr_conv(wskpn_mr* m, int l, const float* in, float* out, int h, int w, cudaStream_t st) {
    const auto& L = mr::LAYERS[l];
    return launch_conv_simt(&in, &out, 1, h, w, L.cin, L.cout, mr::KS, m->w32[l], m->b32[l], L.relu, st, m->err);
}

wskpn_status mr_tc(wskpn_mr* m, int l, const void* in, void* out, int out_cp, int out_c0, int h, int w,
                   cudaStream_t st) {
    const bool head = l == mr::H2 || l == mr::H1 || l == mr::H0;
    return tc_layer_run(m->tcL[l], mr::KS, in, out, out_cp, out_c0, head, mr::LAYERS[l].relu, 1, h, w, m->d_status,
                        m->device, st, m->err);
}

// BF16 U-Net on the tensor cores (hi/lo activations), same outputs as mr_forward.
wskpn_status mr_forward_bf16(wskpn_mr* m, const wskpn_frame* f, int h, int w, cudaStream_t st) {
    const int h1 = (h + 1) / 2, w1 = (w + 1) / 2, h2 = (h1 + 1) / 2, w2 = (w1 + 1) / 2;
    const size_t P0 = (size_t)h * w, P1 = (size_t)h1 * w1, P2 = (size_t)h2 * w2;
    // E0 assembles its input tiles from the frame (Sec. 5.1) inside its own
    // kernel; the assembled input is never stored
    wskpn_status s = tc_layer_run_pin(m->tcL[mr::E0], mr::KS, f, m->cfg.gamma, m->cfg.depth_near, m->cfg.depth_far,
                                      m->bt0, 32, mr::LAYERS[mr::E0].relu, h, w, m->d_status, m->device, st, m->err);
    if (!s) s = mr_tc(m, mr::E0B, m->bt0, m->bc0, 80, 48, h, w, st);  // skip into channels 48..79
    if (!s) {
        mr::pool_nhwc_kernel<<<mr::grid_for(32 * P1), 256, 0, st>>>(m->bc0, 80, 48, 32, h, w, m->bp1);
        s = mr_tc(m, mr::E1, m->bp1, m->bt1, 48, 0, h1, w1, st);
    }
    if (!s) s = mr_tc(m, mr::E1B, m->bt1, m->bc1, 112, 64, h1, w1, st);  // skip into channels 64..111
    if (!s) {
        mr::pool_nhwc_kernel<<<mr::grid_for(48 * P2), 256, 0, st>>>(m->bc1, 112, 64, 48, h1, w1, m->bp2);
        s = mr_tc(m, mr::E2, m->bp2, m->bt2, 64, 0, h2, w2, st);
    }
    if (!s) s = mr_tc(m, mr::E2B, m->bt2, m->be2, 64, 0, h2, w2, st);
    if (!s) s = mr_tc(m, mr::H2, m->be2, m->z2, 16, 0, h2, w2, st);
    if (!s) {
        mr::up_nhwc_kernel<<<mr::grid_for(64 * P1), 256, 0, st>>>(m->be2, 64, h1, w1, 112, 0, m->bc1);
        s = mr_tc(m, mr::D1, m->bc1, m->bt1, 48, 0, h1, w1, st);
    }
    if (!s) s = mr_tc(m, mr::H1, m->bt1, m->z1, 16, 0, h1, w1, st);
    if (!s) {
        mr::up_nhwc_kernel<<<mr::grid_for(48 * P0), 256, 0, st>>>(m->bt1, 48, h, w, 80, 0, m->bc0);
        s = mr_tc(m, mr::D0, m->bc0, m->bt0, 32, 0, h, w, st);
    }
    if (!s) s = mr_tc(m, mr::H0, m->bt0, m->z0, 16, 0, h, w, st);
    if (!s && cudaGetLastError() != cudaSuccess) {
        m->err = "multires forward: kernel launch failed";
        s = WSKPN_ECUDA;
    }
    return s;
}

// U-Net outputs for one frame into m->z0 [5][h][w], m->z1 [5][h1][w1], m->z2 [4][h2][w2].
wskpn_status mr_forward(wskpn_mr* m, const wskpn_frame* f, int h, int w, cudaStream_t st) {
    if (m->cfg.prec == WSKPN_BF16) return mr_forward_bf16(m, f, h, w, st);
    const int h1 = (h + 1) / 2, w1 = (w + 1) / 2, h2 = (h1 + 1) / 2, w2 = (w1 + 1) / 2;
    const size_t P0 = (size_t)h * w, P1 = (size_t)h1 * w1;
    void* x0 = m->x0;
    wskpn_status s = launch_prep(f, 1, h, w, m->cfg.gamma, m->cfg.depth_near, m->cfg.depth_far, &x0, 0, st, m->err);
    float* e0b = m->c0 + 48 * P0;  // skip planes after the 48 upsampled ones
    float* e1b = m->c1 + 64 * P1;
    if (!s) s = mr_conv(m, mr::E0, m->x0, m->t0, h, w, st);
    if (!s) s = mr_conv(m, mr::E0B, m->t0, e0b, h, w, st);
    if (!s) {
        mr::down_kernel<<<mr::grid_for(32 * P1), 256, 0, st>>>(e0b, 32, h, w, m->p1);
        s = mr_conv(m, mr::E1, m->p1, m->t1, h1, w1, st);
    }
    if (!s) s = mr_conv(m, mr::E1B, m->t1, e1b, h1, w1, st);
    if (!s) {
        mr::down_kernel<<<mr::grid_for(48 * (size_t)h2 * w2), 256, 0, st>>>(e1b, 48, h1, w1, m->p2);
        s = mr_conv(m, mr::E2, m->p2, m->t2, h2, w2, st);
    }
    if (!s) s = mr_conv(m, mr::E2B, m->t2, m->e2, h2, w2, st);
    if (!s) s = mr_conv(m, mr::H2, m->e2, m->z2, h2, w2, st);
    if (!s) {
        mr::up_kernel<<<mr::grid_for(64 * P1), 256, 0, st>>>(m->e2, 64, h1, w1, m->c1);
        s = mr_conv(m, mr::D1, m->c1, m->t1, h1, w1, st);
    }
    if (!s) s = mr_conv(m, mr::H1, m->t1, m->z1, h1, w1, st);
    if (!s) {
        mr::up_kernel<<<mr::grid_for(48 * P0), 256, 0, st>>>(m->t1, 48, h, w, m->c0);
        s = mr_conv(m, mr::D0, m->c0, m->t0, h, w, st);
    }
    if (!s) s = mr_conv(m, mr::H0, m->t0, m->z0, h, w, st);
    if (!s && cudaGetLastError() != cudaSuccess) {
        m->err = "multires forward: kernel launch failed";
        s = WSKPN_ECUDA;
    }
    return s;
}

wskpn_status mr_check(wskpn_mr* m, const wskpn_frame* f, int h, int w, const void* out) {
    if (!m) return WSKPN_EINVAL;
    if (!f || !out || !f->radiance || !f->albedo || !f->normal || !f->depth || h < 1 || w < 1 || h > m->cfg.max_h ||
        w > m->cfg.max_w) {
        m->err = "wskpn_mr: invalid frame, output or size";
        return WSKPN_EINVAL;
    }
    cudaSetDevice(m->device);
    return WSKPN_OK;
}
}  // namespace

extern "C" wskpn_status wskpn_mr_logits(wskpn_mr* m, const wskpn_frame* f, int h, int w, float* z0, float* z1,
                                        float* z2, void* stream) {
    wskpn_status s = mr_check(m, f, h, w, z0);
    if (s) return s;
    if (!z1 || !z2) return WSKPN_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    s = mr_forward(m, f, h, w, st);
    if (s) return s;
    const int h1 = (h + 1) / 2, w1 = (w + 1) / 2, h2 = (h1 + 1) / 2, w2 = (w1 + 1) / 2;
    if (cudaMemcpyAsync(z0, m->z0, 5 * (size_t)h * w * sizeof(float), cudaMemcpyDeviceToDevice, st) ||
        cudaMemcpyAsync(z1, m->z1, 5 * (size_t)h1 * w1 * sizeof(float), cudaMemcpyDeviceToDevice, st) ||
        cudaMemcpyAsync(z2, m->z2, 4 * (size_t)h2 * w2 * sizeof(float), cudaMemcpyDeviceToDevice, st)) {
        m->err = "wskpn_mr_logits: copy failed";
        return WSKPN_ECUDA;
    }
    return WSKPN_OK;
}

extern "C" wskpn_status wskpn_mr_denoise(wskpn_mr* m, const wskpn_frame* f, int h, int w, float* out,
                                         void* stream) {
    wskpn_status s = mr_check(m, f, h, w, out);
    if (s) return s;
    cudaStream_t st = (cudaStream_t)stream;
    s = mr_forward(m, f, h, w, st);
    if (s) return s;
    int hs[3] = {h, (h + 1) / 2, 0}, ws[3] = {w, (w + 1) / 2, 0};
    hs[2] = (hs[1] + 1) / 2;
    ws[2] = (ws[1] + 1) / 2;
    // irradiance pyramid
    mr::demod_kernel<<<mr::grid_for(3 * (size_t)h * w), 256, 0, st>>>(f->radiance, f->albedo, m->cfg.albedo_eps,
                                                                     (size_t)h * w, m->y[0]);
    for (int l = 1; l < mr::LEVELS; ++l)
        mr::down_kernel<<<mr::grid_for(3 * (size_t)hs[l] * ws[l]), 256, 0, st>>>(m->y[l - 1], 3, hs[l - 1],
                                                                                 ws[l - 1], m->y[l]);
    // per-level Eq. 3-5 (irradiance mode: no albedo)
    const float* zl[3] = {m->z0, m->z1, m->z2};
    for (int l = 0; l < mr::LEVELS && !s; ++l) {
        const float* yl = m->y[l];
        const float* al = nullptr;
        float* il = m->iv[l];
        s = launch_decode_fuse_fwd(&zl[l], &yl, &al, &il, 1, hs[l], ws[l], mr::M, mr::KSIZES, m->cfg.albedo_eps,
                                   m->d_fallbacks, st, m->err);
    }
    if (s) return s;
    // Eq. 7 from the coarsest level; the last step re-modulates
    mr::combine_kernel<<<mr::grid_for((size_t)hs[1] * ws[1]), 256, 0, st>>>(
        m->iv[1], m->iv[2], m->z1 + 4 * (size_t)hs[1] * ws[1], nullptr, 0.f, hs[1], ws[1], m->o1);
    mr::combine_kernel<<<mr::grid_for((size_t)h * w), 256, 0, st>>>(m->iv[0], m->o1, m->z0 + 4 * (size_t)h * w,
                                                                    f->albedo, m->cfg.albedo_eps, h, w, out);
    if (cudaGetLastError() != cudaSuccess) {
        m->err = "wskpn_mr_denoise: kernel launch failed";
        return WSKPN_ECUDA;
    }
    return WSKPN_OK;
}

extern "C" const char* wskpn_mr_last_error(const wskpn_mr* m) { return m ? m->err.c_str() : ""; }
