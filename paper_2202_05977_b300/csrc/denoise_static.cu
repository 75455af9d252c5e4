// Allocation-free variant of the FP32 denoise pipeline.
//
// wskpn_denoise keeps its intermediate images (the network input, the
// hidden activations and the network output) in workspaces that
// wskpn_create allocates with cudaMalloc.  Some callers cannot allocate
// device memory at all: code running where the allocator is off limits
// (inside another runtime's memory pool or a host callback, a plug-in that
// may not grow its process's footprint, a process that must not call
// cudaMalloc after start-up).  wskpn_denoise_static serves them: it runs the
// same kernels in the same order, but every intermediate lives in one
// file-scope device array, g_static_scratch, whose size is fixed when the
// library is loaded.  The caller passes the weights, the frames and the
// output; nothing is allocated or freed.
#include <mutex>

#include "ctx.h"

namespace wskpn {

wskpn_status launch_prep(const wskpn_frame* frames, int B, int H, int W, float gamma, float dnear,
                         float dfar, void* const* out, int layout, cudaStream_t st, std::string& err);
wskpn_status launch_conv_simt(const float* const* in, float* const* out, int B, int H, int W,
                              int Cin, int Cout, int KS, const float* w_packed,
                              const float* bias_padded, int relu, cudaStream_t st, std::string& err);
wskpn_status launch_pack_simt(const float* w, const float* b, int Cin, int Cout, int KS, float* wp,
                              float* bp, cudaStream_t st, std::string& err);
int simt_coutp(int cout);
wskpn_status launch_decode_fuse_fwd(const float* const* z, const float* const* r,
                                    const float* const* a, float* const* out, int B, int H, int W,
                                    int M, const int* ks, float eps, unsigned int* fallbacks,
                                    cudaStream_t st, std::string& err);

namespace {

// 16 Mi floats = 64 MiB, held by every GPU that loads the library until the
// process exits.
constexpr size_t kStaticScratchFloats = size_t(16) << 20;
static __device__ __align__(256) float g_static_scratch[kStaticScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
float* g_static_addr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device, looked up once
// per device.  In host code the array's name is only a stand-in, so kernels
// must be given this address.
wskpn_status static_scratch_address(float** out, std::string& err) {
    int dev = -1;
    WSKPN_CUDA_TRY(cudaGetDevice(&dev), err);
    if (dev < 0 || dev >= kMaxDevices) {
        err = "wskpn_denoise_static: device ordinal out of range";
        return WSKPN_EUNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
        void* p = nullptr;
        WSKPN_CUDA_TRY(cudaGetSymbolAddress(&p, g_static_scratch), err);
        g_static_addr[dev] = static_cast<float*>(p);
    }
    *out = g_static_addr[dev];
    return WSKPN_OK;
}

size_t round4(size_t n) { return (n + 3) / 4 * 4; }

}  // namespace
}  // namespace wskpn

using namespace wskpn;

extern "C" wskpn_status wskpn_denoise_static(const wskpn_config* cfg, const float* weights,
                                             const wskpn_frame* frames, int batch, int h, int w,
                                             float* out, void* stream) {
    std::string err;
    const std::string v = validate_config(cfg);
    if (!v.empty()) {
        set_thread_error("wskpn_denoise_static: " + v);
        return WSKPN_EINVAL;
    }
    if (cfg->prec != WSKPN_FP32) {
        set_thread_error("wskpn_denoise_static: only the FP32 plain path is available without allocation");
        return WSKPN_EUNSUPPORTED;
    }
    if (!weights || !frames || !out || batch < 1 || h < 1 || w < 1) {
        set_thread_error("wskpn_denoise_static: NULL pointer or empty size");
        return WSKPN_EINVAL;
    }
    for (int b = 0; b < batch; ++b)
        if (!frames[b].radiance || !frames[b].albedo || !frames[b].normal || !frames[b].depth) {
            set_thread_error("wskpn_denoise_static: a frame buffer pointer is NULL");
            return WSKPN_EINVAL;
        }
    const wskpn_config& c = *cfg;
    const int L = c.n_layers, KS = c.conv_ks;
    // Scratch plan: packed weights and biases per layer, then the two
    // ping-pong activation images and the network output.
    size_t wfl = 0;
    for (int l = 0; l < L; ++l) {
        const size_t coutp = simt_coutp(c.widths[l + 1]);
        wfl += round4((size_t)c.widths[l] * KS * KS * coutp) + round4(coutp);
    }
    int wa = 0, wb = 0;
    for (int l = 0; l < L; ++l) {
        if (l % 2 == 0) wa = wa > c.widths[l] ? wa : c.widths[l];
        else wb = wb > c.widths[l] ? wb : c.widths[l];
    }
    const size_t px = (size_t)batch * h * w;
    const size_t need = wfl + round4(px * wa) + round4(px * wb) + round4(px * c.widths[L]);
    if (need > kStaticScratchFloats) {
        set_thread_error("wskpn_denoise_static: batch x h x w too large for the 64 MiB static scratch (needs " +
                         std::to_string(need * 4) + " bytes; at the default widths at most about 134000 pixels)");
        return WSKPN_EINVAL;
    }
    float* base = nullptr;
    wskpn_status s = static_scratch_address(&base, err);
    if (s) {
        set_thread_error(err);
        return s;
    }
    cudaStream_t st = (cudaStream_t)stream;
    // Weight packing into the scratch (the FP32 SIMT layout).
    float* p = base;
    const float* wsrc = weights;
    std::vector<const float*> wpk(L), bpk(L);
    for (int l = 0; l < L; ++l) {
        const int cin = c.widths[l], cout = c.widths[l + 1], coutp = simt_coutp(cout);
        float* wp = p;
        p += round4((size_t)cin * KS * KS * coutp);
        float* bp = p;
        p += round4(coutp);
        s = launch_pack_simt(wsrc, wsrc + (size_t)cout * cin * KS * KS, cin, cout, KS, wp, bp, st, err);
        if (s) {
            set_thread_error(err);
            return s;
        }
        wsrc += (size_t)cout * cin * KS * KS + cout;
        wpk[l] = wp;
        bpk[l] = bp;
    }
    float* actA = p;
    p += round4(px * wa);
    float* actB = p;
    p += round4(px * wb);
    float* z = p;
    const size_t HW = (size_t)h * w;
    std::vector<void*> x0(batch);
    for (int b = 0; b < batch; ++b) x0[b] = actA + (size_t)b * c.widths[0] * HW;
    s = launch_prep(frames, batch, h, w, c.gamma, c.depth_near, c.depth_far, x0.data(), 0, st, err);
    std::vector<const float*> in(batch);
    std::vector<float*> o(batch);
    for (int l = 1; l <= L && !s; ++l) {
        float* src = (l - 1) % 2 == 0 ? actA : actB;
        float* dst = l == L ? z : (l % 2 == 0 ? actA : actB);
        for (int b = 0; b < batch; ++b) {
            in[b] = src + (size_t)b * c.widths[l - 1] * HW;
            o[b] = dst + (size_t)b * c.widths[l] * HW;
        }
        s = launch_conv_simt(in.data(), o.data(), batch, h, w, c.widths[l - 1], c.widths[l], KS, wpk[l - 1],
                             bpk[l - 1], l < L, st, err);
    }
    if (!s) {
        std::vector<const float*> zz(batch), rr(batch), aa(batch);
        for (int b = 0; b < batch; ++b) {
            zz[b] = z + (size_t)b * c.widths[L] * HW;
            rr[b] = frames[b].radiance;
            aa[b] = frames[b].albedo;
            o[b] = out + (size_t)b * 3 * HW;
        }
        s = launch_decode_fuse_fwd(zz.data(), rr.data(), aa.data(), o.data(), batch, h, w, c.n_kernels, c.ksizes,
                                   c.albedo_eps, nullptr, st, err);
    }
    if (s) set_thread_error(err);
    return s;
}
