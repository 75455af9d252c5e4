// C ABI of libwskpn: context lifetime, weight packing, workspaces and the
// per-frame denoise pipeline (Sec. 5.1 prep -> Sec. 4.1 convs -> Eq. 3-5
// reconstruction), all enqueued on the caller's stream.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "ctx.h"

namespace wskpn {

static thread_local std::string g_thread_err;
void set_thread_error(const std::string& msg) { g_thread_err = msg; }
const std::string& thread_error() { return g_thread_err; }

// kernels (other translation units)
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

void prof_begin(wskpn_ctx* ctx, cudaStream_t st) {
    if (!ctx->prof) return;
    const size_t n = ctx->cfg.n_layers + 3;
    if (ctx->prof_used == ctx->prof_sets.size()) {
        std::vector<cudaEvent_t> ev(n);
        for (auto& e : ev) cudaEventCreate(&e);
        ctx->prof_sets.push_back(ev);
    }
    ctx->prof_cur = (int)ctx->prof_used++;
    auto& ev = ctx->prof_sets[ctx->prof_cur];
    for (size_t i = 0; i < n; ++i) cudaEventRecord(ev[i], st);  // stages not run read as 0 ms
}

void prof_mark(wskpn_ctx* ctx, int boundary, cudaStream_t st) {
    if (!ctx->prof || ctx->prof_cur < 0) return;
    auto& ev = ctx->prof_sets[ctx->prof_cur];
    for (size_t i = boundary; i < ev.size(); ++i) cudaEventRecord(ev[i], st);
}

void prof_end(wskpn_ctx* ctx) { ctx->prof_cur = -1; }

std::string validate_config(const wskpn_config* c) {
    if (!c) return "config is NULL";
    if (c->n_layers < 1 || c->n_layers > WSKPN_MAX_LAYERS) return "n_layers out of range [1, 8]";
    if (c->widths[0] != 10) return "widths[0] must be 10 (Sec. 5.1 input channels)";
    for (int l = 1; l <= c->n_layers; ++l)
        if (c->widths[l] < 1 || c->widths[l] > 64) return "layer widths must be in [1, 64]";
    if (c->conv_ks != 3 && c->conv_ks != 5) return "conv_ks must be 3 or 5";
    if (c->n_kernels < 1 || c->n_kernels > WSKPN_MAX_KERNELS) return "n_kernels out of range [1, 8]";
    if (c->widths[c->n_layers] != 2 * c->n_kernels) return "last width must be 2 * n_kernels";
    for (int i = 0; i < c->n_kernels; ++i)
        if (c->ksizes[i] < 1 || c->ksizes[i] > 13 || (c->ksizes[i] & 1) == 0)
            return "ksizes must be odd and in [1, 13]";
    if (!(c->albedo_eps > 0.f)) return "albedo_eps must be > 0";
    if (!(c->gamma > 0.f)) return "gamma must be > 0";
    if (!(c->depth_far > c->depth_near)) return "depth_far must exceed depth_near";
    if (c->max_batch < 1 || c->max_batch > 64) return "max_batch out of range [1, 64]";
    if (c->max_h < 1 || c->max_w < 1 || (long)c->max_h * c->max_w > (1L << 26))
        return "max_h/max_w out of range";
    if (c->prec != WSKPN_FP32 && c->prec != WSKPN_BF16 && c->prec != WSKPN_FP8) return "unknown precision";
    return "";
}

size_t n_weights_of(const wskpn_config* c) {
    size_t n = 0;
    for (int l = 1; l <= c->n_layers; ++l)
        n += (size_t)c->widths[l] * c->widths[l - 1] * c->conv_ks * c->conv_ks + c->widths[l];
    return n;
}

// Weight images from the master weights: the configured precision's now;
// the FP32 SIMT images of a BF16 / FP8 context (used only by its FP32
// training and calibration paths) when one of those next needs them.
wskpn_status ctx_repack(wskpn_ctx* ctx, cudaStream_t st) {
    const wskpn_config& c = ctx->cfg;
    ctx->simt_stale = true;
    if (c.prec == WSKPN_FP32) return ctx_simt_weights(ctx, st);
    for (int l = 0; l < c.n_layers; ++l) {
        const wskpn_status s = tc_pack_layer(ctx, l, st);
        if (s) return s;
    }
    return WSKPN_OK;
}

wskpn_status ctx_simt_weights(wskpn_ctx* ctx, cudaStream_t st) {
    if (!ctx->simt_stale) return WSKPN_OK;
    const wskpn_config& c = ctx->cfg;
    for (int l = 0; l < c.n_layers; ++l) {
        Layer& L = ctx->layers[l];
        const wskpn_status s = launch_pack_simt(ctx->d_master + L.woff, ctx->d_master + L.boff, L.cin, L.cout,
                                                c.conv_ks, L.w32, L.b32, st, ctx->err);
        if (s) return s;
    }
    ctx->simt_stale = false;
    return WSKPN_OK;
}

wskpn_status check_frames(wskpn_ctx* ctx, const wskpn_frame* frames, int batch, int h, int w) {
    if (!frames) {
        ctx->err = "frames is NULL";
        return WSKPN_EINVAL;
    }
    if (batch < 1 || batch > ctx->cfg.max_batch) {
        ctx->err = "batch out of range [1, max_batch]";
        return WSKPN_EINVAL;
    }
    if (h < 1 || w < 1 || h > ctx->cfg.max_h || w > ctx->cfg.max_w || (size_t)batch * h * w > ctx->ws_pixels) {
        ctx->err = "frame size exceeds the context's max_h/max_w/max_batch";
        return WSKPN_EINVAL;
    }
    for (int b = 0; b < batch; ++b)
        if (!frames[b].radiance || !frames[b].albedo || !frames[b].normal || !frames[b].depth) {
            ctx->err = "a frame buffer pointer is NULL";
            return WSKPN_EINVAL;
        }
    return WSKPN_OK;
}

// FP32 plain path: prep -> SIMT convs -> z (planar FP32 [B][2M][H][W]).
static wskpn_status logits_fp32(wskpn_ctx* ctx, const wskpn_frame* frames, int B, int H, int W,
                                float* z, cudaStream_t st) {
    const wskpn_config& c = ctx->cfg;
    const size_t HW = (size_t)H * W;
    std::vector<void*> x0(B);
    for (int b = 0; b < B; ++b) x0[b] = ctx->d_actA + (size_t)b * c.widths[0] * HW;
    wskpn_status s = launch_prep(frames, B, H, W, c.gamma, c.depth_near, c.depth_far, x0.data(), 0, st, ctx->err);
    if (s) return s;
    prof_mark(ctx, 1, st);
    s = ctx_simt_weights(ctx, st);
    if (s) return s;
    std::vector<const float*> in(B);
    std::vector<float*> out(B);
    for (int l = 1; l <= c.n_layers; ++l) {
        float* src = (l - 1) % 2 == 0 ? ctx->d_actA : ctx->d_actB;
        float* dst = l == c.n_layers ? z : (l % 2 == 0 ? ctx->d_actA : ctx->d_actB);
        for (int b = 0; b < B; ++b) {
            in[b] = src + (size_t)b * c.widths[l - 1] * HW;
            out[b] = dst + (size_t)b * c.widths[l] * HW;
        }
        const Layer& L = ctx->layers[l - 1];
        s = launch_conv_simt(in.data(), out.data(), B, H, W, L.cin, L.cout, c.conv_ks, L.w32, L.b32,
                             l < c.n_layers, st, ctx->err);
        if (s) return s;
        prof_mark(ctx, 1 + l, st);
    }
    return WSKPN_OK;
}

wskpn_status ctx_logits(wskpn_ctx* ctx, const wskpn_frame* frames, int B, int H, int W, float* z,
                        cudaStream_t st) {
    if (ctx->cfg.prec == WSKPN_FP32) return logits_fp32(ctx, frames, B, H, W, z, st);
    return tc_logits(ctx, frames, B, H, W, z, st);
}

}  // namespace wskpn

using namespace wskpn;

extern "C" {

const char* wskpn_version(void) { return "wskpn 0.1 (sm_103a)"; }

wskpn_status wskpn_config_default(wskpn_config* cfg) {
    if (!cfg) {
        set_thread_error("cfg is NULL");
        return WSKPN_EINVAL;
    }
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->n_layers = 4;
    const int widths[5] = {10, 32, 48, 64, 12};
    for (int i = 0; i < 5; ++i) cfg->widths[i] = widths[i];
    cfg->conv_ks = 5;
    cfg->n_kernels = 6;
    for (int i = 0; i < 6; ++i) cfg->ksizes[i] = 3 + 2 * i;
    cfg->prec = WSKPN_BF16;
    cfg->albedo_eps = 1e-2f;
    cfg->gamma = 2.2f;
    cfg->depth_near = 1.f;
    cfg->depth_far = 10.f;
    cfg->max_batch = 1;
    cfg->max_h = 1080;
    cfg->max_w = 1920;
    return WSKPN_OK;
}

size_t wskpn_n_weights(const wskpn_config* cfg) {
    if (!validate_config(cfg).empty()) return 0;
    return n_weights_of(cfg);
}

wskpn_status wskpn_create(const wskpn_config* cfg, const float* host_weights, size_t n, wskpn_ctx** out) {
    if (!out) {
        set_thread_error("out is NULL");
        return WSKPN_EINVAL;
    }
    *out = nullptr;
    std::string v = validate_config(cfg);
    if (!v.empty()) {
        set_thread_error(v);
        return WSKPN_EINVAL;
    }
    if (!host_weights || n != n_weights_of(cfg)) {
        set_thread_error("weights NULL or wrong count (see wskpn_n_weights)");
        return WSKPN_EINVAL;
    }
    wskpn_ctx* ctx = new wskpn_ctx();
    ctx->cfg = *cfg;
    ctx->nw = n;
    wskpn_status s = ctx_init(ctx, host_weights);
    if (s) {
        set_thread_error(ctx->err);
        wskpn_destroy(ctx);
        return s;
    }
    *out = ctx;
    return WSKPN_OK;
}

void wskpn_destroy(wskpn_ctx* ctx) {
    if (!ctx) return;
    ctx_free(ctx);
    delete ctx;
}

const char* wskpn_last_error(const wskpn_ctx* ctx) { return ctx ? ctx->err.c_str() : thread_error().c_str(); }

wskpn_status wskpn_set_weights(wskpn_ctx* ctx, const float* weights, size_t n, int on_device, void* stream) {
    if (!ctx) return WSKPN_EINVAL;
    if (!weights || n != ctx->nw) {
        ctx->err = "weights NULL or wrong count";
        return WSKPN_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    WSKPN_CUDA_TRY(cudaMemcpyAsync(ctx->d_master, weights, n * sizeof(float),
                                   on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st),
                   ctx->err);
    if (!on_device) WSKPN_CUDA_TRY(cudaStreamSynchronize(st), ctx->err);  // host buffer may go away
    return ctx_repack(ctx, st);
}

wskpn_status wskpn_get_weights(wskpn_ctx* ctx, float* dev_out, size_t n, void* stream) {
    if (!ctx) return WSKPN_EINVAL;
    if (!dev_out || n != ctx->nw) {
        ctx->err = "dev_out NULL or wrong count";
        return WSKPN_EINVAL;
    }
    WSKPN_CUDA_TRY(cudaMemcpyAsync(dev_out, ctx->d_master, n * sizeof(float), cudaMemcpyDeviceToDevice,
                                   (cudaStream_t)stream),
                   ctx->err);
    return WSKPN_OK;
}

wskpn_status wskpn_logits(wskpn_ctx* ctx, const wskpn_frame* frames, int batch, int h, int w, float* z_out,
                          void* stream) {
    if (!ctx) return WSKPN_EINVAL;
    wskpn_status s = check_frames(ctx, frames, batch, h, w);
    if (s) return s;
    if (!z_out) {
        ctx->err = "z_out is NULL";
        return WSKPN_EINVAL;
    }
    prof_begin(ctx, (cudaStream_t)stream);
    s = ctx_logits(ctx, frames, batch, h, w, z_out, (cudaStream_t)stream);
    prof_end(ctx);
    return s;
}

wskpn_status wskpn_denoise(wskpn_ctx* ctx, const wskpn_frame* frames, int batch, int h, int w, float* out,
                           void* stream) {
    if (!ctx) return WSKPN_EINVAL;
    wskpn_status s = check_frames(ctx, frames, batch, h, w);
    if (s) return s;
    if (!out) {
        ctx->err = "out is NULL";
        return WSKPN_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const wskpn_config& c = ctx->cfg;
    prof_begin(ctx, st);
    s = ctx_logits(ctx, frames, batch, h, w, ctx->d_z, st);
    if (s) {
        prof_end(ctx);
        return s;
    }
    const size_t HW = (size_t)h * w;
    std::vector<const float*> z(batch), r(batch), a(batch);
    std::vector<float*> o(batch);
    for (int b = 0; b < batch; ++b) {
        z[b] = ctx->d_z + (size_t)b * 2 * c.n_kernels * HW;
        r[b] = frames[b].radiance;
        a[b] = frames[b].albedo;
        o[b] = out + (size_t)b * 3 * HW;
    }
    s = launch_decode_fuse_fwd(z.data(), r.data(), a.data(), o.data(), batch, h, w, c.n_kernels, c.ksizes,
                               c.albedo_eps, ctx->d_fallbacks, st, ctx->err);
    prof_mark(ctx, c.n_layers + 2, st);
    prof_end(ctx);
    return s;
}

// Banded host call.  Output rows [y0, y1) of a frame depend only on input
// rows within the receptive field: conv_ks / 2 per layer plus the largest
// window's half, so each band is denoised as a sub-image of its rows plus
// that halo (recomputed per band) and only its central rows are kept.  Band
// j + 1's upload (one copy stream) and band j - 1's download (another)
// overlap band j's compute on the caller's stream.
static int band_halo(const wskpn_config& c) {
    int kmax = 1;
    for (int i = 0; i < c.n_kernels; ++i) kmax = std::max(kmax, c.ksizes[i]);
    return c.n_layers * (c.conv_ks / 2) + kmax / 2;
}

// The network's workspaces (activations, logits) for a call of `px` pixels,
// moved to the second half of the context's buffers while the object lives:
// two band calls of at most ws_pixels / 2 pixels each can then be in flight
// on two streams (kernels take the buffer addresses at launch).  The
// context's device status word and fallback counter are NOT shifted: both
// band streams accumulate into the same two words, which are meant to be
// read only after the call's final synchronisation (a timeout bit or a
// fallback count then covers the whole frame, not one band).
struct WorkspaceShift {
    wskpn_ctx* c;
    void *ta, *tb;
    float *fa, *fb, *z;
    WorkspaceShift(wskpn_ctx* ctx, bool shift, size_t px) : c(ctx) {
        ta = c->d_tcA, tb = c->d_tcB, fa = c->d_actA, fb = c->d_actB, z = c->d_z;
        if (!shift) return;
        const wskpn_config& cfg = c->cfg;
        auto up = [](size_t b) { return (b + 255) / 256 * 256; };  // keep 256-byte alignment
        if (c->d_tcA) c->d_tcA = static_cast<uint8_t*>(ta) + up(px * tc_act_bytes_per_pixel(cfg, 0));
        if (c->d_tcB) c->d_tcB = static_cast<uint8_t*>(tb) + up(px * tc_act_bytes_per_pixel(cfg, 1));
        int wa = 0, wb = 0;
        for (int l = 0; l < cfg.n_layers; ++l) (l % 2 == 0 ? wa : wb) = std::max(l % 2 == 0 ? wa : wb, cfg.widths[l]);
        if (c->d_actA) c->d_actA = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(fa) + up(px * wa * 4));
        if (c->d_actB) c->d_actB = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(fb) + up(px * wb * 4));
        c->d_z = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(z) + up(px * cfg.widths[cfg.n_layers] * 4));
    }
    ~WorkspaceShift() { c->d_tcA = ta, c->d_tcB = tb, c->d_actA = fa, c->d_actB = fb, c->d_z = z; }
};

// wait: return after the results are in host_out; else return once the
// work is queued, with `st` ordered after the last download (a later call's
// bands then wait, through the slot events, only for the slots they reuse).
static wskpn_status denoise_host_banded(wskpn_ctx* ctx, const wskpn_frame* hf, int batch, int h, int w,
                                        float* host_out, int nb, cudaStream_t st, bool wait) {
    const int halo = band_halo(ctx->cfg);
    // band k covers rows [yb[k], yb[k + 1]); the first may be shorter (the
    // first computation starts sooner) and the last (less work after the
    // last upload)
    std::vector<int> yb(nb + 1, h);
    {
        double wgt[64];
        double tot = 0.0;
        for (int k = 0; k < nb; ++k) {
            wgt[k] = nb == 1 ? 1.0 : k == 0 ? ctx->host_first_pct / 100.0 : k == nb - 1 ? ctx->host_last_pct / 100.0 : 1.0;
            tot += wgt[k];
        }
        double acc = 0.0;
        yb[0] = 0;
        for (int k = 1; k < nb; ++k) {
            acc += wgt[k - 1];
            yb[k] = std::max(yb[k - 1] + 1, std::min(h - (nb - k), (int)(h * acc / tot + 0.5)));
        }
    }
    int bh = 0;
    for (int k = 0; k < nb; ++k) bh = std::max(bh, yb[k + 1] - yb[k]);
    const int ext = std::min(h, bh + 2 * halo);  // rows of an extended band
    const size_t need = (size_t)13 * ext * w;
    if (!ctx->up_stream) {
        WSKPN_CUDA_TRY(cudaStreamCreateWithFlags(&ctx->up_stream, cudaStreamNonBlocking), ctx->err);
        WSKPN_CUDA_TRY(cudaStreamCreateWithFlags(&ctx->down_stream, cudaStreamNonBlocking), ctx->err);
        WSKPN_CUDA_TRY(cudaStreamCreateWithFlags(&ctx->halo_stream, cudaStreamNonBlocking), ctx->err);
        ctx->band_events.resize(4 * wskpn_ctx::BAND_SLOTS + 2);
        for (auto& e : ctx->band_events)
            WSKPN_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), ctx->err);
    }
    // consecutive bands compute on two streams (one's tail overlaps the
    // next one's start) when two band workspaces fit in the context's
    // buffers; not while per-stage profiling records events on one stream
    const size_t band_px = (size_t)ext * w;
    const bool two = !ctx->prof && 2 * (band_px + 256) <= ctx->ws_pixels;
    if (two && !ctx->band_stream)
        WSKPN_CUDA_TRY(cudaStreamCreateWithFlags(&ctx->band_stream, cudaStreamNonBlocking), ctx->err);
    cudaEvent_t ev_start = ctx->band_events[4 * wskpn_ctx::BAND_SLOTS];
    cudaEvent_t ev_end = ctx->band_events[4 * wskpn_ctx::BAND_SLOTS + 1];
    // A band buffer holds its inputs from the start and its output past the
    // inputs of the call's tallest band.  A call with another layout (frame
    // width or band height) could write inputs over an output an earlier
    // call has not downloaded yet: its copies into the buffers wait for
    // that call's last download first.  Calls of one size overlap freely.
    if (ctx->band_job > 0 && (ext != ctx->band_ext || w != ctx->band_w)) {
        WSKPN_CUDA_TRY(cudaStreamWaitEvent(ctx->up_stream, ev_end, 0), ctx->err);
        WSKPN_CUDA_TRY(cudaStreamWaitEvent(ctx->halo_stream, ev_end, 0), ctx->err);
    }
    ctx->band_ext = ext;
    ctx->band_w = w;
    if (two) {  // the second stream starts after what the caller queued before
        WSKPN_CUDA_TRY(cudaEventRecord(ev_start, st), ctx->err);
        WSKPN_CUDA_TRY(cudaStreamWaitEvent(ctx->band_stream, ev_start, 0), ctx->err);
    }
    constexpr int NS = wskpn_ctx::BAND_SLOTS;
    if (ctx->band_floats < need) {
        // earlier calls that returned without waiting may still use the slots
        WSKPN_CUDA_TRY(cudaDeviceSynchronize(), ctx->err);
        for (float*& p : ctx->d_band) {
            cudaFree(p);
            p = nullptr;
        }
        ctx->band_floats = 0;
        for (float*& p : ctx->d_band) WSKPN_CUDA_TRY(cudaMalloc(&p, need * sizeof(float)), ctx->err);
        ctx->band_floats = need;
    }
    // events per slot s: uploaded, computed, downloaded, halo rows copied in
    // from the previous band's slot.  With three slots the upload of band j
    // waits only for band j - 3's compute, so the uploads (the host link is
    // the bottleneck) run back to back while bands compute.
    cudaEvent_t* evs = ctx->band_events.data();
    auto EV_UP = [&](int s) { return evs[s]; };
    auto EV_COMP = [&](int s) { return evs[NS + s]; };
    auto EV_DOWN = [&](int s) { return evs[2 * NS + s]; };
    auto EV_HALO = [&](int s) { return evs[3 * NS + s]; };
    const int ch[4] = {3, 3, 3, 1};
    const size_t HW = (size_t)h * w;
    // the job count runs on across calls, so that a call's first bands wait
    // for the slots' previous uses (also those of an earlier call that
    // returned without waiting)
    uint64_t job = ctx->band_job;
    for (int b = 0; b < batch; ++b) {
        const float* src[4] = {hf[b].radiance, hf[b].albedo, hf[b].normal, hf[b].depth};
        int pe0 = 0, pe1 = 0;  // extended rows of this frame's previous band (in the other slot)
        for (int k = 0; k < nb; ++k, ++job) {
            const int slot = (int)(job % NS), pslot = (int)((job + NS - 1) % NS);
            const int y0 = yb[k], y1 = yb[k + 1];
            if (y0 >= y1) break;
            const int e0 = std::max(0, y0 - halo), e1 = std::min(h, y1 + halo), eh = e1 - e0;
            const size_t ePX = (size_t)eh * w;
            float* base = ctx->d_band[slot];
            // the slot's previous band (job - NS) must be computed before its
            // inputs are replaced, and band job - NS + 1 must have copied its
            // halo rows out of this slot
            if (job >= NS) WSKPN_CUDA_TRY(cudaStreamWaitEvent(ctx->up_stream, EV_COMP(slot), 0), ctx->err);
            if (job >= NS - 1)
                WSKPN_CUDA_TRY(cudaStreamWaitEvent(ctx->up_stream, EV_HALO((job - NS + 1) % NS), 0), ctx->err);
            wskpn_frame f{};
            const float** dst[4] = {&f.radiance, &f.albedo, &f.normal, &f.depth};
            // rows [e0, kept) are already on the device in the previous band's
            // slot (its halo overlaps this band's): copied there device to device
            // on a stream of their own, concurrently with this band's upload;
            // only rows [kept, e1) cross the host link, so each input row is
            // uploaded once per frame
            const int kept = k > 0 ? std::max(e0, std::min(e1, pe1)) : e0;
            const size_t pPX = (size_t)(pe1 - pe0) * w;
            const float* prev = ctx->d_band[pslot];
            if (kept > e0) {  // after the previous band's upload and this slot's previous compute
                WSKPN_CUDA_TRY(cudaStreamWaitEvent(ctx->halo_stream, EV_UP(pslot), 0), ctx->err);
                if (job >= NS) WSKPN_CUDA_TRY(cudaStreamWaitEvent(ctx->halo_stream, EV_COMP(slot), 0), ctx->err);
            }
            float* p = base;
            for (int q = 0; q < 4; ++q) {
                *dst[q] = p;
                if (kept > e0)  // ch[q] planes, pPX apart in the previous slot, ePX apart here
                    WSKPN_CUDA_TRY(cudaMemcpy2DAsync(p, ePX * sizeof(float), prev + (size_t)(e0 - pe0) * w,
                                                     pPX * sizeof(float), (size_t)(kept - e0) * w * sizeof(float),
                                                     ch[q], cudaMemcpyDeviceToDevice, ctx->halo_stream),
                                   ctx->err);
                if (e1 > kept)  // one 2D copy per input buffer: ch[q] planes HW apart in the host buffer
                    WSKPN_CUDA_TRY(cudaMemcpy2DAsync(p + (size_t)(kept - e0) * w, ePX * sizeof(float),
                                                     src[q] + (size_t)kept * w, HW * sizeof(float),
                                                     (size_t)(e1 - kept) * w * sizeof(float), ch[q],
                                                     cudaMemcpyHostToDevice, ctx->up_stream),
                                   ctx->err);
                p += (size_t)ch[q] * ePX;
                prev += (size_t)ch[q] * pPX;
            }
            WSKPN_CUDA_TRY(cudaEventRecord(EV_HALO(slot), ctx->halo_stream), ctx->err);
            pe0 = e0;
            pe1 = e1;
            // the output region sits past the inputs of the tallest band, so a
            // later, taller band's upload into this slot cannot reach the rows
            // of this band still waiting for download
            float* dout = base + (size_t)10 * ext * w;
            WSKPN_CUDA_TRY(cudaEventRecord(EV_UP(slot), ctx->up_stream), ctx->err);
            // compute after the upload and the halo copy, and after the slot's
            // previous download; with two compute streams, odd jobs use the
            // second stream and the second half of the workspaces (jobs on
            // one stream run in order, so a workspace half is never shared)
            const bool odd = job & 1;
            cudaStream_t cs = two && odd ? ctx->band_stream : st;
            WSKPN_CUDA_TRY(cudaStreamWaitEvent(cs, EV_UP(slot), 0), ctx->err);
            WSKPN_CUDA_TRY(cudaStreamWaitEvent(cs, EV_HALO(slot), 0), ctx->err);
            if (job >= NS) WSKPN_CUDA_TRY(cudaStreamWaitEvent(cs, EV_DOWN(slot), 0), ctx->err);
            {
                WorkspaceShift shift(ctx, two && odd, band_px);
                wskpn_status s = wskpn_denoise(ctx, &f, 1, eh, w, dout, cs);
                if (s) return s;
            }
            WSKPN_CUDA_TRY(cudaEventRecord(EV_COMP(slot), cs), ctx->err);
            // download the central rows
            WSKPN_CUDA_TRY(cudaStreamWaitEvent(ctx->down_stream, EV_COMP(slot), 0), ctx->err);
            WSKPN_CUDA_TRY(cudaMemcpy2DAsync(host_out + (size_t)b * 3 * HW + (size_t)y0 * w, HW * sizeof(float),
                                             dout + (size_t)(y0 - e0) * w, ePX * sizeof(float),
                                             (size_t)(y1 - y0) * w * sizeof(float), 3, cudaMemcpyDeviceToHost,
                                             ctx->down_stream),
                           ctx->err);
            WSKPN_CUDA_TRY(cudaEventRecord(EV_DOWN(slot), ctx->down_stream), ctx->err);
            ctx->band_job = job + 1;  // issued: a later call (even after an error here) waits for it
        }
    }
    // every download is ordered after its band's compute
    WSKPN_CUDA_TRY(cudaEventRecord(ev_end, ctx->down_stream), ctx->err);
    if (!wait) {
        WSKPN_CUDA_TRY(cudaStreamWaitEvent(st, ev_end, 0), ctx->err);
        return WSKPN_OK;
    }
    WSKPN_CUDA_TRY(cudaStreamSynchronize(ctx->down_stream), ctx->err);
    WSKPN_CUDA_TRY(cudaStreamSynchronize(st), ctx->err);
    if (two) WSKPN_CUDA_TRY(cudaStreamSynchronize(ctx->band_stream), ctx->err);
    return WSKPN_OK;
}

static wskpn_status denoise_host(wskpn_ctx* ctx, const wskpn_frame* host_frames, int batch, int h, int w,
                                 float* host_out, void* stream, bool wait) {
    if (!ctx) return WSKPN_EINVAL;
    wskpn_status s = check_frames(ctx, host_frames, batch, h, w);
    if (s) return s;
    if (!host_out) {
        ctx->err = "host_out is NULL";
        return WSKPN_EINVAL;
    }
    // Frames of at least 432 rows go through the banded pipeline (one band
    // per ~160 rows, at most 12; measured best or within 2 % of the best
    // count at 720p, 1080p and 1440p): the recomputed halos cost less than
    // the copies they let overlap.  Smaller frames: one upload, denoise,
    // download.
    const int nb = ctx->host_bands > 0 ? std::min(ctx->host_bands, h) : h < 432 ? 1 : std::min(12, h / 160);
    if (nb >= 2) return denoise_host_banded(ctx, host_frames, batch, h, w, host_out, nb, (cudaStream_t)stream, wait);
    if (!ctx->d_stage) {
        cudaError_t e = cudaMalloc((void**)&ctx->d_stage, ctx->ws_pixels * 13 * sizeof(float));
        if (e != cudaSuccess) {
            ctx->d_stage = nullptr;
            ctx->err = std::string("staging cudaMalloc: ") + cudaGetErrorString(e);
            return WSKPN_ENOMEM;
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t HW = (size_t)h * w;
    std::vector<wskpn_frame> dev(batch);
    float* p = ctx->d_stage;
    for (int b = 0; b < batch; ++b) {
        const float* src[4] = {host_frames[b].radiance, host_frames[b].albedo, host_frames[b].normal,
                               host_frames[b].depth};
        const int ch[4] = {3, 3, 3, 1};
        const float** dst[4] = {&dev[b].radiance, &dev[b].albedo, &dev[b].normal, &dev[b].depth};
        for (int k = 0; k < 4; ++k) {
            WSKPN_CUDA_TRY(cudaMemcpyAsync(p, src[k], ch[k] * HW * sizeof(float), cudaMemcpyHostToDevice, st),
                           ctx->err);
            *dst[k] = p;
            p += ch[k] * HW;
        }
    }
    float* dout = p;
    s = wskpn_denoise(ctx, dev.data(), batch, h, w, dout, stream);
    if (s) return s;
    WSKPN_CUDA_TRY(cudaMemcpyAsync(host_out, dout, (size_t)batch * 3 * HW * sizeof(float), cudaMemcpyDeviceToHost,
                                   st),
                   ctx->err);
    if (wait) WSKPN_CUDA_TRY(cudaStreamSynchronize(st), ctx->err);
    return WSKPN_OK;
}

wskpn_status wskpn_denoise_host(wskpn_ctx* ctx, const wskpn_frame* host_frames, int batch, int h, int w,
                                float* host_out, void* stream) {
    return denoise_host(ctx, host_frames, batch, h, w, host_out, stream, true);
}

wskpn_status wskpn_denoise_host_async(wskpn_ctx* ctx, const wskpn_frame* host_frames, int batch, int h, int w,
                                      float* host_out, void* stream) {
    return denoise_host(ctx, host_frames, batch, h, w, host_out, stream, false);
}

wskpn_status wskpn_prep(const wskpn_frame* frames, int batch, int h, int w, float gamma, float depth_near,
                        float depth_far, float* x0_out, void* stream) {
    std::string err;
    if (!frames || !x0_out || batch < 1 || h < 1 || w < 1 || !(gamma > 0.f) || !(depth_far > depth_near)) {
        set_thread_error("wskpn_prep: invalid argument");
        return WSKPN_EINVAL;
    }
    std::vector<void*> o(batch);
    for (int b = 0; b < batch; ++b) o[b] = x0_out + (size_t)b * 10 * h * w;
    wskpn_status s =
        launch_prep(frames, batch, h, w, gamma, depth_near, depth_far, o.data(), 0, (cudaStream_t)stream, err);
    if (s) set_thread_error(err);
    return s;
}

wskpn_status wskpn_decode_fuse_fwd(const float* z, const float* radiance, const float* albedo, int batch, int h,
                                   int w, int M, const int* ksizes, float eps, float* out,
                                   unsigned int* fallbacks, void* stream) {
    if (!z || !radiance || !albedo || !out || !ksizes || batch < 1 || h < 1 || w < 1 || M < 1 ||
        M > WSKPN_MAX_KERNELS || !(eps > 0.f)) {
        set_thread_error("wskpn_decode_fuse_fwd: invalid argument");
        return WSKPN_EINVAL;
    }
    for (int i = 0; i < M; ++i)
        if (ksizes[i] < 1 || ksizes[i] > 13 || (ksizes[i] & 1) == 0) {
            set_thread_error("wskpn_decode_fuse_fwd: ksizes must be odd and in [1, 13]");
            return WSKPN_EINVAL;
        }
    const size_t HW = (size_t)h * w;
    std::vector<const float*> zz(batch), rr(batch), aa(batch);
    std::vector<float*> oo(batch);
    for (int b = 0; b < batch; ++b) {
        zz[b] = z + (size_t)b * 2 * M * HW;
        rr[b] = radiance + (size_t)b * 3 * HW;
        aa[b] = albedo + (size_t)b * 3 * HW;
        oo[b] = out + (size_t)b * 3 * HW;
    }
    std::string err;
    wskpn_status s = launch_decode_fuse_fwd(zz.data(), rr.data(), aa.data(), oo.data(), batch, h, w, M, ksizes,
                                            eps, fallbacks, (cudaStream_t)stream, err);
    if (s) set_thread_error(err);
    return s;
}

wskpn_status wskpn_numeric_fallbacks(wskpn_ctx* ctx, uint64_t* count) {
    if (!ctx || !count) return WSKPN_EINVAL;
    unsigned int v = 0;
    WSKPN_CUDA_TRY(cudaDeviceSynchronize(), ctx->err);
    WSKPN_CUDA_TRY(cudaMemcpy(&v, ctx->d_fallbacks, sizeof(v), cudaMemcpyDeviceToHost), ctx->err);
    *count = v;
    return WSKPN_OK;
}

wskpn_status wskpn_profile_enable(wskpn_ctx* ctx, int enable) {
    if (!ctx) return WSKPN_EINVAL;
    ctx->prof = enable != 0;
    return WSKPN_OK;
}

wskpn_status wskpn_profile_read(wskpn_ctx* ctx, float* ms, int cap, int* n_stages, int* calls) {
    if (!ctx || (!ms && cap > 0)) return WSKPN_EINVAL;
    const int n = ctx->cfg.n_layers + 2;
    std::vector<double> acc(n, 0.0);
    for (size_t k = 0; k < ctx->prof_used; ++k) {
        auto& ev = ctx->prof_sets[k];
        WSKPN_CUDA_TRY(cudaEventSynchronize(ev.back()), ctx->err);
        for (int i = 0; i < n; ++i) {
            float t = 0.f;
            WSKPN_CUDA_TRY(cudaEventElapsedTime(&t, ev[i], ev[i + 1]), ctx->err);
            acc[i] += t;
        }
    }
    for (int i = 0; i < n && i < cap; ++i) ms[i] = (float)acc[i];
    if (n_stages) *n_stages = n;
    if (calls) *calls = (int)ctx->prof_used;
    ctx->prof_used = 0;
    return WSKPN_OK;
}

wskpn_status wskpn_set_tuning(wskpn_ctx* ctx, int key, int value) {
    if (!ctx) return WSKPN_EINVAL;
    if (key == WSKPN_TUNE_TC_SPLIT && (value == 0 || value == 1)) {
        ctx->tc_split = value;
        return WSKPN_OK;
    }
    if (key == WSKPN_TUNE_TC_SPLIT_LAYERS && value >= 0) {
        ctx->tc_split_layers = (unsigned)value;
        return WSKPN_OK;
    }
    if (key == WSKPN_TUNE_TRAIN_RECOMPUTE && value >= 0 && value <= 2) {
        ctx->train_tc_recompute = value;
        return WSKPN_OK;
    }
    if (key == WSKPN_TUNE_HOST_BANDS && value >= 0 && value <= 64) {
        ctx->host_bands = value;
        return WSKPN_OK;
    }
    if (key == WSKPN_TUNE_HOST_FIRST_BAND && value >= 10 && value <= 100) {
        ctx->host_first_pct = value;
        return WSKPN_OK;
    }
    if (key == WSKPN_TUNE_HOST_LAST_BAND && value >= 10 && value <= 100) {
        ctx->host_last_pct = value;
        return WSKPN_OK;
    }
    if (key == WSKPN_TUNE_FP8_SPLIT && (value == 0 || value == 1) && ctx->cfg.prec == WSKPN_FP8) {
        if (value == ctx->fp8_split) return WSKPN_OK;
        WSKPN_CUDA_TRY(cudaDeviceSynchronize(), ctx->err);
        ctx->fp8_split = value;
        for (int l = 0; l < ctx->cfg.n_layers; ++l) {
            wskpn_status s = tc_alloc_layer(ctx, l);
            if (s) return s;
        }
        wskpn_status s = ctx_repack(ctx, 0);
        if (s) return s;
        WSKPN_CUDA_TRY(cudaDeviceSynchronize(), ctx->err);
        return WSKPN_OK;
    }
    if (key == WSKPN_TUNE_WAIT_LIMIT_US && value >= 0) {
        ctx->wait_ns = value == 0 ? 2000000000ull : (uint64_t)value * 1000ull;
        return WSKPN_OK;
    }
    if (key == WSKPN_TUNE_WAIT_PROBE && (value == 0 || value == 1) && ctx->cfg.prec != WSKPN_FP32) {
        ctx->wait_probe = value;
        return WSKPN_OK;
    }
    if (key == WSKPN_TUNE_TRAIN_KEEP && (value == 0 || value == 1)) {
        ctx->train_keep = value;
        return WSKPN_OK;
    }
    if (key == WSKPN_TUNE_FUSED_PREP && (value == 0 || value == 1)) {
        ctx->fused_prep = value;
        return WSKPN_OK;
    }
    ctx->err = "wskpn_set_tuning: unknown key or value";
    return WSKPN_EINVAL;
}

wskpn_status wskpn_device_status(wskpn_ctx* ctx, uint32_t* bits) {
    if (!ctx) return WSKPN_EINVAL;
    unsigned int v = 0;
    WSKPN_CUDA_TRY(cudaDeviceSynchronize(), ctx->err);
    WSKPN_CUDA_TRY(cudaMemcpy(&v, ctx->d_status, sizeof(v), cudaMemcpyDeviceToHost), ctx->err);
    WSKPN_CUDA_TRY(cudaMemset(ctx->d_status, 0, sizeof(v)), ctx->err);
    if (bits) *bits = v;
    if (v) {
        ctx->err = "a bounded wait in the tensor-core convolution expired (status " + std::to_string(v) + ")";
        return WSKPN_ETIMEOUT;
    }
    return WSKPN_OK;
}

}  // extern "C"
