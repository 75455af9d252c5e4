// Internal definition of the opaque wskpn_ctx and the helpers shared by the
// library's translation units.
#pragma once

#include <string>
#include <vector>

#include "common.cuh"

struct wskpn_ctx;

namespace wskpn {

struct Layer {
    int cin, cout;
    size_t woff, boff;  // offsets of W and b in the FP32 master blob
    // FP32 SIMT packing
    float* w32 = nullptr;  // [Cin][KS*KS][COUTP]
    float* b32 = nullptr;  // [COUTP]
    // tensor-core packing (BF16 / FP8): the exact shared-memory image of the
    // layer's B operand, plus per-output-channel epilogue scale and bias
    void* wtc = nullptr;
    size_t wtc_bytes = 0;
    float* ep_scale = nullptr;  // [cout_p]  (FP8: act_scale_in * w_scale[o]; BF16: 1)
    float* ep_bias = nullptr;   // [cout_p]
    float* wscale = nullptr;    // [cout_p]  FP8 per-output-channel weight scale
    int cin_p = 0, cout_p = 0;  // padded channel counts of the tensor-core layout
    int groups = 1;             // output-channel groups run as separate passes (weights too large for one)
    int xfold = 0;              // image packed for folded horizontal taps (BF16 last layer, 16 outputs)
    int xf_cr = 0;              // folded: output channels per tap block (12 or 16)
};

std::string validate_config(const wskpn_config* c);
size_t n_weights_of(const wskpn_config* c);

}  // namespace wskpn

struct wskpn_ctx {
    wskpn_config cfg{};
    int device = 0;
    std::string err;
    size_t nw = 0;
    float* d_master = nullptr;  // FP32 weight blob
    wskpn::Layer layers[WSKPN_MAX_LAYERS];
    size_t ws_pixels = 0;       // max_batch * max_h * max_w
    float* d_actA = nullptr;    // FP32 planar ping buffer
    float* d_actB = nullptr;    // FP32 planar pong buffer
    void* d_tcA = nullptr;      // tensor-core NHWC ping buffer
    void* d_tcB = nullptr;      // tensor-core NHWC pong buffer
    float* d_z = nullptr;       // network output [B][2M][H][W]
    float* d_stage = nullptr;   // host-call staging: 10 input + 3 output planes per pixel
    // banded host calls: two copy streams (upload, download) and the staging
    // of two bands in flight
    cudaStream_t up_stream = nullptr, down_stream = nullptr;
    cudaStream_t band_stream = nullptr;  // second compute stream of the host-buffer pipeline
    cudaStream_t halo_stream = nullptr;  // device copies of the halo rows bands share
    static constexpr int BAND_SLOTS = 3;       // band buffers of the host pipeline
    float* d_band[BAND_SLOTS] = {};            // [10 + 3][band_rows][max_w] each
    size_t band_floats = 0;
    std::vector<cudaEvent_t> band_events;   // per band slot: uploaded, computed, downloaded, halo copied;
                                            // then the call's start and end
    uint64_t band_job = 0;                  // bands issued so far (slot = job % BAND_SLOTS, across calls)
    int band_ext = -1, band_w = -1;         // band buffer layout of the last call (extended rows, width)
    unsigned int* d_fallbacks = nullptr;
    unsigned int* d_status = nullptr;  // device status word of the tensor-core kernels
    float act_scale[WSKPN_MAX_LAYERS + 1] = {};  // FP8 per-layer activation scales
    bool fp8_calibrated = false;
    int tc_split = 1;  // BF16 activations as hi/lo pairs (WSKPN_TUNE_TC_SPLIT)
    uint64_t wait_ns = 2000000000ull;  // limit of the convolutions' barrier waits (WSKPN_TUNE_WAIT_LIMIT_US)
    int wait_probe = 0;                 // test hook for the next convolution launch (WSKPN_TUNE_WAIT_PROBE)
    unsigned tc_split_layers = 0xFFFFFFFFu;  // of those, the layer inputs split (bit l; WSKPN_TUNE_TC_SPLIT_LAYERS)
    int fp8_split = 1;  // e4m3 activations and weights as hi/lo pairs (WSKPN_TUNE_FP8_SPLIT)
    bool simt_stale = true;      // FP32 SIMT weight images older than the master weights
    int train_keep = 0;          // wskpn_forward_train keeps the layer inputs for the backward (WSKPN_TUNE_TRAIN_KEEP)
    int fused_prep = 1;          // BF16 inference: the first layer assembles its input (WSKPN_TUNE_FUSED_PREP)
    int train_tc_recompute = 1;  // backward on the tensor cores: 1 recompute + input gradients, 2 recompute only (WSKPN_TUNE_TRAIN_RECOMPUTE)
    int host_bands = 0;         // bands of the host-buffer pipeline, 0 = automatic (WSKPN_TUNE_HOST_BANDS)
    int host_first_pct = 100;   // first band's height in % of the others (WSKPN_TUNE_HOST_FIRST_BAND)
    int host_last_pct = 100;    // last band's height in % of the others (WSKPN_TUNE_HOST_LAST_BAND)
    void* train = nullptr;  // training workspaces (train.cu), allocated by the first training call
    // stage profiling: one event set (n_layers + 3 events) per recorded call
    bool prof = false;
    std::vector<std::vector<cudaEvent_t>> prof_sets;
    size_t prof_used = 0;
    int prof_cur = -1;  // index of the set of the call in flight, -1 = none
};

namespace wskpn {
wskpn_status ctx_init(wskpn_ctx* ctx, const float* host_weights);
void ctx_free(wskpn_ctx* ctx);
void ctx_free_train(wskpn_ctx* ctx);
wskpn_status ctx_repack(wskpn_ctx* ctx, cudaStream_t st);
// Packs the FP32 SIMT weight images if the master weights changed since.
wskpn_status ctx_simt_weights(wskpn_ctx* ctx, cudaStream_t st);
// stage profiling hooks (no-ops unless profiling is enabled)
void prof_begin(wskpn_ctx* ctx, cudaStream_t st);
void prof_mark(wskpn_ctx* ctx, int boundary, cudaStream_t st);  // boundary 1..n_layers+2
void prof_end(wskpn_ctx* ctx);
wskpn_status ctx_logits(wskpn_ctx* ctx, const wskpn_frame* frames, int B, int H, int W, float* z,
                        cudaStream_t st);
// tensor-core path (conv_tc.cu)
size_t tc_act_bytes_per_pixel(const wskpn_config& c, int which /*0 = A, 1 = B*/);
wskpn_status tc_alloc_layer(wskpn_ctx* ctx, int l);
wskpn_status tc_pack_layer(wskpn_ctx* ctx, int l, cudaStream_t st);
// Argument checks shared by the calls that take frames (EINVAL with a message).
wskpn_status check_frames(wskpn_ctx* ctx, const wskpn_frame* frames, int batch, int h, int w);
// Layer l of the context's ImportanceNet on the tensor cores (BF16 / FP8
// activations in the context's layout; the last layer writes planar z).
wskpn_status tc_conv_layer(wskpn_ctx* ctx, int l, const void* in, void* out, int B, int H, int W, cudaStream_t st);
// Whether layer l (BF16, hi/lo input) has a kernel that also writes its
// output's ReLU bits (the training backward's input-gradient masks).
bool tc_relu_bits_supported(const wskpn_ctx* ctx, int l);
wskpn_status tc_logits(wskpn_ctx* ctx, const wskpn_frame* frames, int B, int H, int W, float* z,
                       cudaStream_t st);
wskpn_status tc_layer_alloc(Layer& L, int KS, bool fp8, bool fp8_lo, std::string& err);
// BF16: whether the input of layer l is stored as hi/lo pairs, and whether
// every layer input is (the training recompute needs all of them split).
int tc_split_of(const wskpn_ctx* ctx, int l);
bool tc_split_all(const wskpn_ctx* ctx);
bool tc_fused_prep_supported(const wskpn_ctx* ctx);
// x_0 .. x_{L-1} as NHWC hi/lo into xs[l]; with bits, also the positive-
// channel bits of x_1 .. x_{L-1} into (*bits)[l] (two words per pixel).
wskpn_status tc_recompute_nhwc(wskpn_ctx* ctx, const wskpn_frame* frames, int B, int H, int W,
                               const std::vector<void*>& xs, cudaStream_t st,
                               const std::vector<uint32_t*>* bits = nullptr);
wskpn_status tc_recompute_acts(wskpn_ctx* ctx, const wskpn_frame* frames, int B, int H, int W,
                               const std::vector<std::vector<float*>>& acts, cudaStream_t st);
// BF16 tensor-core layers outside a context (hi/lo activations in and out)
wskpn_status tc_layer_create(Layer& L, int KS, const float* w, const float* b, cudaStream_t st, std::string& err);
void tc_layer_free(Layer& L);
wskpn_status tc_dgrad_layer_alloc(Layer& Lt, int KS, int cin, int cout, std::string& err);
wskpn_status tc_dgrad_layer_pack(Layer& Lt, int KS, const float* w, float* wt, const float* zero_bias,
                                 cudaStream_t st, std::string& err);
wskpn_status tc_layer_run(const Layer& L, int KS, const void* in, void* out, int out_cp, int out_c0, int last,
                          int relu, int B, int H, int W, unsigned int* status, int device, cudaStream_t st,
                          std::string& err);
wskpn_status tc_layer_run_pin(const Layer& L, int KS, const wskpn_frame* frame, float gamma, float dnear, float dfar,
                              void* out, int out_cp, int relu, int H, int W, unsigned int* status, int device,
                              cudaStream_t st, std::string& err);
// The input gradient gx (NHWC BF16, Lt.cout_p channels) of a layer from its
// output gradient g (NHWC BF16) through Lt, times the ReLU derivative of the layer input
// (x_bits: its positive-channel bits, two words per pixel), with per-warp
// bias sums of the result in bias_part [*nparts][64] (channels of gx).
wskpn_status tc_dgrad_run(const Layer& Lt, int KS, const void* g, void* gx, const uint32_t* x_bits, float* bias_part,
                          int* nparts, int B, int H, int W, unsigned int* status, int device, cudaStream_t st,
                          std::string& err);
}  // namespace wskpn

// Temporal accumulation history of one stream (temporal.cu): planes
// [A0 A1 A2 | P0 P1 P2 | n0 n1 n2 | h] of H x W floats, two copies; state[cur]
// holds the latest frame's state.
struct wskpn_temporal {
    wskpn_temporal_config cfg;
    int h = 0, w = 0;
    float* state[2] = {nullptr, nullptr};
    int cur = 0;
};

namespace wskpn {
constexpr int TEMPORAL_PLANES = 10;
bool temporal_config_valid(const wskpn_temporal_config& c);
// Batched step: frame j reads prev[j] (10 planes) and writes next[j] and out[j] (3 planes).
wskpn_status launch_temporal(const wskpn_temporal_config& cfg, const float* const* c, const float* const* P,
                             const float* const* n, const float* const* m, const float* const* prev,
                             float* const* next, float* const* out, int B, int H, int W, cudaStream_t st,
                             std::string& err);
}  // namespace wskpn
