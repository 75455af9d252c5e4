/*
 * wskpn — weight-sharing kernel-prediction Monte Carlo denoiser on one
 * NVIDIA B300 (sm_103a).  C ABI of libwskpn.so.
 *
 * The method (Fan, Wang, Huo, Bao, "Real-time Monte Carlo Denoising with
 * Weight Sharing Kernel Prediction Network", EGSR 2021):
 *   Sec. 5.1  input assembly: gamma tone-mapped radiance, albedo, normal and
 *             depth scaled to [0,1] -> 10 channels;
 *   Sec. 4.1  ImportanceNet: KSxKS conv blocks with ReLU, then an output conv
 *             giving M importance maps I_i (Eq. 2) and M fusion logits;
 *   Eq. 3-4   per-pixel kernels w_p(q) = softmax over the k_i x k_i window
 *             Omega_p of I_i(q), applied to all colour channels;
 *   Eq. 5     fusion of the M filtered images with per-pixel softmax weights
 *             alpha_i; the filter runs on irradiance r / (a + eps) and the
 *             result is multiplied back by (a + eps) (Sec. 4.2).
 *
 * Conventions for every entry point below:
 *   - Images are float32, planar [C][H][W] (x fastest), in DEVICE memory
 *     unless a parameter says "host".  A batch of B frames of one size is
 *     either B separate wskpn_frame pointer sets or one contiguous
 *     [B][C][H][W] tensor, as stated per call.
 *   - The caller owns every buffer it passes; the library never frees or
 *     retains caller pointers beyond the call (asynchronous calls read them
 *     until the enqueued work completes on `stream`).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Compute calls are asynchronous: they enqueue kernels and
 *     return; the caller synchronises the stream before reading results.
 *   - A context belongs to the CUDA device that was current at
 *     wskpn_create; call it with that device current.
 *   - Every call returns a wskpn_status and never aborts or traps.  On
 *     failure wskpn_last_error() describes the cause; nothing is enqueued
 *     when argument validation fails.
 *   - All floating-point work of the denoiser runs in CUDA kernels of this
 *     library; there is no CPU fallback.
 */
#ifndef WSKPN_H
#define WSKPN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    WSKPN_OK = 0,
    WSKPN_EINVAL = 1,       /* bad argument (null pointer, size, config) */
    WSKPN_ENOMEM = 2,       /* device or host allocation failed */
    WSKPN_ECUDA = 3,        /* a CUDA runtime/driver call failed */
    WSKPN_EUNSUPPORTED = 4, /* valid request the library has no kernel for */
    WSKPN_EBUSY = 5,        /* serving: admission refused, queue full */
    WSKPN_ETIMEOUT = 6,     /* a bounded wait ran out */
    WSKPN_ENUMERIC = 7      /* non-finite values detected */
} wskpn_status;

typedef enum {
    WSKPN_FP32 = 0, /* convolutions in FP32 FFMA (SIMT) */
    WSKPN_BF16 = 1, /* convolutions on tcgen05 tensor cores, BF16 in, FP32 accumulate */
    WSKPN_FP8 = 2   /* convolutions on tcgen05, e4m3 operands (as hi/lo pairs by default, see
                       WSKPN_TUNE_FP8_SPLIT), FP32 accumulate, per-channel weight scales */
} wskpn_precision;

#define WSKPN_MAX_LAYERS 8
#define WSKPN_MAX_KERNELS 8
#define WSKPN_MAX_BATCH 16

/* Network and runtime configuration (Sec. 4.1, Sec. 5.3).
 * widths[0] must be 10 (the Sec. 5.1 input channels) and widths[n_layers]
 * must be 2 * n_kernels; every conv layer but the last has a ReLU.
 * ksizes are odd filtering window sizes (paper: k_b = 3, k_s = 2, M = 6 ->
 * 3,5,...,13).  max_batch/max_h/max_w size the context's workspaces. */
typedef struct {
    int n_layers;
    int widths[WSKPN_MAX_LAYERS + 1];
    int conv_ks;        /* 3 or 5 */
    int n_kernels;      /* M */
    int ksizes[WSKPN_MAX_KERNELS];
    wskpn_precision prec;
    float albedo_eps;   /* eps in y = r / (a + eps) */
    float gamma;        /* tone-map exponent 1/gamma */
    float depth_near, depth_far;
    int max_batch, max_h, max_w;
} wskpn_config;

/* One frame's input buffers, float32 planar: radiance [3][H][W],
 * albedo [3][H][W], normal [3][H][W], depth [1][H][W]. */
typedef struct {
    const float* radiance;
    const float* albedo;
    const float* normal;
    const float* depth;
} wskpn_frame;

typedef struct wskpn_ctx wskpn_ctx;

/* Library version string (static storage). */
const char* wskpn_version(void);

/* Fills *cfg with the paper's 3-block configuration (widths 10-32-48-64-12,
 * 5x5 convs, M = 6 sizes 3..13, eps 1e-2, gamma 2.2, depth range [1, 10],
 * BF16, max 1 x 1080 x 1920).  Returns WSKPN_EINVAL if cfg is NULL. */
wskpn_status wskpn_config_default(wskpn_config* cfg);

/* Number of float32 values in the weight blob for cfg: per layer
 * W[Cout][Cin][KS][KS] followed by b[Cout], layers in order.  0 if cfg is
 * invalid. */
size_t wskpn_n_weights(const wskpn_config* cfg);

/* Creates a context on the current CUDA device: validates cfg, copies the
 * host weight blob (n_weights floats, layout as wskpn_n_weights), packs it
 * for the configured precision and allocates workspaces for
 * max_batch x max_h x max_w.  *out receives the context (NULL on failure).
 * Errors: EINVAL (cfg/weights), ENOMEM, ECUDA, EUNSUPPORTED. */
wskpn_status wskpn_create(const wskpn_config* cfg, const float* host_weights, size_t n_weights,
                          wskpn_ctx** out);

/* Frees the context and all its device memory (synchronises its device).
 * NULL is ignored. */
void wskpn_destroy(wskpn_ctx* ctx);

/* Last error message of ctx (or of the calling thread when ctx is NULL). */
const char* wskpn_last_error(const wskpn_ctx* ctx);

/* Replaces the weights from a host blob (same layout as wskpn_create) or a
 * device blob; re-packs them for the configured precision, stream-ordered.
 * The FP8 activation scales are kept. */
wskpn_status wskpn_set_weights(wskpn_ctx* ctx, const float* weights, size_t n, int on_device,
                               void* stream);

/* Copies the context's FP32 master weights to a device buffer of
 * wskpn_n_weights floats (stream-ordered). */
wskpn_status wskpn_get_weights(wskpn_ctx* ctx, float* dev_out, size_t n, void* stream);

/* D_Theta(r, f): denoises `batch` frames of size h x w (Eq. 1-5).
 * frames: host array of `batch` wskpn_frame (device pointers).
 * out:    device float32 [batch][3][h][w].
 * Errors: EINVAL (null pointers, batch < 1 or > max_batch, h or w < 1 or
 * beyond max_h/max_w), ECUDA. */
wskpn_status wskpn_denoise(wskpn_ctx* ctx, const wskpn_frame* frames, int batch, int h, int w,
                           float* out, void* stream);

/* wskpn_denoise from HOST buffers, synchronous: copies each frame's inputs
 * (host float32 planar, pinned memory recommended) into context-owned
 * device staging buffers, denoises, copies the result to host_out
 * ([batch][3][h][w] float32) and waits before returning.  Frames of 432
 * rows or more are processed as horizontal bands of about 160 rows (at
 * most 12; WSKPN_TUNE_HOST_BANDS), each with the receptive-field halo
 * (conv_ks / 2 rows per layer plus the largest window's half) recomputed:
 * three context-owned band buffers rotate so that a band uploads while
 * earlier bands compute (on `stream` and, when two band workspaces fit, a
 * second context-owned stream) and download; each input row crosses the
 * host link once (the halo rows a band shares with the previous one are
 * copied on the device).  The result equals wskpn_denoise up to the
 * reconstruction's per-tile exponent shift (float32 rounding).  Staging
 * (52 bytes per pixel of max_batch x max_h x max_w for unbanded calls, 13
 * floats per pixel of an extended band per buffer for banded ones) is
 * allocated on first use.  Errors as wskpn_denoise, plus ENOMEM. */
wskpn_status wskpn_denoise_host(wskpn_ctx* ctx, const wskpn_frame* host_frames, int batch, int h,
                                int w, float* host_out, void* stream);

/* wskpn_denoise_host without the final wait: queues the same copies and
 * kernels and returns; `stream` is ordered after the last copy into
 * host_out, so the result may be read once `stream` has reached that point
 * (cudaStreamSynchronize, or an event recorded on it after the call).  The
 * host input and output buffers must stay valid and unmodified until then.
 * Successive calls on one context overlap: a call's uploads wait only for
 * the band buffers they reuse, so the next frame's first bands cross the
 * host link while the previous frame's last bands compute and download.
 * Calls of one context are issued from one thread, on one stream.  Errors
 * as wskpn_denoise_host (argument errors before anything is queued). */
wskpn_status wskpn_denoise_host_async(wskpn_ctx* ctx, const wskpn_frame* host_frames, int batch, int h,
                                      int w, float* host_out, void* stream);

/* ImportanceNet only (Sec. 5.1 + Sec. 4.1): writes the network output
 * z [batch][2M][h][w] (channels 0..M-1 importance maps for ksizes[0..M-1],
 * M..2M-1 fusion logits) to device memory.  Errors as wskpn_denoise. */
wskpn_status wskpn_logits(wskpn_ctx* ctx, const wskpn_frame* frames, int batch, int h, int w,
                          float* z_out, void* stream);

/* Sec. 5.1 input assembly alone: x0 [batch][10][h][w] float32 planar:
 * clamp(r,0,1)^(1/gamma), albedo, 0.5 n + 0.5, (d - near)/(far - near). */
wskpn_status wskpn_prep(const wskpn_frame* frames, int batch, int h, int w, float gamma,
                        float depth_near, float depth_far, float* x0_out, void* stream);

/* Reconstruction (Eq. 3-5 with Sec. 4.2 demodulation), stateless:
 *   z        device [batch][2M][h][w]: importance maps then fusion logits;
 *   radiance device [batch][3][h][w]; albedo device [batch][3][h][w];
 *   ksizes   host array of M odd sizes (1..13), M in 1..8;
 *   out      device [batch][3][h][w];
 *   fallbacks optional device uint32 counter, incremented once per
 *            (pixel, size) whose window sum needed the per-window-max path.
 * Windows are clipped to the image.  Errors: EINVAL, ECUDA. */
wskpn_status wskpn_decode_fuse_fwd(const float* z, const float* radiance, const float* albedo,
                                   int batch, int h, int w, int M, const int* ksizes, float eps,
                                   float* out, unsigned int* fallbacks, void* stream);

/* FP8 contexts: sets the static per-layer activation scales.  Runs the
 * FP32 network on the given frames (device, as wskpn_denoise), takes the
 * maximum of each layer's input over all pixels and channels, and sets
 * scale_l = margin * max_l / 448 (the largest finite e4m3 value), so that
 * x / scale_l is stored in e4m3 with satfinite.  Weights carry their own
 * per-output-channel scales (max |W[o]| / 448).  margin >= 1.  Must be
 * called before the first denoise of an FP8 context (which otherwise
 * returns EUNSUPPORTED); allocates and frees temporary device buffers;
 * synchronises `stream`.  batch <= 16.  Errors: EINVAL (not FP8, bad
 * arguments), ENOMEM, ECUDA. */
wskpn_status wskpn_calibrate(wskpn_ctx* ctx, const wskpn_frame* frames, int batch, int h, int w,
                             float margin, void* stream);

/* ---- Differentiation (one training step of Eq. 1) ------------------ */

/* Floats of scratch that wskpn_decode_fuse_bwd needs: (2M + 3) x batch x h
 * x w (0 for invalid sizes). */
size_t wskpn_decode_fuse_bwd_scratch_floats(int batch, int h, int w, int M);

/* Backward of wskpn_decode_fuse_fwd (chain rule through Eq. 3-5):
 *   dout     device [batch][3][h][w], dL/d(out);
 *   dz       device [batch][2M][h][w] output: dL/dz (importance maps, then
 *            fusion logits);
 *   scratch  device buffer of wskpn_decode_fuse_bwd_scratch_floats floats,
 *            owned by the caller and overwritten;
 * other arguments as wskpn_decode_fuse_fwd.  Errors: EINVAL, ECUDA. */
wskpn_status wskpn_decode_fuse_bwd(const float* z, const float* radiance, const float* albedo,
                                   const float* dout, int batch, int h, int w, int M,
                                   const int* ksizes, float eps, float* dz, float* scratch,
                                   unsigned int* fallbacks, void* stream);

/* Forward pass for training: out [batch][3][h][w] as wskpn_denoise, and the
 * network output z_saved [batch][2M][h][w] (device, caller-owned) that
 * wskpn_backward needs.  With WSKPN_TUNE_TRAIN_KEEP = 1 (BF16 context on
 * the tensor-core training path, batch <= 16) the layer inputs are written
 * to the context's training workspace (allocated by the first training
 * call) and kept for a wskpn_backward over the same frame buffers
 * (pointers), batch and size; the values are those of wskpn_logits, and the
 * frame buffers must not change in between.  Otherwise (default) no
 * activation is kept. */
wskpn_status wskpn_forward_train(wskpn_ctx* ctx, const wskpn_frame* frames, int batch, int h, int w,
                                 float* out, float* z_saved, void* stream);

/* Backward pass: from dout = dL/d(out) [batch][3][h][w] and z_saved,
 * writes dL/dweights (device, wskpn_n_weights floats, blob layout) and,
 * if dz_out is not NULL, dL/dz [batch][2M][h][w].  The activations are
 * those kept by wskpn_forward_train (see there), else recomputed from the
 * frames.  BF16 context (default WSKPN_TUNE_TRAIN_RECOMPUTE = 1): kept or
 * recomputed with the context's own tensor-core convolutions; the input
 * gradient of each layer is a tensor-core convolution of the gradient
 * (carried between layers as BF16) with the transposed, flipped BF16
 * weights, the weight
 * gradient a tensor-core GEMM over the pixels (BF16 operands), both with
 * FP32 accumulation and a fixed summation order (the result does not
 * depend on scheduling).  FP32 and FP8 contexts, and the other tuning
 * values: FP32 recompute and FP32 gradient kernels.  The ReLU derivative
 * at 0 is 0.  The first training call on a context allocates its training
 * workspaces (of the order of 1.5 KB per pixel of max_batch x max_h x
 * max_w).  batch <= 16.  Errors: EINVAL, ENOMEM, ECUDA. */
wskpn_status wskpn_backward(wskpn_ctx* ctx, const wskpn_frame* frames, int batch, int h, int w,
                            const float* z_saved, const float* dout, float* dz_out, float* dweights,
                            void* stream);

/* L1 loss over n elements: *loss (device float) = sum |out - target| / n,
 * and, if dout is not NULL, dout = sign(out - target) / n (sign(0) = 0).
 * Deterministic (fixed-order reduction).  Errors: EINVAL, ENOMEM, ECUDA. */
wskpn_status wskpn_l1_loss(wskpn_ctx* ctx, const float* out, const float* target, size_t n,
                           float* loss, float* dout, void* stream);

/* One Adam step (Kingma & Ba; the optimiser of Sec. 5.3) on the context's
 * FP32 master weights with gradient dweights (device, wskpn_n_weights
 * floats); step counts from 1 and drives the bias correction; the moments
 * live in the context (zero at the first call).  Re-packs the weights for
 * the configured precision.  Errors: EINVAL, ENOMEM, ECUDA. */
wskpn_status wskpn_adam_step(wskpn_ctx* ctx, const float* dweights, float lr, float beta1,
                             float beta2, float eps, int step, void* stream);

/* ---- RepVGG re-parameterisation (Sec. 4.1) -------------------------- */

/* Folds one training-time block (5x5, 3x3 and 1x1 conv branches, plus the
 * identity when `identity` is set, which needs cin == cout) into the single
 * 5x5 conv used at inference: W = w5 + pad(w3) + pad(w1) (+ centre 1 on the
 * diagonal), b = b5 + b3 + b1.  Device float32, layouts [cout][cin][k][k]
 * and [cout]; w_out [cout][cin][5][5], b_out [cout].  Errors: EINVAL, ECUDA. */
wskpn_status wskpn_repvgg_fold(const float* w5, const float* b5, const float* w3, const float* b3,
                               const float* w1, const float* b1, int cin, int cout, int identity,
                               float* w_out, float* b_out, void* stream);

/* Gradient of the fold: from dL/dW [cout][cin][5][5] writes dL/dw5 (same
 * shape), dL/dw3 [cout][cin][3][3] and dL/dw1 [cout][cin][1][1] (any may be
 * NULL); every branch bias receives dL/db unchanged.  Errors: EINVAL, ECUDA. */
wskpn_status wskpn_repvgg_fold_grad(const float* gW, int cin, int cout, float* g5, float* g3, float* g1,
                                    void* stream);

/* ---- Temporal accumulation before denoising (Sec. 4.3) -------------- */

/* Per pixel p, the previous frame's accumulated radiance is reprojected to
 * q = p + motion(p) (bilinear over the 4 pixels around q, pixel centres at
 * integer coordinates); a tap is kept when it lies in the image, has
 * history, |P_prev - P|^2 < tau_pos^2 and n_prev . n > tau_normal.  With
 * kept weight W > min_weight: A_prev and the history length are the
 * renormalised kept averages, h = h_prev + 1, alpha = max(1/h, alpha_min),
 * A = A_prev + alpha (c - A_prev); otherwise A = c, h = 1.  The paper gives
 * the steps, not the constants; the defaults are readings. */
typedef struct wskpn_temporal wskpn_temporal;

typedef struct {
    float alpha_min;   /* blend floor; 1/alpha_min frames of running mean (0.2) */
    float tau_pos;     /* world-position distance threshold (0.1) */
    float tau_normal;  /* minimum dot product of the shading normals (0.9) */
    float min_weight;  /* minimum kept bilinear weight (1e-3) */
} wskpn_temporal_config;

void wskpn_temporal_config_default(wskpn_temporal_config* cfg);

/* History of one stream of h x w frames, owned by the library (two device
 * copies of 10 float planes: accumulated radiance, world position, normal,
 * history length), starting empty.  cfg may be NULL (defaults).
 * Errors: EINVAL (size, config), ENOMEM, ECUDA. */
wskpn_status wskpn_temporal_create(const wskpn_temporal_config* cfg, int h, int w, wskpn_temporal** out);

/* One frame: device float32 planar radiance [3][h][w], world position
 * [3][h][w], shading normal [3][h][w] and motion [2][h][w] ((x, y) offset
 * from each pixel to its position in the previous frame); writes the
 * accumulated radiance [3][h][w] (caller-owned, may not alias the inputs)
 * and advances the history.  Calls on one object must be ordered on the
 * GPU (same stream, or synchronised).  Errors: EINVAL, ECUDA. */
wskpn_status wskpn_temporal_step(wskpn_temporal* t, const float* radiance, const float* position,
                                 const float* normal, const float* motion, float* accumulated, void* stream);

/* Copies the current history length plane [h][w] (0 = none) to `history`
 * (device).  Errors: EINVAL, ECUDA. */
wskpn_status wskpn_temporal_history(const wskpn_temporal* t, float* history, void* stream);

/* Forgets the history (the next step restarts every pixel).  Errors: EINVAL, ECUDA. */
wskpn_status wskpn_temporal_reset(wskpn_temporal* t, void* stream);

void wskpn_temporal_destroy(wskpn_temporal* t);

/* ---- Multi-resolution variant (Sec. 5.3 "Implementation", Eq. 7) ----- */

/* The paper's network for high-spp input: a U-Net of 3x3 convolutions
 * predicts, at full, half and quarter resolution, importance maps for
 * kernel sizes 3 and 5, their fusion logits and (full and half) a blending
 * logit; each level filters the demodulated irradiance averaged down to its
 * resolution (Eq. 3-5), and the levels combine from the coarsest as
 * o = i^f - alpha U D i^f + alpha U o^c (Eq. 7, D = 2x2 box average,
 * U = nearest upsampling, alpha = sigmoid of the blending logit); the
 * output is (a + eps) o.  Layers (weight-blob order, each W[cout][cin][3][3]
 * then b[cout]): 10-32, 32-32, 32-48, 48-48, 48-64, 64-64, head 64-4,
 * 112-48 (upsampled 64 + skip 48), head 48-5, 80-32 (upsampled 48 + skip
 * 32), head 32-5.  The architecture is a reading: the paper defers it to a
 * supplement.  The decode, Eq. 7 and re-modulation are FP32 in every mode. */
typedef struct wskpn_mr wskpn_mr;

typedef struct {
    int max_h, max_w;                /* largest frame (workspaces sized for it) */
    float albedo_eps, gamma, depth_near, depth_far;  /* as wskpn_config */
    wskpn_precision prec;            /* WSKPN_FP32 (SIMT convolutions) or WSKPN_BF16
                                        (tcgen05, hi/lo activations); default FP32 */
} wskpn_mr_config;

void wskpn_mr_config_default(wskpn_mr_config* cfg);
size_t wskpn_mr_n_weights(void);

/* Copies the FP32 weights (wskpn_mr_n_weights() floats, host) to the device
 * and allocates the workspaces.  cfg may be NULL (defaults: 1080 x 1920).
 * Errors: EINVAL, ENOMEM, ECUDA. */
wskpn_status wskpn_mr_create(const wskpn_mr_config* cfg, const float* host_weights, size_t n, wskpn_mr** out);

/* Denoises one frame (device planar float32 buffers as wskpn_denoise) into
 * out [3][h][w] (device).  Calls on one object must not overlap on the GPU.
 * Errors: EINVAL (size beyond the config, NULL pointers), ECUDA. */
wskpn_status wskpn_mr_denoise(wskpn_mr* m, const wskpn_frame* frame, int h, int w, float* out, void* stream);

/* The U-Net outputs of one frame: z0 [5][h][w], z1 [5][h1][w1],
 * z2 [4][h2][w2] (h1 = ceil(h/2), h2 = ceil(h1/2), same for w); device. */
wskpn_status wskpn_mr_logits(wskpn_mr* m, const wskpn_frame* frame, int h, int w, float* z0, float* z1, float* z2,
                             void* stream);

const char* wskpn_mr_last_error(const wskpn_mr* m);
void wskpn_mr_destroy(wskpn_mr* m);

/* ---- Serving: continuous batching of frame-denoise requests --------- */

typedef struct wskpn_server wskpn_server;

typedef struct {
    int n_workers;        /* GPU batches in flight at once, one CUDA stream and
                             one context each (default 4) */
    int max_batch;        /* frames of one size per batch (default 4, <= 16) */
    int max_queue;        /* queued requests beyond which submit returns
                             EBUSY (default 8192) */
    size_t mem_budget;    /* bytes of device memory that admitted requests may
                             occupy at once (their footprint: workspace and
                             staging per pixel); 0 = 8 GiB */
    int use_graphs;       /* 1 = replay one captured CUDA graph per
                             (worker, h, w, batch) (default 1) */
    int batch_window_us;  /* how long the oldest request may wait for
                             companions of its size (default 200) */
    wskpn_temporal_config temporal;  /* constants of the per-stream temporal
                             accumulation (wskpn_serve_submit_temporal);
                             default wskpn_temporal_config_default */
} wskpn_serve_config;

typedef struct {
    uint64_t submitted, completed, rejected, failed;
    uint64_t batches, graph_launches, graph_captures;
    double p50_ms, p99_ms, mean_ms, max_ms;  /* submit -> delivery latency */
    double fps;                              /* completed / (last delivery - first submit) */
    double mean_batch;
    size_t mem_in_use, mem_peak;             /* admitted footprint, bytes */
    uint64_t temporal_frames;                /* frames accumulated with their stream's history */
    uint64_t temporal_streams;               /* streams holding a temporal history */
    size_t temporal_bytes;                   /* device bytes of those histories */
} wskpn_serve_stats;

/* Fills the defaults above. */
wskpn_status wskpn_serve_config_default(wskpn_serve_config* scfg);

/* Starts a server: cfg/weights as wskpn_create (cfg's max_h/max_w bound
 * the request sizes; its max_batch is replaced by scfg->max_batch), one
 * context, CUDA stream and staging slots per worker on the current device,
 * and a scheduler thread.  Requests of equal size are batched; requests
 * that arrive while others run are admitted as workers and memory budget
 * free up, and their batches run concurrently on the workers' streams.
 * Errors: EINVAL, ENOMEM, ECUDA. */
wskpn_status wskpn_serve_start(const wskpn_config* cfg, const float* host_weights, size_t n_weights,
                               const wskpn_serve_config* scfg, wskpn_server** out);

/* Queues one frame (device pointers, planar float32) of size h x w for
 * stream `stream_id` (any integer naming a client stream); the result is
 * written to `out` (device [3][h][w]).  The caller keeps the frame and out
 * buffers alive and unmodified until the ticket is delivered.  Results are
 * delivered in submission order per stream.  Errors: EINVAL (size beyond
 * the server's limits, NULL pointers), EBUSY (queue full or the request's
 * footprint alone exceeds the budget). */
wskpn_status wskpn_serve_submit(wskpn_server* srv, int stream_id, const wskpn_frame* frame, int h, int w,
                                float* out, uint64_t* ticket);

/* As wskpn_serve_submit, with temporal accumulation (Sec. 4.3) before the
 * denoise: the frame's radiance is blended with the reprojected history of
 * stream `stream_id` (kept by the server on the device, created on the
 * stream's first temporal frame and restarted when its size changes or
 * reset_history is set).  position [3][h][w] is the world position of each
 * pixel, motion [2][h][w] its (x, y) offset to the previous frame; the
 * constants are scfg->temporal.  Frames of one temporal stream run one at a
 * time in submission order; frames of different streams batch together.
 * Errors: as wskpn_serve_submit. */
wskpn_status wskpn_serve_submit_temporal(wskpn_server* srv, int stream_id, const wskpn_frame* frame,
                                         const float* position, const float* motion, int reset_history, int h,
                                         int w, float* out, uint64_t* ticket);

/* Waits up to timeout_ms (0 = poll, < 0 = no limit) for a ticket.  Returns
 * OK when delivered, ETIMEOUT when the limit ran out, EINVAL for an unknown
 * ticket, or the request's own failure status. */
wskpn_status wskpn_serve_wait(wskpn_server* srv, uint64_t ticket, int timeout_ms);

/* Timeline of one delivered request, in milliseconds of the host's
 * steady clock since wskpn_serve_start: when it was submitted, when its
 * batch was handed to a worker (dispatch_ms; -1 if it never ran), and when
 * the scheduler saw that batch complete (done_ms, polled every ~20 us);
 * the worker index, the frames in its batch and its size. */
typedef struct {
    int h, w, worker, batch;
    double submit_ms, dispatch_ms, done_ms;
} wskpn_serve_ticket_info;

/* As wskpn_serve_wait; on delivery also fills *info (NULL is ignored). */
wskpn_status wskpn_serve_wait_info(wskpn_server* srv, uint64_t ticket, int timeout_ms,
                                   wskpn_serve_ticket_info* info);

/* Pauses (1) or resumes (0) admission of queued requests (batches already
 * on the GPU finish).  Used to drain or to build a queue deterministically. */
wskpn_status wskpn_serve_pause(wskpn_server* srv, int paused);

/* Snapshot of the counters and latency percentiles so far. */
wskpn_status wskpn_serve_stats_get(wskpn_server* srv, wskpn_serve_stats* st);

/* Finishes queued and running work, stops the scheduler and frees the
 * server.  NULL is ignored. */
void wskpn_serve_stop(wskpn_server* srv);

/* Numeric fallback counter of ctx (pixels x sizes that took the slow exact
 * softmax path since creation); synchronises the context's device. */
wskpn_status wskpn_numeric_fallbacks(wskpn_ctx* ctx, uint64_t* count);

/* Per-stage device timing (the paper reports prediction and reconstruction
 * time separately, Sec. 6.2, Table "time").  While enabled, every
 * wskpn_denoise / wskpn_logits call records CUDA events on its own stream
 * at each stage boundary.  Stages: 0 = input assembly (Sec. 5.1),
 * 1..n_layers = conv layers (Sec. 4.1), n_layers + 1 = reconstruction
 * (Eq. 3-5).  Errors: EINVAL (ctx NULL). */
wskpn_status wskpn_profile_enable(wskpn_ctx* ctx, int enable);

/* Waits for every call recorded since the last read, writes the summed
 * milliseconds of each stage to ms[0 .. min(cap, n_layers + 2) - 1], the
 * stage count (n_layers + 2) to *n_stages and the number of recorded calls
 * to *calls, then clears the record.  Stages a call did not run add 0. */
wskpn_status wskpn_profile_read(wskpn_ctx* ctx, float* ms, int cap, int* n_stages, int* calls);

/* Tuning knobs (for tests and benchmarks).
 *   WSKPN_TUNE_TC_SPLIT (BF16 only): 1 = store every BF16 activation as a
 *     hi/lo pair (x = hi + lo, both BF16) and run the K loop over both
 *     halves against the same BF16 weights, which removes the activation
 *     rounding error at twice the MMA work (default); 0 = one BF16 value.
 *   WSKPN_TUNE_TC_SPLIT_LAYERS (BF16 only, with TC_SPLIT = 1): bit l set =
 *     the input of layer l is stored as a hi/lo pair, clear = as one BF16
 *     value (half the MMA work of that layer, its input rounded to BF16);
 *     default all bits set.  The training backward on the tensor cores
 *     needs every bit set (otherwise it recomputes in FP32).
 *   WSKPN_TUNE_TRAIN_RECOMPUTE (BF16 only): how wskpn_backward recomputes
 *     the activations and forms the input gradients: 1 = activations with
 *     the context's own tensor-core convolutions, as the forward computed
 *     them, and each layer's input gradient as a tensor-core convolution of
 *     the gradient (BF16 values) with the transposed, flipped BF16
 *     weights (default; needs TC_SPLIT = 1); 2 = the same activations, input
 *     gradients in FP32 SIMT with the FP32 weights; 0 = everything in FP32
 *     with the FP32 weights (the ReLU masks are then those of the FP32
 *     network, which brings the gradient closer to the FP32/FP64 one).
 *     Weight gradients: tensor-core GEMMs over the pixels in mode 1, FP32
 *     SIMT in modes 0 and 2.
 *   WSKPN_TUNE_FP8_SPLIT (FP8 only): 1 = every e4m3 activation and weight
 *     is a hi/lo pair in one scale (x / s = hi + lo, lo = e4m3 of the
 *     residual) and each convolution sums A_hi W_hi + A_lo W_hi + A_hi W_lo,
 *     three e4m3 products (default: the e4m3 rounding of the single term,
 *     about 6 % per operand, compounds through the layers and the exp of
 *     Eq. 3); 0 = one e4m3 value per operand.  Changing it re-packs the
 *     weights (synchronises the device).
 *   WSKPN_TUNE_HOST_BANDS: bands of the wskpn_denoise_host pipeline; 0 =
 *     automatic (one per ~160 rows, at most 12, none below 432 rows), 1 =
 *     no banding, n = n bands.
 *   WSKPN_TUNE_HOST_FIRST_BAND, WSKPN_TUNE_HOST_LAST_BAND: height of the
 *     pipeline's first / last band in % of the others (10 .. 100; defaults
 *     100 and 100).
 *   WSKPN_TUNE_WAIT_LIMIT_US: limit, in microseconds, of every shared-memory
 *     barrier wait of the context's tensor-core convolutions (0 = the
 *     default, 2 s).  An expired wait sets a bit of the device status word
 *     (wskpn_device_status) and the kernel winds down: every role stops,
 *     waits (for at most 2 s, whatever this limit) for the copies and MMAs
 *     it has issued, and the CTA frees its tensor memory and returns; the
 *     launch's output is then invalid.
 *   WSKPN_TUNE_WAIT_PROBE (BF16 / FP8 only): test hook for that path.  1 =
 *     in the next tensor-core convolution launch of the context (one launch;
 *     the key then reads 0 again), each epilogue warp first waits on a
 *     barrier that nothing signals, so that its wait limit expires.
 *   WSKPN_TUNE_TRAIN_KEEP (BF16 only, with TRAIN_RECOMPUTE = 1): 0 = the
 *     backward recomputes the layer inputs (default); 1 = wskpn_forward_train
 *     keeps them for the backward (see there), at 4 bytes per channel of
 *     every layer input per pixel (0.64 GB for 16 crops of 256 x 256).
 *   WSKPN_TUNE_FUSED_PREP (BF16 / FP8 inference): 1 = the first
 *     convolution assembles its own input tiles from the FP32 frame buffers
 *     (the Sec. 5.1 tone map and scalings, split into BF16 or e4m3 hi/lo
 *     pairs, written to shared memory by four extra warps of that kernel)
 *     and the assembled input is never stored (default; applies when the
 *     first layer's input is a hi/lo pair and a kernel is built for its
 *     shape, 10 -> 32); 0 = a separate assembly kernel stores the input in
 *     HBM and the first convolution reads it back.  Both give the same bits.
 * Errors: EINVAL for an unknown key or value. */
#define WSKPN_TUNE_TC_SPLIT 2
#define WSKPN_TUNE_TRAIN_RECOMPUTE 3
#define WSKPN_TUNE_FP8_SPLIT 4
#define WSKPN_TUNE_HOST_BANDS 5
#define WSKPN_TUNE_HOST_FIRST_BAND 6
#define WSKPN_TUNE_HOST_LAST_BAND 7
#define WSKPN_TUNE_TC_SPLIT_LAYERS 8
#define WSKPN_TUNE_WAIT_LIMIT_US 9
#define WSKPN_TUNE_WAIT_PROBE 10
#define WSKPN_TUNE_TRAIN_KEEP 11
#define WSKPN_TUNE_FUSED_PREP 12
wskpn_status wskpn_set_tuning(wskpn_ctx* ctx, int key, int value);

/* Reads and clears the context's device status word after synchronising
 * the device.  Bits 0..2: a bounded wait inside the tensor-core convolution
 * expired in its TMA, MMA or epilogue role (the kernel gave up instead of
 * hanging; its output is invalid).  Returns WSKPN_ETIMEOUT when any bit
 * was set, WSKPN_OK otherwise. */
wskpn_status wskpn_device_status(wskpn_ctx* ctx, uint32_t* bits);

/* Allocation-free FP32 denoise (the paper has no counterpart: this is a
 * deployment feature).  For callers that may not allocate device memory,
 * for example code running inside another runtime's memory pool, a host
 * callback, or a plug-in that must not grow its process's device
 * footprint.  It runs the same kernels as wskpn_denoise with prec = FP32,
 * but needs no context: every intermediate (packed weights, activations,
 * network output) lives in one static device array of 64 MiB that each GPU
 * loading this library holds until the process exits.  No cudaMalloc,
 * cudaFree or allocating library call is made.
 *   cfg      configuration as for wskpn_create, validated the same way
 *            (max_batch/max_h/max_w must hold valid values although they
 *            do not limit this call); prec must be WSKPN_FP32 (else
 *            EUNSUPPORTED);
 *   weights  DEVICE float32 blob in the wskpn_create layout;
 *   frames   host array of `batch` wskpn_frame (device pointers);
 *   out      device float32 [batch][3][h][w].
 * Limit: the whole call must fit the 64 MiB array (packed weights plus
 * (max even-layer width + max odd-layer width + 2M) floats per pixel of
 * batch x h x w; at the default widths about 134,000 pixels, e.g. one
 * 512 x 256 frame); larger requests return EINVAL with the size needed.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current.  With lazy module
 * loading (the CUDA default) that lookup is also when the driver loads the
 * module and commits the 64 MiB on that device, so the first call can fail
 * with ECUDA (out of memory) where memory is short: make it at start-up,
 * before any stream capture.  The address is cached per device for the
 * life of the process; cudaDeviceReset invalidates it and is not supported
 * between calls.  All calls share the array and it keeps the
 * last call's contents: calls whose work overlaps on the GPU (different
 * streams or devices' threads racing on one device) corrupt each other, so
 * serialise them.  Asynchronous on `stream` like wskpn_denoise. */
wskpn_status wskpn_denoise_static(const wskpn_config* cfg, const float* weights,
                                  const wskpn_frame* frames, int batch, int h, int w, float* out,
                                  void* stream);

#ifdef __cplusplus
}
#endif

#endif /* WSKPN_H */
