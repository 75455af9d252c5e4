// Context set-up and tear-down: master weights, per-precision packings and
// workspaces sized for max_batch x max_h x max_w.
#include <algorithm>

#include "ctx.h"

namespace wskpn {

int simt_coutp(int cout);

static wskpn_status dalloc(void** p, size_t bytes, std::string& err) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        err = std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e);
        *p = nullptr;
        return e == cudaErrorMemoryAllocation ? WSKPN_ENOMEM : WSKPN_ECUDA;
    }
    return WSKPN_OK;
}

wskpn_status ctx_init(wskpn_ctx* ctx, const float* host_weights) {
    const wskpn_config& c = ctx->cfg;
    WSKPN_CUDA_TRY(cudaGetDevice(&ctx->device), ctx->err);
    wskpn_status s = dalloc((void**)&ctx->d_master, ctx->nw * sizeof(float), ctx->err);
    if (s) return s;
    WSKPN_CUDA_TRY(cudaMemcpy(ctx->d_master, host_weights, ctx->nw * sizeof(float), cudaMemcpyHostToDevice),
                   ctx->err);
    size_t off = 0;
    for (int l = 0; l < c.n_layers; ++l) {
        Layer& L = ctx->layers[l];
        L.cin = c.widths[l];
        L.cout = c.widths[l + 1];
        L.woff = off;
        L.boff = off + (size_t)L.cout * L.cin * c.conv_ks * c.conv_ks;
        off = L.boff + L.cout;
        const int coutp = simt_coutp(L.cout);
        s = dalloc((void**)&L.w32, (size_t)L.cin * c.conv_ks * c.conv_ks * coutp * sizeof(float), ctx->err);
        if (s) return s;
        s = dalloc((void**)&L.b32, coutp * sizeof(float), ctx->err);
        if (s) return s;
        if (c.prec != WSKPN_FP32) {
            s = tc_alloc_layer(ctx, l);
            if (s) return s;
        }
    }
    ctx->ws_pixels = (size_t)c.max_batch * c.max_h * c.max_w;
    int wa = 0, wb = 0;
    for (int l = 0; l < c.n_layers; ++l) {
        if (l % 2 == 0) wa = std::max(wa, c.widths[l]);
        else wb = std::max(wb, c.widths[l]);
    }
    if (c.prec == WSKPN_FP32) {
        s = dalloc((void**)&ctx->d_actA, ctx->ws_pixels * wa * sizeof(float), ctx->err);
        if (s) return s;
        if (wb) {
            s = dalloc((void**)&ctx->d_actB, ctx->ws_pixels * wb * sizeof(float), ctx->err);
            if (s) return s;
        }
    } else {
        s = dalloc(&ctx->d_tcA, ctx->ws_pixels * tc_act_bytes_per_pixel(c, 0) + 256, ctx->err);
        if (s) return s;
        s = dalloc(&ctx->d_tcB, ctx->ws_pixels * tc_act_bytes_per_pixel(c, 1) + 256, ctx->err);
        if (s) return s;
    }
    s = dalloc((void**)&ctx->d_z, ctx->ws_pixels * c.widths[c.n_layers] * sizeof(float), ctx->err);
    if (s) return s;
    s = dalloc((void**)&ctx->d_fallbacks, 2 * sizeof(unsigned int), ctx->err);
    if (s) return s;
    ctx->d_status = ctx->d_fallbacks + 1;
    WSKPN_CUDA_TRY(cudaMemset(ctx->d_fallbacks, 0, 2 * sizeof(unsigned int)), ctx->err);
    s = ctx_repack(ctx, 0);
    if (s) return s;
    WSKPN_CUDA_TRY(cudaDeviceSynchronize(), ctx->err);
    return WSKPN_OK;
}

void ctx_free(wskpn_ctx* ctx) {
    cudaDeviceSynchronize();
    ctx_free_train(ctx);
    for (int l = 0; l < WSKPN_MAX_LAYERS; ++l) {
        Layer& L = ctx->layers[l];
        cudaFree(L.w32);
        cudaFree(L.b32);
        cudaFree(L.wtc);
        cudaFree(L.ep_scale);
        cudaFree(L.ep_bias);
        cudaFree(L.wscale);
    }
    cudaFree(ctx->d_master);
    cudaFree(ctx->d_actA);
    cudaFree(ctx->d_actB);
    cudaFree(ctx->d_tcA);
    cudaFree(ctx->d_tcB);
    cudaFree(ctx->d_z);
    cudaFree(ctx->d_stage);
    for (float* p : ctx->d_band) cudaFree(p);
    for (cudaEvent_t e : ctx->band_events) cudaEventDestroy(e);
    if (ctx->up_stream) cudaStreamDestroy(ctx->up_stream);
    if (ctx->down_stream) cudaStreamDestroy(ctx->down_stream);
    if (ctx->band_stream) cudaStreamDestroy(ctx->band_stream);
    if (ctx->halo_stream) cudaStreamDestroy(ctx->halo_stream);
    cudaFree(ctx->d_fallbacks);
    for (auto& set : ctx->prof_sets)
        for (auto e : set) cudaEventDestroy(e);
}

}  // namespace wskpn
