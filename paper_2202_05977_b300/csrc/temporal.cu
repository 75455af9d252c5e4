// Temporal accumulation before denoising (Sec. 4.3): the previous frame's
// accumulated radiance is reprojected with the motion vectors (bilinear, 4
// taps), each tap is kept only if its world position and shading normal
// agree with the current pixel, and the current 1-spp radiance is blended
// with the renormalised kept history; a pixel without consistent history
// restarts from its 1-spp value.
//
// Per pixel p = (x, y), with q = p + m(p), x0 = floor(q):
//   kept taps t in {(0,0),(1,0),(0,1),(1,1)}: inside, h_prev > 0,
//     |P_prev - P|^2 < tau_pos^2, n_prev . n > tau_normal
//   W = sum of kept bilinear weights; if W > min_weight:
//     A_prev = sum w A_prev / W,  h = sum w h_prev / W + 1,
//     alpha = max(1 / h, alpha_min),  A = A_prev + alpha (c - A_prev)
//   else A = c, h = 1.
// Every quantity a branch depends on (q, floor(q), the tap weights, W and the
// two consistency measures) is computed with one rounding per operation in a
// fixed order (no contraction into fused multiply-adds), so the decisions are
// reproducible bit for bit by any float32 implementation of the same order.
//
// State per stream: planes [A0 A1 A2 | P0 P1 P2 | n0 n1 n2 | h] of H x W
// floats, two copies (read previous, write current), swapped every step.
// One thread per pixel; all accesses of a warp are to consecutive pixels
// except the 4 gathered taps, which hit the same few cache lines.
#include "ctx.h"

namespace wskpn {

struct TemporalArgs {
    PtrBatch<const float*> c, P, n, m;   // current frame: radiance, position, normal (3 planes), motion (2)
    PtrBatch<const float*> prev;         // previous state (10 planes)
    PtrBatch<float*> next;               // new state (10 planes)
    PtrBatch<float*> out;                // accumulated radiance (3 planes)
    int H, W;
    float alpha_min, tau_pos2, tau_normal, min_weight;
};

__global__ void __launch_bounds__(256) temporal_kernel(TemporalArgs a) {
    const int b = blockIdx.y;
    const int H = a.H, W = a.W;
    const size_t HW = (size_t)H * W;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= HW) return;
    const int x = (int)(i % W), y = (int)(i / W);
    const float* __restrict__ c = a.c.p[b];
    const float* __restrict__ P = a.P.p[b];
    const float* __restrict__ n = a.n.p[b];
    const float* __restrict__ m = a.m.p[b];
    const float* __restrict__ prev = a.prev.p[b];
    float* __restrict__ next = a.next.p[b];
    float* __restrict__ out = a.out.p[b];

    float cv[3], Pv[3], nv[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        cv[k] = c[k * HW + i];
        Pv[k] = P[k * HW + i];
        nv[k] = n[k * HW + i];
    }
    const float qx = __fadd_rn((float)x, m[i]);
    const float qy = __fadd_rn((float)y, m[HW + i]);
    const float flx = floorf(qx), fly = floorf(qy);
    const float fx = __fsub_rn(qx, flx), fy = __fsub_rn(qy, fly);
    const float ax = __fsub_rn(1.f, fx), ay = __fsub_rn(1.f, fy);
    const float wt[4] = {__fmul_rn(ax, ay), __fmul_rn(fx, ay), __fmul_rn(ax, fy), __fmul_rn(fx, fy)};
    // integer corner; q far outside the image gives taps that fail the inside test
    const int x0 = (int)fmaxf(fminf(flx, (float)W + 1.f), -2.f);
    const int y0 = (int)fmaxf(fminf(fly, (float)H + 1.f), -2.f);

    float Wsum = 0.f, Aacc[3] = {0.f, 0.f, 0.f}, hacc = 0.f;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int tx = x0 + (t & 1), ty = y0 + (t >> 1);
        if (tx < 0 || tx >= W || ty < 0 || ty >= H) continue;
        const size_t g = (size_t)ty * W + tx;
        const float hp = prev[9 * HW + g];
        if (!(hp > 0.f)) continue;
        const float d0 = __fsub_rn(prev[3 * HW + g], Pv[0]);
        const float d1 = __fsub_rn(prev[4 * HW + g], Pv[1]);
        const float d2 = __fsub_rn(prev[5 * HW + g], Pv[2]);
        const float dist2 = __fadd_rn(__fadd_rn(__fmul_rn(d0, d0), __fmul_rn(d1, d1)), __fmul_rn(d2, d2));
        const float dot = __fadd_rn(__fadd_rn(__fmul_rn(prev[6 * HW + g], nv[0]), __fmul_rn(prev[7 * HW + g], nv[1])),
                                    __fmul_rn(prev[8 * HW + g], nv[2]));
        if (!(dist2 < a.tau_pos2) || !(dot > a.tau_normal)) continue;
        const float w = wt[t];
        Wsum = __fadd_rn(Wsum, w);
#pragma unroll
        for (int k = 0; k < 3; ++k) Aacc[k] = fmaf(w, prev[k * HW + g], Aacc[k]);
        hacc = fmaf(w, hp, hacc);
    }
    float A[3], h;
    if (Wsum > a.min_weight) {
        const float inv = 1.f / Wsum;
        h = hacc * inv + 1.f;
        const float alpha = fmaxf(1.f / h, a.alpha_min);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float Ap = Aacc[k] * inv;
            A[k] = fmaf(alpha, cv[k] - Ap, Ap);
        }
    } else {
        h = 1.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) A[k] = cv[k];
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        next[k * HW + i] = A[k];
        next[(3 + k) * HW + i] = Pv[k];
        next[(6 + k) * HW + i] = nv[k];
        out[k * HW + i] = A[k];
    }
    next[9 * HW + i] = h;
}

}  // namespace wskpn

using namespace wskpn;

namespace wskpn {
bool temporal_config_valid(const wskpn_temporal_config& c) {
    return c.alpha_min > 0.f && c.alpha_min <= 1.f && c.tau_pos >= 0.f && c.tau_normal >= -1.f &&
           c.min_weight >= 0.f && c.min_weight < 1.f;
}
}  // namespace wskpn

extern "C" void wskpn_temporal_config_default(wskpn_temporal_config* cfg) {
    if (!cfg) return;
    cfg->alpha_min = 0.2f;
    cfg->tau_pos = 0.1f;
    cfg->tau_normal = 0.9f;
    cfg->min_weight = 1e-3f;
}

extern "C" wskpn_status wskpn_temporal_create(const wskpn_temporal_config* cfg, int h, int w,
                                              wskpn_temporal** out) {
    if (!out || h < 1 || w < 1 || (size_t)h * w > ((size_t)1 << 31)) {
        set_thread_error("wskpn_temporal_create: invalid size or NULL output");
        return WSKPN_EINVAL;
    }
    *out = nullptr;
    wskpn_temporal_config c;
    wskpn_temporal_config_default(&c);
    if (cfg) c = *cfg;
    if (!temporal_config_valid(c)) {
        set_thread_error("wskpn_temporal_create: alpha_min in (0,1], tau_pos >= 0, tau_normal >= -1, "
                         "min_weight in [0,1)");
        return WSKPN_EINVAL;
    }
    auto* t = new (std::nothrow) wskpn_temporal;
    if (!t) return WSKPN_ENOMEM;
    t->cfg = c;
    t->h = h;
    t->w = w;
    const size_t bytes = (size_t)TEMPORAL_PLANES * h * w * sizeof(float);
    for (int k = 0; k < 2; ++k) {
        if (cudaMalloc(&t->state[k], bytes) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(t->state[0]);
            delete t;
            set_thread_error("wskpn_temporal_create: device allocation failed");
            return WSKPN_ENOMEM;
        }
    }
    // no history yet: h = 0 everywhere (all planes zero)
    if (cudaMemset(t->state[0], 0, bytes) != cudaSuccess || cudaMemset(t->state[1], 0, bytes) != cudaSuccess) {
        cudaFree(t->state[0]);
        cudaFree(t->state[1]);
        delete t;
        set_thread_error("wskpn_temporal_create: CUDA error");
        return WSKPN_ECUDA;
    }
    *out = t;
    return WSKPN_OK;
}

extern "C" void wskpn_temporal_destroy(wskpn_temporal* t) {
    if (!t) return;
    cudaFree(t->state[0]);
    cudaFree(t->state[1]);
    delete t;
}

extern "C" wskpn_status wskpn_temporal_reset(wskpn_temporal* t, void* stream) {
    if (!t) return WSKPN_EINVAL;
    const size_t bytes = (size_t)TEMPORAL_PLANES * t->h * t->w * sizeof(float);
    if (cudaMemsetAsync(t->state[t->cur], 0, bytes, (cudaStream_t)stream) != cudaSuccess) {
        set_thread_error("wskpn_temporal_reset: CUDA error");
        return WSKPN_ECUDA;
    }
    return WSKPN_OK;
}

namespace wskpn {
wskpn_status launch_temporal(const wskpn_temporal_config& cfg, const float* const* c, const float* const* P,
                             const float* const* n, const float* const* m, const float* const* prev,
                             float* const* next, float* const* out, int B, int H, int W, cudaStream_t st,
                             std::string& err) {
    for (int b0 = 0; b0 < B; b0 += WSKPN_MAX_BATCH) {
        const int nb = B - b0 < WSKPN_MAX_BATCH ? B - b0 : WSKPN_MAX_BATCH;
        TemporalArgs a{};
        for (int j = 0; j < nb; ++j) {
            a.c.p[j] = c[b0 + j];
            a.P.p[j] = P[b0 + j];
            a.n.p[j] = n[b0 + j];
            a.m.p[j] = m[b0 + j];
            a.prev.p[j] = prev[b0 + j];
            a.next.p[j] = next[b0 + j];
            a.out.p[j] = out[b0 + j];
        }
        a.H = H;
        a.W = W;
        a.alpha_min = cfg.alpha_min;
        a.tau_pos2 = cfg.tau_pos * cfg.tau_pos;  // one float32 rounding
        a.tau_normal = cfg.tau_normal;
        a.min_weight = cfg.min_weight;
        const size_t HW = (size_t)H * W;
        dim3 grid((unsigned)((HW + 255) / 256), nb);
        temporal_kernel<<<grid, 256, 0, st>>>(a);
        WSKPN_CUDA_TRY(cudaGetLastError(), err);
    }
    return WSKPN_OK;
}

wskpn_status temporal_step_into(wskpn_temporal* t, const float* radiance, const float* position,
                                const float* normal, const float* motion, float* out, cudaStream_t st,
                                std::string& err) {
    const float* prev = t->state[t->cur];
    float* next = t->state[t->cur ^ 1];
    wskpn_status s = launch_temporal(t->cfg, &radiance, &position, &normal, &motion, &prev, &next, &out, 1, t->h,
                                     t->w, st, err);
    if (!s) t->cur ^= 1;
    return s;
}
}  // namespace wskpn

extern "C" wskpn_status wskpn_temporal_step(wskpn_temporal* t, const float* radiance, const float* position,
                                            const float* normal, const float* motion, float* accumulated,
                                            void* stream) {
    if (!t || !radiance || !position || !normal || !motion || !accumulated) {
        set_thread_error("wskpn_temporal_step: NULL argument");
        return WSKPN_EINVAL;
    }
    std::string err;
    const wskpn_status s =
        temporal_step_into(t, radiance, position, normal, motion, accumulated, (cudaStream_t)stream, err);
    if (s) set_thread_error("wskpn_temporal_step: " + err);
    return s;
}

extern "C" wskpn_status wskpn_temporal_history(const wskpn_temporal* t, float* history, void* stream) {
    if (!t || !history) {
        set_thread_error("wskpn_temporal_history: NULL argument");
        return WSKPN_EINVAL;
    }
    const size_t HW = (size_t)t->h * t->w;
    if (cudaMemcpyAsync(history, t->state[t->cur] + 9 * HW, HW * sizeof(float), cudaMemcpyDeviceToDevice,
                        (cudaStream_t)stream) != cudaSuccess) {
        set_thread_error("wskpn_temporal_history: CUDA error");
        return WSKPN_ECUDA;
    }
    return WSKPN_OK;
}
