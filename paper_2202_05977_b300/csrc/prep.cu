// Input assembly (Sec. 5.1): the ImportanceNet's 10 input channels are the
// gamma tone-mapped LDR radiance clamp(r,0,1)^(1/gamma), the albedo, the
// normal linearly scaled from [-1,1] to [0,1] and the depth linearly scaled
// from [near,far] to [0,1].
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "common.cuh"
#include "prep.cuh"
#include "quant.cuh"

namespace wskpn {

struct PrepArgs {
    FrameBatch f;
    PtrBatch<void*> out;
    int H, W;
    float inv_gamma, dnear, dscale;  // dscale = 1 / (far - near)
    float qscale;                    // e4m3 layout: 1 / activation scale
};

// The 10 input channels of pixel g of frame b (prep.cuh).
template <bool FAST = false>
__device__ __forceinline__ void prep_pixel(const PrepArgs& a, int b, size_t g, size_t HW, float* v) {
    float raw[10];
    prep_load_raw(a.f.r.p[b], a.f.a.p[b], a.f.n.p[b], a.f.d.p[b], g, HW, raw);
    prep_from_raw<FAST>(raw, PrepConst{a.inv_gamma, a.dnear, a.dscale}, v);
}

// Planar FP32 output [10][H][W] (the FP32 path's layout).
__global__ void prep_planar_kernel(PrepArgs a) {
    const int b = blockIdx.y;
    const size_t HW = (size_t)a.H * a.W;
    float* out = static_cast<float*>(a.out.p[b]);
    for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < HW; g += (size_t)gridDim.x * blockDim.x) {
        float v[10];
        prep_pixel(a, b, g, HW, v);
#pragma unroll
        for (int c = 0; c < 10; ++c) out[c * HW + g] = v[c];
    }
}

// Channels-last BF16 output [H][W][16] (channels 10..15 zero): the tensor
// core path's layout, one 32-byte row per pixel.
__global__ void prep_nhwc16_bf16_kernel(PrepArgs a) {
    const int b = blockIdx.y;
    const size_t HW = (size_t)a.H * a.W;
    uint4* out = static_cast<uint4*>(a.out.p[b]);
    for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < HW; g += (size_t)gridDim.x * blockDim.x) {
        float v[10];
        prep_pixel<true>(a, b, g, HW, v);
        __nv_bfloat162 h[8];
#pragma unroll
        for (int j = 0; j < 5; ++j) h[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
#pragma unroll
        for (int j = 5; j < 8; ++j) h[j] = __floats2bfloat162_rn(0.f, 0.f);
        const uint4* hv = reinterpret_cast<const uint4*>(h);
        out[2 * g] = hv[0];
        out[2 * g + 1] = hv[1];
    }
}

// Channels-last BF16 hi/lo output [H][W][32]: channels 0..15 = bf16(v),
// 16..31 = bf16(v - bf16(v)) (the split-BF16 activation format).
__global__ void prep_nhwc16_bf16x2_kernel(PrepArgs a) {
    const int b = blockIdx.y;
    const size_t HW = (size_t)a.H * a.W;
    uint4* out = static_cast<uint4*>(a.out.p[b]);
    for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < HW; g += (size_t)gridDim.x * blockDim.x) {
        float v[16];
        prep_pixel<true>(a, b, g, HW, v);
#pragma unroll
        for (int j = 10; j < 16; ++j) v[j] = 0.f;
        uint4 q[4];
        bf16_hilo16(v, q);
        out[4 * g] = q[0];
        out[4 * g + 1] = q[1];
        out[4 * g + 2] = q[2];
        out[4 * g + 3] = q[3];
    }
}

// Channels-last e4m3 output [H][W][32] (channels 10..31 zero), values
// divided by the layer-0 activation scale (FP8 tensor-core path).
__global__ void prep_nhwc32_fp8_kernel(PrepArgs a) {
    const int b = blockIdx.y;
    const size_t HW = (size_t)a.H * a.W;
    uint4* out = static_cast<uint4*>(a.out.p[b]);
    for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < HW; g += (size_t)gridDim.x * blockDim.x) {
        float v[16];
        prep_pixel<true>(a, b, g, HW, v);
#pragma unroll
        for (int j = 10; j < 16; ++j) v[j] = 0.f;
        uint32_t wds[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const __nv_fp8x2_storage_t lo =
                __nv_cvt_float2_to_fp8x2(make_float2(v[4 * j] * a.qscale, v[4 * j + 1] * a.qscale), __NV_SATFINITE, __NV_E4M3);
            const __nv_fp8x2_storage_t hi = __nv_cvt_float2_to_fp8x2(
                make_float2(v[4 * j + 2] * a.qscale, v[4 * j + 3] * a.qscale), __NV_SATFINITE, __NV_E4M3);
            wds[j] = (uint32_t)lo | ((uint32_t)hi << 16);
        }
        out[2 * g] = make_uint4(wds[0], wds[1], wds[2], wds[3]);
        out[2 * g + 1] = make_uint4(0u, 0u, 0u, 0u);
    }
}

// Channels-last e4m3 hi/lo pairs of the values divided by the layer-0
// activation scale (the FP8 hi/lo tensor-core path): per pixel
// [hi(16) | hi(16) again | lo(16) | 0 (16)], the 10 channels (6 zeros after
// them) being the first layer's trailing half chunk.
__global__ void prep_nhwc32_fp8x2_kernel(PrepArgs a) {
    const int b = blockIdx.y;
    const size_t HW = (size_t)a.H * a.W;
    uint4* out = static_cast<uint4*>(a.out.p[b]);
    for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < HW; g += (size_t)gridDim.x * blockDim.x) {
        float v[16];
        prep_pixel<true>(a, b, g, HW, v);
#pragma unroll
        for (int j = 10; j < 16; ++j) v[j] = 0.f;
        uint4 hi, lo;
        fp8_pack16(v, a.qscale, hi, &lo);
        const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
        out[4 * g] = hi;
        out[4 * g + 1] = hi;
        out[4 * g + 2] = lo;
        out[4 * g + 3] = zero;
    }
}

static thread_local float g_prep_qscale = 1.f;

wskpn_status launch_prep(const wskpn_frame* frames, int B, int H, int W, float gamma, float dnear,
                         float dfar, void* const* out, int layout, cudaStream_t st, std::string& err) {
    for (int b0 = 0; b0 < B; b0 += WSKPN_MAX_BATCH) {
        const int nb = B - b0 < WSKPN_MAX_BATCH ? B - b0 : WSKPN_MAX_BATCH;
        PrepArgs a{};
        for (int j = 0; j < nb; ++j) {
            a.f.r.p[j] = frames[b0 + j].radiance;
            a.f.a.p[j] = frames[b0 + j].albedo;
            a.f.n.p[j] = frames[b0 + j].normal;
            a.f.d.p[j] = frames[b0 + j].depth;
            a.out.p[j] = out[b0 + j];
        }
        a.H = H;
        a.W = W;
        a.inv_gamma = (float)(1.0 / (double)gamma);
        a.dnear = dnear;
        a.dscale = (float)(1.0 / ((double)dfar - (double)dnear));
        a.qscale = g_prep_qscale;
        const size_t HW = (size_t)H * W;
        int blocks = (int)((HW + 255) / 256);
        if (blocks > 148 * 8) blocks = 148 * 8;
        dim3 grid(blocks, nb);
        if (layout == 0)
            prep_planar_kernel<<<grid, 256, 0, st>>>(a);
        else if (layout == 1)
            prep_nhwc16_bf16_kernel<<<grid, 256, 0, st>>>(a);
        else if (layout == 2)
            prep_nhwc16_bf16x2_kernel<<<grid, 256, 0, st>>>(a);
        else if (layout == 3)
            prep_nhwc32_fp8_kernel<<<grid, 256, 0, st>>>(a);
        else
            prep_nhwc32_fp8x2_kernel<<<grid, 256, 0, st>>>(a);
        WSKPN_CUDA_TRY(cudaGetLastError(), err);
    }
    return WSKPN_OK;
}

// layout 3: e4m3 NHWC32 with values / act_scale; layout 4 (hilo): e4m3 hi/lo pairs
wskpn_status launch_prep_fp8(const wskpn_frame* frames, int B, int H, int W, float gamma, float dnear, float dfar,
                             void* const* out, float act_scale, int hilo, cudaStream_t st, std::string& err) {
    g_prep_qscale = 1.f / act_scale;
    const wskpn_status s = launch_prep(frames, B, H, W, gamma, dnear, dfar, out, hilo ? 4 : 3, st, err);
    g_prep_qscale = 1.f;
    return s;
}

}  // namespace wskpn
