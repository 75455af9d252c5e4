// Input assembly of one pixel (Sec. 5.1) and its BF16 hi/lo storage form,
// shared by the input-assembly kernels and by the first tensor-core layer
// when it assembles its own input tiles: both paths run these same
// functions, so they store the same bits.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

namespace wskpn {

__device__ __forceinline__ float exp2f_fast(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Tone-map exponent and depth range of the assembly: LDR radiance
// clamp(r, 0, 1)^(1/gamma), depth (d - near) / (far - near).
struct PrepConst {
    float inv_gamma, dnear, dscale;  // dscale = 1 / (far - near)
};

// The 10 input channels from the raw values of one pixel, in the order
// radiance RGB, albedo RGB, normal XYZ, depth: tone-mapped radiance,
// albedo as is, the normal scaled from [-1, 1] to [0, 1], the depth from
// [near, far] to [0, 1].  FAST (layouts stored as BF16 or e4m3, whose
// rounding is 2^-9 or coarser): t^(1/gamma) as 2^(log2(t) / gamma) with the
// hardware's approximate log2 and exp2 (relative error near 2^-21 for t in
// (0, 1]; t = 0 gives 0); otherwise powf.
template <bool FAST>
__device__ __forceinline__ void prep_from_raw(const float (&raw)[10], const PrepConst& k, float* v) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float t = fminf(fmaxf(raw[c], 0.f), 1.f);
        v[c] = FAST ? exp2f_fast(__log2f(t) * k.inv_gamma) : powf(t, k.inv_gamma);
        v[3 + c] = raw[3 + c];
        v[6 + c] = 0.5f * raw[6 + c] + 0.5f;
    }
    v[9] = (raw[9] - k.dnear) * k.dscale;
}

// Raw values of pixel g of planar [C][HW] frame buffers.
__device__ __forceinline__ void prep_load_raw(const float* __restrict__ r, const float* __restrict__ al,
                                              const float* __restrict__ n, const float* __restrict__ d, size_t g,
                                              size_t HW, float (&raw)[10]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        raw[c] = __ldg(r + c * HW + g);
        raw[3 + c] = __ldg(al + c * HW + g);
        raw[6 + c] = __ldg(n + c * HW + g);
    }
    raw[9] = __ldg(d + g);
}

// The split-BF16 storage of 16 channels (10 assembled, 6 zero): q[0..1] =
// bf16(v) (channels 0-7, 8-15), q[2..3] = bf16(v - bf16(v)).
__device__ __forceinline__ void bf16_hilo16(const float (&v)[16], uint4 (&q)[4]) {
    __nv_bfloat162 h[8], l[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        h[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
        const float2 hf = __bfloat1622float2(h[j]);
        l[j] = __floats2bfloat162_rn(v[2 * j] - hf.x, v[2 * j + 1] - hf.y);
    }
    const uint4* hv = reinterpret_cast<const uint4*>(h);
    const uint4* lv = reinterpret_cast<const uint4*>(l);
    q[0] = hv[0];
    q[1] = hv[1];
    q[2] = lv[0];
    q[3] = lv[1];
}

}  // namespace wskpn
