// Activation quantisation helpers shared by the input assembly and the
// tensor-core epilogues (e4m3 storage formats).
#pragma once

#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <cstdint>

namespace wskpn {

// 16 values v * qs as e4m3 (satfinite), channel j in byte j; with lo, also
// the residuals v * qs - e4m3(v * qs) rounded to e4m3 (the lo half of an
// e4m3 hi/lo pair; the subtraction is exact in FP32).
__device__ __forceinline__ void fp8_pack16(const float (&v)[16], float qs, uint4& hi, uint4* lo) {
    uint32_t wh[4] = {0u, 0u, 0u, 0u}, wl[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float2 x = make_float2(v[2 * j] * qs, v[2 * j + 1] * qs);
        const __nv_fp8x2_storage_t h = __nv_cvt_float2_to_fp8x2(x, __NV_SATFINITE, __NV_E4M3);
        wh[j >> 1] |= (uint32_t)h << ((j & 1) * 16);
        if (lo) {
            const __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2(h, __NV_E4M3);
            const float2 hf = __half22float2(*reinterpret_cast<const __half2*>(&hr));
            const __nv_fp8x2_storage_t l =
                __nv_cvt_float2_to_fp8x2(make_float2(x.x - hf.x, x.y - hf.y), __NV_SATFINITE, __NV_E4M3);
            wl[j >> 1] |= (uint32_t)l << ((j & 1) * 16);
        }
    }
    hi = make_uint4(wh[0], wh[1], wh[2], wh[3]);
    if (lo) *lo = make_uint4(wl[0], wl[1], wl[2], wl[3]);
}

}  // namespace wskpn
