// Shared helpers of libwskpn (device + host).  No method arithmetic here.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>

#include "wskpn.h"

namespace wskpn {

// Per-launch table of per-frame pointers, passed by value as a kernel
// parameter (B <= WSKPN_MAX_BATCH frames of one size per launch).
template <typename T>
struct PtrBatch {
    T p[WSKPN_MAX_BATCH];
};

struct FrameBatch {
    PtrBatch<const float*> r, a, n, d;  // radiance, albedo, normal, depth
};

// Error state: per-thread message used when no context is at hand.
void set_thread_error(const std::string& msg);
const std::string& thread_error();

#define WSKPN_CUDA_TRY(expr, errstr)                                                     \
    do {                                                                                 \
        cudaError_t e__ = (expr);                                                        \
        if (e__ != cudaSuccess) {                                                        \
            errstr = std::string(#expr) + ": " + cudaGetErrorString(e__);                \
            return WSKPN_ECUDA;                                                          \
        }                                                                                \
    } while (0)

inline int cdiv(long a, long b) { return (int)((a + b - 1) / b); }

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace wskpn
