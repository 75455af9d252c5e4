// RepVGG re-parameterisation (Sec. 4.1): the training-time block's 5x5, 3x3
// and 1x1 conv branches (+ identity when Cin == Cout) are linear, so they
// fold into one 5x5 conv: kernels zero-padded to 5x5 and summed, biases
// summed.  The gradient of the fold maps dL/dW back to the branches.
#include "common.cuh"

namespace wskpn {

__global__ void repvgg_fold_kernel(const float* __restrict__ w5, const float* __restrict__ b5,
                                   const float* __restrict__ w3, const float* __restrict__ b3,
                                   const float* __restrict__ w1, const float* __restrict__ b1, int cin, int cout,
                                   int identity, float* __restrict__ W, float* __restrict__ b) {
    const int n = cout * cin * 25;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int dx = i % 5, dy = (i / 5) % 5, c = (i / 25) % cin, o = i / (25 * cin);
        float v = w5[i];
        if (dy >= 1 && dy <= 3 && dx >= 1 && dx <= 3) v += w3[((o * cin + c) * 3 + (dy - 1)) * 3 + (dx - 1)];
        if (dy == 2 && dx == 2) {
            v += w1[o * cin + c];
            if (identity && o == c) v += 1.f;
        }
        W[i] = v;
    }
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < cout; o += gridDim.x * blockDim.x)
        b[o] = b5[o] + b3[o] + b1[o];
}

__global__ void repvgg_fold_grad_kernel(const float* __restrict__ gW, int cin, int cout, float* __restrict__ g5,
                                        float* __restrict__ g3, float* __restrict__ g1) {
    const int n = cout * cin * 25;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int dx = i % 5, dy = (i / 5) % 5, c = (i / 25) % cin, o = i / (25 * cin);
        const float g = gW[i];
        if (g5) g5[i] = g;
        if (g3 && dy >= 1 && dy <= 3 && dx >= 1 && dx <= 3) g3[((o * cin + c) * 3 + (dy - 1)) * 3 + (dx - 1)] = g;
        if (g1 && dy == 2 && dx == 2) g1[o * cin + c] = g;
    }
}

}  // namespace wskpn

using namespace wskpn;

extern "C" wskpn_status wskpn_repvgg_fold(const float* w5, const float* b5, const float* w3, const float* b3,
                                          const float* w1, const float* b1, int cin, int cout, int identity,
                                          float* w_out, float* b_out, void* stream) {
    if (!w5 || !b5 || !w3 || !b3 || !w1 || !b1 || !w_out || !b_out || cin < 1 || cout < 1 ||
        (identity && cin != cout)) {
        set_thread_error("wskpn_repvgg_fold: invalid argument (identity needs cin == cout)");
        return WSKPN_EINVAL;
    }
    repvgg_fold_kernel<<<64, 256, 0, (cudaStream_t)stream>>>(w5, b5, w3, b3, w1, b1, cin, cout, identity, w_out,
                                                              b_out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_thread_error(std::string("wskpn_repvgg_fold: ") + cudaGetErrorString(e));
        return WSKPN_ECUDA;
    }
    return WSKPN_OK;
}

extern "C" wskpn_status wskpn_repvgg_fold_grad(const float* gW, int cin, int cout, float* g5, float* g3, float* g1,
                                               void* stream) {
    if (!gW || cin < 1 || cout < 1) {
        set_thread_error("wskpn_repvgg_fold_grad: invalid argument");
        return WSKPN_EINVAL;
    }
    repvgg_fold_grad_kernel<<<64, 256, 0, (cudaStream_t)stream>>>(gW, cin, cout, g5, g3, g1);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_thread_error(std::string("wskpn_repvgg_fold_grad: ") + cudaGetErrorString(e));
        return WSKPN_ECUDA;
    }
    return WSKPN_OK;
}
