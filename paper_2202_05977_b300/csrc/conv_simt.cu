// FP32 plain path of the ImportanceNet convolutions (Sec. 4.1): one KSxKS
// conv (zero padding KS/2, cross-correlation) + bias (+ ReLU), true FP32 FFMA.
//
// Activations are planar [C][H][W] per frame.  A CTA computes a 32 x 8 pixel
// tile for all output channels: lane = x, each warp owns 4 rows and a
// quarter of the (padded) output channels, each thread 4 rows x CPT channels
// in registers.  Input channels are staged 8 at a time in shared memory
// ([c][TH+KS-1][TW+KS-1]) next to the matching weights ([c][tap][Cout],
// broadcast-read as float4).  Accumulation order per output is fixed
// (channel, then dx, then dy), so results do not depend on the launch.
#include "common.cuh"

namespace wskpn {

namespace cs {
constexpr int TW = 32, TH = 8, THREADS = 256, CC = 8;
}

struct ConvSimtArgs {
    PtrBatch<const float*> in;
    PtrBatch<float*> out;
    PtrBatch<const float*> mask;  // optional [Cout][H][W]: output zeroed where mask <= 0 (ReLU backward)
    const float* w;     // [Cin][KS*KS][COUTP]
    const float* bias;  // [COUTP]
    int H, W, Cin, Cout, relu, has_mask;
};

template <int KS, int CPT>
__global__ void __launch_bounds__(cs::THREADS, 2) conv_simt_kernel(ConvSimtArgs a) {
    constexpr int COUTP = 4 * CPT;
    constexpr int IW = cs::TW + KS - 1, IH = cs::TH + KS - 1;
    constexpr int PAD = KS / 2;
    extern __shared__ float4 smem4[];
    float* sIn = reinterpret_cast<float*>(smem4);             // [CC][IH][IW]
    float* sW = sIn + ((cs::CC * IH * IW + 3) / 4) * 4;        // [CC][KS*KS][COUTP]

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rg = warp & 1, cg = warp >> 1;
    const int b = blockIdx.z;
    const int H = a.H, W = a.W, Cin = a.Cin;
    const size_t HW = (size_t)H * W;
    const int x0 = blockIdx.x * cs::TW, y0 = blockIdx.y * cs::TH;
    const float* __restrict__ in = a.in.p[b];

    float acc[4][CPT];
#pragma unroll
    for (int j = 0; j < CPT; ++j) {
        const float bj = a.bias[cg * CPT + j];
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[r][j] = bj;
    }

    for (int c0 = 0; c0 < Cin; c0 += cs::CC) {
        const int cc = min(cs::CC, Cin - c0);
        __syncthreads();
        for (int i = tid; i < cc * IH * IW; i += cs::THREADS) {
            const int c = i / (IH * IW), rem = i % (IH * IW);
            const int iy = rem / IW, ix = rem % IW;
            const int gy = y0 + iy - PAD, gx = x0 + ix - PAD;
            const bool inb = gy >= 0 && gy < H && gx >= 0 && gx < W;
            sIn[i] = inb ? in[(size_t)(c0 + c) * HW + (size_t)gy * W + gx] : 0.f;
        }
        {
            const float4* src = reinterpret_cast<const float4*>(a.w + (size_t)c0 * KS * KS * COUTP);
            float4* dst = reinterpret_cast<float4*>(sW);
            for (int i = tid; i < cc * KS * KS * COUTP / 4; i += cs::THREADS) dst[i] = src[i];
        }
        __syncthreads();
        for (int c = 0; c < cc; ++c) {
            const float* si = sIn + c * IH * IW + (rg * 4) * IW + lane;
            const float* sw = sW + c * KS * KS * COUTP + cg * CPT;
#pragma unroll
            for (int dx = 0; dx < KS; ++dx) {
                float v[4 + KS - 1];
#pragma unroll
                for (int r = 0; r < 4 + KS - 1; ++r) v[r] = si[r * IW + dx];
#pragma unroll
                for (int dy = 0; dy < KS; ++dy) {
                    float wv[CPT];
                    const float4* w4 = reinterpret_cast<const float4*>(sw + (dy * KS + dx) * COUTP);
#pragma unroll
                    for (int j = 0; j < CPT / 4; ++j) {
                        const float4 t = w4[j];
                        wv[4 * j] = t.x;
                        wv[4 * j + 1] = t.y;
                        wv[4 * j + 2] = t.z;
                        wv[4 * j + 3] = t.w;
                    }
#pragma unroll
                    for (int r = 0; r < 4; ++r)
#pragma unroll
                        for (int j = 0; j < CPT; ++j) acc[r][j] = fmaf(v[r + dy], wv[j], acc[r][j]);
                }
            }
        }
    }

    float* __restrict__ out = a.out.p[b];
    const int gx = x0 + lane;
    if (gx >= W) return;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int gy = y0 + rg * 4 + r;
        if (gy >= H) continue;
#pragma unroll
        for (int j = 0; j < CPT; ++j) {
            const int o = cg * CPT + j;
            if (o < a.Cout) {
                float v = acc[r][j];
                if (a.relu) v = fmaxf(v, 0.f);
                const size_t g = (size_t)o * HW + (size_t)gy * W + gx;
                if (a.has_mask && !(a.mask.p[b][g] > 0.f)) v = 0.f;
                out[g] = v;
            }
        }
    }
}

template <int KS, int CPT>
static wskpn_status launch_simt_t(const ConvSimtArgs& a, int nb, cudaStream_t st, std::string& err) {
    constexpr int IW = cs::TW + KS - 1, IH = cs::TH + KS - 1;
    const size_t smem = (((cs::CC * IH * IW + 3) / 4) * 4 + cs::CC * KS * KS * 4 * CPT) * sizeof(float);
    WSKPN_CUDA_TRY(cudaFuncSetAttribute(conv_simt_kernel<KS, CPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem),
                   err);
    dim3 grid(cdiv(a.W, cs::TW), cdiv(a.H, cs::TH), nb);
    conv_simt_kernel<KS, CPT><<<grid, cs::THREADS, smem, st>>>(a);
    WSKPN_CUDA_TRY(cudaGetLastError(), err);
    return WSKPN_OK;
}

// Output channels padded to a multiple of 16 (4 channel groups x CPT, CPT % 4 == 0).
int simt_coutp(int cout) { return ((cout + 15) / 16) * 16; }

wskpn_status launch_conv_simt_masked(const float* const* in, float* const* out, const float* const* mask, int B,
                                     int H, int W, int Cin, int Cout, int KS, const float* w_packed,
                                     const float* bias_padded, int relu, cudaStream_t st, std::string& err) {
    const int cpt = simt_coutp(Cout) / 4;
    for (int b0 = 0; b0 < B; b0 += WSKPN_MAX_BATCH) {
        const int nb = B - b0 < WSKPN_MAX_BATCH ? B - b0 : WSKPN_MAX_BATCH;
        ConvSimtArgs a{};
        for (int j = 0; j < nb; ++j) {
            a.in.p[j] = in[b0 + j];
            a.out.p[j] = out[b0 + j];
            a.mask.p[j] = mask ? mask[b0 + j] : nullptr;
        }
        a.has_mask = mask != nullptr;
        a.w = w_packed;
        a.bias = bias_padded;
        a.H = H;
        a.W = W;
        a.Cin = Cin;
        a.Cout = Cout;
        a.relu = relu;
        wskpn_status s;
#define WSKPN_SIMT_CASE(ks_, cpt_) \
    if (KS == ks_ && cpt == cpt_) { s = launch_simt_t<ks_, cpt_>(a, nb, st, err); if (s) return s; continue; }
        WSKPN_SIMT_CASE(5, 4) WSKPN_SIMT_CASE(5, 8) WSKPN_SIMT_CASE(5, 12) WSKPN_SIMT_CASE(5, 16)
        WSKPN_SIMT_CASE(3, 4) WSKPN_SIMT_CASE(3, 8) WSKPN_SIMT_CASE(3, 12) WSKPN_SIMT_CASE(3, 16)
#undef WSKPN_SIMT_CASE
        err = "conv_simt: unsupported KS/Cout combination";
        return WSKPN_EUNSUPPORTED;
    }
    return WSKPN_OK;
}

wskpn_status launch_conv_simt(const float* const* in, float* const* out, int B, int H, int W, int Cin, int Cout,
                              int KS, const float* w_packed, const float* bias_padded, int relu, cudaStream_t st,
                              std::string& err) {
    return launch_conv_simt_masked(in, out, nullptr, B, H, W, Cin, Cout, KS, w_packed, bias_padded, relu, st, err);
}

// Packs an OIHW FP32 layer ([Cout][Cin][KS][KS] + bias[Cout]) into the SIMT
// layout [Cin][KS*KS][COUTP] and a zero-padded bias [COUTP].
__global__ void pack_simt_kernel(const float* __restrict__ w, const float* __restrict__ b, int Cin,
                                 int Cout, int KS, int COUTP, float* __restrict__ wp,
                                 float* __restrict__ bp) {
    const int n = Cin * KS * KS * COUTP;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int o = i % COUTP, t = (i / COUTP) % (KS * KS), c = i / (COUTP * KS * KS);
        wp[i] = o < Cout ? w[((size_t)o * Cin + c) * KS * KS + t] : 0.f;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < COUTP; i += gridDim.x * blockDim.x)
        bp[i] = i < Cout ? b[i] : 0.f;
}

wskpn_status launch_pack_simt(const float* w, const float* b, int Cin, int Cout, int KS, float* wp,
                              float* bp, cudaStream_t st, std::string& err) {
    pack_simt_kernel<<<64, 256, 0, st>>>(w, b, Cin, Cout, KS, simt_coutp(Cout), wp, bp);
    WSKPN_CUDA_TRY(cudaGetLastError(), err);
    return WSKPN_OK;
}

}  // namespace wskpn
