// Backward of the ImportanceNet convolutions (FP32), for one training step
// of Eq. 1.  For y = b + W * x (KSxKS cross-correlation, zero padding) and
// the pre-activation gradient gy:
//   dL/dx[c](q)     = sum_{o,t} W[o][c][t] gy[o](q - t + pad)
//                   = a forward conv of gy with W transposed and flipped,
//                     followed by the ReLU mask of x (x > 0);
//   dL/dW[o][c][t]  = sum_p gy[o](p) x[c](p + t - pad);
//   dL/db[o]        = sum_p gy[o](p).
// The weight gradient is a reduction over every pixel of the batch: CTAs
// accumulate partial sums over a fixed set of pixel tiles, write them to a
// workspace, and a second kernel adds the partials in a fixed order, so
// the result does not depend on scheduling.
#include "common.cuh"

namespace wskpn {

int simt_coutp(int cout);

// W[o][c][t] (OIHW) -> packed [o][t'][coutp(Cin)] with t' the flipped tap:
// the SIMT conv layout of the transposed layer (Cin' = Cout, Cout' = Cin).
__global__ void pack_simt_transposed_kernel(const float* __restrict__ w, int Cin, int Cout, int KS, int coutp,
                                            float* __restrict__ wp, float* __restrict__ bp) {
    const int KK = KS * KS;
    const int n = Cout * KK * coutp;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int c = i % coutp, t = (i / coutp) % KK, o = i / (coutp * KK);
        wp[i] = c < Cin ? w[((size_t)o * Cin + c) * KK + (KK - 1 - t)] : 0.f;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < coutp; i += gridDim.x * blockDim.x) bp[i] = 0.f;
}

wskpn_status launch_pack_simt_transposed(const float* w, int Cin, int Cout, int KS, float* wp, float* bp,
                                         cudaStream_t st, std::string& err) {
    pack_simt_transposed_kernel<<<64, 256, 0, st>>>(w, Cin, Cout, KS, simt_coutp(Cin), wp, bp);
    WSKPN_CUDA_TRY(cudaGetLastError(), err);
    return WSKPN_OK;
}

namespace wg {
constexpr int TW = 32, TH = 8, THREADS = 256, CC = 8, MAXO = 64;
}

struct WgradArgs {
    PtrBatch<const float*> x;   // [Cin][H][W]
    PtrBatch<const float*> gy;  // [Cout][H][W]
    float* part;                // [G][Cin_chunks*CC][KS*KS][MAXO] then db [G][MAXO]
    int B, H, W, Cin, Cout, tiles_x, tiles_y, ntiles, G;
};

// Grid (G, Cin chunks).  Lane = output channel (o, and o + 32 when NO = 64
// output channels are kept; NO = 32 serves layers of at most 32), warp w
// owns KS of the CC x KS (channel, dy) pairs; each thread keeps NO / 32 x KS
// x KS partial sums and slides a KS-wide window of x along each tile row.
// NO = 16 (at most 16 output channels): each half-warp is one set of 16
// channels and owns its own pairs, and a chunk holds 2 CC input channels.
template <int KS, int NO>
__global__ void __launch_bounds__(wg::THREADS) wgrad_kernel(WgradArgs a) {
    constexpr bool HALF = NO == 16;
    constexpr int U = HALF ? 1 : NO / 32;        // output channels per lane
    constexpr int CCT = HALF ? 2 * wg::CC : wg::CC;  // input channels per chunk
    constexpr int PAD = KS / 2, IW = wg::TW + KS - 1, IH = wg::TH + KS - 1;
    constexpr int COMBOS = CCT * KS;             // (c, dy) pairs per chunk
    constexpr int GROUPS = (wg::THREADS / 32) * (HALF ? 2 : 1);  // warps, or half-warps
    constexpr int CPW = COMBOS / GROUPS;         // pairs per warp (half-warp)
    static_assert(COMBOS % GROUPS == 0, "pairs per warp");
    extern __shared__ float wg_smem[];
    float (*sx)[IH][IW] = reinterpret_cast<float (*)[IH][IW]>(wg_smem);                    // [CCT][IH][IW]
    float (*sg)[wg::MAXO] = reinterpret_cast<float (*)[wg::MAXO]>(wg_smem + CCT * IH * IW);  // [TH*TW][MAXO]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int grp = HALF ? warp * 2 + (lane >> 4) : warp;  // owner of pairs grp * CPW ..
    const int ol = HALF ? lane & 15 : lane;                // this lane's output channel
    const int g = blockIdx.x, c0 = blockIdx.y * CCT;
    const int H = a.H, W = a.W;
    const size_t HW = (size_t)H * W;
    float acc[U][CPW][KS];
    float dbacc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) dbacc[u] = 0.f;
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
        for (int k = 0; k < CPW; ++k)
#pragma unroll
            for (int d = 0; d < KS; ++d) acc[u][k][d] = 0.f;

    for (int t = g; t < a.ntiles; t += a.G) {
        const int tx = t % a.tiles_x, ty = (t / a.tiles_x) % a.tiles_y, b = t / (a.tiles_x * a.tiles_y);
        const int x0 = tx * wg::TW, y0 = ty * wg::TH;
        const float* __restrict__ xb = a.x.p[b];
        const float* __restrict__ gb = a.gy.p[b];
        __syncthreads();
        for (int i = tid; i < CCT * IH * IW; i += wg::THREADS) {
            const int c = i / (IH * IW), rem = i % (IH * IW), iy = rem / IW, ix = rem % IW;
            const int gy = y0 + iy - PAD, gx = x0 + ix - PAD;
            const bool in = c0 + c < a.Cin && gy >= 0 && gy < H && gx >= 0 && gx < W;
            sx[c][iy][ix] = in ? xb[(size_t)(c0 + c) * HW + (size_t)gy * W + gx] : 0.f;
        }
        for (int i = tid; i < wg::TH * wg::TW * NO; i += wg::THREADS) {
            const int o = i / (wg::TH * wg::TW), p = i % (wg::TH * wg::TW);
            const int gy = y0 + p / wg::TW, gx = x0 + p % wg::TW;
            const bool in = o < a.Cout && gy < H && gx < W;
            sg[p][o] = in ? gb[(size_t)o * HW + (size_t)gy * W + gx] : 0.f;
        }
        __syncthreads();
        for (int py = 0; py < wg::TH; ++py) {
            float win[CPW][KS];
#pragma unroll
            for (int k = 0; k < CPW; ++k) {
                const int combo = grp * CPW + k, c = combo / KS, dy = combo % KS;
#pragma unroll
                for (int d = 0; d < KS - 1; ++d) win[k][d] = sx[c][py + dy][d];
            }
#pragma unroll
            for (int px = 0; px < wg::TW; ++px) {
                float gv[U];
#pragma unroll
                for (int u = 0; u < U; ++u) gv[u] = sg[py * wg::TW + px][ol + 32 * u];
                if (blockIdx.y == 0 && grp == 0)
#pragma unroll
                    for (int u = 0; u < U; ++u) dbacc[u] += gv[u];
#pragma unroll
                for (int k = 0; k < CPW; ++k) {
                    const int combo = grp * CPW + k, c = combo / KS, dy = combo % KS;
                    win[k][(px + KS - 1) % KS] = sx[c][py + dy][px + KS - 1];
#pragma unroll
                    for (int d = 0; d < KS; ++d) {
                        const float xv = win[k][(px + d) % KS];
#pragma unroll
                        for (int u = 0; u < U; ++u) acc[u][k][d] = fmaf(gv[u], xv, acc[u][k][d]);
                    }
                }
            }
        }
    }
    // partial [g][c][dy*KS+dx][o]
    // (entries of channels o >= NO are never read: the layer has fewer)
    const int cpad = gridDim.y * CCT;
    float* part = a.part + (size_t)g * cpad * KS * KS * wg::MAXO;
#pragma unroll
    for (int k = 0; k < CPW; ++k) {
        const int combo = grp * CPW + k, c = c0 + combo / KS, dy = combo % KS;
#pragma unroll
        for (int d = 0; d < KS; ++d)
#pragma unroll
            for (int u = 0; u < U; ++u) part[((size_t)c * KS * KS + dy * KS + d) * wg::MAXO + ol + 32 * u] = acc[u][k][d];
    }
    if (blockIdx.y == 0 && grp == 0) {
        float* pdb = a.part + (size_t)a.G * cpad * KS * KS * wg::MAXO + (size_t)g * wg::MAXO;
#pragma unroll
        for (int u = 0; u < U; ++u) pdb[ol + 32 * u] = dbacc[u];
    }
}

// dW[o][c][t] = sum_g part[g][c][t][o];  db[o] = sum_g pdb[g][o] (fixed order)
__global__ void wgrad_reduce_kernel(const float* __restrict__ part, int G, int cpad, int Cin, int Cout, int KK,
                                    float* __restrict__ dw, float* __restrict__ db) {
    const int n = Cout * Cin * KK;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n + Cout; i += gridDim.x * blockDim.x) {
        float s = 0.f;
        if (i < n) {
            const int t = i % KK, c = (i / KK) % Cin, o = i / (KK * Cin);
            for (int g = 0; g < G; ++g) s += part[(((size_t)g * cpad + c) * KK + t) * wg::MAXO + o];
            dw[i] = s;
        } else {
            const int o = i - n;
            const float* pdb = part + (size_t)G * cpad * KK * wg::MAXO;
            for (int g = 0; g < G; ++g) s += pdb[(size_t)g * wg::MAXO + o];
            db[o] = s;
        }
    }
}

size_t wgrad_part_floats(int Cin, int KS, int G) {
    const int cpad = (Cin + 2 * wg::CC - 1) / (2 * wg::CC) * (2 * wg::CC);  // chunks of CC or 2 CC channels
    return (size_t)G * cpad * KS * KS * wg::MAXO + (size_t)G * wg::MAXO;
}

wskpn_status launch_wgrad(const float* const* x, const float* const* gy, int B, int H, int W, int Cin, int Cout,
                          int KS, int G, float* part, float* dw, float* db, cudaStream_t st, std::string& err) {
    if (Cout > wg::MAXO || B > WSKPN_MAX_BATCH) {
        err = "wgrad: Cout > 64 or batch > 16";
        return WSKPN_EUNSUPPORTED;
    }
    WgradArgs a{};
    for (int b = 0; b < B; ++b) {
        a.x.p[b] = x[b];
        a.gy.p[b] = gy[b];
    }
    a.part = part;
    a.B = B;
    a.H = H;
    a.W = W;
    a.Cin = Cin;
    a.Cout = Cout;
    a.tiles_x = cdiv(W, wg::TW);
    a.tiles_y = cdiv(H, wg::TH);
    a.ntiles = a.tiles_x * a.tiles_y * B;
    a.G = G;
    // layers of at most 16 / 32 output channels keep them on half-warps / one per lane
    const int no = Cout <= 16 ? 16 : Cout <= 32 ? 32 : 64;
    const int cct = no == 16 ? 2 * wg::CC : wg::CC;  // input channels per chunk
    const int nchunks = cdiv(Cin, cct);
    dim3 grid(G, nchunks);
    const size_t smem = (size_t)(cct * (wg::TH + KS - 1) * (wg::TW + KS - 1) + wg::TH * wg::TW * wg::MAXO) * sizeof(float);
    void (*kern)(WgradArgs) = KS == 5 ? (no == 16 ? wgrad_kernel<5, 16> : no == 32 ? wgrad_kernel<5, 32> : wgrad_kernel<5, 64>)
                                      : (no == 16 ? wgrad_kernel<3, 16> : no == 32 ? wgrad_kernel<3, 32> : wgrad_kernel<3, 64>);
    WSKPN_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), err);
    kern<<<grid, wg::THREADS, smem, st>>>(a);
    WSKPN_CUDA_TRY(cudaGetLastError(), err);
    wgrad_reduce_kernel<<<148, 256, 0, st>>>(part, G, nchunks * cct, Cin, Cout, KS * KS, dw, db);
    WSKPN_CUDA_TRY(cudaGetLastError(), err);
    return WSKPN_OK;
}

}  // namespace wskpn
