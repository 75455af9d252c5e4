// Reconstruction phase (Sec. 4.2): kernel construction from importance maps
// (Eq. 3), filtering (Eq. 4), multi-size fusion (Eq. 5) and albedo
// re-modulation, fused into one streaming kernel that never materialises the
// H x W x k^2 kernel map.
//
// Per output pixel p and size i (window Omega_i(p) clipped to the image):
//   R_i(p) = sum_q exp(I_i(q)) y(q) / sum_q exp(I_i(q)),  y = r / (a + eps)
// i.e. Eq. 3-4 written as the ratio of two window sums N_i / D_i.  The sums
// are separable box sums, evaluated from a shared-memory tile with a 6-pixel
// halo.  The exponent is shifted by the maximum of I_i over the tile's
// window footprint; the shift cancels in N/D for every pixel.  A pixel whose
// D_i falls below 1e-30 (the footprint's logit range exceeds ~69) is
// recomputed exactly with its own window maximum and counted.
#include "common.cuh"

namespace wskpn {

namespace df {
constexpr int TW = 64;              // tile width (output pixels)
constexpr int TH = 16;              // tile height
constexpr int HALO = 6;             // largest half window (k = 13)
constexpr int RW = TW + 2 * HALO;   // 76
constexpr int RH = TH + 2 * HALO;   // 28
constexpr int RP = RW + 1;          // odd row pitch: column-walking lanes hit distinct banks
constexpr int HP = TW + 1;          // pitch of the horizontal-sum rows
constexpr int THREADS = 256;
constexpr int PPT = TW * TH / THREADS;  // output pixels per thread (4)
constexpr int SMEM_FLOATS = 3 * RH * RP + 4 * RH * RP + 4 * RH * HP;
constexpr size_t SMEM_BYTES = SMEM_FLOATS * sizeof(float);
constexpr float DMIN = 1e-30f;
}  // namespace df

struct DecodeArgs {
    PtrBatch<const float*> z, r, a;
    PtrBatch<float*> out;
    int H, W, M;
    int ks[WSKPN_MAX_KERNELS];
    float eps;
    unsigned int* fallbacks;
};

// Horizontal window sums of the 4 planes (E, E*y0, E*y1, E*y2) for the rows
// the vertical pass needs.  One thread walks one (plane, row, 16-pixel
// segment) and keeps the 16 + K - 1 inputs in registers.
template <int K>
__device__ __forceinline__ void hpass(const float* __restrict__ sE, float* __restrict__ sH, int tid) {
    constexpr int h = K / 2;
    constexpr int NR = df::TH + 2 * h;
    constexpr int SEG = 16;                 // outputs per item
    constexpr int NSEG = df::TW / SEG;      // 4
    for (int it = tid; it < 4 * NSEG * NR; it += df::THREADS) {
        const int row = it % NR;
        const int seg = (it / NR) % NSEG;
        const int ch = it / (NSEG * NR);
        const int ry = df::HALO - h + row;
        const float* src = sE + (ch * df::RH + ry) * df::RP + (df::HALO - h) + seg * SEG;
        float* dst = sH + (ch * df::RH + ry) * df::HP + seg * SEG;
        float win[SEG + K - 1];
#pragma unroll
        for (int j = 0; j < SEG + K - 1; ++j) win[j] = src[j];
#pragma unroll
        for (int x = 0; x < SEG; ++x) {
            float s = win[x];
#pragma unroll
            for (int d = 1; d < K; ++d) s += win[x + d];
            dst[x] = s;
        }
    }
}

// Vertical window sums of the horizontal sums -> sV[4][TH][TW].
template <int K>
__device__ __forceinline__ void vpass(const float* __restrict__ sH, float* __restrict__ sV, int tid) {
    constexpr int h = K / 2;
    const int x = tid % df::TW;
    const int ch = tid / df::TW;  // THREADS == 4 * TW
    const float* src = sH + (ch * df::RH + (df::HALO - h)) * df::HP + x;
    float col[df::TH + K - 1];
#pragma unroll
    for (int j = 0; j < df::TH + K - 1; ++j) col[j] = src[j * df::HP];
#pragma unroll
    for (int y = 0; y < df::TH; ++y) {
        float s = col[y];
#pragma unroll
        for (int d = 1; d < K; ++d) s += col[y + d];
        sV[(ch * df::TH + y) * df::TW + x] = s;
    }
}

template <int K>
__device__ __forceinline__ void box_sums(const float* sE, float* sH, float* sV, int tid) {
    hpass<K>(sE, sH, tid);
    __syncthreads();
    vpass<K>(sH, sV, tid);
}

// Exact per-window evaluation of Eq. 3-4 for one pixel (slow path).
__device__ __noinline__ void window_exact(const float* __restrict__ z, const float* __restrict__ r,
                             const float* __restrict__ a, int H, int W, int k, float eps, int px,
                             int py, float R[3]) {
    const int h = k / 2;
    const size_t HW = (size_t)H * W;
    const int y0 = max(py - h, 0), y1 = min(py + h, H - 1);
    const int x0 = max(px - h, 0), x1 = min(px + h, W - 1);
    float m = -INFINITY;
    for (int qy = y0; qy <= y1; ++qy)
        for (int qx = x0; qx <= x1; ++qx) m = fmaxf(m, z[(size_t)qy * W + qx]);
    float D = 0.f, N0 = 0.f, N1 = 0.f, N2 = 0.f;
    for (int qy = y0; qy <= y1; ++qy)
        for (int qx = x0; qx <= x1; ++qx) {
            const size_t g = (size_t)qy * W + qx;
            const float e = expf(z[g] - m);
            D += e;
            N0 += e * (r[g] / (a[g] + eps));
            N1 += e * (r[HW + g] / (a[HW + g] + eps));
            N2 += e * (r[2 * HW + g] / (a[2 * HW + g] + eps));
        }
    R[0] = N0 / D;
    R[1] = N1 / D;
    R[2] = N2 / D;
}

// Every load of a thread is issued before any is used (one memory latency
// per phase instead of one per loop iteration).
constexpr int REGION_PER_THREAD = (df::RH * df::RW + df::THREADS - 1) / df::THREADS;  // 9

__device__ __forceinline__ void load_irradiance(float* __restrict__ sY, const float* __restrict__ r,
                                                const float* __restrict__ a, int H, int W, int tx0, int ty0,
                                                float eps, int tid) {
    const size_t HW = (size_t)H * W;
    float rv[REGION_PER_THREAD][3], av[REGION_PER_THREAD][3];
#pragma unroll
    for (int j = 0; j < REGION_PER_THREAD; ++j) {
        const int i = tid + j * df::THREADS;
        const int ry = i / df::RW, rx = i % df::RW;
        const int gy = ty0 - df::HALO + ry, gx = tx0 - df::HALO + rx;
        const bool in = i < df::RH * df::RW && gy >= 0 && gy < H && gx >= 0 && gx < W;
        const size_t g = in ? (size_t)gy * W + gx : 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            rv[j][c] = in ? __ldg(r + c * HW + g) : 0.f;
            av[j][c] = in ? __ldg(a + c * HW + g) : 0.f;
        }
    }
#pragma unroll
    for (int j = 0; j < REGION_PER_THREAD; ++j) {
        const int i = tid + j * df::THREADS;
        if (i >= df::RH * df::RW) continue;
        const int ry = i / df::RW, rx = i % df::RW;
#pragma unroll
        for (int c = 0; c < 3; ++c) sY[(c * df::RH + ry) * df::RP + rx] = rv[j][c] / (av[j][c] + eps);
    }
}

// For one window size K (compile-time, so all index arithmetic divides by
// constants): load I_i on the footprint of the tile's windows, shift by its
// maximum m, form E = exp(I - m) and E*y in smem (E = 0 outside the image)
// and take the K x K window sums into sV.  Returns m.
template <int K>
__device__ __noinline__ float size_sums(float* __restrict__ sE, float* __restrict__ sH, float* __restrict__ sV,
                                           const float* __restrict__ sY, float* __restrict__ red,
                                           const float* __restrict__ zi, int H, int W, int tx0, int ty0, int tid) {
    constexpr int h = K / 2, NR = df::TH + 2 * h, NC = df::TW + 2 * h, NT = NR * NC;
    constexpr int PER = (NT + df::THREADS - 1) / df::THREADS;
    float v[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int t = tid + j * df::THREADS;
        const int gy = ty0 - h + t / NC, gx = tx0 - h + t % NC;
        const bool in = t < NT && gy >= 0 && gy < H && gx >= 0 && gx < W;
        v[j] = in ? __ldg(zi + (size_t)gy * W + gx) : -INFINITY;
    }
    float m = -INFINITY;
#pragma unroll
    for (int j = 0; j < PER; ++j) m = fmaxf(m, v[j]);
    m = warp_max(m);
    if ((tid & 31) == 0) red[tid >> 5] = m;
    __syncthreads();
    m = red[0];
#pragma unroll
    for (int w = 1; w < df::THREADS / 32; ++w) m = fmaxf(m, red[w]);
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int t = tid + j * df::THREADS;
        if (PER * df::THREADS > NT && t >= NT) continue;
        const int o = (df::HALO - h + t / NC) * df::RP + (df::HALO - h + t % NC);
        const float e = expf(v[j] - m);
        sE[o] = e;
#pragma unroll
        for (int c = 0; c < 3; ++c) sE[(1 + c) * df::RH * df::RP + o] = e * sY[c * df::RH * df::RP + o];
    }
    __syncthreads();
    box_sums<K>(sE, sH, sV, tid);
    return m;
}

__device__ __forceinline__ float size_sums_k(int k, float* sE, float* sH, float* sV, const float* sY, float* red,
                                             const float* zi, int H, int W, int tx0, int ty0, int tid) {
    switch (k) {
        case 1: return size_sums<1>(sE, sH, sV, sY, red, zi, H, W, tx0, ty0, tid);
        case 3: return size_sums<3>(sE, sH, sV, sY, red, zi, H, W, tx0, ty0, tid);
        case 5: return size_sums<5>(sE, sH, sV, sY, red, zi, H, W, tx0, ty0, tid);
        case 7: return size_sums<7>(sE, sH, sV, sY, red, zi, H, W, tx0, ty0, tid);
        case 9: return size_sums<9>(sE, sH, sV, sY, red, zi, H, W, tx0, ty0, tid);
        case 11: return size_sums<11>(sE, sH, sV, sY, red, zi, H, W, tx0, ty0, tid);
        default: return size_sums<13>(sE, sH, sV, sY, red, zi, H, W, tx0, ty0, tid);
    }
}

__global__ void __launch_bounds__(df::THREADS, 2) decode_fuse_fwd_kernel(DecodeArgs args) {
    extern __shared__ float smem[];
    float* sY = smem;                          // [3][RH][RP]  irradiance y
    float* sE = sY + 3 * df::RH * df::RP;      // [4][RH][RP]  E, E*y  (reused as sV)
    float* sH = sE + 4 * df::RH * df::RP;      // [4][RH][HP]  horizontal sums
    float* sV = sE;                            // [4][TH][TW]
    __shared__ float red[df::THREADS / 32];

    const int tid = threadIdx.x;
    const int b = blockIdx.z;
    const int H = args.H, W = args.W, M = args.M;
    const size_t HW = (size_t)H * W;
    const int tx0 = blockIdx.x * df::TW, ty0 = blockIdx.y * df::TH;
    const float* __restrict__ z = args.z.p[b];
    const float* __restrict__ r = args.r.p[b];
    const float* __restrict__ a = args.a.p[b];
    const float eps = args.eps;

    // Demodulated irradiance on the tile + halo (0 outside the image).
    load_irradiance(sY, r, a, H, W, tx0, ty0, eps, tid);

    // Fusion weights alpha_i(p) = exp(l_i - lmax) / sum_j exp(l_j - lmax)
    // over the M logits of each own pixel; only lmax and 1/sum are kept.
    float lmax[df::PPT], linv[df::PPT];
    float acc[df::PPT][3];
#pragma unroll
    for (int j = 0; j < df::PPT; ++j) {
        const int p = tid + j * df::THREADS;
        const int gy = ty0 + p / df::TW, gx = tx0 + p % df::TW;
        const bool in = gy < H && gx < W;
        const size_t g = in ? (size_t)gy * W + gx : 0;
        float m = -INFINITY;
        for (int i = 0; i < M; ++i) m = fmaxf(m, in ? __ldg(z + (size_t)(M + i) * HW + g) : 0.f);
        float sum = 0.f;
        for (int i = 0; i < M; ++i) sum += in ? expf(__ldg(z + (size_t)(M + i) * HW + g) - m) : 1.f;
        lmax[j] = m;
        linv[j] = 1.f / sum;
        acc[j][0] = acc[j][1] = acc[j][2] = 0.f;
    }

    for (int i = 0; i < M; ++i) {
        const int k = args.ks[i];
        const float* __restrict__ zi = z + (size_t)i * HW;
        // E_i = exp(I_i - m) and E_i * y on the footprint, then window sums
        size_sums_k(k, sE, sH, sV, sY, red, zi, H, W, tx0, ty0, tid);
        __syncthreads();
#pragma unroll
        for (int j = 0; j < df::PPT; ++j) {
            const int p = tid + j * df::THREADS;
            const int ly = p / df::TW, lx = p % df::TW;
            const int gy = ty0 + ly, gx = tx0 + lx;
            if (gy >= H || gx >= W) continue;
            const float D = sV[ly * df::TW + lx];
            float R[3];
            if (D >= df::DMIN) {
                const float invD = 1.f / D;
#pragma unroll
                for (int c = 0; c < 3; ++c) R[c] = sV[((1 + c) * df::TH + ly) * df::TW + lx] * invD;
            } else {
                window_exact(zi, r, a, H, W, k, eps, gx, gy, R);
                if (args.fallbacks) atomicAdd(args.fallbacks, 1u);
            }
            const float al = expf(__ldg(z + (size_t)(M + i) * HW + (size_t)gy * W + gx) - lmax[j]) * linv[j];
#pragma unroll
            for (int c = 0; c < 3; ++c) acc[j][c] = fmaf(al, R[c], acc[j][c]);
        }
        __syncthreads();
    }

    // Re-modulation and store.
    float* __restrict__ out = args.out.p[b];
#pragma unroll
    for (int j = 0; j < df::PPT; ++j) {
        const int p = tid + j * df::THREADS;
        const int gy = ty0 + p / df::TW, gx = tx0 + p % df::TW;
        if (gy >= H || gx >= W) continue;
        const size_t g = (size_t)gy * W + gx;
#pragma unroll
        for (int c = 0; c < 3; ++c) out[c * HW + g] = (a[c * HW + g] + eps) * acc[j][c];
    }
}

// Host launcher: z/r/a/out given per frame.
wskpn_status launch_decode_fuse_fwd(const float* const* z, const float* const* r,
                                    const float* const* a, float* const* out, int B, int H, int W,
                                    int M, const int* ks, float eps, unsigned int* fallbacks,
                                    cudaStream_t st, std::string& err) {
    WSKPN_CUDA_TRY(cudaFuncSetAttribute(decode_fuse_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)df::SMEM_BYTES),
                   err);
    for (int b0 = 0; b0 < B; b0 += WSKPN_MAX_BATCH) {
        const int nb = B - b0 < WSKPN_MAX_BATCH ? B - b0 : WSKPN_MAX_BATCH;
        DecodeArgs args{};
        for (int j = 0; j < nb; ++j) {
            args.z.p[j] = z[b0 + j];
            args.r.p[j] = r[b0 + j];
            args.a.p[j] = a[b0 + j];
            args.out.p[j] = out[b0 + j];
        }
        args.H = H;
        args.W = W;
        args.M = M;
        for (int i = 0; i < M; ++i) args.ks[i] = ks[i];
        args.eps = eps;
        args.fallbacks = fallbacks;
        dim3 grid(cdiv(W, df::TW), cdiv(H, df::TH), nb);
        decode_fuse_fwd_kernel<<<grid, df::THREADS, df::SMEM_BYTES, st>>>(args);
        WSKPN_CUDA_TRY(cudaGetLastError(), err);
    }
    return WSKPN_OK;
}


// ======================================================================
// Backward of the reconstruction (chain rule through Eq. 3-5).
//
// With g_c = (a_c + eps) dL/dout_c, h_ic = g_c alpha_i, E_i = exp(I_i),
// D_i(p) = sum_{Omega_i(p)} E_i and R_ic = N_ic / D_i:
//   dL/dalpha-logit_i(p) = alpha_i (da_i - sum_j alpha_j da_j),  da_i = sum_c g_c R_ic
//   dL/dI_i(q) = sum_{p in Omega_i(q)} exp(I_i(q) - LSE_i(p)) sum_c h_ic(p) (y_c(q) - R_ic(p))
// (windows are symmetric: q in Omega(p) <=> p in Omega(q)), where
// LSE_i(p) = log D_i(p) is carried exactly, so the two kernels need no
// common exponent shift.
//   kernel 1 (per pixel p): R_ic, LSE_i, alpha_i, g_c -> scratch; the
//            fusion-logit gradients -> dz;
//   kernel 2 (per pixel q): window sums over p of u(p) h_ic(p) and
//            u(p) sum_c h_ic(p) R_ic(p) with u = exp(s - LSE), s the
//            footprint's minimum LSE, then
//            dz_i(q) = exp(I_i(q) - s) (sum_c y_c(q) S_c(q) - S_B(q)).
// Footprints whose LSE range exceeds 80 take an exact per-window loop.
// Scratch layout per frame: planes [LSE_0..M-1, alpha_0..M-1,
// R_{0,0..2}, ..., R_{M-1,0..2}, g_0..2] = 5M + 3 planes of H x W.
// ======================================================================

struct DecodeBwdArgs {
    PtrBatch<const float*> z, r, a, G;
    PtrBatch<float*> dz, scratch;
    int H, W, M;
    int ks[WSKPN_MAX_KERNELS];
    float eps;
    unsigned int* fallbacks;
};

__global__ void __launch_bounds__(df::THREADS, 2) decode_fuse_bwd1_kernel(DecodeBwdArgs args) {
    extern __shared__ float smem[];
    float* sY = smem;
    float* sE = sY + 3 * df::RH * df::RP;
    float* sH = sE + 4 * df::RH * df::RP;
    float* sV = sE;
    __shared__ float red[df::THREADS / 32];

    const int tid = threadIdx.x;
    const int b = blockIdx.z;
    const int H = args.H, W = args.W, M = args.M;
    const size_t HW = (size_t)H * W;
    const int tx0 = blockIdx.x * df::TW, ty0 = blockIdx.y * df::TH;
    const float* __restrict__ z = args.z.p[b];
    const float* __restrict__ r = args.r.p[b];
    const float* __restrict__ a = args.a.p[b];
    const float* __restrict__ G = args.G.p[b];
    float* __restrict__ sc = args.scratch.p[b];
    float* __restrict__ dz = args.dz.p[b];
    const float eps = args.eps;

    load_irradiance(sY, r, a, H, W, tx0, ty0, eps, tid);

    float alpha[df::PPT][WSKPN_MAX_KERNELS];
    float dal[df::PPT][WSKPN_MAX_KERNELS];
    float gc[df::PPT][3];
#pragma unroll
    for (int j = 0; j < df::PPT; ++j) {
        const int p = tid + j * df::THREADS;
        const int gy = ty0 + p / df::TW, gx = tx0 + p % df::TW;
        const bool in = gy < H && gx < W;
        const size_t g = (size_t)gy * W + gx;
        float m = -INFINITY;
#pragma unroll
        for (int i = 0; i < WSKPN_MAX_KERNELS; ++i) {
            alpha[j][i] = (i < M && in) ? z[(size_t)(M + i) * HW + g] : -INFINITY;
            m = fmaxf(m, alpha[j][i]);
            dal[j][i] = 0.f;
        }
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < WSKPN_MAX_KERNELS; ++i) {
            alpha[j][i] = (i < M && in) ? expf(alpha[j][i] - m) : 0.f;
            s += alpha[j][i];
        }
#pragma unroll
        for (int i = 0; i < WSKPN_MAX_KERNELS; ++i) alpha[j][i] = in ? alpha[j][i] / s : 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) gc[j][c] = in ? (a[c * HW + g] + eps) * G[c * HW + g] : 0.f;
        if (in) {
#pragma unroll
            for (int i = 0; i < WSKPN_MAX_KERNELS; ++i)
                if (i < M) sc[(size_t)(M + i) * HW + g] = alpha[j][i];
#pragma unroll
            for (int c = 0; c < 3; ++c) sc[(size_t)(5 * M + c) * HW + g] = gc[j][c];
        }
    }

    for (int i = 0; i < M; ++i) {
        const int k = args.ks[i];
        const int h = k / 2;
        const float* __restrict__ zi = z + (size_t)i * HW;
        const float m = size_sums_k(k, sE, sH, sV, sY, red, zi, H, W, tx0, ty0, tid);
        __syncthreads();
#pragma unroll
        for (int j = 0; j < df::PPT; ++j) {
            const int p = tid + j * df::THREADS;
            const int ly = p / df::TW, lx = p % df::TW;
            const int gy = ty0 + ly, gx = tx0 + lx;
            if (gy >= H || gx >= W) continue;
            const size_t g = (size_t)gy * W + gx;
            const float D = sV[ly * df::TW + lx];
            float R[3], L;
            if (D >= df::DMIN) {
#pragma unroll
                for (int c = 0; c < 3; ++c) R[c] = sV[((1 + c) * df::TH + ly) * df::TW + lx] / D;
                L = m + logf(D);
            } else {
                window_exact(zi, r, a, H, W, k, eps, gx, gy, R);
                // exact log-sum-exp of the window
                const int y0 = max(gy - h, 0), y1 = min(gy + h, H - 1), x0 = max(gx - h, 0), x1 = min(gx + h, W - 1);
                float mw = -INFINITY, Dw = 0.f;
                for (int qy = y0; qy <= y1; ++qy)
                    for (int qx = x0; qx <= x1; ++qx) mw = fmaxf(mw, zi[(size_t)qy * W + qx]);
                for (int qy = y0; qy <= y1; ++qy)
                    for (int qx = x0; qx <= x1; ++qx) Dw += expf(zi[(size_t)qy * W + qx] - mw);
                L = mw + logf(Dw);
                if (args.fallbacks) atomicAdd(args.fallbacks, 1u);
            }
            sc[(size_t)i * HW + g] = L;
#pragma unroll
            for (int c = 0; c < 3; ++c) sc[(size_t)(2 * M + 3 * i + c) * HW + g] = R[c];
            const float d = gc[j][0] * R[0] + gc[j][1] * R[1] + gc[j][2] * R[2];
#pragma unroll
            for (int q = 0; q < WSKPN_MAX_KERNELS; ++q)
                if (q == i) dal[j][q] = d;
        }
        __syncthreads();
    }

    // fusion-logit gradients
#pragma unroll
    for (int j = 0; j < df::PPT; ++j) {
        const int p = tid + j * df::THREADS;
        const int gy = ty0 + p / df::TW, gx = tx0 + p % df::TW;
        if (gy >= H || gx >= W) continue;
        const size_t g = (size_t)gy * W + gx;
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < WSKPN_MAX_KERNELS; ++i) s += alpha[j][i] * dal[j][i];
#pragma unroll
        for (int i = 0; i < WSKPN_MAX_KERNELS; ++i)
            if (i < M) dz[(size_t)(M + i) * HW + g] = alpha[j][i] * (dal[j][i] - s);
    }
}

__global__ void __launch_bounds__(df::THREADS, 2) decode_fuse_bwd2_kernel(DecodeBwdArgs args) {
    extern __shared__ float smem[];
    float* sE = smem;                       // [4][RH][RP]: u h_0, u h_1, u h_2, u sum_c h_c R_c
    float* sH = sE + 4 * df::RH * df::RP;   // [4][RH][HP]
    float* sV = sE;
    __shared__ float red[2][df::THREADS / 32];

    const int tid = threadIdx.x;
    const int b = blockIdx.z;
    const int H = args.H, W = args.W, M = args.M;
    const size_t HW = (size_t)H * W;
    const int tx0 = blockIdx.x * df::TW, ty0 = blockIdx.y * df::TH;
    const float* __restrict__ z = args.z.p[b];
    const float* __restrict__ r = args.r.p[b];
    const float* __restrict__ a = args.a.p[b];
    const float* __restrict__ sc = args.scratch.p[b];
    float* __restrict__ dz = args.dz.p[b];
    const float eps = args.eps;

    float yq[df::PPT][3];
#pragma unroll
    for (int j = 0; j < df::PPT; ++j) {
        const int p = tid + j * df::THREADS;
        const int gy = ty0 + p / df::TW, gx = tx0 + p % df::TW;
        const bool in = gy < H && gx < W;
        const size_t g = (size_t)gy * W + gx;
#pragma unroll
        for (int c = 0; c < 3; ++c) yq[j][c] = in ? r[c * HW + g] / (a[c * HW + g] + eps) : 0.f;
    }

    for (int i = 0; i < M; ++i) {
        const int k = args.ks[i];
        const int h = k / 2;
        const int nr = df::TH + 2 * h, nc = df::TW + 2 * h;
        const float* __restrict__ Li = sc + (size_t)i * HW;
        const float* __restrict__ Ai = sc + (size_t)(M + i) * HW;
        const float* __restrict__ Ri = sc + (size_t)(2 * M + 3 * i) * HW;
        const float* __restrict__ gcp = sc + (size_t)(5 * M) * HW;
        // footprint minimum and maximum of LSE
        float mn = INFINITY, mx = -INFINITY;
        for (int t = tid; t < nr * nc; t += df::THREADS) {
            const int gy = ty0 - h + t / nc, gx = tx0 - h + t % nc;
            if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
                const float v = Li[(size_t)gy * W + gx];
                mn = fminf(mn, v);
                mx = fmaxf(mx, v);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
        if ((tid & 31) == 0) {
            red[0][tid >> 5] = mn;
            red[1][tid >> 5] = mx;
        }
        __syncthreads();
        mn = red[0][0];
        mx = red[1][0];
#pragma unroll
        for (int w = 1; w < df::THREADS / 32; ++w) {
            mn = fminf(mn, red[0][w]);
            mx = fmaxf(mx, red[1][w]);
        }
        const bool exact = mx - mn > 80.f;  // block-uniform
        if (!exact) {
            for (int t = tid; t < nr * nc; t += df::THREADS) {
                const int ry = df::HALO - h + t / nc, rx = df::HALO - h + t % nc;
                const int gy = ty0 - df::HALO + ry, gx = tx0 - df::HALO + rx;
                const int o = ry * df::RP + rx;
                float v0 = 0.f, v1 = 0.f, v2 = 0.f, v3 = 0.f;
                if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
                    const size_t g = (size_t)gy * W + gx;
                    const float u = expf(mn - Li[g]) * Ai[g];
                    const float h0 = u * gcp[g], h1 = u * gcp[HW + g], h2 = u * gcp[2 * HW + g];
                    v0 = h0;
                    v1 = h1;
                    v2 = h2;
                    v3 = h0 * Ri[g] + h1 * Ri[HW + g] + h2 * Ri[2 * HW + g];
                }
                sE[o] = v0;
                sE[df::RH * df::RP + o] = v1;
                sE[2 * df::RH * df::RP + o] = v2;
                sE[3 * df::RH * df::RP + o] = v3;
            }
            __syncthreads();
            switch (k) {
                case 1: box_sums<1>(sE, sH, sV, tid); break;
                case 3: box_sums<3>(sE, sH, sV, tid); break;
                case 5: box_sums<5>(sE, sH, sV, tid); break;
                case 7: box_sums<7>(sE, sH, sV, tid); break;
                case 9: box_sums<9>(sE, sH, sV, tid); break;
                case 11: box_sums<11>(sE, sH, sV, tid); break;
                default: box_sums<13>(sE, sH, sV, tid); break;
            }
            __syncthreads();
        }
#pragma unroll
        for (int j = 0; j < df::PPT; ++j) {
            const int p = tid + j * df::THREADS;
            const int ly = p / df::TW, lx = p % df::TW;
            const int gy = ty0 + ly, gx = tx0 + lx;
            if (gy >= H || gx >= W) continue;
            const size_t g = (size_t)gy * W + gx;
            const float zq = z[(size_t)i * HW + g];
            float v;
            if (!exact) {
                const float S0 = sV[ly * df::TW + lx], S1 = sV[(df::TH + ly) * df::TW + lx];
                const float S2 = sV[(2 * df::TH + ly) * df::TW + lx], SB = sV[(3 * df::TH + ly) * df::TW + lx];
                v = expf(zq - mn) * (yq[j][0] * S0 + yq[j][1] * S1 + yq[j][2] * S2 - SB);
            } else {
                v = 0.f;
                for (int py = max(gy - h, 0); py <= min(gy + h, H - 1); ++py)
                    for (int px = max(gx - h, 0); px <= min(gx + h, W - 1); ++px) {
                        const size_t gp = (size_t)py * W + px;
                        const float al = Ai[gp];
                        float t = 0.f;
#pragma unroll
                        for (int c = 0; c < 3; ++c) t += gcp[c * HW + gp] * al * (yq[j][c] - Ri[c * HW + gp]);
                        v += expf(zq - Li[gp]) * t;
                    }
                if (args.fallbacks) atomicAdd(args.fallbacks, 1u);
            }
            dz[(size_t)i * HW + g] = v;
        }
        __syncthreads();
    }
}

constexpr size_t DF_BWD2_SMEM = (4 * df::RH * df::RP + 4 * df::RH * df::HP) * sizeof(float);

wskpn_status launch_decode_fuse_bwd(const float* const* z, const float* const* r, const float* const* a,
                                    const float* const* G, float* const* dz, float* const* scratch, int B, int H,
                                    int W, int M, const int* ks, float eps, unsigned int* fallbacks,
                                    cudaStream_t st, std::string& err) {
    WSKPN_CUDA_TRY(cudaFuncSetAttribute(decode_fuse_bwd1_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)df::SMEM_BYTES),
                   err);
    WSKPN_CUDA_TRY(cudaFuncSetAttribute(decode_fuse_bwd2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)DF_BWD2_SMEM),
                   err);
    for (int b0 = 0; b0 < B; b0 += WSKPN_MAX_BATCH) {
        const int nb = B - b0 < WSKPN_MAX_BATCH ? B - b0 : WSKPN_MAX_BATCH;
        DecodeBwdArgs args{};
        for (int j = 0; j < nb; ++j) {
            args.z.p[j] = z[b0 + j];
            args.r.p[j] = r[b0 + j];
            args.a.p[j] = a[b0 + j];
            args.G.p[j] = G[b0 + j];
            args.dz.p[j] = dz[b0 + j];
            args.scratch.p[j] = scratch[b0 + j];
        }
        args.H = H;
        args.W = W;
        args.M = M;
        for (int i = 0; i < M; ++i) args.ks[i] = ks[i];
        args.eps = eps;
        args.fallbacks = fallbacks;
        dim3 grid(cdiv(W, df::TW), cdiv(H, df::TH), nb);
        decode_fuse_bwd1_kernel<<<grid, df::THREADS, df::SMEM_BYTES, st>>>(args);
        WSKPN_CUDA_TRY(cudaGetLastError(), err);
        decode_fuse_bwd2_kernel<<<grid, df::THREADS, DF_BWD2_SMEM, st>>>(args);
        WSKPN_CUDA_TRY(cudaGetLastError(), err);
    }
    return WSKPN_OK;
}

}  // namespace wskpn
