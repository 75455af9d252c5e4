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

// s[x] = sum_{d < K} w[x + d], x < NOUT (K <= 15): sums of 2, 4 and 8
// consecutive inputs are formed once and each window is assembled from the
// binary digits of K (all terms of one sign, so no cancellation); values no
// output needs are never computed (the arrays are fully unrolled).
template <int K, int NOUT>
__device__ __forceinline__ void box_sum1(const float (&w)[NOUT + K - 1], float (&s)[NOUT]) {
    constexpr int N1 = NOUT + K - 1;
    constexpr int B8 = K & 8, B4 = K & 4, B2 = K & 2, B1 = K & 1;
    constexpr int O4 = B8, O2 = B8 + B4, O1 = B8 + B4 + B2;
    static_assert(K >= 1 && K <= 15, "window");
    float p2[N1 > 1 ? N1 - 1 : 1], p4[N1 > 3 ? N1 - 3 : 1], p8[N1 > 7 ? N1 - 7 : 1];
#pragma unroll
    for (int j = 0; j + 1 < N1; ++j) p2[j] = w[j] + w[j + 1];
#pragma unroll
    for (int j = 0; j + 3 < N1; ++j) p4[j] = p2[j] + p2[j + 2];
#pragma unroll
    for (int j = 0; j + 7 < N1; ++j) p8[j] = p4[j] + p4[j + 4];
#pragma unroll
    for (int x = 0; x < NOUT; ++x) {
        float t = 0.f;
        if constexpr (B8 != 0) t = p8[x];
        if constexpr (B4 != 0) {
            if constexpr (O4 != 0) t += p4[x + O4];
            else t = p4[x];
        }
        if constexpr (B2 != 0) {
            if constexpr (O2 != 0) t += p2[x + O2];
            else t = p2[x];
        }
        if constexpr (B1 != 0) {
            if constexpr (O1 != 0) t += w[x + O1];
            else t = w[x];
        }
        s[x] = t;
    }
}

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
        float win[SEG + K - 1], out[SEG];
#pragma unroll
        for (int j = 0; j < SEG + K - 1; ++j) win[j] = src[j];
        box_sum1<K, SEG>(win, out);
#pragma unroll
        for (int x = 0; x < SEG; ++x) dst[x] = out[x];
    }
}

// Vertical window sums of the horizontal sums -> sV[4][TH][TW].
template <int K>
__device__ __forceinline__ void vpass(const float* __restrict__ sH, float* __restrict__ sV, int tid) {
    constexpr int h = K / 2;
    const int x = tid % df::TW;
    const int ch = tid / df::TW;  // THREADS == 4 * TW
    const float* src = sH + (ch * df::RH + (df::HALO - h)) * df::HP + x;
    float col[df::TH + K - 1], out[df::TH];
#pragma unroll
    for (int j = 0; j < df::TH + K - 1; ++j) col[j] = src[j * df::HP];
    box_sum1<K, df::TH>(col, out);
#pragma unroll
    for (int y = 0; y < df::TH; ++y) sV[(ch * df::TH + y) * df::TW + x] = out[y];
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
            N0 += e * (a ? r[g] / (a[g] + eps) : r[g]);
            N1 += e * (a ? r[HW + g] / (a[HW + g] + eps) : r[HW + g]);
            N2 += e * (a ? r[2 * HW + g] / (a[2 * HW + g] + eps) : r[2 * HW + g]);
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

// ---------------------------------------------------------------- forward
// With a NULL albedo the kernel takes r as the irradiance itself and writes
// the fused filtered irradiance (no demodulation, no re-modulation): the
// per-level filtering of the multi-resolution variant.
// The forward kernel uses 64 x 32 output tiles (6-pixel halo, 512 threads,
// one CTA per SM: the halo overhead of a tile is 1.6x its area for the
// largest window instead of 2.1x with 64 x 16) and organises each size's
// work for instruction economy:
//  * the horizontal pass forms E and E*y on the fly from the E and y planes
//    and handles the four planes as two packed pairs (D, N0) and (N1, N2)
//    with paired FP32 adds;
//  * a K-wide window sum is built from sums of 2, 4 and 8 neighbours taken
//    once per row segment and combined by the binary digits of K (all
//    terms positive, so no cancellation);
//  * the vertical pass of one column produces D and N directly for the
//    thread's own 4 pixels, which accumulate alpha_i R_i in registers;
//  * alpha (Eq. 5) is computed once per pixel into shared memory.
namespace dfw {
constexpr int TW = 64;                  // tile width (output pixels)
constexpr int TH = 32;                  // tile height
constexpr int HALO = 6;                 // largest half window (k = 13)
constexpr int RW = TW + 2 * HALO;       // 76: region pitch in floats (76 / 4 odd: row-strided 16-byte accesses are conflict-free)
constexpr int RH = TH + 2 * HALO;       // 44
constexpr int SEG = 8;                  // horizontal-pass outputs per item
constexpr int NSEG = TW / SEG;          // 8
constexpr int HP2 = TW + 2;             // pitch of the packed horizontal-sum rows in float2 (132 floats, 132 / 4 odd)
constexpr int THREADS = 512;
constexpr int RPT = TH * TW / THREADS;  // 4 output pixels per thread, one column
static_assert(THREADS / TW * RPT == TH, "vertical-pass mapping");
static_assert(RH * NSEG <= THREADS, "one horizontal item per thread");
constexpr int MAXK = WSKPN_MAX_KERNELS;
// shared memory in floats: y [3][RH][RW] | E [RH][RW] | hsum [2][RH][HP2] float2 | alpha [MAXK][TH][TW] |
// acc [RPT * 3][THREADS]
constexpr int OFF_Y = 0;
constexpr int OFF_E = OFF_Y + 3 * RH * RW;
constexpr int OFF_H = OFF_E + RH * RW;
constexpr int OFF_A = OFF_H + 2 * RH * HP2 * 2;
constexpr int OFF_ACC = OFF_A + MAXK * TH * TW;
constexpr int SMEM_FLOATS = OFF_ACC + RPT * 3 * THREADS;
constexpr size_t SMEM_BYTES = SMEM_FLOATS * sizeof(float);
static_assert(OFF_E % 4 == 0 && OFF_H % 4 == 0 && OFF_A % 4 == 0, "16-byte aligned planes");
}  // namespace dfw

// s[x] = sum_{d < K} w[x + d], x < NOUT, for two planes at once.  Sums of 2,
// 4 and 8 consecutive inputs are formed once and the window is assembled
// from the binary digits of K (K <= 15); values no output needs are never
// computed (the arrays are fully unrolled).
template <int K, int NOUT>
__device__ __forceinline__ void box_sum2(const float2 (&w)[NOUT + K - 1], float2 (&s)[NOUT]) {
    constexpr int N1 = NOUT + K - 1;
    constexpr int B8 = K & 8, B4 = K & 4, B2 = K & 2, B1 = K & 1;
    constexpr int O4 = B8, O2 = B8 + B4, O1 = B8 + B4 + B2;
    static_assert(K >= 1 && K <= 15, "window");
    float2 p2[N1 > 1 ? N1 - 1 : 1], p4[N1 > 3 ? N1 - 3 : 1], p8[N1 > 7 ? N1 - 7 : 1];
#pragma unroll
    for (int j = 0; j + 1 < N1; ++j) p2[j] = __fadd2_rn(w[j], w[j + 1]);
#pragma unroll
    for (int j = 0; j + 3 < N1; ++j) p4[j] = __fadd2_rn(p2[j], p2[j + 2]);
#pragma unroll
    for (int j = 0; j + 7 < N1; ++j) p8[j] = __fadd2_rn(p4[j], p4[j + 4]);
#pragma unroll
    for (int x = 0; x < NOUT; ++x) {
        float2 t = make_float2(0.f, 0.f);
        if constexpr (B8 != 0) t = p8[x];
        if constexpr (B4 != 0) {
            if constexpr (O4 != 0) t = __fadd2_rn(t, p4[x + O4]);
            else t = p4[x];
        }
        if constexpr (B2 != 0) {
            if constexpr (O2 != 0) t = __fadd2_rn(t, p2[x + O2]);
            else t = p2[x];
        }
        if constexpr (B1 != 0) {
            if constexpr (O1 != 0) t = __fadd2_rn(t, w[x + O1]);
            else t = w[x];
        }
        s[x] = t;
    }
}

// Horizontal window sums of (E, E y0) and (E y1, E y2) for the NR footprint
// rows of size K: one thread per (row, 8-pixel segment).  Inputs are read
// as 16-byte vectors from the aligned column at or before the footprint's
// first column; rows of consecutive threads are one region pitch apart.
template <int K>
__device__ __forceinline__ void fwd_hpass(const float* __restrict__ sE, const float* __restrict__ sY,
                                          float2* __restrict__ sH, int tid) {
    constexpr int h = K / 2, NR = dfw::TH + 2 * h;
    constexpr int C0 = dfw::HALO - h;
    constexpr int A0 = C0 & ~3;
    constexpr int OFF = C0 - A0;
    constexpr int NIN = dfw::SEG + K - 1;
    constexpr int NV = (OFF + NIN + 3) / 4;
    static_assert(A0 + (dfw::NSEG - 1) * dfw::SEG + 4 * NV <= dfw::RW, "aligned row reads stay in the region");
    if (tid >= NR * dfw::NSEG) return;
    const int row = tid % NR, seg = tid / NR;
    const int base = (dfw::HALO - h + row) * dfw::RW + seg * dfw::SEG + A0;
    float e[4 * NV], y[4 * NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const float4 t = *reinterpret_cast<const float4*>(sE + base + 4 * v);
        e[4 * v] = t.x; e[4 * v + 1] = t.y; e[4 * v + 2] = t.z; e[4 * v + 3] = t.w;
    }
    float2 w[NIN], s01[dfw::SEG], s23[dfw::SEG];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const float4 t = *reinterpret_cast<const float4*>(sY + base + 4 * v);
        y[4 * v] = t.x; y[4 * v + 1] = t.y; y[4 * v + 2] = t.z; y[4 * v + 3] = t.w;
    }
#pragma unroll
    for (int j = 0; j < NIN; ++j) w[j] = make_float2(e[OFF + j], e[OFF + j] * y[OFF + j]);
    box_sum2<K, dfw::SEG>(w, s01);
    float y2[4 * NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const float4 t = *reinterpret_cast<const float4*>(sY + dfw::RH * dfw::RW + base + 4 * v);
        const float4 u = *reinterpret_cast<const float4*>(sY + 2 * dfw::RH * dfw::RW + base + 4 * v);
        y[4 * v] = t.x; y[4 * v + 1] = t.y; y[4 * v + 2] = t.z; y[4 * v + 3] = t.w;
        y2[4 * v] = u.x; y2[4 * v + 1] = u.y; y2[4 * v + 2] = u.z; y2[4 * v + 3] = u.w;
    }
#pragma unroll
    for (int j = 0; j < NIN; ++j)
        w[j] = __fmul2_rn(make_float2(e[OFF + j], e[OFF + j]), make_float2(y[OFF + j], y2[OFF + j]));
    box_sum2<K, dfw::SEG>(w, s23);
    float2* d01 = sH + row * dfw::HP2 + seg * dfw::SEG;
    float2* d23 = d01 + dfw::RH * dfw::HP2;
#pragma unroll
    for (int x = 0; x < dfw::SEG; x += 2) {
        *reinterpret_cast<float4*>(d01 + x) = make_float4(s01[x].x, s01[x].y, s01[x + 1].x, s01[x + 1].y);
        *reinterpret_cast<float4*>(d23 + x) = make_float4(s23[x].x, s23[x].y, s23[x + 1].x, s23[x + 1].y);
    }
}

// One window size K: footprint logits and their maximum, E = exp(I_i - m)
// (0 outside the image), horizontal then vertical window sums, and
// acc += alpha_i R_i for the thread's own pixels (column x, rows
// RPT * rg ...), kept in shared memory [RPT * 3][THREADS] so that each size
// is a separate function with its own register allocation.  Three block
// barriers; the next size's first barrier orders this size's reads of E and
// the sums before they are overwritten.
template <int K>
__device__ __noinline__ void fwd_size(float* __restrict__ sE, float2* __restrict__ sH,
                                         const float* __restrict__ sY, const float* __restrict__ sAl,
                                         float* __restrict__ red, const float* __restrict__ zi,
                                         const float* __restrict__ r, const float* __restrict__ a, int H, int W,
                                         int tx0, int ty0, int tid, float eps, unsigned int* fallbacks,
                                         float* __restrict__ sAcc) {
    constexpr int h = K / 2, NR = dfw::TH + 2 * h, NC = dfw::TW + 2 * h, NT = NR * NC;
    constexpr int PER = (NT + dfw::THREADS - 1) / dfw::THREADS;
    float v[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int t = tid + j * dfw::THREADS;
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
    for (int w = 1; w < dfw::THREADS / 32; ++w) m = fmaxf(m, red[w]);
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int t = tid + j * dfw::THREADS;
        if (PER * dfw::THREADS > NT && t >= NT) continue;
        sE[(dfw::HALO - h + t / NC) * dfw::RW + (dfw::HALO - h + t % NC)] = expf(v[j] - m);
    }
    __syncthreads();
    fwd_hpass<K>(sE, sY, sH, tid);
    __syncthreads();

    const int x = tid % dfw::TW, rg = tid / dfw::TW;
    constexpr int NIN = dfw::RPT + K - 1;
    float2 c[NIN], s01[dfw::RPT], s23[dfw::RPT];
#pragma unroll
    for (int j = 0; j < NIN; ++j) c[j] = sH[(rg * dfw::RPT + j) * dfw::HP2 + x];
    box_sum2<K, dfw::RPT>(c, s01);
#pragma unroll
    for (int j = 0; j < NIN; ++j) c[j] = sH[(dfw::RH + rg * dfw::RPT + j) * dfw::HP2 + x];
    box_sum2<K, dfw::RPT>(c, s23);
    const int gx = tx0 + x;
#pragma unroll
    for (int j = 0; j < dfw::RPT; ++j) {
        const int ly = rg * dfw::RPT + j, gy = ty0 + ly;
        if (gy >= H || gx >= W) continue;
        float R[3];
        const float D = s01[j].x;
        if (D >= df::DMIN) {
            const float invD = 1.f / D;
            R[0] = s01[j].y * invD;
            R[1] = s23[j].x * invD;
            R[2] = s23[j].y * invD;
        } else {
            window_exact(zi, r, a, H, W, K, eps, gx, gy, R);
            if (fallbacks) atomicAdd(fallbacks, 1u);
        }
        const float al = sAl[ly * dfw::TW + x];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float* p = sAcc + (j * 3 + ch) * dfw::THREADS + tid;
            *p = fmaf(al, R[ch], *p);
        }
    }
}

template <bool DEMOD>
__global__ void __launch_bounds__(dfw::THREADS, 1) decode_fuse_fwd_kernel(DecodeArgs args) {
    extern __shared__ float4 dsm4[];
    float* smem = reinterpret_cast<float*>(dsm4);
    float* sY = smem + dfw::OFF_Y;
    float* sE = smem + dfw::OFF_E;
    float2* sH = reinterpret_cast<float2*>(smem + dfw::OFF_H);
    float* sAl = smem + dfw::OFF_A;
    float* sAcc = smem + dfw::OFF_ACC;
    __shared__ float red[dfw::THREADS / 32];

    const int tid = threadIdx.x;
    const int b = blockIdx.z;
    const int H = args.H, W = args.W, M = args.M;
    const size_t HW = (size_t)H * W;
    const int tx0 = blockIdx.x * dfw::TW, ty0 = blockIdx.y * dfw::TH;
    const float* __restrict__ z = args.z.p[b];
    const float* __restrict__ r = args.r.p[b];
    const float* __restrict__ a = DEMOD ? args.a.p[b] : nullptr;
    const float eps = args.eps;

    // Demodulated irradiance y = r / (a + eps) on tile + halo (0 outside the image);
    // every load of the phase is issued before any is used.
    {
        constexpr int NREG = dfw::RH * dfw::RW;
        constexpr int PER = (NREG + dfw::THREADS - 1) / dfw::THREADS;
        float rv[PER][3], av[PER][3];
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const int t = tid + j * dfw::THREADS;
            const int gy = ty0 - dfw::HALO + t / dfw::RW, gx = tx0 - dfw::HALO + t % dfw::RW;
            const bool in = t < NREG && gy >= 0 && gy < H && gx >= 0 && gx < W;
            const size_t g = in ? (size_t)gy * W + gx : 0;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                rv[j][ch] = in ? __ldg(r + ch * HW + g) : 0.f;
                av[j][ch] = in && DEMOD ? __ldg(a + ch * HW + g) : 1.f - eps;
            }
        }
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const int t = tid + j * dfw::THREADS;
            if (PER * dfw::THREADS > NREG && t >= NREG) continue;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) sY[ch * NREG + t] = DEMOD ? rv[j][ch] / (av[j][ch] + eps) : rv[j][ch];
        }
    }

    // Fusion weights alpha_i(p) = softmax_i of the M fusion logits (Eq. 5),
    // once per own pixel, into shared memory [i][TH][TW].
    const int x = tid % dfw::TW, rg = tid / dfw::TW;
    const int gx = tx0 + x;
#pragma unroll
    for (int j = 0; j < dfw::RPT; ++j) {
        const int ly = rg * dfw::RPT + j, gy = ty0 + ly;
        if (gy >= H || gx >= W) continue;
        const size_t g = (size_t)gy * W + gx;
        float l[dfw::MAXK];
        float m = -INFINITY;
#pragma unroll
        for (int i = 0; i < dfw::MAXK; ++i) {
            l[i] = i < M ? __ldg(z + (size_t)(M + i) * HW + g) : -INFINITY;
            m = fmaxf(m, l[i]);
        }
        float sum = 0.f;
#pragma unroll
        for (int i = 0; i < dfw::MAXK; ++i) {
            l[i] = i < M ? expf(l[i] - m) : 0.f;
            sum += l[i];
        }
        const float inv = 1.f / sum;
#pragma unroll
        for (int i = 0; i < dfw::MAXK; ++i)
            if (i < M) sAl[(i * dfw::TH + ly) * dfw::TW + x] = l[i] * inv;
    }
#pragma unroll
    for (int j = 0; j < dfw::RPT * 3; ++j) sAcc[j * dfw::THREADS + tid] = 0.f;
    __syncthreads();

    for (int i = 0; i < M; ++i) {
        const float* __restrict__ zi = z + (size_t)i * HW;
        const float* __restrict__ al = sAl + i * dfw::TH * dfw::TW;
#define WSKPN_FWD_SIZE(K_) \
    case K_: fwd_size<K_>(sE, sH, sY, al, red, zi, r, a, H, W, tx0, ty0, tid, eps, args.fallbacks, sAcc); break;
        switch (args.ks[i]) {
            WSKPN_FWD_SIZE(1) WSKPN_FWD_SIZE(3) WSKPN_FWD_SIZE(5) WSKPN_FWD_SIZE(7) WSKPN_FWD_SIZE(9)
            WSKPN_FWD_SIZE(11)
            default: fwd_size<13>(sE, sH, sY, al, red, zi, r, a, H, W, tx0, ty0, tid, eps, args.fallbacks, sAcc);
        }
#undef WSKPN_FWD_SIZE
    }

    // Re-modulation and store.
    float* __restrict__ out = args.out.p[b];
#pragma unroll
    for (int j = 0; j < dfw::RPT; ++j) {
        const int gy = ty0 + rg * dfw::RPT + j;
        if (gy >= H || gx >= W) continue;
        const size_t g = (size_t)gy * W + gx;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch)
            out[ch * HW + g] = (DEMOD ? __ldg(a + ch * HW + g) + eps : 1.f) * sAcc[(j * 3 + ch) * dfw::THREADS + tid];
    }
}

// Host launcher: z/r/a/out given per frame.
wskpn_status launch_decode_fuse_fwd(const float* const* z, const float* const* r,
                                    const float* const* a, float* const* out, int B, int H, int W,
                                    int M, const int* ks, float eps, unsigned int* fallbacks,
                                    cudaStream_t st, std::string& err) {
    WSKPN_CUDA_TRY(cudaFuncSetAttribute(decode_fuse_fwd_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)dfw::SMEM_BYTES),
                   err);
    WSKPN_CUDA_TRY(cudaFuncSetAttribute(decode_fuse_fwd_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)dfw::SMEM_BYTES),
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
        dim3 grid(cdiv(W, dfw::TW), cdiv(H, dfw::TH), nb);
        if (a[b0])  // every frame of a call either has an albedo or none
            decode_fuse_fwd_kernel<true><<<grid, dfw::THREADS, dfw::SMEM_BYTES, st>>>(args);
        else
            decode_fuse_fwd_kernel<false><<<grid, dfw::THREADS, dfw::SMEM_BYTES, st>>>(args);
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
// Scratch layout per frame: planes [LSE_0..M-1, hR_0..M-1,
// h_{0,0..2}, ..., h_{M-1,0..2}, (3 unused)] = 5M + 3 planes of H x W, with
// h_ic = alpha_i g_c and hR_i = sum_c h_ic R_ic: kernel 2 reads four
// planes per footprint pixel besides LSE.
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
            float al = 0.f;  // alpha_i of this pixel (registers indexed by constants only)
#pragma unroll
            for (int q = 0; q < WSKPN_MAX_KERNELS; ++q)
                if (q == i) al = alpha[j][q];
            sc[(size_t)i * HW + g] = L;
            float hR = 0.f;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float hc = al * gc[j][c];
                sc[(size_t)(2 * M + 3 * i + c) * HW + g] = hc;
                hR += hc * R[c];
            }
            sc[(size_t)(M + i) * HW + g] = hR;
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
        const float* __restrict__ HRi = sc + (size_t)(M + i) * HW;
        const float* __restrict__ Hi = sc + (size_t)(2 * M + 3 * i) * HW;
        // footprint minimum and maximum of LSE; the footprint's LSE values
        // stay in registers for the plane pass (all loads issued first)
        constexpr int FPER = ((df::TH + 2 * df::HALO) * (df::TW + 2 * df::HALO) + df::THREADS - 1) / df::THREADS;
        float lv[FPER];
        float mn = INFINITY, mx = -INFINITY;
#pragma unroll
        for (int u = 0; u < FPER; ++u) {
            const int t = tid + u * df::THREADS;
            const int gy = ty0 - h + t / nc, gx = tx0 - h + t % nc;
            const bool in = t < nr * nc && gy >= 0 && gy < H && gx >= 0 && gx < W;
            lv[u] = in ? Li[(size_t)gy * W + gx] : 0.f;
            if (in) {
                mn = fminf(mn, lv[u]);
                mx = fmaxf(mx, lv[u]);
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
#pragma unroll
            for (int u = 0; u < FPER; ++u) {
                const int t = tid + u * df::THREADS;
                if (t >= nr * nc) break;
                const int ry = df::HALO - h + t / nc, rx = df::HALO - h + t % nc;
                const int gy = ty0 - df::HALO + ry, gx = tx0 - df::HALO + rx;
                const int o = ry * df::RP + rx;
                float v0 = 0.f, v1 = 0.f, v2 = 0.f, v3 = 0.f;
                if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
                    const size_t g = (size_t)gy * W + gx;
                    const float e = expf(mn - lv[u]);
                    v0 = e * Hi[g];
                    v1 = e * Hi[HW + g];
                    v2 = e * Hi[2 * HW + g];
                    v3 = e * HRi[g];
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
                        float t = -HRi[gp];
#pragma unroll
                        for (int c = 0; c < 3; ++c) t += Hi[c * HW + gp] * yq[j][c];
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
