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
__device__ __forceinline__ void window_exact_inl(const float* __restrict__ z, const float* __restrict__ r,
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

__device__ __noinline__ void window_exact(const float* __restrict__ z, const float* __restrict__ r,
                                          const float* __restrict__ a, int H, int W, int k, float eps, int px, int py,
                                          float R[3]) {
    window_exact_inl(z, r, a, H, W, k, eps, px, py, R);
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
//
// Organisation (64 x 32 output tiles, 256 threads, two CTAs per SM):
//  * set-up: the radiance and albedo of the tile's 44 x 80 footprint (rows
//    -6..37, columns -8..71 around the tile) are staged by cp.async while
//    the fusion logits load, and the demodulated irradiance y = r / (a + eps)
//    (0 outside the image) is formed in place as three planes;
//    each horizontal-pass thread keeps, for its 8 pixels, the maximum c of
//    their fusion logits (the shift of Eq. 5's softmax) in registers;
//  * per window size K (two block barriers):
//      - the importance map I_i of the footprint was staged in shared
//        memory by cp.async during the previous size's phase (two buffers),
//        and its maximum m_i (the exponent shift, over the whole staged
//        block) reduced at the end of that phase;
//      - vertical pass, one task per (footprint column, half tile): the
//        thread walks 16 + K - 1 rows, forms E = exp(I - m_i) once per
//        element, (E y0, E) and (E y1, E y2), and keeps their K-row window
//        sums as streaming binary-digit partial sums in registers;
//      - horizontal pass, one task per (row, 8 pixels): K-column sums of
//        (E y0, E), giving w = exp(l_i - c) / D_i (the fusion logits l_i
//        were loaded into registers one phase ahead), acc0 += w N0 and
//        S += w D (= exp(l_i - c)); then of (E y1, E y2): acc1 += w N1,
//        acc2 += w N2;
//  * out = (a + eps) acc / S, with the tile's albedo staged by cp.async
//    into the y planes during the last horizontal pass.
// The exponent shift cancels in N/D for every window; a pixel whose D_i
// falls below 1e-30 is recomputed exactly (window_exact) and counted.
namespace dfv {
constexpr int TW = 64;                  // tile width (output pixels)
constexpr int TH = 32;                  // tile height
constexpr int HALO = 6;                 // largest half window (k = 13)
constexpr int XOFF = 8;                 // staged columns start 8 left of the tile (16-byte aligned)
constexpr int FW = TW + 2 * XOFF;       // 80 staged columns
constexpr int FH = TH + 2 * HALO;       // 44 staged rows
constexpr int NCH = FH * FW / 4;        // 880 four-column chunks
constexpr int THREADS = 256;
constexpr int NWARP = THREADS / 32;
constexpr int RV = TH / 2;              // vertical-pass output rows per task
constexpr int SEG = 8;                  // horizontal-pass output pixels per task
constexpr int VP = TW + 2 * HALO + 1;   // 77: pitch of the window-sum planes in float2 (odd: conflict-free)
constexpr int LP = TW + 4;              // 68: pitch of the per-pixel planes (16-byte aligned rows)
constexpr int CPT = (NCH + THREADS - 1) / THREADS;  // chunks per thread (4)
static_assert(TH == 32 && TW / SEG == NWARP, "horizontal pass: lane = row, warp = segment");
static_assert(2 * (TW + 2 * HALO) < THREADS, "vertical pass: one task per thread, some threads idle");
constexpr size_t PLANE = sizeof(float) * FH * FW;                // one staged [FH][FW] plane (14,080 B)
constexpr size_t OFF_Y = 0;                                       // float [3][FH][FW]: y0, y1, y2
constexpr size_t OFF_Z = OFF_Y + 3 * PLANE;                      // float [2][FH][FW]: I_i, I_{i+1}
constexpr size_t OFF_V = OFF_Z + 2 * PLANE;                      // float2 [2][TH][VP]: (N0, D) | (N1, N2)
constexpr size_t OFF_R = OFF_V + sizeof(float2) * 2 * TH * VP;   // int [2]: shifts of sizes i, i + 1
constexpr size_t SMEM_BYTES = OFF_R + sizeof(int) * 4;
// set-up: the radiance footprint is staged in the second z buffer and the
// window-sum planes (idle until the first size), the albedo footprint in
// the y planes, where y = r / (a + eps) then replaces it element by element
constexpr size_t OFF_RSTAGE = OFF_Z + PLANE;
static_assert(OFF_RSTAGE + 3 * PLANE <= OFF_R, "staged radiance fits before the shifts");
static_assert(OFF_V % 16 == 0 && OFF_Z % 16 == 0 && PLANE % 16 == 0, "16-byte aligned planes");
static_assert(3 * TH * LP * sizeof(float) <= 2 * PLANE, "staged albedo fits the y1, y2 planes");
static_assert(2 * (SMEM_BYTES + 1024) <= 228 * 1024, "two CTAs per SM");
constexpr float LOG2E = 1.4426950408889634f;
}  // namespace dfv

// 2^x with the SFU's approximate exponential (flushes subnormal results to
// 0).  exp(t) is formed as 2^(t log2 e); the caller folds the constant
// shift into one FMA, so only the product's final rounding enters.
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Order-preserving map between float and int (so integer max reductions
// give the float maximum; -inf maps below every finite value).
__device__ __forceinline__ int f2ord(float f) {
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float ord2f(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(sdst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(__cvta_generic_to_global(gsrc))
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void* sdst, const void* gsrc) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(sdst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(__cvta_generic_to_global(gsrc))
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Window sums s[y] = sum_{d < K} w[y + d] of NP float pairs, y < NOUT,
// streamed in input order: in(j, w) yields input j of every pair,
// out(y, s) takes output y as soon as its last input has arrived.  Sums of
// 2, 4 and 8 consecutive inputs are formed once; a window is assembled
// from the binary digits of K (all terms of one sign: no cancellation).
// Every array index is a compile-time constant, so the arrays live in
// registers and entries no output needs are never computed; at step j only
// the partial sums later outputs still need are live (about 16 pairs per
// plane pair for K = 13).
template <int K, int NOUT, int NP, typename In, typename Out>
__device__ __forceinline__ void box_stream(In in, Out out) {
    constexpr int N1 = NOUT + K - 1;
    constexpr int B8 = K & 8, B4 = K & 4, B2 = K & 2, B1 = K & 1;
    constexpr int O4 = B8, O2 = B8 + B4, O1 = B8 + B4 + B2;
    static_assert(K >= 1 && K <= 15, "window");
    float2 w[N1][NP], p2[N1][NP], p4[N1][NP], p8[N1][NP];
#pragma unroll
    for (int j = 0; j < N1; ++j) {
        in(j, w[j]);
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            if (j >= 1) p2[j - 1][q] = __fadd2_rn(w[j - 1][q], w[j][q]);
            if (j >= 3) p4[j - 3][q] = __fadd2_rn(p2[j - 3][q], p2[j - 1][q]);
            if (j >= 7) p8[j - 7][q] = __fadd2_rn(p4[j - 7][q], p4[j - 3][q]);
        }
        const int y = j - (K - 1);
        if (y >= 0) {
            float2 t[NP];
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                bool set = false;
                if constexpr (B8 != 0) {
                    t[q] = p8[y][q];
                    set = true;
                }
                if constexpr (B4 != 0) {
                    t[q] = set ? __fadd2_rn(t[q], p4[y + O4][q]) : p4[y + O4][q];
                    set = true;
                }
                if constexpr (B2 != 0) {
                    t[q] = set ? __fadd2_rn(t[q], p2[y + O2][q]) : p2[y + O2][q];
                    set = true;
                }
                if constexpr (B1 != 0) t[q] = set ? __fadd2_rn(t[q], w[y + O1][q]) : w[y + O1][q];
            }
            out(y, t);
        }
    }
}

// Stage one logit plane's footprint block [FH][FW] into sZ (cp.async;
// -inf outside the image) and return the maximum of what this thread
// staged once its copies have landed (call finish_stage for that).
template <bool VEC>
__device__ __forceinline__ void stage_plane(float* __restrict__ sZ, const float* __restrict__ zi, int H, int W,
                                            int tx0, int ty0, int tid) {
    if constexpr (VEC) {
#pragma unroll
        for (int u = 0; u < dfv::CPT; ++u) {
            const int c = tid + u * dfv::THREADS;
            if (dfv::CPT * dfv::THREADS > dfv::NCH && c >= dfv::NCH) break;
            const int row = c / (dfv::FW / 4), c4 = c % (dfv::FW / 4);
            const int gy = ty0 - dfv::HALO + row, gx = tx0 - dfv::XOFF + 4 * c4;
            float* dst = sZ + row * dfv::FW + 4 * c4;
            if (gy >= 0 && gy < H && gx >= 0 && gx < W)  // W % 4 == 0: a chunk is wholly in or out
                cp_async16(dst, zi + (size_t)gy * W + gx);
            else
                *reinterpret_cast<float4*>(dst) = make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY);
        }
    } else {
        for (int e = tid; e < dfv::FH * dfv::FW; e += dfv::THREADS) {
            const int row = e / dfv::FW, col = e % dfv::FW;
            const int gy = ty0 - dfv::HALO + row, gx = tx0 - dfv::XOFF + col;
            if (gy >= 0 && gy < H && gx >= 0 && gx < W)
                cp_async4(sZ + e, zi + (size_t)gy * W + gx);
            else
                sZ[e] = -INFINITY;
        }
    }
    cp_async_commit();
}

// Wait for this thread's copies, take the maximum of the elements it
// staged and fold the warp's maximum into *red (order-preserving int).
template <bool VEC>
__device__ __forceinline__ void finish_stage(const float* __restrict__ sZ, int* __restrict__ red, int tid) {
    cp_async_wait_all();
    float m = -INFINITY;
    if constexpr (VEC) {
#pragma unroll
        for (int u = 0; u < dfv::CPT; ++u) {
            const int c = tid + u * dfv::THREADS;
            if (dfv::CPT * dfv::THREADS > dfv::NCH && c >= dfv::NCH) break;
            const float4 v = reinterpret_cast<const float4*>(sZ)[c];
            m = fmaxf(m, fmaxf(fmaxf(v.x, v.y), fmaxf(v.z, v.w)));
        }
    } else {
        for (int e = tid; e < dfv::FH * dfv::FW; e += dfv::THREADS) m = fmaxf(m, sZ[e]);
    }
    const int w = __reduce_max_sync(0xffffffffu, f2ord(m));
    if ((tid & 31) == 0) atomicMax(red, w);
}

// The fusion logits of one row's 8 consecutive pixels (0 outside the image).
template <bool VEC>
__device__ __forceinline__ void load_fusion_logits(float (&l)[dfv::SEG], const float* __restrict__ zl, int H, int W,
                                                   int gy, int gx0) {
    if (VEC && gy < H && gx0 + dfv::SEG <= W) {
        const float4* p = reinterpret_cast<const float4*>(zl + (size_t)gy * W + gx0);
        const float4 u = __ldg(p), v = __ldg(p + 1);
        l[0] = u.x, l[1] = u.y, l[2] = u.z, l[3] = u.w, l[4] = v.x, l[5] = v.y, l[6] = v.z, l[7] = v.w;
    } else {
#pragma unroll
        for (int x = 0; x < dfv::SEG; ++x)
            l[x] = (gy < H && gx0 + x < W) ? __ldg(zl + (size_t)gy * W + gx0 + x) : 0.f;
    }
}
// Vertical pass of size K: task (half, col), t < 2 (64 + K - 1), walks
// footprint column col (image column tx0 - h + col) over rows
// 16 half - h .. 16 half + 15 + h of the tile, forming E once per element,
// and writes the 16 K-row sums of (E y0, E) to sVA and of (E y1, E y2) to
// sVB at [16 half + r][col].  sY holds the planes y0, y1, y2.
template <int K>
__device__ __forceinline__ void fwd_vpass(const float* __restrict__ sZ, const float* __restrict__ sY,
                                          float2* __restrict__ sVA, float2* __restrict__ sVB, float ml2e, int t) {
    constexpr int h = K / 2, NCOL = dfv::TW + 2 * h;
    constexpr int PL = dfv::FH * dfv::FW;
    const int half = t >= NCOL ? 1 : 0;
    const int col = t - half * NCOL;
    const int o = (dfv::HALO + dfv::RV * half - h) * dfv::FW + dfv::XOFF - h + col;
    const int v = dfv::RV * half * dfv::VP + col;
    box_stream<K, dfv::RV, 2>(
        [&](int j, float2(&w)[2]) {
            const int q = o + j * dfv::FW;
            const float e = ex2_approx(fmaf(sZ[q], dfv::LOG2E, -ml2e));
            w[0] = make_float2(e * sY[q], e);
            w[1] = __fmul2_rn(make_float2(e, e), make_float2(sY[PL + q], sY[2 * PL + q]));
        },
        [&](int y, const float2(&s)[2]) {
            sVA[v + y * dfv::VP] = s[0];
            sVB[v + y * dfv::VP] = s[1];
        });
}

// Per-thread state of the horizontal-pass task (row, 8 pixels) across the
// sizes i: acc_c = sum_i w_i N_ic and S = sum_i w_i D_i = sum_i exp(l_i - c)
// with w_i = exp(l_i - c) / D_i; cl = c log2(e) (c = max_i l_i) and l, the
// fusion logits of the size being processed (loaded one phase ahead).
struct HState {
    float acc[dfv::SEG][3];
    float S[dfv::SEG];
    float cl[dfv::SEG];
    float l[dfv::SEG];
};

// Horizontal pass of size K for the thread's row and 8-pixel segment.
// Returns the mask of pixels whose D underflowed (their exact evaluation
// is deferred to the end of the kernel, out of the unrolled code).
template <int K>
__device__ __forceinline__ unsigned fwd_hpass(const float2* __restrict__ sVA, const float2* __restrict__ sVB,
                                              HState& st, int row, int seg) {
    const int v = row * dfv::VP + seg * dfv::SEG;
    float w[dfv::SEG];
    bool bad = false;
    box_stream<K, dfv::SEG, 1>([&](int j, float2(&in)[1]) { in[0] = sVA[v + j]; },
                               [&](int x, const float2(&t)[1]) {
                                   const float D = t[0].y;
                                   const bool ok = D >= df::DMIN;
                                   bad |= !ok;
                                   const float e = ex2_approx(fmaf(st.l[x], dfv::LOG2E, -st.cl[x]));
                                   w[x] = ok ? e * __fdividef(1.f, D) : 0.f;
                                   st.acc[x][0] = fmaf(w[x], t[0].x, st.acc[x][0]);
                                   st.S[x] = fmaf(w[x], D, st.S[x]);
                               });
    box_stream<K, dfv::SEG, 1>([&](int j, float2(&in)[1]) { in[0] = sVB[v + j]; },
                               [&](int x, const float2(&t)[1]) {
                                   st.acc[x][1] = fmaf(w[x], t[0].x, st.acc[x][1]);
                                   st.acc[x][2] = fmaf(w[x], t[0].y, st.acc[x][2]);
                               });
    unsigned exact = 0;
    if (bad) {  // rare: find the pixels again
#pragma unroll 1
        for (int x = 0; x < dfv::SEG; ++x) {
            float D = 0.f;
#pragma unroll 1
            for (int j = 0; j < K; ++j) D += sVA[v + x + j].y;
            if (!(D >= df::DMIN)) exact |= 1u << x;
        }
    }
    return exact;
}

// The tile's albedo [3][TH][TW] into sA [3][TH][LP] (cp.async, 16-byte
// chunks; chunks outside the image are not copied and never used).
__device__ __forceinline__ void stage_albedo(float* __restrict__ sA, const float* __restrict__ a, int H, int W,
                                             int tx0, int ty0, int tid) {
    const size_t HW = (size_t)H * W;
    constexpr int NC = 3 * dfv::TH * (dfv::TW / 4);
#pragma unroll
    for (int c = tid; c < NC; c += dfv::THREADS) {
        const int ch = c / (dfv::TH * dfv::TW / 4), rc = c % (dfv::TH * dfv::TW / 4);
        const int row = rc / (dfv::TW / 4), c4 = rc % (dfv::TW / 4);
        const int gy = ty0 + row, gx = tx0 + 4 * c4;
        if (gy < H && gx < W) cp_async16(sA + (ch * dfv::TH + row) * dfv::LP + 4 * c4, a + ch * HW + (size_t)gy * W + gx);
    }
    cp_async_commit();
}

// One window size K.  Phase layout: I_{i+1} is staged into the other z
// buffer at the start (it has the whole phase to land); the vertical pass
// reads I_i; after the barrier the horizontal pass consumes this size's
// fusion logits, the next size's are loaded, and the next shift is reduced.
template <int K, bool VEC>
__device__ __forceinline__ unsigned fwd_size(const float* __restrict__ sZcur, float* __restrict__ sZnext,
                                             float* __restrict__ sY, float2* __restrict__ sVA,
                                             float2* __restrict__ sVB,
                                             int* __restrict__ red, int* __restrict__ red_next, HState& st,
                                             const float* __restrict__ znext, const float* __restrict__ zlnext,
                                             const float* __restrict__ a_stage, int H, int W, int tx0, int ty0,
                                             int tid) {
    constexpr int NCOL = dfv::TW + 2 * (K / 2);
    const float ml2e = ord2f(*red) * dfv::LOG2E;
    if (tid == 0) *red_next = INT_MIN;  // its last reader finished before the previous barrier
    if (znext) stage_plane<VEC>(sZnext, znext, H, W, tx0, ty0, tid);
    if (tid < 2 * NCOL) fwd_vpass<K>(sZcur, sY, sVA, sVB, ml2e, tid);
    __syncthreads();
    // after the last vertical pass the y planes are free: the albedo of the
    // re-modulation is staged in the y1, y2 planes while the horizontal pass runs
    if (a_stage) stage_albedo(sY + dfv::FH * dfv::FW, a_stage, H, W, tx0, ty0, tid);
    const int row = tid & 31, seg = tid >> 5;
    const unsigned exact = fwd_hpass<K>(sVA, sVB, st, row, seg);
    if (zlnext) load_fusion_logits<VEC>(st.l, zlnext, H, W, ty0 + row, tx0 + seg * dfv::SEG);
    if (znext) finish_stage<VEC>(sZnext, red_next, tid);
    if (a_stage) cp_async_wait_all();
    __syncthreads();
    return exact;
}

template <bool DEMOD, bool VEC>
__global__ void __launch_bounds__(dfv::THREADS, 2) decode_fuse_fwd_kernel(const __grid_constant__ DecodeArgs args) {
    extern __shared__ float4 dsm4[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(dsm4);
    float* sY = reinterpret_cast<float*>(smem + dfv::OFF_Y);
    float* sRst = reinterpret_cast<float*>(smem + dfv::OFF_RSTAGE);
    float* sZ = reinterpret_cast<float*>(smem + dfv::OFF_Z);
    float2* sVA = reinterpret_cast<float2*>(smem + dfv::OFF_V);
    float2* sVB = sVA + dfv::TH * dfv::VP;
    int* red = reinterpret_cast<int*>(smem + dfv::OFF_R);

    const int tid = threadIdx.x;
    const int b = blockIdx.z;
    const int H = args.H, W = args.W, M = args.M;
    const size_t HW = (size_t)H * W;
    const int tx0 = blockIdx.x * dfv::TW, ty0 = blockIdx.y * dfv::TH;
    const float* __restrict__ z = args.z.p[b];
    const float* __restrict__ r = args.r.p[b];
    const float* __restrict__ a = DEMOD ? args.a.p[b] : nullptr;
    const float eps = args.eps;
    const int row = tid & 31, seg = tid >> 5;
    const int gy = ty0 + row, gx0 = tx0 + seg * dfv::SEG;

    // Set-up, with every DRAM read in flight at once: the first importance
    // map's footprint into sZ[0]; the radiance and albedo footprints by
    // cp.async (the radiance into space idle until the first size, the
    // albedo into the y planes); the fusion logits of the thread's own
    // pixels into registers.
    constexpr int PL = dfv::FH * dfv::FW;
    if (tid == 0) red[0] = INT_MIN;
    stage_plane<VEC>(sZ, z, H, W, tx0, ty0, tid);
    {
        // chunk (VEC: 4 columns, else 1 element) c of plane ch: image rows and
        // columns outside the frame are written as 0 (y = 0 there)
        float* rdst = DEMOD ? sRst : sY;
        if constexpr (VEC) {
#pragma unroll
            for (int u = 0; u < dfv::CPT; ++u) {
                const int c = tid + u * dfv::THREADS;
                if (dfv::CPT * dfv::THREADS > dfv::NCH && c >= dfv::NCH) break;
                const int cr = c / (dfv::FW / 4), c4 = c % (dfv::FW / 4);
                const int yy = ty0 - dfv::HALO + cr, xx = tx0 - dfv::XOFF + 4 * c4;
                const bool in = yy >= 0 && yy < H && xx >= 0 && xx < W;
                const size_t g = (size_t)yy * W + xx;
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    float* dr = rdst + ch * PL + 4 * c;
                    float* da = sY + ch * PL + 4 * c;
                    if (in) {
                        cp_async16(dr, r + ch * HW + g);
                        if (DEMOD) cp_async16(da, a + ch * HW + g);
                    } else {
                        *reinterpret_cast<float4*>(dr) = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (DEMOD) *reinterpret_cast<float4*>(da) = make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
            }
        } else {
            for (int e = tid; e < PL; e += dfv::THREADS) {
                const int er = e / dfv::FW, ec = e % dfv::FW;
                const int yy = ty0 - dfv::HALO + er, xx = tx0 - dfv::XOFF + ec;
                const bool in = yy >= 0 && yy < H && xx >= 0 && xx < W;
                const size_t g = (size_t)yy * W + xx;
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    if (in) {
                        cp_async4(rdst + ch * PL + e, r + ch * HW + g);
                        if (DEMOD) cp_async4(sY + ch * PL + e, a + ch * HW + g);
                    } else {
                        rdst[ch * PL + e] = 0.f;
                        if (DEMOD) sY[ch * PL + e] = 0.f;
                    }
                }
            }
        }
        cp_async_commit();
    }
    __syncthreads();  // red[0] initialised before any thread folds its maximum in

    // Shift of the fusion softmax per own pixel (Eq. 5): c = max_i l_i (all
    // loads issued at once, while the copies above are in flight); the first
    // size's logits stay in st.l.
    HState st;
    {
        float l[WSKPN_MAX_KERNELS][dfv::SEG];
#pragma unroll
        for (int i = 0; i < WSKPN_MAX_KERNELS; ++i)
            if (i < M) load_fusion_logits<VEC>(l[i], z + (size_t)(M + i) * HW, H, W, gy, gx0);
#pragma unroll
        for (int x = 0; x < dfv::SEG; ++x) {
            float c = l[0][x];
#pragma unroll
            for (int i = 1; i < WSKPN_MAX_KERNELS; ++i)
                if (i < M) c = fmaxf(c, l[i][x]);
            st.cl[x] = c * dfv::LOG2E;
            st.l[x] = l[0][x];
            st.acc[x][0] = st.acc[x][1] = st.acc[x][2] = st.S[x] = 0.f;
        }
    }

    // Demodulated irradiance y = r / (a + eps), in place of the albedo: each
    // thread converts exactly the elements it staged, after its own copies
    // landed (outside the frame r = a = 0, so y = 0).
    cp_async_wait_all();
    if constexpr (DEMOD) {
        if constexpr (VEC) {
#pragma unroll
            for (int u = 0; u < dfv::CPT; ++u) {
                const int c = tid + u * dfv::THREADS;
                if (dfv::CPT * dfv::THREADS > dfv::NCH && c >= dfv::NCH) break;
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    const float4 rv = reinterpret_cast<const float4*>(sRst + ch * PL)[c];
                    float4& yv = reinterpret_cast<float4*>(sY + ch * PL)[c];
                    const float4 av = yv;
                    yv = make_float4(__fdividef(rv.x, av.x + eps), __fdividef(rv.y, av.y + eps),
                                     __fdividef(rv.z, av.z + eps), __fdividef(rv.w, av.w + eps));
                }
            }
        } else {
            for (int e = tid; e < PL; e += dfv::THREADS)
#pragma unroll
                for (int ch = 0; ch < 3; ++ch)
                    sY[ch * PL + e] = __fdividef(sRst[ch * PL + e], sY[ch * PL + e] + eps);
        }
    }

    finish_stage<VEC>(sZ, red, tid);
    __syncthreads();

    unsigned long long exact = 0;  // bit 8 i + x: pixel x's D_i underflowed
    for (int i = 0; i < M; ++i) {
        const bool more = i + 1 < M;
        const float* znext = more ? z + (size_t)(i + 1) * HW : nullptr;
        const float* zlnext = more ? z + (size_t)(M + i + 1) * HW : nullptr;
        float* zc = sZ + (i & 1) * dfv::FH * dfv::FW;
        float* zn = sZ + ((i + 1) & 1) * dfv::FH * dfv::FW;
        int* rd = red + (i & 1);
        int* rn = red + ((i + 1) & 1);
        const float* astage = DEMOD && VEC && i + 1 == M ? a : nullptr;
        unsigned ex = 0;
#define WSKPN_FWD_SIZE(K_)                                                                                      \
    case K_:                                                                                                    \
        ex = fwd_size<K_, VEC>(zc, zn, sY, sVA, sVB, rd, rn, st, znext, zlnext, astage, H, W, tx0, ty0, tid); \
        break;
        switch (args.ks[i]) {
            WSKPN_FWD_SIZE(1) WSKPN_FWD_SIZE(3) WSKPN_FWD_SIZE(5) WSKPN_FWD_SIZE(7) WSKPN_FWD_SIZE(9)
            WSKPN_FWD_SIZE(11) WSKPN_FWD_SIZE(13)
        }
#undef WSKPN_FWD_SIZE
        exact |= (unsigned long long)ex << (8 * i);
    }

    // Pixels whose window sum underflowed for some size: exact per-window
    // evaluation (rare); that size contributed nothing on the fast path.
    if (exact) {
#pragma unroll 1
        for (int i = 0; i < M; ++i) {
#pragma unroll 1
            for (int x = 0; x < dfv::SEG; ++x) {
                if (!((exact >> (8 * i + x)) & 1ull) || gy >= H || gx0 + x >= W) continue;  // outside: never stored
                float R[3];
                window_exact_inl(z + (size_t)i * HW, r, a, H, W, args.ks[i], eps, gx0 + x, gy, R);
                if (args.fallbacks) atomicAdd(args.fallbacks, 1u);
                const float l = __ldg(z + (size_t)(M + i) * HW + (size_t)gy * W + gx0 + x);
#pragma unroll
                for (int q = 0; q < dfv::SEG; ++q)
                    if (q == x) {
                        const float e = ex2_approx(fmaf(l, dfv::LOG2E, -st.cl[q]));
                        st.acc[q][0] = fmaf(e, R[0], st.acc[q][0]);
                        st.acc[q][1] = fmaf(e, R[1], st.acc[q][1]);
                        st.acc[q][2] = fmaf(e, R[2], st.acc[q][2]);
                        st.S[q] += e;
                    }
            }
        }
    }

    // Re-modulation and store: out = (a + eps) acc / S.
    float* __restrict__ out = args.out.p[b];
    if (gy >= H) return;
    float inv[dfv::SEG];
#pragma unroll
    for (int x = 0; x < dfv::SEG; ++x) inv[x] = __fdividef(1.f, st.S[x]);
    const size_t g0 = (size_t)gy * W + gx0;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        float o[dfv::SEG];
#pragma unroll
        for (int x = 0; x < dfv::SEG; ++x) o[x] = st.acc[x][ch] * inv[x];
        if (VEC && gx0 + dfv::SEG <= W) {
            if constexpr (DEMOD) {
                const float4* pa = reinterpret_cast<const float4*>(sY + PL + (ch * dfv::TH + row) * dfv::LP +
                                                                   seg * dfv::SEG);
                const float4 u = pa[0], v = pa[1];
                const float m[dfv::SEG] = {u.x, u.y, u.z, u.w, v.x, v.y, v.z, v.w};
#pragma unroll
                for (int x = 0; x < dfv::SEG; ++x) o[x] *= m[x] + eps;
            }
            float4* po = reinterpret_cast<float4*>(out + ch * HW + g0);
            po[0] = make_float4(o[0], o[1], o[2], o[3]);
            po[1] = make_float4(o[4], o[5], o[6], o[7]);
        } else {
#pragma unroll
            for (int x = 0; x < dfv::SEG; ++x) {
                if (gx0 + x >= W) break;
                out[ch * HW + g0 + x] = (DEMOD ? __ldg(a + ch * HW + g0 + x) + eps : 1.f) * o[x];
            }
        }
    }
}

template <bool DEMOD, bool VEC>
static wskpn_status launch_fwd_variant(const DecodeArgs& args, int nb, cudaStream_t st, std::string& err) {
    WSKPN_CUDA_TRY(cudaFuncSetAttribute(decode_fuse_fwd_kernel<DEMOD, VEC>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dfv::SMEM_BYTES),
                   err);
    dim3 grid(cdiv(args.W, dfv::TW), cdiv(args.H, dfv::TH), nb);
    decode_fuse_fwd_kernel<DEMOD, VEC><<<grid, dfv::THREADS, dfv::SMEM_BYTES, st>>>(args);
    WSKPN_CUDA_TRY(cudaGetLastError(), err);
    return WSKPN_OK;
}

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// Host launcher: z/r/a/out given per frame.  The vectorised variant (16-byte
// loads, stores and copies) runs when W is a multiple of 4 and every plane
// pointer is 16-byte aligned, so that each 4-pixel chunk of a row lies
// wholly inside or outside the image.
wskpn_status launch_decode_fuse_fwd(const float* const* z, const float* const* r,
                                    const float* const* a, float* const* out, int B, int H, int W,
                                    int M, const int* ks, float eps, unsigned int* fallbacks,
                                    cudaStream_t st, std::string& err) {
    for (int b0 = 0; b0 < B; b0 += WSKPN_MAX_BATCH) {
        const int nb = B - b0 < WSKPN_MAX_BATCH ? B - b0 : WSKPN_MAX_BATCH;
        DecodeArgs args{};
        bool vec = W % 4 == 0;
        for (int j = 0; j < nb; ++j) {
            args.z.p[j] = z[b0 + j];
            args.r.p[j] = r[b0 + j];
            args.a.p[j] = a[b0 + j];
            args.out.p[j] = out[b0 + j];
            vec = vec && aligned16(z[b0 + j]) && aligned16(r[b0 + j]) && aligned16(out[b0 + j]) &&
                  (!a[b0 + j] || aligned16(a[b0 + j]));
        }
        args.H = H;
        args.W = W;
        args.M = M;
        for (int i = 0; i < M; ++i) args.ks[i] = ks[i];
        args.eps = eps;
        args.fallbacks = fallbacks;
        wskpn_status s;
        if (a[b0])  // every frame of a call either has an albedo or none
            s = vec ? launch_fwd_variant<true, true>(args, nb, st, err) : launch_fwd_variant<true, false>(args, nb, st, err);
        else
            s = vec ? launch_fwd_variant<false, true>(args, nb, st, err)
                    : launch_fwd_variant<false, false>(args, nb, st, err);
        if (s) return s;
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
