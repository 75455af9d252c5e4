// Reconstruction phase (Sec. 4.2): kernel construction from importance maps
// (Eq. 3), filtering (Eq. 4), multi-size fusion (Eq. 5) and albedo
// re-modulation, fused into one streaming kernel that never materialises the
// H x W x k^2 kernel map.
//
// Per output pixel p and size i (window Omega_i(p) clipped to the image):
//   R_i(p) = sum_q exp(I_i(q)) y(q) / sum_q exp(I_i(q)),  y = r / (a + eps)
// i.e. Eq. 3-4 written as the ratio of two window sums N_i / D_i.  The sums
// are separable box sums, evaluated from a shared-memory tile with a 6-pixel
// halo (64 x 32 output pixels per tile).  The exponent is shifted by the maximum of I_i over the tile's
// window footprint; the shift cancels in N/D for every pixel.  A pixel whose
// D_i falls below 1e-30 (the footprint's logit range exceeds ~69) is
// recomputed exactly with its own window maximum and counted.
#include "common.cuh"

namespace wskpn {

namespace df {
constexpr float DMIN = 1e-30f;  // smallest window sum D_i the fast paths divide by
}  // namespace df

struct DecodeArgs {
    PtrBatch<const float*> z, r, a;
    PtrBatch<float*> out;
    int H, W, M;
    int ks[WSKPN_MAX_KERNELS];
    float eps;
    unsigned int* fallbacks;
};

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
// 78: pitch of the window-sum planes in float2; even, so that a horizontal-
// pass row starts on 16 bytes and its inputs load in pairs; the lanes of a
// warp (rows, 624 bytes apart) then hit 8 distinct 16-byte bank groups
constexpr int VP = TW + 2 * HALO + 2;
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
static_assert(VP % 2 == 0 && SEG % 2 == 0 && (TH * VP) % 2 == 0, "paired loads of the window-sum planes");
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
__device__ __forceinline__ void box_stream(In in, Out out);

// Input of a horizontal pass: element j of a plane row starting at p (16-
// byte aligned), for j = 0, 1, 2, ... in order, two per 16-byte load.
struct PairLoader {
    const float2* p;
    float2 nxt;
    __device__ __forceinline__ void operator()(int j, float2 (&in)[1]) {
        if ((j & 1) == 0) {
            const float4 q = *reinterpret_cast<const float4*>(p + j);
            in[0] = make_float2(q.x, q.y);
            nxt = make_float2(q.z, q.w);
        } else {
            in[0] = nxt;
        }
    }
};

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

// Stage one plane's footprint block [FH][FW] into sZ (cp.async; `fill`
// outside the image, -inf for logits); finish_stage (or, in the backward,
// finish_minmax) waits for the copies and reduces what landed.
template <bool VEC>
__device__ __forceinline__ void stage_plane(float* __restrict__ sZ, const float* __restrict__ zi, int H, int W,
                                            int tx0, int ty0, int tid, float fill) {
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
                *reinterpret_cast<float4*>(dst) = make_float4(fill, fill, fill, fill);
        }
    } else {
        for (int e = tid; e < dfv::FH * dfv::FW; e += dfv::THREADS) {
            const int row = e / dfv::FW, col = e % dfv::FW;
            const int gy = ty0 - dfv::HALO + row, gx = tx0 - dfv::XOFF + col;
            if (gy >= 0 && gy < H && gx >= 0 && gx < W)
                cp_async4(sZ + e, zi + (size_t)gy * W + gx);
            else
                sZ[e] = fill;
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

// 8 consecutive pixels of one row of a plane (0 outside the image): the
// fusion logits of a horizontal-pass task, its radiance, albedo, ...
template <bool VEC>
__device__ __forceinline__ void load_row8(float (&l)[dfv::SEG], const float* __restrict__ zl, int H, int W, int gy,
                                          int gx0) {
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
// Vertical pass of size K: task (segment, col), t < 3 (64 + K - 1), walks
// footprint column col (image column tx0 - h + col) over the rows r0 - h ..
// r0 + 10 + h of the tile, r0 = 0, 11, 21 for segments 0, 1, 2 (three
// segments of 11 rows keep 3 (64 + K - 1) of the 256 threads busy, each
// walking 11 + K - 1 rows), forming E once per element, and writes the 11
// K-row sums of (E y0, E) to sVA and of (E y1, E y2) to sVB at
// [r0 + r][col] (row 21, the last of segment 1, is written by segment 1
// only).  sY holds the planes y0, y1, y2.
template <int K>
__device__ __forceinline__ void fwd_vpass(const float* __restrict__ sZ, const float* __restrict__ sY,
                                          float2* __restrict__ sVA, float2* __restrict__ sVB, float ml2e, int t) {
    constexpr int h = K / 2, NCOL = dfv::TW + 2 * h;
    constexpr int PL = dfv::FH * dfv::FW;
    constexpr int RS = 11;  // output rows per segment
    static_assert(2 * RS <= dfv::TH && dfv::TH - RS <= 2 * RS && 3 * (dfv::TW + 12) <= dfv::THREADS,
                  "three segments cover the tile rows; every task has a thread");
    const int seg = t >= 2 * NCOL ? 2 : t >= NCOL ? 1 : 0;
    const int col = t - seg * NCOL;
    const int r0 = seg == 2 ? dfv::TH - RS : seg * RS;
    const int o = (dfv::HALO + r0 - h) * dfv::FW + dfv::XOFF - h + col;
    const int v = r0 * dfv::VP + col;
    const int y_first = seg == 2 ? 2 * RS - r0 : 0;  // rows before it belong to segment 1
    box_stream<K, RS, 2>(
        [&](int j, float2(&w)[2]) {
            const int q = o + j * dfv::FW;
            const float e = ex2_approx(fmaf(sZ[q], dfv::LOG2E, -ml2e));
            w[0] = make_float2(e * sY[q], e);
            w[1] = __fmul2_rn(make_float2(e, e), make_float2(sY[PL + q], sY[2 * PL + q]));
        },
        [&](int y, const float2(&s)[2]) {
            if (y >= y_first) {
                sVA[v + y * dfv::VP] = s[0];
                sVB[v + y * dfv::VP] = s[1];
            }
        });
}

// Radiance and albedo of the footprint block [3][FH][FW] by cp.async: the
// radiance into sR, the albedo into sY (DEMOD; without an albedo the
// radiance goes straight into sY as the irradiance).  Chunks (VEC: 4
// columns, else 1 element) outside the frame are written as 0, so y = 0
// there.
template <bool DEMOD, bool VEC>
__device__ __forceinline__ void stage_irradiance(float* __restrict__ sY, float* __restrict__ sR,
                                                 const float* __restrict__ r, const float* __restrict__ a, int H,
                                                 int W, int tx0, int ty0, int tid) {
    constexpr int PL = dfv::FH * dfv::FW;
    const size_t HW = (size_t)H * W;
    float* rdst = DEMOD ? sR : sY;
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

// Demodulated irradiance y = r / (a + eps) in place of the staged albedo:
// each thread converts exactly the elements it staged, once its own copies
// have landed (outside the frame r = a = 0, so y = 0).
template <bool VEC>
__device__ __forceinline__ void form_irradiance(float* __restrict__ sY, const float* __restrict__ sR, float eps,
                                                int tid) {
    constexpr int PL = dfv::FH * dfv::FW;
    if constexpr (VEC) {
#pragma unroll
        for (int u = 0; u < dfv::CPT; ++u) {
            const int c = tid + u * dfv::THREADS;
            if (dfv::CPT * dfv::THREADS > dfv::NCH && c >= dfv::NCH) break;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                const float4 rv = reinterpret_cast<const float4*>(sR + ch * PL)[c];
                float4& yv = reinterpret_cast<float4*>(sY + ch * PL)[c];
                const float4 av = yv;
                yv = make_float4(__fdividef(rv.x, av.x + eps), __fdividef(rv.y, av.y + eps),
                                 __fdividef(rv.z, av.z + eps), __fdividef(rv.w, av.w + eps));
            }
        }
    } else {
        for (int e = tid; e < PL; e += dfv::THREADS)
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) sY[ch * PL + e] = __fdividef(sR[ch * PL + e], sY[ch * PL + e] + eps);
    }
}

// Per-thread state of the horizontal-pass task (row, 8 pixels) across the
// sizes i: acc_c = sum_i w_i N_ic and S = sum_i w_i D_i = sum_i exp(l_i - c)
// with w_i = exp(l_i - c) / D_i; cl = c log2(e), c the largest fusion logit
// of the sizes so far (a running maximum: when a size raises it, acc and S
// are rescaled by exp(c_old - c_new) first, so every size's exponential is
// at most 1), and l, the fusion logits of the size being processed (loaded
// one phase ahead).
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
    box_stream<K, dfv::SEG, 1>(PairLoader{sVA + v, {}},
                               [&](int x, const float2(&t)[1]) {
                                   const float D = t[0].y;
                                   const bool ok = D >= df::DMIN;
                                   bad |= !ok;
                                   // running softmax shift (Eq. 5): rescale what the
                                   // earlier sizes accumulated when this one raises it
                                   const float lx = st.l[x] * dfv::LOG2E;
                                   const float cn = fmaxf(st.cl[x], lx);
                                   const float sc = ex2_approx(st.cl[x] - cn);
                                   st.cl[x] = cn;
                                   st.acc[x][0] *= sc;
                                   st.acc[x][1] *= sc;
                                   st.acc[x][2] *= sc;
                                   st.S[x] *= sc;
                                   const float e = ex2_approx(lx - cn);
                                   w[x] = ok ? e * __fdividef(1.f, D) : 0.f;
                                   st.acc[x][0] = fmaf(w[x], t[0].x, st.acc[x][0]);
                                   st.S[x] = fmaf(w[x], D, st.S[x]);
                               });
    box_stream<K, dfv::SEG, 1>(PairLoader{sVB + v, {}},
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
    if (znext) stage_plane<VEC>(sZnext, znext, H, W, tx0, ty0, tid, -INFINITY);
    if (tid < 3 * NCOL) fwd_vpass<K>(sZcur, sY, sVA, sVB, ml2e, tid);
    __syncthreads();
    // after the last vertical pass the y planes are free: the albedo of the
    // re-modulation is staged in the y1, y2 planes while the horizontal pass runs
    if (a_stage) stage_albedo(sY + dfv::FH * dfv::FW, a_stage, H, W, tx0, ty0, tid);
    const int row = tid & 31, seg = tid >> 5;
    const unsigned exact = fwd_hpass<K>(sVA, sVB, st, row, seg);
    if (zlnext) load_row8<VEC>(st.l, zlnext, H, W, ty0 + row, tx0 + seg * dfv::SEG);
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
    // tiles bottom row first: the logits the convolution wrote last (the
    // bottom of the frame) are the ones still in L2 when this kernel starts
    const int tx0 = blockIdx.x * dfv::TW, ty0 = (gridDim.y - 1 - blockIdx.y) * dfv::TH;
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
    stage_plane<VEC>(sZ, z, H, W, tx0, ty0, tid, -INFINITY);
    stage_irradiance<DEMOD, VEC>(sY, sRst, r, a, H, W, tx0, ty0, tid);
    __syncthreads();  // red[0] initialised before any thread folds its maximum in

    // The first size's fusion logits (loaded while the copies above are in
    // flight); the softmax shift of Eq. 5 is a running maximum over the
    // sizes (HState), so the other sizes' logits are read once, one size
    // ahead of their horizontal pass.
    HState st;
    load_row8<VEC>(st.l, z + (size_t)M * HW, H, W, gy, gx0);
#pragma unroll
    for (int x = 0; x < dfv::SEG; ++x) {
        st.cl[x] = -INFINITY;
        st.acc[x][0] = st.acc[x][1] = st.acc[x][2] = st.S[x] = 0.f;
    }

    // Demodulated irradiance y = r / (a + eps), in place of the albedo: each
    // thread converts exactly the elements it staged, after its own copies
    // landed (outside the frame r = a = 0, so y = 0).
    cp_async_wait_all();
    if constexpr (DEMOD) form_irradiance<VEC>(sY, sRst, eps, tid);
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
// With g_c = (a_c + eps) dL/dout_c, E_i = exp(I_i), D_i(p) = sum over
// Omega_i(p) of E_i, R_ic = N_ic / D_i, LSE_i = log D_i, fusion weights
// alpha_i and d_i = sum_c g_c R_ic:
//   dL/dl_i(p) = alpha_i (d_i - sum_j alpha_j d_j)              (fusion logits)
//   dL/dI_i(q) = sum over p in Omega_i(q) of
//                alpha_i(p) exp(I_i(q) - LSE_i(p)) (sum_c g_c(p) y_c(q) - d_i(p))
// (windows are symmetric: q in Omega(p) <=> p in Omega(q)).  With
// Lp_i = LSE_i - ln alpha_i the second is exp(I_i(q) - s) times the window
// sums over p of e(p) g_c(p) and e(p) d_i(p), e = exp(s - Lp_i(p)), for any
// shift s; s is the minimum of Lp_i over the tile's staged block.
//   kernel 1 (the forward's tiles and window sums): Lp_i, d_i and g_c ->
//            scratch, the fusion-logit gradients -> dz;
//   kernel 2 (the same tiles): per size, the window sums of
//            (e g0, e g1 | e g2, e d) -> dz_i.
// Scratch per frame: planes [Lp_0..M-1 | d_0..M-1 | g_0 g_1 g_2] of H x W.
// A pixel whose D_i underflows takes an exact window loop in kernel 1; a
// tile whose staged Lp_i spans more than 80 takes one in kernel 2 (there the
// factors exp(I - s) and exp(s - Lp) stay inside the FP32 range).
// ======================================================================

struct DecodeBwdArgs {
    PtrBatch<const float*> z, r, a, G;
    PtrBatch<float*> dz, scratch;
    int H, W, M;
    int ks[WSKPN_MAX_KERNELS];
    float eps;
    unsigned int* fallbacks;
};

namespace dfv {
constexpr float LN2 = 0.6931471805599453f;
constexpr float RANGE = 80.f;  // widest staged Lp range of kernel 2's window-sum path
}  // namespace dfv

// 8 results of a horizontal-pass task into one row of a plane.
template <bool VEC>
__device__ __forceinline__ void store_row8(float* __restrict__ p, int H, int W, int gy, int gx0,
                                           const float (&v)[dfv::SEG]) {
    if (gy >= H) return;
    if (VEC && gx0 + dfv::SEG <= W) {
        float4* q = reinterpret_cast<float4*>(p + (size_t)gy * W + gx0);
        q[0] = make_float4(v[0], v[1], v[2], v[3]);
        q[1] = make_float4(v[4], v[5], v[6], v[7]);
    } else {
#pragma unroll
        for (int x = 0; x < dfv::SEG; ++x)
            if (gx0 + x < W) p[(size_t)gy * W + gx0 + x] = v[x];
    }
}

// log-sum-exp of I over the window of size k around (px, py), clipped to
// the image (exact, shifted by the window's own maximum).
__device__ __noinline__ float window_lse(const float* __restrict__ zi, int H, int W, int k, int px, int py) {
    const int h = k / 2;
    const int y0 = max(py - h, 0), y1 = min(py + h, H - 1), x0 = max(px - h, 0), x1 = min(px + h, W - 1);
    float m = -INFINITY, D = 0.f;
    for (int qy = y0; qy <= y1; ++qy)
        for (int qx = x0; qx <= x1; ++qx) m = fmaxf(m, zi[(size_t)qy * W + qx]);
    for (int qy = y0; qy <= y1; ++qy)
        for (int qx = x0; qx <= x1; ++qx) D += expf(zi[(size_t)qy * W + qx] - m);
    return m + logf(D);
}

// Kernel-1 state of a horizontal-pass task across the sizes.
struct BState {
    float g[dfv::SEG][3];  // g_c = (a_c + eps) dL/dout_c
    float Sd[dfv::SEG];    // sum over the sizes so far of alpha_i d_i
    float cl[dfv::SEG];    // (c + ln S) log2 e, so that alpha_i = 2^(l_i log2 e - cl)
    float l[dfv::SEG];     // fusion logits of the size being processed
};

// Kernel 1, horizontal pass of size K: from the window sums (N0, D) and
// (N1, N2), d = sum_c g_c N_c / D and Lp = LSE - ln alpha (LSE = m + ln D,
// m the size's exponent shift, ml2e = m log2 e); Sd += alpha d.  Returns the
// mask of pixels whose D underflowed (their d, Lp are redone exactly).
template <int K>
__device__ __forceinline__ unsigned bwd1_hpass(const float2* __restrict__ sVA, const float2* __restrict__ sVB,
                                               BState& st, float ml2e, int row, int seg, float (&Lp)[dfv::SEG],
                                               float (&d)[dfv::SEG]) {
    const int v = row * dfv::VP + seg * dfv::SEG;
    float inv[dfv::SEG];
    bool bad = false;
    box_stream<K, dfv::SEG, 1>(PairLoader{sVA + v, {}},
                               [&](int x, const float2(&t)[1]) {
                                   const float D = t[0].y;
                                   const bool ok = D >= df::DMIN;
                                   bad |= !ok;
                                   inv[x] = ok ? __fdividef(1.f, D) : 0.f;
                                   d[x] = st.g[x][0] * t[0].x;
                                   // log2 alpha = l log2 e - cl
                                   Lp[x] = (ml2e + __log2f(D) - fmaf(st.l[x], dfv::LOG2E, -st.cl[x])) * dfv::LN2;
                               });
    box_stream<K, dfv::SEG, 1>(PairLoader{sVB + v, {}},
                               [&](int x, const float2(&t)[1]) {
                                   d[x] = (d[x] + fmaf(st.g[x][1], t[0].x, st.g[x][2] * t[0].y)) * inv[x];
                               });
#pragma unroll
    for (int x = 0; x < dfv::SEG; ++x)
        st.Sd[x] = fmaf(ex2_approx(fmaf(st.l[x], dfv::LOG2E, -st.cl[x])), d[x], st.Sd[x]);
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

// Kernel 1, one window size K: the forward's phase (I_{i+1} staged during
// this size's vertical pass, the next fusion logits and shift after the
// horizontal pass), storing Lp_i and d_i of the task's 8 pixels.
template <int K, bool VEC>
__device__ __forceinline__ unsigned bwd1_size(const float* __restrict__ sZcur, float* __restrict__ sZnext,
                                              const float* __restrict__ sY, float2* __restrict__ sVA,
                                              float2* __restrict__ sVB, int* __restrict__ red,
                                              int* __restrict__ red_next, BState& st,
                                              const float* __restrict__ znext, const float* __restrict__ zlnext,
                                              float* __restrict__ Lp_out, float* __restrict__ d_out, int H, int W,
                                              int tx0, int ty0, int tid) {
    constexpr int NCOL = dfv::TW + 2 * (K / 2);
    const float ml2e = ord2f(*red) * dfv::LOG2E;
    if (tid == 0) *red_next = INT_MIN;  // its last reader finished before the previous barrier
    if (znext) stage_plane<VEC>(sZnext, znext, H, W, tx0, ty0, tid, -INFINITY);
    if (tid < 3 * NCOL) fwd_vpass<K>(sZcur, sY, sVA, sVB, ml2e, tid);
    __syncthreads();
    const int row = tid & 31, seg = tid >> 5;
    float Lp[dfv::SEG], d[dfv::SEG];
    const unsigned exact = bwd1_hpass<K>(sVA, sVB, st, ml2e, row, seg, Lp, d);
    store_row8<VEC>(Lp_out, H, W, ty0 + row, tx0 + seg * dfv::SEG, Lp);
    store_row8<VEC>(d_out, H, W, ty0 + row, tx0 + seg * dfv::SEG, d);
    if (zlnext) load_row8<VEC>(st.l, zlnext, H, W, ty0 + row, tx0 + seg * dfv::SEG);
    if (znext) finish_stage<VEC>(sZnext, red_next, tid);
    __syncthreads();
    return exact;
}

template <bool VEC>
__global__ void __launch_bounds__(dfv::THREADS, 2) decode_fuse_bwd1_kernel(const __grid_constant__ DecodeBwdArgs args) {
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
    const float* __restrict__ a = args.a.p[b];
    const float* __restrict__ G = args.G.p[b];
    float* const sc = args.scratch.p[b];  // written here and read back by the same threads
    float* __restrict__ dz = args.dz.p[b];
    const float eps = args.eps;
    const int row = tid & 31, seg = tid >> 5;
    const int gy = ty0 + row, gx0 = tx0 + seg * dfv::SEG;

    // Set-up as the forward's; besides the fusion softmax's shift each task
    // keeps the shift that also normalises it, and g_c of its pixels.
    if (tid == 0) red[0] = INT_MIN;
    stage_plane<VEC>(sZ, z, H, W, tx0, ty0, tid, -INFINITY);
    stage_irradiance<true, VEC>(sY, sRst, r, a, H, W, tx0, ty0, tid);
    __syncthreads();  // red[0] initialised before any thread folds its maximum in
    BState st;
    {
        float l[WSKPN_MAX_KERNELS][dfv::SEG];
#pragma unroll
        for (int i = 0; i < WSKPN_MAX_KERNELS; ++i)
            if (i < M) load_row8<VEC>(l[i], z + (size_t)(M + i) * HW, H, W, gy, gx0);
#pragma unroll
        for (int x = 0; x < dfv::SEG; ++x) {
            float c = l[0][x];
#pragma unroll
            for (int i = 1; i < WSKPN_MAX_KERNELS; ++i)
                if (i < M) c = fmaxf(c, l[i][x]);
            const float c2 = c * dfv::LOG2E;
            float S = 0.f;  // >= 1: the largest term is 2^0
#pragma unroll
            for (int i = 0; i < WSKPN_MAX_KERNELS; ++i)
                if (i < M) S += ex2_approx(fmaf(l[i][x], dfv::LOG2E, -c2));
            st.cl[x] = c2 + __log2f(S);
            st.l[x] = l[0][x];
            st.Sd[x] = 0.f;
        }
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float av[dfv::SEG], gv[dfv::SEG];
            load_row8<VEC>(av, a + ch * HW, H, W, gy, gx0);
            load_row8<VEC>(gv, G + ch * HW, H, W, gy, gx0);
#pragma unroll
            for (int x = 0; x < dfv::SEG; ++x) st.g[x][ch] = (av[x] + eps) * gv[x];
        }
    }
    cp_async_wait_all();
    form_irradiance<VEC>(sY, sRst, eps, tid);
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
        float* Lp_out = sc + (size_t)i * HW;
        float* d_out = sc + (size_t)(M + i) * HW;
        unsigned ex = 0;
#define WSKPN_BWD1_SIZE(K_)                                                                                  \
    case K_:                                                                                                 \
        ex = bwd1_size<K_, VEC>(zc, zn, sY, sVA, sVB, rd, rn, st, znext, zlnext, Lp_out, d_out, H, W, tx0, ty0, \
                                tid);                                                                        \
        break;
        switch (args.ks[i]) {
            WSKPN_BWD1_SIZE(1) WSKPN_BWD1_SIZE(3) WSKPN_BWD1_SIZE(5) WSKPN_BWD1_SIZE(7) WSKPN_BWD1_SIZE(9)
            WSKPN_BWD1_SIZE(11) WSKPN_BWD1_SIZE(13)
        }
#undef WSKPN_BWD1_SIZE
        exact |= (unsigned long long)ex << (8 * i);
    }
    if (gy >= H) return;

    // Pixels whose D_i underflowed: exact R and LSE of the window (rare); the
    // fast path left d = 0 out of Sd and stored values replaced here.
    if (exact) {
#pragma unroll 1
        for (int i = 0; i < M; ++i) {
#pragma unroll 1
            for (int x = 0; x < dfv::SEG; ++x) {
                const int px = gx0 + x;
                if (!((exact >> (8 * i + x)) & 1ull) || px >= W) continue;
                const float* zi = z + (size_t)i * HW;
                float R[3];
                window_exact_inl(zi, r, a, H, W, args.ks[i], eps, px, gy, R);
                const float L = window_lse(zi, H, W, args.ks[i], px, gy);
                if (args.fallbacks) atomicAdd(args.fallbacks, 1u);
                const size_t g = (size_t)gy * W + px;
                const float l = __ldg(z + (size_t)(M + i) * HW + g);
#pragma unroll
                for (int q = 0; q < dfv::SEG; ++q)
                    if (q == x) {
                        const float la2 = fmaf(l, dfv::LOG2E, -st.cl[q]);  // log2 alpha_i
                        const float dv = st.g[q][0] * R[0] + st.g[q][1] * R[1] + st.g[q][2] * R[2];
                        sc[(size_t)i * HW + g] = L - la2 * dfv::LN2;
                        sc[(size_t)(M + i) * HW + g] = dv;
                        st.Sd[q] = fmaf(ex2_approx(la2), dv, st.Sd[q]);
                    }
            }
        }
    }

    // g_c for kernel 2, and the fusion-logit gradients alpha_i (d_i - Sd)
    // (d_i read back from this thread's own stores).
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        float gv[dfv::SEG];
#pragma unroll
        for (int x = 0; x < dfv::SEG; ++x) gv[x] = st.g[x][ch];
        store_row8<VEC>(sc + (size_t)(2 * M + ch) * HW, H, W, gy, gx0, gv);
    }
    // three sizes per round, every load of a round issued before any use
    constexpr int GRP = 3;
    for (int i0 = 0; i0 < M; i0 += GRP) {
        float l[GRP][dfv::SEG], dv[GRP][dfv::SEG];
#pragma unroll
        for (int j = 0; j < GRP; ++j) {
            if (i0 + j >= M) break;
            load_row8<VEC>(l[j], z + (size_t)(M + i0 + j) * HW, H, W, gy, gx0);
            const float* dp = sc + (size_t)(M + i0 + j) * HW + (size_t)gy * W + gx0;
            if (VEC && gx0 + dfv::SEG <= W) {
                const float4 u = reinterpret_cast<const float4*>(dp)[0], v = reinterpret_cast<const float4*>(dp)[1];
                dv[j][0] = u.x, dv[j][1] = u.y, dv[j][2] = u.z, dv[j][3] = u.w;
                dv[j][4] = v.x, dv[j][5] = v.y, dv[j][6] = v.z, dv[j][7] = v.w;
            } else {
#pragma unroll
                for (int x = 0; x < dfv::SEG; ++x) dv[j][x] = gx0 + x < W ? dp[x] : 0.f;
            }
        }
#pragma unroll
        for (int j = 0; j < GRP; ++j) {
            if (i0 + j >= M) break;
            float o[dfv::SEG];
#pragma unroll
            for (int x = 0; x < dfv::SEG; ++x)
                o[x] = ex2_approx(fmaf(l[j][x], dfv::LOG2E, -st.cl[x])) * (dv[j][x] - st.Sd[x]);
            store_row8<VEC>(dz + (size_t)(M + i0 + j) * HW, H, W, gy, gx0, o);
        }
    }
}

// Kernel 2: wait for this thread's copies of the staged Lp block, and fold
// the warp's minimum and largest finite value into red[0], red[1]
// (order-preserving ints; outside the image Lp is +inf).
template <bool VEC>
__device__ __forceinline__ void finish_minmax(const float* __restrict__ sL, int* __restrict__ red, int tid) {
    cp_async_wait_all();
    float mn = INFINITY, mx = -INFINITY;
    auto take = [&](float v) {
        mn = fminf(mn, v);
        if (v < INFINITY) mx = fmaxf(mx, v);
    };
    if constexpr (VEC) {
#pragma unroll
        for (int u = 0; u < dfv::CPT; ++u) {
            const int c = tid + u * dfv::THREADS;
            if (dfv::CPT * dfv::THREADS > dfv::NCH && c >= dfv::NCH) break;
            const float4 v = reinterpret_cast<const float4*>(sL)[c];
            take(v.x), take(v.y), take(v.z), take(v.w);
        }
    } else {
        for (int e = tid; e < dfv::FH * dfv::FW; e += dfv::THREADS) take(sL[e]);
    }
    const int wmn = __reduce_min_sync(0xffffffffu, f2ord(mn));
    const int wmx = __reduce_max_sync(0xffffffffu, f2ord(mx));
    if ((tid & 31) == 0) {
        atomicMin(red, wmn);
        atomicMax(red + 1, wmx);
    }
}

// Kernel 2, vertical pass of size K (tasks as the forward's): e =
// exp(s - Lp) once per element (s = mn2 / log2 e), and the K-row sums of
// (e g0, e g1) into sVA and of (e g2, e d) into sVB.  sS holds the Lp and d
// blocks, sG the g blocks.
template <int K>
__device__ __forceinline__ void bwd2_vpass(const float* __restrict__ sS, const float* __restrict__ sG,
                                           float2* __restrict__ sVA, float2* __restrict__ sVB, float mn2, int t) {
    constexpr int h = K / 2, NCOL = dfv::TW + 2 * h;
    constexpr int PL = dfv::FH * dfv::FW;
    const int half = t >= NCOL ? 1 : 0;
    const int col = t - half * NCOL;
    const int o = (dfv::HALO + dfv::RV * half - h) * dfv::FW + dfv::XOFF - h + col;
    const int v = dfv::RV * half * dfv::VP + col;
    box_stream<K, dfv::RV, 2>(
        [&](int j, float2(&w)[2]) {
            const int q = o + j * dfv::FW;
            const float e = ex2_approx(fmaf(sS[q], -dfv::LOG2E, mn2));
            w[0] = __fmul2_rn(make_float2(e, e), make_float2(sG[q], sG[PL + q]));
            w[1] = __fmul2_rn(make_float2(e, e), make_float2(sG[2 * PL + q], sS[PL + q]));
        },
        [&](int y, const float2(&s)[2]) {
            sVA[v + y * dfv::VP] = s[0];
            sVB[v + y * dfv::VP] = s[1];
        });
}

// Kernel 2, horizontal pass of size K: the window sums S_c (of e g_c) and
// S_d (of e d) of the task's 8 pixels q give
// dL/dI(q) = exp(I(q) - s) (sum_c y_c(q) S_c - S_d).
template <int K>
__device__ __forceinline__ void bwd2_hpass(const float2* __restrict__ sVA, const float2* __restrict__ sVB,
                                           const float (&y)[dfv::SEG][3], const float (&zq)[dfv::SEG], float mn2,
                                           int row, int seg, float (&o)[dfv::SEG]) {
    const int v = row * dfv::VP + seg * dfv::SEG;
    box_stream<K, dfv::SEG, 1>(PairLoader{sVA + v, {}},
                               [&](int x, const float2(&t)[1]) { o[x] = fmaf(y[x][0], t[0].x, y[x][1] * t[0].y); });
    box_stream<K, dfv::SEG, 1>(PairLoader{sVB + v, {}},
                               [&](int x, const float2(&t)[1]) {
                                   const float f = ex2_approx(fmaf(zq[x], dfv::LOG2E, -mn2));
                                   o[x] = f * (fmaf(y[x][2], t[0].x, o[x]) - t[0].y);
                               });
}

// Kernel 2's exact path for one pixel q (a tile whose staged Lp range is too
// wide): the window loop over p of exp(I(q) - Lp(p)) (sum_c g_c(p) y_c(q) - d(p)).
__device__ __noinline__ float bwd2_exact(const float* __restrict__ sc, int M, int i, int H, int W, int k, float zq,
                                         float y0, float y1, float y2, int px, int py) {
    const size_t HW = (size_t)H * W;
    const float* Lp = sc + (size_t)i * HW;
    const float* d = sc + (size_t)(M + i) * HW;
    const float* g = sc + (size_t)(2 * M) * HW;
    const int h = k / 2;
    float v = 0.f;
    for (int qy = max(py - h, 0); qy <= min(py + h, H - 1); ++qy)
        for (int qx = max(px - h, 0); qx <= min(px + h, W - 1); ++qx) {
            const size_t p = (size_t)qy * W + qx;
            const float t = fmaf(__ldg(g + p), y0, fmaf(__ldg(g + HW + p), y1, __ldg(g + 2 * HW + p) * y2)) - __ldg(d + p);
            v += expf(zq - __ldg(Lp + p)) * t;
        }
    return v;
}

// Kernel 2, one window size K.  Phase: the vertical pass reads the staged
// Lp_i, d_i blocks; after the barrier Lp_{i+1}, d_{i+1} are staged into the
// same buffer while the horizontal pass runs, then their range is reduced.
// Returns true (block-uniform) when the staged range is too wide for the
// window sums: the size's gradients are then left to the exact loop.
template <int K, bool VEC>
__device__ __forceinline__ bool bwd2_size(float* __restrict__ sS, const float* __restrict__ sG,
                                          float2* __restrict__ sVA, float2* __restrict__ sVB, int* __restrict__ red,
                                          int* __restrict__ red_next, const float (&y)[dfv::SEG][3],
                                          float (&zq)[dfv::SEG], const float* __restrict__ sc, int M, int i,
                                          const float* __restrict__ zi_next, float* __restrict__ dzi, int H, int W,
                                          int tx0, int ty0, int tid) {
    constexpr int NCOL = dfv::TW + 2 * (K / 2);
    constexpr int PL = dfv::FH * dfv::FW;
    const float mn = ord2f(red[0]), mx = ord2f(red[1]);
    const float mn2 = mn * dfv::LOG2E;
    const bool wide = !(mx - mn <= dfv::RANGE);  // block-uniform
    if (tid == 0) {  // their last readers finished before the previous barrier
        red_next[0] = INT_MAX;
        red_next[1] = INT_MIN;
    }
    if (!wide && tid < 2 * NCOL) bwd2_vpass<K>(sS, sG, sVA, sVB, mn2, tid);
    __syncthreads();
    const bool more = zi_next != nullptr;
    const size_t HW = (size_t)H * W;
    if (more) {
        stage_plane<VEC>(sS, sc + (size_t)(i + 1) * HW, H, W, tx0, ty0, tid, INFINITY);
        stage_plane<VEC>(sS + PL, sc + (size_t)(M + i + 1) * HW, H, W, tx0, ty0, tid, 0.f);
    }
    const int row = tid & 31, seg = tid >> 5;
    const int gy = ty0 + row, gx0 = tx0 + seg * dfv::SEG;
    if (!wide) {
        float o[dfv::SEG];
        bwd2_hpass<K>(sVA, sVB, y, zq, mn2, row, seg, o);
        store_row8<VEC>(dzi, H, W, gy, gx0, o);
    }
    if (more) load_row8<VEC>(zq, zi_next, H, W, gy, gx0);
    if (more) finish_minmax<VEC>(sS, red_next, tid);
    __syncthreads();
    return wide;
}

template <bool VEC>
__global__ void __launch_bounds__(dfv::THREADS, 2) decode_fuse_bwd2_kernel(const __grid_constant__ DecodeBwdArgs args) {
    extern __shared__ float4 dsm4[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(dsm4);
    float* sG = reinterpret_cast<float*>(smem + dfv::OFF_Y);  // [3][FH][FW]: g0, g1, g2
    float* sS = reinterpret_cast<float*>(smem + dfv::OFF_Z);  // [2][FH][FW]: Lp_i, d_i
    float2* sVA = reinterpret_cast<float2*>(smem + dfv::OFF_V);
    float2* sVB = sVA + dfv::TH * dfv::VP;
    int* red = reinterpret_cast<int*>(smem + dfv::OFF_R);  // [2][min, max]
    constexpr int PL = dfv::FH * dfv::FW;

    const int tid = threadIdx.x;
    const int b = blockIdx.z;
    const int H = args.H, W = args.W, M = args.M;
    const size_t HW = (size_t)H * W;
    const int tx0 = blockIdx.x * dfv::TW, ty0 = blockIdx.y * dfv::TH;
    const float* __restrict__ z = args.z.p[b];
    const float* __restrict__ r = args.r.p[b];
    const float* __restrict__ a = args.a.p[b];
    const float* __restrict__ sc = args.scratch.p[b];
    float* __restrict__ dz = args.dz.p[b];
    const float eps = args.eps;
    const int row = tid & 31, seg = tid >> 5;
    const int gy = ty0 + row, gx0 = tx0 + seg * dfv::SEG;

    // Set-up: the g blocks and the first size's Lp, d blocks by cp.async;
    // y and I_0 of the task's own pixels into registers.
    if (tid == 0) {
        red[0] = INT_MAX;
        red[1] = INT_MIN;
    }
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) stage_plane<VEC>(sG + ch * PL, sc + (size_t)(2 * M + ch) * HW, H, W, tx0, ty0, tid, 0.f);
    stage_plane<VEC>(sS, sc, H, W, tx0, ty0, tid, INFINITY);
    stage_plane<VEC>(sS + PL, sc + (size_t)M * HW, H, W, tx0, ty0, tid, 0.f);
    float y[dfv::SEG][3], zq[dfv::SEG];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        float rv[dfv::SEG], av[dfv::SEG];
        load_row8<VEC>(rv, r + ch * HW, H, W, gy, gx0);
        load_row8<VEC>(av, a + ch * HW, H, W, gy, gx0);
#pragma unroll
        for (int x = 0; x < dfv::SEG; ++x) y[x][ch] = __fdividef(rv[x], av[x] + eps);
    }
    load_row8<VEC>(zq, z, H, W, gy, gx0);
    __syncthreads();  // red initialised before any thread folds its range in
    finish_minmax<VEC>(sS, red, tid);
    __syncthreads();

    unsigned wide = 0;  // bit i: size i's staged Lp range was too wide
    for (int i = 0; i < M; ++i) {
        int* rd = red + 2 * (i & 1);
        int* rn = red + 2 * ((i + 1) & 1);
        const float* zi_next = i + 1 < M ? z + (size_t)(i + 1) * HW : nullptr;
        float* dzi = dz + (size_t)i * HW;
        bool wi = false;
#define WSKPN_BWD2_SIZE(K_)                                                                                   \
    case K_:                                                                                                  \
        wi = bwd2_size<K_, VEC>(sS, sG, sVA, sVB, rd, rn, y, zq, sc, M, i, zi_next, dzi, H, W, tx0, ty0, tid); \
        break;
        switch (args.ks[i]) {
            WSKPN_BWD2_SIZE(1) WSKPN_BWD2_SIZE(3) WSKPN_BWD2_SIZE(5) WSKPN_BWD2_SIZE(7) WSKPN_BWD2_SIZE(9)
            WSKPN_BWD2_SIZE(11) WSKPN_BWD2_SIZE(13)
        }
#undef WSKPN_BWD2_SIZE
        wide |= (unsigned)wi << i;
    }

    // Sizes whose range was too wide: the exact window loop per own pixel
    // (rare; y and I reloaded, out of the unrolled code above).
    if (wide && gy < H) {
#pragma unroll 1
        for (int i = 0; i < M; ++i) {
            if (!((wide >> i) & 1u)) continue;
#pragma unroll 1
            for (int x = 0; x < dfv::SEG; ++x) {
                if (gx0 + x >= W) break;
                const size_t g = (size_t)gy * W + gx0 + x;
                float yc[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) yc[c] = __fdividef(__ldg(r + c * HW + g), __ldg(a + c * HW + g) + eps);
                dz[(size_t)i * HW + g] = bwd2_exact(sc, M, i, H, W, args.ks[i], __ldg(z + (size_t)i * HW + g), yc[0],
                                                    yc[1], yc[2], gx0 + x, gy);
                if (args.fallbacks) atomicAdd(args.fallbacks, 1u);
            }
        }
    }
}

template <bool VEC>
static wskpn_status launch_bwd_variant(const DecodeBwdArgs& args, int nb, cudaStream_t st, std::string& err) {
    WSKPN_CUDA_TRY(cudaFuncSetAttribute(decode_fuse_bwd1_kernel<VEC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)dfv::SMEM_BYTES),
                   err);
    WSKPN_CUDA_TRY(cudaFuncSetAttribute(decode_fuse_bwd2_kernel<VEC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)dfv::SMEM_BYTES),
                   err);
    dim3 grid(cdiv(args.W, dfv::TW), cdiv(args.H, dfv::TH), nb);
    decode_fuse_bwd1_kernel<VEC><<<grid, dfv::THREADS, dfv::SMEM_BYTES, st>>>(args);
    WSKPN_CUDA_TRY(cudaGetLastError(), err);
    decode_fuse_bwd2_kernel<VEC><<<grid, dfv::THREADS, dfv::SMEM_BYTES, st>>>(args);
    WSKPN_CUDA_TRY(cudaGetLastError(), err);
    return WSKPN_OK;
}

// Host launcher; the vectorised variant under the forward's condition (W a
// multiple of 4, every plane pointer 16-byte aligned).
wskpn_status launch_decode_fuse_bwd(const float* const* z, const float* const* r, const float* const* a,
                                    const float* const* G, float* const* dz, float* const* scratch, int B, int H,
                                    int W, int M, const int* ks, float eps, unsigned int* fallbacks,
                                    cudaStream_t st, std::string& err) {
    for (int b0 = 0; b0 < B; b0 += WSKPN_MAX_BATCH) {
        const int nb = B - b0 < WSKPN_MAX_BATCH ? B - b0 : WSKPN_MAX_BATCH;
        DecodeBwdArgs args{};
        bool vec = W % 4 == 0;
        for (int j = 0; j < nb; ++j) {
            args.z.p[j] = z[b0 + j];
            args.r.p[j] = r[b0 + j];
            args.a.p[j] = a[b0 + j];
            args.G.p[j] = G[b0 + j];
            args.dz.p[j] = dz[b0 + j];
            args.scratch.p[j] = scratch[b0 + j];
            vec = vec && aligned16(z[b0 + j]) && aligned16(r[b0 + j]) && aligned16(a[b0 + j]) &&
                  aligned16(G[b0 + j]) && aligned16(dz[b0 + j]) && aligned16(scratch[b0 + j]);
        }
        args.H = H;
        args.W = W;
        args.M = M;
        for (int i = 0; i < M; ++i) args.ks[i] = ks[i];
        args.eps = eps;
        args.fallbacks = fallbacks;
        const wskpn_status s = vec ? launch_bwd_variant<true>(args, nb, st, err) : launch_bwd_variant<false>(args, nb, st, err);
        if (s) return s;
    }
    return WSKPN_OK;
}

}  // namespace wskpn
