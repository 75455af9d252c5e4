// Weight gradient of the ImportanceNet convolutions on the tensor cores
// (tcgen05, BF16 operands, FP32 accumulators in tensor memory), for the
// training step of Eq. 1.  For y = b + W * x (KS x KS cross-correlation,
// zero padding KS / 2) and the pre-activation gradient gy:
//   dL/dW[o][c][dy][dx] = sum_{b,y,x} gy[o](y, x) x[c](y + dy - pad, x + dx - pad)
// (the bias gradient, the plain sum of gy, is formed where gy is packed).
//
// GEMM view: K = pixels.  A work item is one segment of 128 pixels of one
// gy row; it meets the KS x rows y + dy - pad.  Both operands are read
// MN-major straight from channels-last BF16 tiles (TMA boxes of 32-byte
// pixel rows, 16 channels each, 32-byte swizzle):
//   A = x:  M = 128 rows (s, c) = 8 horizontal shifts s x 16 channels of one
//           channel chunk; the shift is the leading-dimension stride of
//           one 32-byte pixel row, so row (s, c) at K index k reads pixel
//           x0 - pad + k + s of the same box (shifts s >= KS are computed
//           and discarded);
//   B = gy: N = the layer's padded output channels, 16-channel chunks in
//           separate boxes.
// Where KS x N fits one MMA the vertical taps are folded into N instead: a
// work item is an x row, B stacks the KS gy rows it meets (see the kernel).
// One accumulator per (dy, channel chunk) of N columns stays in TMEM for the
// whole kernel; each CTA walks a fixed set of work items (split K) and
// writes its sums as partials, which a second kernel adds in a fixed order,
// so the result does not depend on scheduling.
//
// Roles: warp 0 issues TMA, warp 1 owns TMEM and issues the MMAs (one
// thread), warps 2-5 zero the accumulators at the start and write the
// partials at the end.  Every mbarrier wait is bounded; on expiry the CTA
// records a status bit, drains what it has in flight, frees its TMEM and
// returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <string>

#include "common.cuh"
#include "tma.cuh"

namespace wskpn {

namespace wgtc {
constexpr int TPX = 128;                  // pixels of a gy row segment (K of one work item)
constexpr int XROWS = TPX + 8;            // x box rows: TPX + up to 7 shifts
constexpr int THREADS = 192;
constexpr uint32_t ROWB = 32;             // bytes of one pixel row of one 16-channel chunk
constexpr uint32_t GY_BOX = TPX * ROWB;   // 4096
constexpr uint32_t X_BOX = XROWS * ROWB;  // 4352
constexpr uint32_t X_SLOT = 5120;         // X_BOX rounded up to 1024 bytes
constexpr uint32_t SMEM_MAX = 232448;
constexpr unsigned ST_TIMEOUT = 8u;       // device status bit of this kernel's waits

__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// MN-major operand with 32-byte swizzle: 16 elements of M (or N) per 32-byte
// row, one row per K index, 8-row groups SBO bytes apart, 16-element groups
// of M (N) LBO bytes apart.
__device__ __forceinline__ uint64_t mn_desc_sw32(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
    d |= (uint64_t)6 << 61;  // 32-byte swizzle
    return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, 1, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc)
        : "memory");
}
__device__ __forceinline__ void commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_zero16(uint32_t taddr) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
        "%1};" ::"r"(taddr),
        "r"(0u)
        : "memory");
}

// Shared-memory bytes of one stage: the gy boxes (GR rows, or with folded
// vertical taps the KS rows an x row meets), then the x boxes (the GR + KS - 1
// rows those gy rows meet, NCC chunks each, or one row with folded taps).
__host__ __device__ constexpr uint32_t gy_part_bytes(int KS, int CPG, bool FOLD, int GR = 1) {
    return (uint32_t)((FOLD ? KS : GR) * (CPG / 16)) * GY_BOX;
}
__host__ __device__ constexpr int x_boxes(int KS, int NCC, bool FOLD, int GR = 1) {
    return FOLD ? NCC : (GR + KS - 1) * NCC;
}
__host__ __device__ constexpr uint32_t stage_bytes(int KS, int CPG, int NCC, bool FOLD, int GR = 1) {
    return gy_part_bytes(KS, CPG, FOLD, GR) + (uint32_t)x_boxes(KS, NCC, FOLD, GR) * X_SLOT;
}
__host__ __device__ constexpr uint32_t tmem_alloc_cols(int cols) {
    return cols <= 32 ? 32 : cols <= 64 ? 64 : cols <= 128 ? 128 : cols <= 256 ? 256 : 512;
}
}  // namespace wgtc

struct WgTcArgs {
    float* part;          // [gridDim.y][gridDim.x][KS * NCC][CPG][128] partial sums
    int H, W;
    int tiles_x, nitems;  // work items: (frame, row or group of GR rows, 128-pixel segment)
    int stages;
    unsigned int* status;
};

// Grid (split-K CTAs, channel-chunk groups); group blockIdx.y takes x chunks
// blockIdx.y * NCC .. + NCC - 1.
// Without FOLD a work item is a gy row y meeting the KS x rows y + dy - pad:
// one MMA (N = CPG) per (dy, chunk, K step), accumulators ordered (dy, chunk).
// With FOLD (KS x CPG <= 256) a work item is an x row y' meeting the KS gy
// rows y' - dy + pad: the B operand stacks those rows' gradients along N
// (N = KS x CPG, the boxes one LBO apart), so one MMA per (chunk, K step)
// covers every vertical tap and reads its A tile once; accumulators ordered
// (chunk, dy).  Every (x row, gy row) pair is met exactly once either way.
// With GR > 1 (unfolded) a work item is GR consecutive gy rows y0 .. y0 + GR
// - 1 and the GR + KS - 1 x rows they meet: x row xr (image row y0 - pad +
// xr) meets gy rows g in [xr - KS + 1, xr] (dy = xr - g), whose boxes sit in
// shared memory in descending g, one LBO apart, so one MMA per (x row,
// chunk, K step) takes them all (N = count x CPG <= 256) into the adjacent
// accumulators of dy = xr - g_hi .. xr - g_lo; accumulators ordered (chunk,
// dy) as with FOLD.  Each x tile is read once per item instead of once per
// gy row.
template <int KS, int CPG, int NCC, bool FOLD, int GR = 1>
__global__ void __launch_bounds__(wgtc::THREADS, 1)
    wgrad_tc_kernel(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap gmap,
                    const WgTcArgs a) {
    using namespace wgtc;
    static_assert(GR >= 1 && !(FOLD && GR > 1), "row groups: unfolded form only");
    static_assert(GR == 1 || (GR < KS ? GR : KS) * CPG <= 256, "row groups: MMA N");
    constexpr int PAD = KS / 2;
    constexpr int NACC = KS * NCC;              // accumulators (dy, chunk)
    constexpr int NCOL = NACC * CPG;            // TMEM columns used
    constexpr uint32_t ALLOC = tmem_alloc_cols(NCOL);
    constexpr uint32_t SB = stage_bytes(KS, CPG, NCC, FOLD, GR);
    constexpr uint32_t GYB = gy_part_bytes(KS, CPG, FOLD, GR);  // gy part of a stage
    constexpr int NXB = x_boxes(KS, NCC, FOLD, GR);
    constexpr uint32_t TX = GYB + (uint32_t)NXB * X_BOX;    // bytes a stage's loads deliver
    // folded: DYP vertical taps per MMA (N = DYP x CPG <= 256), the last MMA
    // of a K step takes the remaining DYL taps
    constexpr int DYP = FOLD ? (KS * CPG <= 256 ? KS : 256 / CPG) : 1;
    constexpr int NPART = FOLD ? (KS + DYP - 1) / DYP : 1;
    constexpr int DYL = KS - (NPART - 1) * DYP;
    constexpr int N = FOLD ? DYP * CPG : CPG;  // MMA N (all but the last part)
    static_assert(KS <= 8, "horizontal shifts per A operand");
    static_assert(N % 16 == 0 && N >= 16 && N <= 256, "MMA N");
    static_assert(NCOL <= 512, "TMEM columns");
    // kind::f16, D F32, A and B BF16, both MN-major, M = 128
    constexpr uint32_t IDESC0 = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                                ((uint32_t)(128 >> 4) << 24);
    constexpr uint32_t IDESC = IDESC0 | ((uint32_t)(N >> 3) << 17);
    constexpr uint32_t IDESC_L = IDESC0 | ((uint32_t)((FOLD ? DYL * CPG : CPG) >> 3) << 17);

    extern __shared__ __align__(1024) uint8_t dsmem[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dsmem) + 1023) & ~uintptr_t(1023));
    const int S = a.stages;
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + (size_t)S * SB);
    uint64_t* empty = full + S;
    uint64_t* done = empty + S;
    volatile uint32_t* tmem_holder = reinterpret_cast<volatile uint32_t*>(done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(done + 1) + 1;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        mbar_init(smem_u32(done), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32((const void*)tmem_holder)),
                     "r"(ALLOC)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_holder;
    if (warp >= 2) {  // accumulators start at zero: every MMA accumulates
        const uint32_t lb = (uint32_t)((warp & 3) * 32) << 16;
#pragma unroll 1
        for (int c = 0; c < NCOL; c += 16) tmem_zero16(tmem + lb + (uint32_t)c);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        fence_before();
    }
    __syncthreads();
    fence_after();

    const int chunk0 = blockIdx.y * NCC;
    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            uint32_t it = 0;
            bool ok = true;
            for (int w = blockIdx.x; w < a.nitems; w += gridDim.x, ++it) {
                const int s = it % S;
                if (!mbar_wait(smem_u32(&empty[s]), ((it / S) & 1u) ^ 1u, abort_flag)) {
                    ok = false;
                    break;
                }
                const int HG = (a.H + GR - 1) / GR;  // row groups per frame
                const int xt = w % a.tiles_x, y = (w / a.tiles_x) % HG * GR, b = w / (a.tiles_x * HG);
                const int x0 = xt * TPX;
                const uint32_t fb = smem_u32(&full[s]);
                const uint32_t dst = smem_u32(sm + (size_t)s * SB);
                mbar_expect_tx(fb, TX);
                // rows and pixels outside the image read as zeros
                if constexpr (FOLD) {
#pragma unroll
                    for (int dy = 0; dy < KS; ++dy)
#pragma unroll
                        for (int j = 0; j < CPG / 16; ++j)
                            tma_load_4d(dst + (dy * (CPG / 16) + j) * GY_BOX, &gmap, 16 * j, x0, y - dy + PAD, b,
                                        fb);
#pragma unroll
                    for (int ci = 0; ci < NCC; ++ci)
                        tma_load_4d(dst + GYB + ci * X_SLOT, &xmap, (chunk0 + ci) * 16, x0 - PAD, y, b, fb);
                } else {
                    // gy rows y .. y + GR - 1 in descending order (rows past the
                    // image read as zeros), then the x rows they meet
#pragma unroll
                    for (int g = 0; g < GR; ++g)
#pragma unroll
                        for (int j = 0; j < CPG / 16; ++j)
                            tma_load_4d(dst + ((GR - 1 - g) * (CPG / 16) + j) * GY_BOX, &gmap, 16 * j, x0, y + g, b,
                                        fb);
#pragma unroll
                    for (int xr = 0; xr < GR + KS - 1; ++xr)
#pragma unroll
                        for (int ci = 0; ci < NCC; ++ci)
                            tma_load_4d(dst + GYB + (xr * NCC + ci) * X_SLOT, &xmap, (chunk0 + ci) * 16, x0 - PAD,
                                        y + xr - PAD, b, fb);
                }
            }
            if (!ok) {
                atomicOr(a.status, ST_TIMEOUT);
                *abort_flag = 1;
            }
            // Drain: every issued stage's load must have landed before exit
            // (also after an abort: these waits ignore the abort flag).
            const uint32_t n_in_flight = it < (uint32_t)S ? it : (uint32_t)S;
            for (uint32_t k = 0; k < n_in_flight; ++k) {
                const uint32_t j = it - 1 - k;
                mbar_wait_drain(smem_u32(&full[j % S]), (j / S) & 1u);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            // descriptors are linear in the start address (16-byte units)
            const uint64_t ad0 = mn_desc_sw32(smem_u32(sm + GYB), ROWB, 8 * ROWB);
            const uint64_t bd0 = mn_desc_sw32(smem_u32(sm), GY_BOX, 8 * ROWB);
            bool ok = true;
            uint32_t it = 0;
            for (int w = blockIdx.x; w < a.nitems; w += gridDim.x, ++it) {
                const int s = it % S;
                if (!mbar_wait(smem_u32(&full[s]), (it / S) & 1u, abort_flag)) {
                    ok = false;
                    break;
                }
                fence_after();
                const uint64_t as = ad0 + (uint64_t)(s * (SB >> 4));
                const uint64_t bs = bd0 + (uint64_t)(s * (SB >> 4));
                // K steps of 16 pixels = 16 rows of 32 bytes
                if constexpr (FOLD) {
#pragma unroll
                    for (int ci = 0; ci < NCC; ++ci)
#pragma unroll
                        for (int j = 0; j < TPX / 16; ++j)
#pragma unroll
                            for (int pt = 0; pt < NPART; ++pt)
                                mma_bf16(tmem + (uint32_t)((ci * KS + pt * DYP) * CPG),
                                         as + (uint64_t)(ci * (X_SLOT >> 4) + j * 32),
                                         bs + (uint64_t)(pt * DYP * (CPG / 16) * (GY_BOX >> 4) + j * 32),
                                         pt == NPART - 1 ? IDESC_L : IDESC);
                } else if constexpr (GR == 1) {
#pragma unroll
                    for (int k = 0; k < NACC; ++k)
#pragma unroll
                        for (int j = 0; j < TPX / 16; ++j)
                            mma_bf16(tmem + (uint32_t)(k * CPG), as + (uint64_t)(k * (X_SLOT >> 4) + j * 32),
                                     bs + (uint64_t)(j * 32), IDESC);
                } else {
#pragma unroll
                    for (int xr = 0; xr < GR + KS - 1; ++xr) {
                        const int g_lo = xr - KS + 1 > 0 ? xr - KS + 1 : 0;
                        const int g_hi = xr < GR - 1 ? xr : GR - 1;
                        const uint32_t idesc = IDESC0 | ((uint32_t)(((g_hi - g_lo + 1) * CPG) >> 3) << 17);
#pragma unroll
                        for (int ci = 0; ci < NCC; ++ci)
#pragma unroll
                            for (int j = 0; j < TPX / 16; ++j)
                                mma_bf16(tmem + (uint32_t)((ci * KS + xr - g_hi) * CPG),
                                         as + (uint64_t)((xr * NCC + ci) * (X_SLOT >> 4) + j * 32),
                                         bs + (uint64_t)((GR - 1 - g_hi) * (CPG / 16) * (GY_BOX >> 4) + j * 32), idesc);
                    }
                }
                commit(smem_u32(&empty[s]));  // frees the stage when these MMAs finish
            }
            if (!ok) {
                atomicOr(a.status, ST_TIMEOUT);
                *abort_flag = 1;
            }
            // arrives when every issued MMA has completed; TMEM is released
            // only after that, whether or not the writers aborted
            commit(smem_u32(done));
            mbar_wait_drain(smem_u32(done), 0);
        }
    } else {
        // ------------------------------------------------ partial-sum writers, warps 2..5
        const int q = warp & 3;  // TMEM lane quarter this warp may access
        const int row = q * 32 + lane;
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        int ok = 1;
        if (lane == 0) ok = mbar_wait(smem_u32(done), 0, abort_flag);
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) {
            if (lane == 0) {
                atomicOr(a.status, ST_TIMEOUT);
                *abort_flag = 1;
            }
        } else {
            fence_after();
            float* part = a.part + (size_t)(blockIdx.y * gridDim.x + blockIdx.x) * NCOL * 128;
#pragma unroll 1
            for (int c = 0; c < NCOL; c += 16) {
                float v[16];
                tmem_ld16(tmem + lane_base + (uint32_t)c, v);
#pragma unroll
                for (int o = 0; o < 16; ++o) part[(size_t)(c + o) * 128 + row] = v[o];
            }
        }
        fence_before();
    }
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ALLOC) : "memory");
    }
}

// dW[o][c][dy][dx] = sum over the split-K CTAs g of partial
// [group][g][k][o][dx * 16 + c % 16], chunk c / 16 = group * NCC + ci and
// accumulator k = dy * NCC + ci, or ci * KS + dy with folded vertical taps.
// A block takes 32 consecutive partial entries (one warp-wide coalesced
// read per CTA g); warp w sums the CTAs g = w, w + 8, ... in that order and
// the 8 warp sums are added in warp order, so the result does not depend on
// scheduling.  Entries of shifts >= KS or padding channels are skipped.
constexpr int WG_RED_SLICES = 8;
__global__ void __launch_bounds__(32 * WG_RED_SLICES) wgrad_tc_reduce_kernel(const float* __restrict__ part, int Gk,
                                                                             int groups, int KS, int NCC, int CPG,
                                                                             int fold, int Cin, int Cout,
                                                                             float* __restrict__ dw) {
    __shared__ float red[WG_RED_SLICES][33];
    const size_t blk = (size_t)KS * NCC * CPG * 128;  // floats of one CTA's partials
    const size_t n = (size_t)groups * blk;
    const int lane = threadIdx.x & 31, sl = threadIdx.x >> 5;
    for (size_t base = (size_t)blockIdx.x * 32; base < n; base += (size_t)gridDim.x * 32) {
        const size_t i = base + lane;
        float s = 0.f;
        if (i < n) {
            const float* p = part + (i / blk) * Gk * blk + (i % blk);
#pragma unroll 4
            for (int g = sl; g < Gk; g += WG_RED_SLICES) s += p[(size_t)g * blk];
        }
        red[sl][lane] = s;
        __syncthreads();
        if (sl == 0 && i < n) {
            float t = red[0][lane];
#pragma unroll
            for (int k = 1; k < WG_RED_SLICES; ++k) t += red[k][lane];
            const int row = (int)(i % 128), o = (int)((i / 128) % CPG), k = (int)((i / (128 * (size_t)CPG)) % (KS * NCC));
            const int grp = (int)(i / blk);
            const int dx = row / 16, c16 = row % 16;
            const int dy = fold ? k % KS : k / NCC, ci = fold ? k / KS : k % NCC;
            const int c = (grp * NCC + ci) * 16 + c16;
            if (dx < KS && c < Cin && o < Cout) dw[(((size_t)o * Cin + c) * KS + dy) * KS + dx] = t;
        }
        __syncthreads();
    }
}

// Channel chunks per CTA group: the largest divisor of the chunk count whose
// accumulators fit in TMEM (KS x NCC x CPG <= 512 columns), at most 4.
static int wgrad_tc_ncc(int KS, int nchunks, int cpg) {
    for (int ncc = nchunks < 4 ? nchunks : 4; ncc >= 1; --ncc)
        if (nchunks % ncc == 0 && KS * ncc * cpg <= 512) return ncc;
    return 0;
}

using WgLaunch = cudaError_t (*)(const CUtensorMap&, const CUtensorMap&, const WgTcArgs&, dim3, size_t,
                                 cudaStream_t);

template <int KS, int CPG, int NCC, bool FOLD, int GR>
static cudaError_t launch_wg(const CUtensorMap& xm, const CUtensorMap& gm, const WgTcArgs& a, dim3 grid, size_t smem,
                             cudaStream_t st) {
    const cudaError_t e = cudaFuncSetAttribute(wgrad_tc_kernel<KS, CPG, NCC, FOLD, GR>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    wgrad_tc_kernel<KS, CPG, NCC, FOLD, GR><<<grid, wgtc::THREADS, smem, st>>>(xm, gm, a);
    return cudaGetLastError();
}

// Vertical taps folded into N where KS x CPG fits one MMA (<= 256).  For
// wider layers (5 x 64) the fold with two MMAs per K step (4 + 1 taps)
// measured no faster than the unfolded form (278 vs 271 us for 48 -> 64 at
// 16 x 256^2): each gradient row is then fetched KS times from L2.  Those
// layers take groups of WG_ROWS gy rows per work item instead (see the
// kernel), up to 256 / CPG rows meeting one x row per MMA.
constexpr int WG_ROWS = 4;
static constexpr bool wg_fold(int KS, int cpg) { return KS * cpg <= 256; }
static constexpr int wg_rows(int KS, int cpg) {
    return wg_fold(KS, cpg) ? 1 : (256 / cpg < WG_ROWS ? 256 / cpg : WG_ROWS);
}

static WgLaunch select_wg(int KS, int cpg, int ncc) {
#define WSKPN_WG_CASE(ks_, n_, c_) \
    if (KS == ks_ && cpg == n_ && ncc == c_) return launch_wg<ks_, n_, c_, wg_fold(ks_, n_), wg_rows(ks_, n_)>;
    // widths 10-32-48-64-12 and 64-64: (output channels, x chunks per CTA)
    WSKPN_WG_CASE(5, 32, 1) WSKPN_WG_CASE(5, 48, 2) WSKPN_WG_CASE(5, 64, 1) WSKPN_WG_CASE(5, 16, 4)
    WSKPN_WG_CASE(3, 32, 1) WSKPN_WG_CASE(3, 48, 2) WSKPN_WG_CASE(3, 64, 1) WSKPN_WG_CASE(3, 16, 4)
    WSKPN_WG_CASE(3, 64, 2)
#undef WSKPN_WG_CASE
    return nullptr;
}

// Geometry of one layer's tensor-core weight gradient.
struct WgPlan {
    int cpx, cpg, nchunks, ncc, groups, gk, stages, rows;  // rows: gy rows per work item
    size_t smem, part_floats;
};

static bool wgrad_tc_plan(int KS, int Cin, int Cout, int B, int H, int W, int nsm, WgPlan& p) {
    p.cpx = (Cin + 15) / 16 * 16;
    p.cpg = (Cout + 15) / 16 * 16;
    p.nchunks = p.cpx / 16;
    p.ncc = wgrad_tc_ncc(KS, p.nchunks, p.cpg);
    if (!p.ncc || !select_wg(KS, p.cpg, p.ncc)) return false;
    p.groups = p.nchunks / p.ncc;
    p.rows = wg_rows(KS, p.cpg);
    const int nitems = cdiv(W, wgtc::TPX) * cdiv(H, p.rows) * B;
    p.gk = nsm / p.groups;
    if (p.gk < 1) p.gk = 1;
    if (p.gk > nitems) p.gk = nitems;
    const uint32_t sb = wgtc::stage_bytes(KS, p.cpg, p.ncc, wg_fold(KS, p.cpg), p.rows);
    const uint32_t fixed = 1024 + 256;  // alignment slack, barriers
    const int s = (int)((wgtc::SMEM_MAX - fixed) / sb);
    if (s < 2) return false;
    p.stages = s < 4 ? s : 4;
    p.smem = fixed + (size_t)p.stages * sb;
    if (p.smem < 120 * 1024) p.smem = 120 * 1024;  // one CTA (one TMEM allocation) per SM
    p.part_floats = (size_t)p.groups * p.gk * KS * p.ncc * p.cpg * 128;
    return true;
}

// Whether a layer's weight gradient can run on the tensor cores, and the
// partial-sum floats it needs for batch x h x w on nsm SMs (at most; fewer
// for smaller calls).
bool wgrad_tc_supported(int KS, int Cin, int Cout, int B, int H, int W, int nsm, size_t* part_floats) {
    WgPlan p;
    if (!wgrad_tc_plan(KS, Cin, Cout, B, H, W, nsm, p)) return false;
    if (part_floats) *part_floats = p.part_floats;
    return true;
}

// x: channels-last BF16 [B][H][W][xcp] whose first round16(Cin) channels are
// the layer input (channels past Cin zero; e.g. the hi half of a hi/lo
// pair); gy_nhwc: the same for the gradient, [B][H][W][gcp_stride] with
// round16(Cout) gradient channels.  part: at least the partial-sum floats
// wgrad_tc_supported reports for a grid of nsm CTAs.  Writes dw (OIHW); the
// bias gradient is formed where the gradient is packed.
wskpn_status launch_wgrad_tc(const void* x, int xcp, const void* gy_nhwc, int gcp_stride, int B, int H, int W,
                             int Cin, int Cout, int KS, float* part, size_t part_cap, float* dw, unsigned int* status,
                             int device, cudaStream_t st, std::string& err) {
    if (B > WSKPN_MAX_BATCH) {
        err = "wgrad_tc: batch > 16";
        return WSKPN_EUNSUPPORTED;
    }
    int nsm = 148;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
    WgPlan p;
    if (!wgrad_tc_plan(KS, Cin, Cout, B, H, W, nsm, p) || p.part_floats > part_cap || xcp < p.cpx ||
        gcp_stride < p.cpg) {
        err = "wgrad_tc: layer shape not supported or workspace too small";
        return WSKPN_EUNSUPPORTED;
    }
    PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder(err);
    if (!encode) return WSKPN_EUNSUPPORTED;
    CUtensorMap xm, gm;
    {
        cuuint64_t gdim[4] = {(cuuint64_t)xcp, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
        cuuint64_t gstr[3] = {(cuuint64_t)xcp * 2, (cuuint64_t)W * xcp * 2, (cuuint64_t)H * W * xcp * 2};
        cuuint32_t box[4] = {16, (cuuint32_t)wgtc::XROWS, 1, 1};
        cuuint32_t estr[4] = {1, 1, 1, 1};
        const CUresult cr = encode(&xm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(x), gdim, gstr, box,
                                   estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (cr != CUDA_SUCCESS) {
            err = "wgrad_tc: cuTensorMapEncodeTiled (x) failed (" + std::to_string((int)cr) + ")";
            return WSKPN_ECUDA;
        }
    }
    {
        cuuint64_t gdim[4] = {(cuuint64_t)gcp_stride, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
        cuuint64_t gstr[3] = {(cuuint64_t)gcp_stride * 2, (cuuint64_t)W * gcp_stride * 2,
                              (cuuint64_t)H * W * gcp_stride * 2};
        cuuint32_t box[4] = {16, (cuuint32_t)wgtc::TPX, 1, 1};
        cuuint32_t estr[4] = {1, 1, 1, 1};
        const CUresult cr = encode(&gm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(gy_nhwc), gdim, gstr,
                                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (cr != CUDA_SUCCESS) {
            err = "wgrad_tc: cuTensorMapEncodeTiled (gy) failed (" + std::to_string((int)cr) + ")";
            return WSKPN_ECUDA;
        }
    }
    WgTcArgs a{};
    a.part = part;
    a.H = H;
    a.W = W;
    a.tiles_x = cdiv(W, wgtc::TPX);
    a.nitems = a.tiles_x * cdiv(H, p.rows) * B;
    a.stages = p.stages;
    a.status = status;
    const WgLaunch launch = select_wg(KS, p.cpg, p.ncc);
    WSKPN_CUDA_TRY(launch(xm, gm, a, dim3(p.gk, p.groups), p.smem, st), err);
    {
        const size_t n = (size_t)p.groups * KS * p.ncc * p.cpg * 128;
        const unsigned blocks = (unsigned)std::min<size_t>((n + 31) / 32, 148 * 16);
        wgrad_tc_reduce_kernel<<<blocks, 32 * WG_RED_SLICES, 0, st>>>(part, p.gk, p.groups, KS, p.ncc, p.cpg,
                                                                      wg_fold(KS, p.cpg) || p.rows > 1 ? 1 : 0, Cin,
                                                                      Cout, dw);
    }
    WSKPN_CUDA_TRY(cudaGetLastError(), err);
    return WSKPN_OK;
}

}  // namespace wskpn
