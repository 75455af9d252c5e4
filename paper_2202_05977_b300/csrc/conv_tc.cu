// Tensor-core path of the ImportanceNet convolutions (Sec. 4.1) on sm_103a:
// implicit-GEMM KSxKS conv + bias (+ ReLU) with tcgen05.mma, operands staged
// by TMA, FP32 accumulators in tensor memory.
//
// GEMM view of one tile: M = 128 consecutive pixels of an image row (TMEM
// lanes), N = padded output channels, K = KS*KS taps x input channels,
// consumed 32 bytes (16 BF16 or 32 e4m3 channels) per MMA.  A CTA owns
// R output rows x 128 pixels (R = 16, 8, 5, 4 for at most 16, 32, 48, 64
// output channels) and keeps R accumulators (one per output row) in TMEM,
// double-buffered across tiles so the epilogue of one tile
// overlaps the MMAs of the next.  Each input row is fetched once per tile
// (one TMA box of 128 + KS - 1 pixels per 32-byte channel chunk) and
// serves every tap that reads it: the KS horizontal taps through operand
// descriptors shifted by whole pixel rows, the KS vertical taps by
// accumulating into the matching output row.  The layer's weights stay
// resident in shared memory (pre-swizzled image, one bulk copy per CTA).
//
// BF16 activations may be stored as hi/lo pairs (x = hi + lo): the K loop
// then runs over both halves against the same weight chunk, which removes
// the activation rounding error at twice the MMA work.
//
// Issue path: one pipeline stage holds up to four input rows with all
// their channel chunks (as many as let two stages fit next to the weights);
// the MMAs of a row are a compile-time unrolled, branch-free sequence, and
// a stage ends with one commit (a branch or commit between MMAs roughly
// doubles their issue time on this part, and every stage costs the MMA
// thread a barrier wait).  Layers whose weight image leaves no room for two
// stages run as output-channel groups, each a pass over the input.
//
// Roles: warp 0 issues TMA, warp 1 owns TMEM and issues the MMAs (one
// thread), warps 2-5 drain TMEM (bias, ReLU, requantise) and store NHWC
// activations, or planar FP32 network outputs for the last layer.
//
// Every mbarrier wait is bounded (2 s of %globaltimer); on expiry the CTA
// records a status bit, drains what it has in flight, frees its TMEM and
// returns instead of hanging.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <cstring>
#include <mutex>
#include <vector>

#include "ctx.h"
#include "prep.cuh"
#include "quant.cuh"
#include "tma.cuh"

namespace wskpn {

namespace tc {
constexpr int BM = 128;            // pixels per tile row = MMA M = TMEM lanes
// Output rows per tile: as many as two buffers of R row accumulators allow
// in TMEM (2 R COUT_P <= 512 columns), at most 16.  More rows per tile means
// fewer MMAs per output row, since an input row's MMA serves up to
// min(R, KS) output rows, and fewer re-fetched halo rows.
__host__ __device__ constexpr int rows_per_tile(int cout_p) {
    return cout_p <= 16 ? 16 : cout_p <= 32 ? 8 : cout_p <= 48 ? 5 : 4;
}
constexpr int THREADS = 192;
// PIN kernels add four warps that assemble the input tiles (Sec. 5.1)
constexpr int THREADS_PIN = THREADS + 128;
constexpr int ROWB = 32;           // bytes of one pixel row of one K chunk
constexpr uint32_t SMEM_MAX = 232448;  // also the limit tc_rows_per_item tests against
constexpr unsigned ST_TIMEOUT_PRODUCER = 1u, ST_TIMEOUT_MMA = 2u, ST_TIMEOUT_EPILOGUE = 4u;
}  // namespace tc

struct TcArgs {
    const void* wimg;        // shared-memory image of the layer's weights
    uint32_t wbytes;
    const float* ep_scale;   // [COUT_P] multiplier of the accumulator
    const float* ep_bias;    // [COUT_P]
    void* out;               // NHWC activations, or planar FP32 [B][cout][H][W] for the last layer
    int B, H, W;
    int cout;                // real output channels of the layer
    int out_cp;              // padded output channels per stored pixel (all groups)
    int zero_c0, zero_n;     // storage channels [zero_c0, zero_c0 + zero_n) this launch writes as zeros
    int dup_src, dup_dst;    // e4m3 hi/lo: the hi bytes of channels [dup_src, dup_src + 16) are also
                             // written at dup_dst (the next layer's trailing half chunk); -1: none
    int out_c0;              // first output channel of this group
    int relu, last;
    int split_out;           // write BF16 hi/lo pairs: [hi(COUT_P) | lo(COUT_P)]
    float out_qscale;        // FP8 activations: 1 / scale of the output activation
    int stages;
    uint32_t box_stride;     // bytes between the chunk boxes of a row
    uint32_t row_bytes;      // bytes of one input row in a stage
    uint32_t stage_bytes;
    int tiles_x, tiles_y, ntiles;
    unsigned int* status;
    uint64_t wait_ns;        // limit of every wait but the drains
    int probe;               // test hook: the epilogue first waits on a barrier nothing signals
    // GM kernels (input gradients of the training step): the ReLU derivative
    // of the layer input as bits, two words per pixel (bit c set: channel c
    // positive, as written through relu_bits by the layer that produced it),
    // and per-warp bias-gradient sums bias_part [gridDim.x * 4][64] of the
    // masked values
    const uint32_t* gbits;
    float* bias_part;
    // BF16 ReLU layers, optional: two words per pixel, bit out_c0 + c set
    // when the stored hi half of output channel c is positive (then x = hi +
    // lo > 0, and only then); this launch writes the words its channels
    // occupy
    uint32_t* relu_bits;
    // PIN (the first layer assembling its own input, Sec. 5.1): the FP32
    // planar frame buffers of this launch's B frames and the assembly
    // constants; the layer input is then never stored
    FrameBatch frames;
    PrepConst prep;
    float in_qscale;  // PIN, e4m3 input: 1 / the input's activation scale
};

// ------------------------------------------------------------- primitives
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// K-major operand, 32-byte swizzle: rows of 32 bytes, 8-row groups 256 B apart.
// The swizzle follows the absolute shared-memory address bits (as the TMA
// writes it), so a start address shifted by whole 32-byte rows addresses
// the shifted matrix with the base-offset field left at 0.
__device__ __forceinline__ uint64_t sdesc_sw32(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;              // leading byte offset (unused for this layout)
    d |= (uint64_t)(256 >> 4) << 32;     // stride byte offset: 8 rows x 32 B
    d |= (uint64_t)1 << 46;              // descriptor version for tcgen05
    d |= (uint64_t)6 << 61;              // 32-byte swizzle
    return d;
}

// K-major operand with rows of RB = 32, 64 or 128 bytes and the matching
// swizzle (32B, 64B, 128B); one MMA reads 32 bytes of each row, selected by
// adding the byte offset within the row to the start address.
template <int RB>
__device__ __forceinline__ uint64_t sdesc_rows(uint32_t saddr) {
    constexpr uint64_t layout = RB == 128 ? 2 : (RB == 64 ? 4 : 6);
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)((8 * RB) >> 4) << 32;  // 8-row groups
    d |= (uint64_t)1 << 46;
    d |= layout << 61;
    return d;
}

// Channel chunks per TMA box: the widest of 4, 2, 1 that divides the chunk count.
__host__ __device__ constexpr int chunks_per_box(int ncc_in) { return ncc_in % 4 == 0 ? 4 : (ncc_in % 2 == 0 ? 2 : 1); }

// Shared-memory bytes of one input row in a stage (its channel-chunk boxes,
// each 1024-byte aligned), and of everything but the stages (weight image of
// one output-channel group, barriers, epilogue scale and bias).
__host__ __device__ constexpr uint32_t tc_row_bytes(int KS, int ncc_in) {
    return (uint32_t)(ncc_in / chunks_per_box(ncc_in)) *
           (uint32_t)(((128 + KS - 1) * 32 * chunks_per_box(ncc_in) + 1023) / 1024 * 1024);
}
// Folded horizontal taps (XF, the last layer): TMEM columns and weight-image
// rows of one output row's accumulators, the KS horizontal taps of cr
// output channels each (cr = 12 or 16), padded to a multiple of 16.
__host__ __device__ constexpr int xf_ncb(int KS, int cr) { return (KS * cr + 15) / 16 * 16; }
// Weight-image bytes of one output-channel group (xf_cr: folded, cr channels per tap block; 0: not folded).
__host__ __device__ constexpr size_t tc_wimg_bytes(int KS, int cout_g, int ncc_w, int xf_cr = 0) {
    return xf_cr ? (size_t)KS * ncc_w * xf_ncb(KS, xf_cr) * 32 : (size_t)KS * KS * ncc_w * cout_g * 32;
}
__host__ __device__ constexpr size_t tc_fixed_bytes(int KS, int cout_g, int ncc_w, int xf_cr = 0) {
    return 1024 + (tc_wimg_bytes(KS, cout_g, ncc_w, xf_cr) + 1023) / 1024 * 1024 + 256 + 2 * 64 * sizeof(float);
}
// Folded horizontal taps (XF, the last layer with 16 output channels): the
// epilogue warps exchange the partial sums of their edge pixels through
// shared memory, [2 rows][4 warps][KS - 1 lanes][KS - 1 taps][16 (+1 pad)]
// floats, plus 2 x 4 flags.
__host__ __device__ constexpr size_t tc_xf_bytes(int KS) {
    return (size_t)2 * 4 * (KS - 1) * (KS - 1) * 17 * sizeof(float) + 64;
}
// Output rows per tile of the folded form: N = (vertical taps) x xf_ncb <= 256
// (and two buffers of that many accumulator slots fill at most 512 columns).
__host__ __device__ constexpr int xf_rows_per_tile(int KS, int cr = 16) { return 256 / xf_ncb(KS, cr); }
// Input rows per pipeline stage: the most of 4, 3, 2 for which two such
// stages fit (one barrier wait and one commit per stage instead of per row:
// conv1 0.158 -> 0.130, conv2 0.269 -> 0.232, conv4 0.381 -> 0.341 ms at
// 1080p), else one.
// extra: further fixed bytes of the kernel (the epilogue staging, below).
__host__ __device__ constexpr int tc_rows_per_item(int KS, int cout_g, int ncc_in, int ncc_w, size_t extra = 0,
                                                   int xf_cr = 0) {
    return tc_fixed_bytes(KS, cout_g, ncc_w, xf_cr) + extra + 8 * (size_t)tc_row_bytes(KS, ncc_in) <= 232448   ? 4
           : tc_fixed_bytes(KS, cout_g, ncc_w, xf_cr) + extra + 6 * (size_t)tc_row_bytes(KS, ncc_in) <= 232448 ? 3
           : tc_fixed_bytes(KS, cout_g, ncc_w, xf_cr) + extra + 4 * (size_t)tc_row_bytes(KS, ncc_in) <= 232448 ? 2
                                                                                                                : 1;
}
// Epilogue staging (STG): each epilogue warp writes a row's 32 output
// pixels of hi/lo pairs (4 x cout bytes each for BF16, 2 x cout for e4m3)
// into shared memory at a pitch of an odd number of 16-byte units
// (conflict-free per lane), then stores them back as 512-byte contiguous
// pieces per warp instruction, instead of one 16-byte piece per lane a
// pixel apart (a partial sector per lane).  Built for BF16 layers of at
// most 48 output channels and e4m3 layers of 32 whose weights, staging and
// two input stages fit in shared memory.
__host__ __device__ constexpr size_t tc_stg_pitch(int cout_g, bool fp8 = false) {
    return (size_t)(fp8 ? 2 : 4) * cout_g + 16;
}
__host__ __device__ constexpr size_t tc_stg_bytes(int cout_g, bool fp8 = false) {
    return 4 * 32 * tc_stg_pitch(cout_g, fp8) + 16;
}
__host__ __device__ constexpr bool tc_stg_fits(int KS, int cout_g, int ncc_in, int ncc_w, bool fp8 = false) {
    return (fp8 ? cout_g == 32 : cout_g <= 48) &&
           tc_fixed_bytes(KS, cout_g, ncc_w) + tc_stg_bytes(cout_g, fp8) + 2 * (size_t)tc_row_bytes(KS, ncc_in) <=
               232448;
}
// The accumulate flag is a compile-time constant: a predicate computed at
// run time costs about twice the issue time of the MMA itself.
template <bool FP8, bool ACC>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc) {
    if constexpr (FP8) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "n"(ACC ? 1 : 0)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "n"(ACC ? 1 : 0)
            : "memory");
    }
}
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
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

// tcgen05.ld of 16 columns without waiting; tmem_wait16 waits for the loads in
// flight and ties these registers to the wait (so nothing reads them before)
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait16(uint32_t (&r)[16]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
}

__device__ __forceinline__ void tmem_zero16(uint32_t taddr) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
        "%1};" ::"r"(taddr),
        "r"(0u)
        : "memory");
}

template <int COUT_P, int R>
__host__ __device__ constexpr uint32_t tmem_cols() {
    return 2 * R * COUT_P <= 32 ? 32 : 2 * R * COUT_P <= 64 ? 64 : 2 * R * COUT_P <= 128 ? 128
           : 2 * R * COUT_P <= 256 ? 256 : 512;
}

// All MMAs of input row ri of a tile.  Input row ri feeds output rows
// ro = ri - dy for the vertical taps dy in [dy0, dy1] (those with
// 0 <= ro < R).  For each channel chunk and horizontal tap dx, ONE MMA
// covers all of them: the weight image stores the KS vertical taps of a
// (dx, chunk) pair as consecutive N blocks, and the accumulators of the R
// output rows sit in TMEM in descending row order (row ro at column block
// R - 1 - ro), so N = (dy1 - dy0 + 1) x COUT_P columns are contiguous.
// Accumulators are zeroed by the epilogue, so every MMA accumulates.  The
// row's tap range (hence N, the accumulator column and the weight offset)
// is computed at run time; the NCC_IN x KS MMAs themselves are an unrolled,
// branch-free sequence, so one body serves every row of any tile height.
template <int KS, int COUT_P, int NCC_IN, int NCC_W, bool FP8, int R, int WM, bool XF>
__device__ __forceinline__ void issue_item(int ri, uint32_t dbase, uint64_t ad, uint64_t bd, uint32_t box_step) {
    if constexpr (XF) {
        // Folded horizontal taps: one MMA per (activation chunk, weight chunk)
        // product covers the input row's vertical taps dy0..dy1 and all KS
        // horizontal taps, N = nb x NCB columns ordered (dy, dx, channel),
        // NCB = KS x COUT_P rounded up to 16 (COUT_P = 12 or 16 channels per
        // tap block); accumulator row slots hold NCB columns, and the
        // epilogue adds the dx-shifted partial sums.  The A operand is the
        // unshifted row window (input pixels x0 - PAD ..).  Products as below.
        constexpr int NCB = xf_ncb(KS, COUT_P);
        static_assert(NCB * (R < KS ? R : KS) <= 256, "MMA N");
        const int dy0 = ri - (R - 1) > 0 ? ri - (R - 1) : 0;
        const int dy1 = ri < KS - 1 ? ri : KS - 1;
        const int nb = dy1 - dy0 + 1;
        if (nb <= 0) return;
        constexpr uint32_t IDESC0 =
            (1u << 4) | (FP8 ? 0u : ((1u << 7) | (1u << 10))) | ((uint32_t)(tc::BM >> 4) << 24);
        const uint32_t idesc = IDESC0 | ((uint32_t)((nb * NCB) >> 3) << 17);
        constexpr uint32_t b_blk = (NCB * tc::ROWB) >> 4;  // one dy block (all dx) of a chunk, 16-byte units
        constexpr int CPB = chunks_per_box(NCC_IN);
        const uint32_t d = dbase + (uint32_t)((R - 1 - (ri - dy0)) * NCB);
        constexpr int nA = NCC_IN / 2;
        constexpr int NF = WM == 2 ? nA - 1 : nA;
        constexpr int NP = WM == 0 ? NCC_IN : 3 * NF + (WM == 2 ? 2 : 0);
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            int ca, cw;
            if (WM == 0) {
                ca = p;
                cw = p % NCC_W;
            } else if (p < 3 * NF) {
                const int c = NF > 0 ? p % NF : 0, kind = NF > 0 ? p / NF : 0;
                ca = kind == 1 ? nA + c : c;
                cw = kind == 2 ? NF + c : c;
            } else {
                ca = p == 3 * NF ? NF : nA + NF;
                cw = 2 * NF;
            }
            const uint64_t a = ad + (uint64_t)((ca / CPB) * box_step + (ca % CPB) * (tc::ROWB >> 4));
            const uint64_t b = bd + (uint64_t)((cw * KS + dy0) * b_blk);
            mma<FP8, true>(d, a, b, idesc);
        }
        return;
    } else {
    static_assert(COUT_P % 16 == 0 && COUT_P * (R < KS ? R : KS) <= 256, "MMA N");
    const int dy0 = ri - (R - 1) > 0 ? ri - (R - 1) : 0;
    const int dy1 = ri < KS - 1 ? ri : KS - 1;
    const int nb = dy1 - dy0 + 1;  // output rows fed by this input row
    if (nb <= 0) return;           // rows past R + KS - 1 loaded to fill a stage
    constexpr uint32_t IDESC0 = (1u << 4) | (FP8 ? 0u : ((1u << 7) | (1u << 10))) | ((uint32_t)(tc::BM >> 4) << 24);
    const uint32_t idesc = IDESC0 | ((uint32_t)((nb * COUT_P) >> 3) << 17);
    constexpr uint32_t b_blk = (COUT_P * tc::ROWB) >> 4;  // one (dx, chunk, dy) block, 16-byte units
    constexpr int CPB = chunks_per_box(NCC_IN);
    constexpr uint32_t a_dx = (CPB * tc::ROWB) >> 4;       // one pixel row of a box
    const uint32_t d = dbase + (uint32_t)((R - 1 - (ri - dy0)) * COUT_P);
    const uint64_t b0 = bd + (uint64_t)(dy0 * b_blk);
    // The (activation chunk, weight chunk) products of the row.  WM = 0:
    // every activation chunk meets its weight chunk (the lo half of a BF16
    // hi/lo activation reuses the hi weights).  WM = 1 (e4m3 hi/lo
    // activations and weights, NF chunks each): A_hi W_hi + A_lo W_hi +
    // A_hi W_lo per chunk, the lo x lo term being below the e4m3 rounding of
    // the rest.  WM = 2: the same for NF full chunks plus a trailing chunk of
    // at most 16 channels t, whose activation chunks are [A_hi(t) | A_hi(t)]
    // and [A_lo(t) | 0] and whose one weight chunk is [W_hi(t) | W_lo(t)]: two
    // MMAs give A_hi W_hi + A_hi W_lo + A_lo W_hi of the tail.  Weight chunks:
    // W_hi of the full chunks, their W_lo, then the tail chunk.
    constexpr int nA = NCC_IN / 2;                  // activation chunks per half (hi or lo)
    constexpr int NF = WM == 2 ? nA - 1 : nA;       // full chunks
    constexpr int NP = WM == 0 ? NCC_IN : 3 * NF + (WM == 2 ? 2 : 0);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        int ca, cw;
        if (WM == 0) {
            ca = p;
            cw = p % NCC_W;
        } else if (p < 3 * NF) {
            const int c = NF > 0 ? p % NF : 0, kind = NF > 0 ? p / NF : 0;
            ca = kind == 1 ? nA + c : c;
            cw = kind == 2 ? NF + c : c;
        } else {
            ca = p == 3 * NF ? NF : nA + NF;
            cw = 2 * NF;
        }
#pragma unroll
        for (int dx = 0; dx < KS; ++dx) {
            const uint64_t a = ad + (uint64_t)((ca / CPB) * box_step + (ca % CPB) * (tc::ROWB >> 4) + dx * a_dx);
            const uint64_t b = b0 + (uint64_t)((dx * NCC_W + cw) * KS * b_blk);
            mma<FP8, true>(d, a, b, idesc);
        }
    }
    }
}

// ----------------------------------------------------------------- kernel
// EPI: 0 plain epilogue; 1 (GM) input gradient with the ReLU mask of the
// layer input and bias sums; 2 (RB) also writes the output's ReLU bits.
template <int KS, int COUT_P, int NCC_IN, int NCC_W, bool FP8, int R, int WM, bool XF, int EPI, bool PIN = false>
__global__ void __launch_bounds__(PIN ? tc::THREADS_PIN : tc::THREADS, 1)
    conv_tc_kernel(const __grid_constant__ CUtensorMap tmap, const TcArgs a) {
    constexpr bool GM = EPI == 1, RB = EPI == 2;
    static_assert(!PIN || (!XF && EPI == 0 && NCC_IN == 2 && NCC_W == 1 && (!FP8 || WM == 2)),
                  "input assembly in the producer: the first layer with hi/lo input pairs (BF16, or e4m3 with "
                  "the trailing half chunk)");
    constexpr int PAD = KS / 2;
    constexpr int CH = FP8 ? 32 : 16;  // channels per K chunk
    constexpr int NCB = XF ? xf_ncb(KS, COUT_P) : COUT_P;  // TMEM columns of one output row's accumulators
    constexpr int TPX = XF ? tc::BM - (KS - 1) : tc::BM;  // output pixels per tile row
    static_assert(!XF || COUT_P == 16 || COUT_P == 12, "folded taps: 12 or 16 output channels per tap block");
    static_assert(!GM || (!XF && !FP8 && COUT_P <= 64), "gradient mask: BF16, at most 64 channels");
    static_assert(!RB || (!XF && !FP8 && COUT_P <= 64), "ReLU bits: BF16, at most 64 channels");
    constexpr uint32_t NCOL = tmem_cols<NCB, R>();
    constexpr int ROWS_IN = R + KS - 1;
    constexpr int CPB = chunks_per_box(NCC_IN);
    constexpr int NBOX = NCC_IN / CPB;
    constexpr uint32_t BOX_BYTES = (tc::BM + KS - 1) * tc::ROWB * CPB;
    constexpr bool STG = !XF && EPI == 0 && tc_stg_fits(KS, COUT_P, NCC_IN, NCC_W, FP8);
    constexpr int RPI =
        tc_rows_per_item(KS, COUT_P, NCC_IN, NCC_W, STG ? tc_stg_bytes(COUT_P, FP8) : 0, XF ? COUT_P : 0);
    static_assert(XF || (COUT_P % 16 == 0 && COUT_P >= 16 && COUT_P <= 256), "MMA N");
    static_assert(2 * R * NCB <= 512, "TMEM columns");

    extern __shared__ __align__(1024) uint8_t dsmem[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dsmem) + 1023) & ~uintptr_t(1023));
    uint8_t* sW = sm;
    uint8_t* sA = sm + ((a.wbytes + 1023u) & ~1023u);
    const int S = a.stages;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sA + (size_t)S * a.stage_bytes);
    uint64_t* full = bars;
    uint64_t* empty = bars + S;
    uint64_t* accf = bars + 2 * S;
    uint64_t* acce = accf + 2;
    uint64_t* wbar = acce + 2;
    uint64_t* fin = wbar + 1;
    uint64_t* dead = fin + 1;  // never signalled: the bounded-wait test hook (a.probe)
    volatile uint32_t* tmem_holder = reinterpret_cast<volatile uint32_t*>(dead + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(dead + 1) + 1;
    // [COUT_P], 16-byte aligned for vector loads
    float* s_scale = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(dead + 2) + 15) & ~uintptr_t(15));
    float* s_bias = s_scale + COUT_P;                     // [COUT_P]
    // XF: edge partial sums and the epilogue warps' tile flags, after the 2 x 64 floats
    float* const sEdge = reinterpret_cast<float*>(
        (reinterpret_cast<uintptr_t>(s_scale) + 2 * 64 * sizeof(float) + 15) & ~uintptr_t(15));
    volatile int* const sOk = reinterpret_cast<volatile int*>(sEdge + 2 * 4 * (KS - 1) * (KS - 1) * 17);
    // STG: the epilogue warps' staging rows, after the 2 x 64 floats
    uint8_t* const sStg = reinterpret_cast<uint8_t*>(sEdge);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // Every CTA of this persistent grid is resident from the start, so the
    // next kernel on the stream may launch now: its CTAs take an SM as this
    // grid's CTAs leave and set up (weights, barriers, TMEM) while it drains.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    for (int i = tid; i < COUT_P; i += tc::THREADS) {
        s_scale[i] = a.ep_scale[i];
        s_bias[i] = a.ep_bias[i];
    }
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(smem_u32(&full[s]), PIN ? 4 : 1);  // PIN: one arrival per assembling warp
            mbar_init(smem_u32(&empty[s]), 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(smem_u32(&accf[i]), 1);
            mbar_init(smem_u32(&acce[i]), 4);
        }
        mbar_init(smem_u32(wbar), 1);
        mbar_init(smem_u32(fin), 1);
        mbar_init(smem_u32(dead), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32((const void*)tmem_holder)),
                     "r"(NCOL)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;
    if (warp >= 2 && warp < 6) {
        // accumulators start at zero: every MMA accumulates
        const uint32_t lb = (uint32_t)((warp & 3) * 32) << 16;
#pragma unroll 1
        for (int c = 0; c < 2 * R * NCB; c += 16) tmem_zero16(tmem + lb + (uint32_t)c);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        tc_fence_before();
    }
    __syncthreads();
    tc_fence_after();

    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            const uint32_t wb = smem_u32(wbar);
            mbar_expect_tx(wb, a.wbytes);
            for (uint32_t off = 0; off < a.wbytes; off += 32768u) {
                const uint32_t n = a.wbytes - off < 32768u ? a.wbytes - off : 32768u;
                bulk_load(smem_u32(sW + off), static_cast<const uint8_t*>(a.wimg) + off, n, wb);
            }
            if constexpr (PIN) {
                // the assembling warps stage the activations: only the weight
                // copy is this warp's to see land before exit
                mbar_wait_drain(wb, 0);
            } else {
                // the activations are the previous kernel's output: wait for that
                // grid to complete (returns at once without a programmatic
                // dependency).  Everything else this CTA reads or writes in global
                // memory follows from these loads.
                asm volatile("griddepcontrol.wait;" ::: "memory");
                uint32_t it = 0;
                bool ok = true;
                for (int t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x) {
                    const int tx = t % a.tiles_x, ty = (t / a.tiles_x) % a.tiles_y, b = t / (a.tiles_x * a.tiles_y);
                    const int x0 = tx * TPX, y0 = ty * R;
                    for (int r0 = 0; r0 < ROWS_IN; r0 += RPI, ++it) {
                        const int s = it % S;
                        if (!mbar_wait(smem_u32(&empty[s]), ((it / S) & 1u) ^ 1u, abort_flag, a.wait_ns)) {
                            ok = false;
                            break;
                        }
                        const uint32_t fb = smem_u32(&full[s]);
                        const uint32_t dst = smem_u32(sA + (size_t)s * a.stage_bytes);
                        mbar_expect_tx(fb, (uint32_t)RPI * NBOX * BOX_BYTES);
#pragma unroll
                        for (int j = 0; j < RPI; ++j)  // rows past the tile read as zeros
#pragma unroll
                            for (int bx = 0; bx < NBOX; ++bx)
                                tma_load_4d(dst + j * a.row_bytes + bx * a.box_stride, &tmap, bx * CPB * CH, x0 - PAD,
                                            y0 - PAD + r0 + j, b, fb);
                    }
                }
                if (!ok) {
                    atomicOr(a.status, tc::ST_TIMEOUT_PRODUCER);
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
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            bool ok = mbar_wait(smem_u32(wbar), 0, abort_flag, a.wait_ns);
            // Descriptors are linear in the start address (16-byte units in
            // the low bits): stages, chunks and taps are offsets from two bases.
            const uint64_t wdesc0 = sdesc_sw32(smem_u32(sW));
            const uint64_t adesc0 = sdesc_rows<CPB * tc::ROWB>(smem_u32(sA));
            const uint32_t a_stage = a.stage_bytes >> 4;
            const uint32_t a_row = a.row_bytes >> 4;
            const uint32_t box_step = a.box_stride >> 4;
            uint32_t it = 0;
            int lt = 0;
            for (int t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x, ++lt) {
                const int buf = lt & 1;
                if (!mbar_wait(smem_u32(&acce[buf]), ((lt >> 1) & 1) ^ 1, abort_flag, a.wait_ns)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t dbase = tmem + (uint32_t)(buf * R * NCB);
                for (int r0 = 0; r0 < ROWS_IN; r0 += RPI, ++it) {
                    const int s = it % S;
                    if (!mbar_wait(smem_u32(&full[s]), (it / S) & 1u, abort_flag, a.wait_ns)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
#pragma unroll
                    for (int j = 0; j < RPI; ++j)
                        issue_item<KS, COUT_P, NCC_IN, NCC_W, FP8, R, WM, XF>(
                            r0 + j, dbase, adesc0 + (uint64_t)(s * a_stage + j * a_row), wdesc0, box_step);
                    mma_commit(smem_u32(&empty[s]));  // frees the stage when these MMAs finish
                }
                if (ok) mma_commit(smem_u32(&accf[buf]));
            }
            if (!ok) {
                atomicOr(a.status, tc::ST_TIMEOUT_MMA);
                *abort_flag = 1;
            }
            // Every issued MMA must complete before TMEM is released (also
            // after an abort: the drain wait ignores the abort flag).
            mma_commit(smem_u32(fin));
            mbar_wait_drain(smem_u32(fin), 0);
        }
    } else if (PIN && warp >= 6) {
        // ------------------------------------------------ input assembly (PIN), warps 6..9
        // The first layer's input tiles straight from the FP32 frame buffers
        // (Sec. 5.1 assembly, the same functions and bits as the separate
        // assembly kernel): each stage row holds the 128 + KS - 1 input pixels
        // of one tile row as 64-byte rows, [hi(16) | lo(16)] BF16 or
        // [hi(16) | hi(16) | lo(16) | 0(16)] e4m3, in the 64-byte
        // swizzle (16-byte unit u of a row at unit u ^ (address bits 7-8)),
        // which is what the TMA writes from the stored NHWC input, so the MMA
        // side is unchanged.  Pixels outside the image are the convolution's
        // zero padding.  All raw loads of a stage are issued before any is used.
        if constexpr (PIN) {
            constexpr int NPX = tc::BM + KS - 1;
            constexpr int NPT = (RPI * NPX + 127) / 128;  // pixels per thread per stage
            const int ct = tid - tc::THREADS;              // 0..127
            const size_t HW = (size_t)a.H * a.W;
            // the frames may be the previous kernel's output
            asm volatile("griddepcontrol.wait;" ::: "memory");
            uint32_t it = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x) {
                const int tx = t % a.tiles_x, ty = (t / a.tiles_x) % a.tiles_y, b = t / (a.tiles_x * a.tiles_y);
                const int x0 = tx * TPX, y0 = ty * R;
                const float* const fr = a.frames.r.p[b];
                const float* const fa = a.frames.a.p[b];
                const float* const fn = a.frames.n.p[b];
                const float* const fd = a.frames.d.p[b];
                for (int r0 = 0; r0 < ROWS_IN; r0 += RPI, ++it) {
                    const int s = it % S;
                    int w = 1;
                    if (lane == 0) w = mbar_wait(smem_u32(&empty[s]), ((it / S) & 1u) ^ 1u, abort_flag, a.wait_ns);
                    if (!__shfl_sync(0xffffffffu, w, 0)) {
                        ok = false;
                        break;
                    }
                    uint8_t* const stg = sA + (size_t)s * a.stage_bytes;
                    float raw[NPT][10];
                    bool inside[NPT];
#pragma unroll
                    for (int k = 0; k < NPT; ++k) {
                        const int i = ct + 128 * k;
                        const int j = i / NPX, px = i - j * NPX;
                        const int yy = y0 - PAD + r0 + j, xx = x0 - PAD + px;
                        inside[k] = i < RPI * NPX && r0 + j < ROWS_IN && yy >= 0 && yy < a.H && xx >= 0 && xx < a.W;
                        if (inside[k]) prep_load_raw(fr, fa, fn, fd, (size_t)yy * a.W + xx, HW, raw[k]);
                    }
#pragma unroll
                    for (int k = 0; k < NPT; ++k) {
                        const int i = ct + 128 * k;
                        const int j = i / NPX, px = i - j * NPX;
                        if (i >= RPI * NPX || r0 + j >= ROWS_IN) continue;  // rows no MMA reads
                        uint4 qv[4] = {make_uint4(0u, 0u, 0u, 0u), make_uint4(0u, 0u, 0u, 0u),
                                       make_uint4(0u, 0u, 0u, 0u), make_uint4(0u, 0u, 0u, 0u)};
                        if (inside[k]) {
                            float v[16];
                            prep_from_raw<true>(raw[k], a.prep, v);
#pragma unroll
                            for (int c = 10; c < 16; ++c) v[c] = 0.f;
                            if constexpr (FP8) {
                                // e4m3 hi/lo of v / scale: [hi | hi | lo | 0], the
                                // layer's trailing half chunk (as the assembly kernel)
                                fp8_pack16(v, a.in_qscale, qv[0], &qv[2]);
                                qv[1] = qv[0];
                            } else {
                                bf16_hilo16(v, qv);
                            }
                        }
                        uint8_t* const row = stg + (size_t)j * a.row_bytes + (size_t)px * 64;
                        const int sw = (px >> 1) & 3;
#pragma unroll
                        for (int u = 0; u < 4; ++u) *reinterpret_cast<uint4*>(row + ((u ^ sw) << 4)) = qv[u];
                    }
                    // generic-proxy writes made visible to the tensor core's reads
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&full[s]));
                }
            }
            if (!ok && lane == 0) {
                atomicOr(a.status, tc::ST_TIMEOUT_PRODUCER);
                *abort_flag = 1;
            }
        }
    } else {
        // ------------------------------------------------ epilogue warps 2..5
        const int q = warp & 3;  // TMEM lane quarter this warp may access
        const int p = q * 32 + lane;
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        int lt = 0, rowc = 0;
        // STG: the whole stored pixel is this launch's (one group, no padding
        // channels, BF16 hi/lo output of a hidden layer)
        const bool coal = STG && !a.last && a.split_out && a.out_c0 == 0 && a.out_cp == COUT_P && a.zero_n == 0 &&
                          a.dup_src < 0;
        (void)coal;
        // GM: this thread's sums of its masked gradient values per channel,
        // over its pixels in tile and row order
        float bsum[GM ? COUT_P : 1];
#pragma unroll
        for (int c = 0; c < (GM ? COUT_P : 1); ++c) bsum[c] = 0.f;
        for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++lt) {
            const int buf = lt & 1;
            int ok = 1;
            if (lane == 0) {
                // test hook: a wait that nothing completes, so the limit expires
                if (a.probe && lt == 0) ok = mbar_wait(smem_u32(dead), 0, abort_flag, a.wait_ns);
                if (ok) ok = mbar_wait(smem_u32(&accf[buf]), (lt >> 1) & 1, abort_flag, a.wait_ns);
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if constexpr (XF) {
                // the rows below hold barriers of the 4 epilogue warps: all of
                // them take this tile or all give up
                if (lane == 0) sOk[(lt & 1) * 4 + q] = ok;
                asm volatile("bar.sync 1, 128;" ::: "memory");
                ok = sOk[(lt & 1) * 4] & sOk[(lt & 1) * 4 + 1] & sOk[(lt & 1) * 4 + 2] & sOk[(lt & 1) * 4 + 3];
            }
            if (!ok) {
                if (lane == 0) {
                    atomicOr(a.status, tc::ST_TIMEOUT_EPILOGUE);
                    *abort_flag = 1;
                }
                break;
            }
            tc_fence_after();
            const int tx = t % a.tiles_x, ty = (t / a.tiles_x) % a.tiles_y, b = t / (a.tiles_x * a.tiles_y);
            const int x = tx * TPX + p;
            // bytes per stored pixel of an NHWC output (BF16 hi/lo pairs double it)
            const size_t pix_bytes = (size_t)a.out_cp * (FP8 ? 1 : 2) * (a.split_out ? 2 : 1);
            if constexpr (XF) {
                // output pixel p = sum over dx of the accumulator of TMEM lane
                // (window pixel) p + dx, block dx; lanes p + dx beyond this warp
                // come from the next warp's first KS - 1 lanes via shared memory
#pragma unroll 1
                for (int r = 0; r < R; ++r, ++rowc) {
                    const int y = ty * R + r;
                    const uint32_t col = (uint32_t)(buf * R * NCB + (R - 1 - r) * NCB);
                    // the slot's NCB columns: tap dx's channel o at column dx COUT_P + o
                    constexpr int NL = NCB / 16;
                    uint32_t u[NL][16];
#pragma unroll
                    for (int c = 0; c < NL; ++c) tmem_ld16_async(tmem + lane_base + col + c * 16, u[c]);
#pragma unroll
                    for (int c = 0; c < NL; ++c) tmem_wait16(u[c]);
#pragma unroll
                    for (int c = 0; c < NL; ++c) tmem_zero16(tmem + lane_base + col + c * 16);
                    float v[KS][COUT_P];
#pragma unroll
                    for (int dx = 0; dx < KS; ++dx)
#pragma unroll
                        for (int o = 0; o < COUT_P; ++o)
                            v[dx][o] = __uint_as_float(u[(dx * COUT_P + o) / 16][(dx * COUT_P + o) % 16]);
                    float* const eb = sEdge + (rowc & 1) * (4 * (KS - 1) * (KS - 1) * 17);
                    if (lane < KS - 1) {
#pragma unroll
                        for (int dx = 1; dx < KS; ++dx)
#pragma unroll
                            for (int o = 0; o < COUT_P; ++o)
                                eb[((q * (KS - 1) + lane) * (KS - 1) + dx - 1) * 17 + o] = v[dx][o];
                    }
                    asm volatile("bar.sync 1, 128;" ::: "memory");
                    float acc[COUT_P];
#pragma unroll
                    for (int o = 0; o < COUT_P; ++o) acc[o] = v[0][o];
#pragma unroll
                    for (int dx = 1; dx < KS; ++dx) {
                        const int src = lane + dx - 32;  // >= 0: lane src of the next warp
#pragma unroll
                        for (int o = 0; o < COUT_P; ++o) {
                            float sv = __shfl_down_sync(0xffffffffu, v[dx][o], dx);
                            if (src >= 0) sv = q < 3 ? eb[(((q + 1) * (KS - 1) + src) * (KS - 1) + dx - 1) * 17 + o] : 0.f;
                            acc[o] += sv;
                        }
                    }
                    if (p < TPX && x < a.W && y < a.H) {
                        const size_t HW = (size_t)a.H * a.W;
                        float* z = static_cast<float*>(a.out) + (size_t)b * a.cout * HW + (size_t)y * a.W + x;
#pragma unroll
                        for (int o = 0; o < COUT_P; ++o)
                            if (o < a.cout) z[(size_t)o * HW] = fmaf(acc[o], s_scale[o], s_bias[o]);
                    }
                }
            } else {
            bool staged = false;
            if constexpr (STG) {
                if (coal) {
                    staged = true;
                    constexpr int PB = (FP8 ? 2 : 4) * COUT_P;  // bytes of a stored pixel: hi then lo
                    constexpr int NU = PB / 16;                 // its 16-byte units
                    constexpr uint32_t PITCH = (uint32_t)tc_stg_pitch(COUT_P, FP8);
                    uint8_t* const stw = sStg + (size_t)q * 32 * PITCH;  // this warp's 32 pixel slots
                    uint8_t* const slot = stw + (size_t)lane * PITCH;
                    const int xw = tx * TPX + q * 32;  // the warp's first pixel
#pragma unroll 1
                    for (int r = 0; r < R; ++r) {
                        const int y = ty * R + r;
                        const uint32_t col = (uint32_t)(buf * R * NCB + (R - 1 - r) * NCB);
                        uint32_t u[COUT_P / 16][16];
#pragma unroll
                        for (int c16 = 0; c16 < COUT_P / 16; ++c16)
                            tmem_ld16_async(tmem + lane_base + col + c16 * 16, u[c16]);
#pragma unroll
                        for (int c16 = 0; c16 < COUT_P / 16; ++c16) tmem_wait16(u[c16]);
#pragma unroll
                        for (int c16 = 0; c16 < COUT_P / 16; ++c16)
                            tmem_zero16(tmem + lane_base + col + c16 * 16);  // ready for the buffer's next tile
                        if (y >= a.H) continue;  // warp-uniform
#pragma unroll
                        for (int c16 = 0; c16 < COUT_P / 16; ++c16) {
                            float v[16];
                            const float4* b4 = reinterpret_cast<const float4*>(s_bias + c16 * 16);
                            const float4* s4 = reinterpret_cast<const float4*>(s_scale + c16 * 16);
#pragma unroll
                            for (int j4 = 0; j4 < 4; ++j4) {
                                const float4 bb = b4[j4];
                                if constexpr (FP8) {  // e4m3 accumulators carry the weight and input scales
                                    const float4 ss = s4[j4];
                                    v[4 * j4] = fmaf(__uint_as_float(u[c16][4 * j4]), ss.x, bb.x);
                                    v[4 * j4 + 1] = fmaf(__uint_as_float(u[c16][4 * j4 + 1]), ss.y, bb.y);
                                    v[4 * j4 + 2] = fmaf(__uint_as_float(u[c16][4 * j4 + 2]), ss.z, bb.z);
                                    v[4 * j4 + 3] = fmaf(__uint_as_float(u[c16][4 * j4 + 3]), ss.w, bb.w);
                                } else {
                                    v[4 * j4] = __uint_as_float(u[c16][4 * j4]) + bb.x;
                                    v[4 * j4 + 1] = __uint_as_float(u[c16][4 * j4 + 1]) + bb.y;
                                    v[4 * j4 + 2] = __uint_as_float(u[c16][4 * j4 + 2]) + bb.z;
                                    v[4 * j4 + 3] = __uint_as_float(u[c16][4 * j4 + 3]) + bb.w;
                                }
                            }
                            (void)s4;
                            if (a.relu)
#pragma unroll
                                for (int j = 0; j < 16; ++j) v[j] = fmaxf(v[j], 0.f);
                            if constexpr (FP8) {
                                // [hi(cout) | lo(cout)] e4m3 of v / the output's scale
                                uint4 hq, lq;
                                fp8_pack16(v, a.out_qscale, hq, &lq);
                                reinterpret_cast<uint4*>(slot)[c16] = hq;
                                reinterpret_cast<uint4*>(slot)[NU / 2 + c16] = lq;
                                continue;
                            }
                            __nv_bfloat162 h2[8], l2[8];
#pragma unroll
                            for (int j = 0; j < 8; ++j) {
                                h2[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                                const float2 hf = __bfloat1622float2(h2[j]);
                                l2[j] = __floats2bfloat162_rn(v[2 * j] - hf.x, v[2 * j + 1] - hf.y);
                            }
                            const uint4* hs = reinterpret_cast<const uint4*>(h2);
                            const uint4* ls = reinterpret_cast<const uint4*>(l2);
                            uint4* const sh = reinterpret_cast<uint4*>(slot) + 2 * c16;
                            uint4* const sl = reinterpret_cast<uint4*>(slot) + NU / 2 + 2 * c16;
                            sh[0] = hs[0];
                            sh[1] = hs[1];
                            sl[0] = ls[0];
                            sl[1] = ls[1];
                        }
                        __syncwarp();
                        // the warp's pixels are contiguous in the NHWC output:
                        // unit g of the run is pixel g / NU, unit g % NU
                        uint8_t* const orow =
                            static_cast<uint8_t*>(a.out) + (((size_t)b * a.H + y) * a.W + xw) * (size_t)PB;
#pragma unroll
                        for (int k = 0; k < NU; ++k) {
                            const int g = k * 32 + lane;
                            const int pp = g / NU, uu = g - pp * NU;
                            const uint4 val = *reinterpret_cast<const uint4*>(stw + (size_t)pp * PITCH + uu * 16);
                            if (xw + pp < a.W) *reinterpret_cast<uint4*>(orow + (size_t)g * 16) = val;
                        }
                        __syncwarp();
                    }
                }
            }
            if (!staged)
#pragma unroll 1
            for (int r = 0; r < R; ++r) {
                const int y = ty * R + r;
                const bool valid = x < a.W && y < a.H;
                const uint32_t col = (uint32_t)(buf * R * NCB + (R - 1 - r) * NCB);
                const size_t pix = ((size_t)b * a.H + y) * a.W + x;
                // this group's first channel of the pixel (hi half for BF16)
                uint8_t* const pbase = static_cast<uint8_t*>(a.out) + pix * pix_bytes + (size_t)a.out_c0 * (FP8 ? 1 : 2);
                // GM: the layer input's positive channels at this pixel, loaded
                // before the accumulators are read
                uint64_t mbits = 0;
                if constexpr (GM) {
                    if (valid) {
                        const uint2 m = reinterpret_cast<const uint2*>(a.gbits)[pix];
                        mbits = (((uint64_t)m.y << 32) | m.x) >> a.out_c0;
                    }
                }
                uint64_t rbits = 0;  // relu_bits of this pixel (channels of this launch)
#pragma unroll
                for (int c16 = 0; c16 < COUT_P / 16; ++c16) {
                    float v[16];
                    tmem_ld16(tmem + lane_base + col + c16 * 16, v);
                    tmem_zero16(tmem + lane_base + col + c16 * 16);  // ready for the buffer's next tile
                    if (!valid) continue;
                    {
                        // BF16 accumulators need no rescale (the scale is 1)
                        const float4* b4 = reinterpret_cast<const float4*>(s_bias + c16 * 16);
                        const float4* s4 = reinterpret_cast<const float4*>(s_scale + c16 * 16);
#pragma unroll
                        for (int j4 = 0; j4 < 4; ++j4) {
                            const float4 bb = b4[j4];
                            const float bj[4] = {bb.x, bb.y, bb.z, bb.w};
                            if constexpr (FP8) {
                                const float4 ss = s4[j4];
                                const float sj[4] = {ss.x, ss.y, ss.z, ss.w};
#pragma unroll
                                for (int k = 0; k < 4; ++k) v[4 * j4 + k] = fmaf(v[4 * j4 + k], sj[k], bj[k]);
                            } else {
#pragma unroll
                                for (int k = 0; k < 4; ++k) v[4 * j4 + k] += bj[k];
                            }
                        }
                        if (a.relu)
#pragma unroll
                            for (int j = 0; j < 16; ++j) v[j] = fmaxf(v[j], 0.f);
                    }
                    if constexpr (GM) {
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (!((mbits >> (c16 * 16 + j)) & 1ull)) v[j] = 0.f;
#pragma unroll
                        for (int j = 0; j < 16; ++j) bsum[c16 * 16 + j] += v[j];
                    }
                    if (a.last) {
                        const size_t HW = (size_t)a.H * a.W;
                        const int o0 = a.out_c0 + c16 * 16;  // first of these 16 output channels
                        float* z = static_cast<float*>(a.out) + ((size_t)b * a.cout + o0) * HW + (size_t)y * a.W + x;
                        const int nvalid = a.cout - o0;
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (j < nvalid) z[(size_t)j * HW] = v[j];
                    } else if constexpr (FP8) {
                        uint4 hq, lq;
                        fp8_pack16(v, a.out_qscale, hq, a.split_out ? &lq : nullptr);
                        *reinterpret_cast<uint4*>(pbase + c16 * 16) = hq;
                        if (a.split_out) *reinterpret_cast<uint4*>(pbase + a.out_cp + c16 * 16) = lq;
                        if (a.out_c0 + c16 * 16 == a.dup_src)
                            *reinterpret_cast<uint4*>(pbase + (a.dup_dst - a.out_c0)) = hq;
                    } else {
                        __nv_bfloat162 h2[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) h2[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                        uint4* dst = reinterpret_cast<uint4*>(pbase + c16 * 32);
                        const uint4* src = reinterpret_cast<const uint4*>(h2);
                        dst[0] = src[0];
                        dst[1] = src[1];
                        if constexpr (RB) {
                            // a positive finite BF16 has bits in [0x0001, 0x7F80]
#pragma unroll
                            for (int j = 0; j < 8; ++j) {
                                const uint32_t hw = reinterpret_cast<const uint32_t*>(h2)[j];
                                if ((hw & 0xFFFFu) - 1u < 0x7F80u) rbits |= 1ull << (c16 * 16 + 2 * j);
                                if ((hw >> 16) - 1u < 0x7F80u) rbits |= 1ull << (c16 * 16 + 2 * j + 1);
                            }
                        }
                        if (a.split_out) {
                            // residual v - bf16(v), itself rounded to BF16
                            __nv_bfloat162 l2[8];
#pragma unroll
                            for (int j = 0; j < 8; ++j) {
                                const float2 hf = __bfloat1622float2(h2[j]);
                                l2[j] = __floats2bfloat162_rn(v[2 * j] - hf.x, v[2 * j + 1] - hf.y);
                            }
                            uint4* dlo = reinterpret_cast<uint4*>(pbase + (size_t)a.out_cp * 2 + c16 * 32);
                            const uint4* slo = reinterpret_cast<const uint4*>(l2);
                            dlo[0] = slo[0];
                            dlo[1] = slo[1];
                        }
                    }
                }
                if constexpr (RB) {
                    if (valid) {
                        uint32_t* rb = a.relu_bits + pix * 2 + (a.out_c0 >> 5);
                        rb[0] = (uint32_t)rbits;
                        if (COUT_P > 32) rb[1] = (uint32_t)(rbits >> 32);
                    }
                }
                if (a.zero_n && valid) {  // storage padding past the layer's channels
                    constexpr int EB = FP8 ? 1 : 2;
                    uint8_t* const zb = static_cast<uint8_t*>(a.out) + pix * pix_bytes + (size_t)a.zero_c0 * EB;
                    const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
                    for (int zc = 0; zc < a.zero_n * EB; zc += 16) {
                        if (a.dup_src < 0) *reinterpret_cast<uint4*>(zb + zc) = zero;  // else the tail copy
                        if (a.split_out) *reinterpret_cast<uint4*>(zb + (size_t)a.out_cp * EB + zc) = zero;
                    }
                }
            }
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&acce[buf]));
        }
        if constexpr (GM) {
            // the warp's per-channel sums (a fixed butterfly over its lanes);
            // lane c % 32 stores channel c
            __syncwarp();
            float* const dst = a.bias_part + ((size_t)blockIdx.x * 4 + q) * 64 + a.out_c0;
#pragma unroll
            for (int c = 0; c < COUT_P; ++c) {
                float s = bsum[c];
#pragma unroll
                for (int m = 16; m > 0; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
                if (lane == (c & 31)) dst[c] = s;
            }
        }
    }
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOL) : "memory");
    }
}

// ------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder(std::string& err) {
    static std::mutex mu;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !p) {
            err = "cuTensorMapEncodeTiled is not available from the CUDA driver";
            return nullptr;
        }
        fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

static int chan_pad(int c, bool fp8) { return fp8 ? (c + 31) / 32 * 32 : (c + 15) / 16 * 16; }
// e4m3 hi/lo weight mode of a layer with cin input channels: 2 when the
// last 32-channel chunk holds at most 16 channels (trailing half chunk,
// stored twice in the hi half of the activations), else 1.
static int fp8_weight_mode(int cin) { return cin % 32 != 0 && cin % 32 <= 16 ? 2 : 1; }
// Output channels of a layer's MMAs (N per vertical tap): a multiple of 16.
// Its stored pixels may be wider (e4m3 activations are stored in 32-channel
// chunks); the epilogue writes the padding as zeros.
static int cout_pad(const wskpn_config& c, int l) { return (c.widths[l + 1] + 15) / 16 * 16; }

// Activations are stored as hi/lo pairs: BF16 (4 bytes per channel) or e4m3
// (2 bytes per channel; the single-term e4m3 form uses half of it).
size_t tc_act_bytes_per_pixel(const wskpn_config& c, int which) {
    const bool fp8 = c.prec == WSKPN_FP8;
    size_t m = 0;
    for (int l = 0; l < c.n_layers; ++l)
        if (l % 2 == which) {
            const size_t b = (size_t)chan_pad(c.widths[l], fp8) * (fp8 ? 2 : 4);
            m = b > m ? b : m;
        }
    return m;
}

// Output-channel groups and device buffers of a tensor-core layer whose
// cin_p / cout_p are set: the smallest power-of-two group count whose weight
// image leaves room for two input stages (hi/lo activations assumed), each
// group a multiple of 16 channels.  fp8_lo: e4m3 weights as hi/lo pairs
// (weight mode fp8_weight_mode(cin), the chunk counts of fp8_chunks).
wskpn_status tc_layer_alloc(Layer& L, int KS, bool fp8, bool fp8_lo, std::string& err) {
    const int nch = L.cin_p / (fp8 ? 32 : 16);
    const int wm = fp8 && fp8_lo ? fp8_weight_mode(L.cin) : 0;
    const int ncc_in = 2 * nch;
    const int ncc_w = wm == 1 ? ncc_in : wm == 2 ? ncc_in - 1 : nch;
    cudaFree(L.wtc);
    cudaFree(L.ep_scale);
    cudaFree(L.ep_bias);
    cudaFree(L.wscale);
    L.wtc = nullptr;
    L.ep_scale = L.ep_bias = L.wscale = nullptr;
    L.wtc_bytes = (size_t)KS * KS * ncc_w * L.cout_p * tc::ROWB;
    L.groups = 1;
    while (true) {
        const size_t fixed = tc_fixed_bytes(KS, L.cout_p / L.groups, ncc_w);
        if (fixed + 2 * (size_t)tc_row_bytes(KS, ncc_in) <= tc::SMEM_MAX) break;
        if (L.cout_p / (2 * L.groups) < 16 || (L.cout_p / (2 * L.groups)) % 16) {
            err = "conv_tc: layer weights do not fit in shared memory";
            return WSKPN_EUNSUPPORTED;
        }
        L.groups *= 2;
    }
    WSKPN_CUDA_TRY(cudaMalloc(&L.wtc, L.wtc_bytes), err);
    WSKPN_CUDA_TRY(cudaMalloc(&L.ep_scale, L.cout_p * sizeof(float)), err);
    WSKPN_CUDA_TRY(cudaMalloc(&L.ep_bias, L.cout_p * sizeof(float)), err);
    WSKPN_CUDA_TRY(cudaMalloc(&L.wscale, L.cout_p * sizeof(float)), err);
    return WSKPN_OK;
}

wskpn_status tc_alloc_layer(wskpn_ctx* ctx, int l) {
    const wskpn_config& c = ctx->cfg;
    Layer& L = ctx->layers[l];
    const bool fp8 = c.prec == WSKPN_FP8;
    L.cin_p = chan_pad(L.cin, fp8);
    L.cout_p = cout_pad(c, l);
    if (L.cout_p > 64) {
        ctx->err = "tensor-core path supports at most 64 output channels per layer";
        return WSKPN_EUNSUPPORTED;
    }
    return tc_layer_alloc(L, c.conv_ks, fp8, fp8 && ctx->fp8_split, ctx->err);
}

// Builds the shared-memory image of a layer's B operand, one image per
// output-channel group of cg = cout_p / groups channels: block
// ((dx * ncc + cc) * KS + dy) of a group holds its cg rows of 32 bytes
// (K-major) of tap (dy, dx) and channel chunk cc, so the KS vertical taps of
// one (dx, cc) pair are consecutive N blocks.  32-byte swizzled like the TMA
// writes A: byte o of a block goes to o ^ (((o >> 7) & 1) << 4).  With xf
// (folded horizontal taps, xf = channels per tap block, 12 or 16) the rows
// of a chunk are ordered (dy, dx, channel) instead: row ((cc * KS + dy) *
// xf_ncb + dx * xf + n), rows past KS * xf of each dy block zero (the image
// is cleared first).  e4m3
// weight modes (lo = e4m3(w / s - e4m3(w / s)), s the channel's scale):
// wm 1: chunks nf .. 2 nf - 1 hold the lo halves of chunks 0 .. nf - 1;
// wm 2: the same for nf = (ncc - 1) / 2 full chunks, then one chunk with
// the hi (bytes 0..15) and lo (16..31) of the at most 16 trailing channels.
__global__ void pack_tc_kernel(const float* __restrict__ w, const float* __restrict__ bias, int Cin, int Cout,
                               int KS, int cout_p, int groups, int ncc, int fp8, int wm, int xf,
                               const float* __restrict__ wscale, float act_in_scale, uint8_t* __restrict__ img,
                               float* __restrict__ ep_scale, float* __restrict__ ep_bias) {
    const int ch = fp8 ? 32 : 16;
    const int cg = cout_p / groups;
    const int nf = wm == 1 ? ncc / 2 : wm == 2 ? (ncc - 1) / 2 : ncc;
    const int n_el = KS * KS * ncc * cout_p * ch;
    const size_t group_bytes = (size_t)KS * KS * ncc * cg * 32;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_el; i += gridDim.x * blockDim.x) {
        const int k = i % ch;
        const int nl = (i / ch) % cg;
        const int chunk = (i / (ch * cg)) % (KS * KS * ncc);
        const int g = i / (ch * cg * KS * KS * ncc);
        const int n = g * cg + nl;
        // block order (dx, cc, dy), or (cc, dy, dx) for folded horizontal taps
        const int dy = xf ? (chunk / KS) % KS : chunk % KS;
        const int cc = xf ? chunk / (KS * KS) : (chunk / KS) % ncc;
        const int dx = xf ? chunk % KS : chunk / (KS * ncc);
        if (xf && nl >= xf) continue;  // channels past the tap block: not stored
        bool lo;
        int cin;
        if (wm == 2 && cc == 2 * nf) {  // trailing half chunk: hi | lo
            lo = k >= 16;
            cin = nf * ch + (k & 15);
        } else {
            lo = wm != 0 && cc >= nf;
            cin = (lo ? cc - nf : cc) * ch + k;
        }
        const float v = (n < Cout && cin < Cin) ? w[((size_t)n * Cin + cin) * KS * KS + dy * KS + dx] : 0.f;
        const uint32_t o = (uint32_t)(nl * 32 + k * (fp8 ? 1 : 2));
        size_t phys = g * group_bytes + (size_t)chunk * cg * 32 + (o ^ (((o >> 7) & 1u) << 4));
        if (xf) {  // one group; swizzle on the absolute byte offset (the image is 1024-aligned)
            const size_t oa = ((size_t)(cc * KS + dy) * xf_ncb(KS, xf) + dx * xf + nl) * 32 + k * (fp8 ? 1 : 2);
            phys = oa ^ (((oa >> 7) & 1u) << 4);
        }
        if (fp8) {
            const float q = v / wscale[n];
            const __nv_fp8_storage_t h = __nv_cvt_float_to_fp8(q, __NV_SATFINITE, __NV_E4M3);
            if (lo) {
                const __half_raw hr = __nv_cvt_fp8_to_halfraw(h, __NV_E4M3);
                img[phys] = (uint8_t)__nv_cvt_float_to_fp8(q - __half2float(*reinterpret_cast<const __half*>(&hr)),
                                                           __NV_SATFINITE, __NV_E4M3);
            } else {
                img[phys] = (uint8_t)h;
            }
        } else {
            *reinterpret_cast<__nv_bfloat16*>(img + phys) = __float2bfloat16_rn(v);
        }
    }
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < cout_p; n += gridDim.x * blockDim.x) {
        ep_bias[n] = n < Cout ? bias[n] : 0.f;
        ep_scale[n] = fp8 ? act_in_scale * wscale[n] : 1.f;
    }
}

// Per-output-channel weight scale for FP8: max |W[n]| / 448 (1 if all zero).
__global__ void wscale_kernel(const float* __restrict__ w, int Cin, int Cout, int KS, int cout_p,
                              float* __restrict__ wscale) {
    const int n = blockIdx.x;
    float m = 0.f;
    if (n < Cout)
        for (int i = threadIdx.x; i < Cin * KS * KS; i += blockDim.x) m = fmaxf(m, fabsf(w[(size_t)n * Cin * KS * KS + i]));
    __shared__ float red[32];
    m = warp_max(m);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int j = 1; j < (int)(blockDim.x >> 5); ++j) m = fmaxf(m, red[j]);
        m = fmaxf(m, red[0]);
        wscale[n] = m > 0.f ? m / 448.f : 1.f;
    }
}

wskpn_status tc_pack_layer(wskpn_ctx* ctx, int l, cudaStream_t st) {
    const wskpn_config& c = ctx->cfg;
    Layer& L = ctx->layers[l];
    const bool fp8 = c.prec == WSKPN_FP8;
    const int wm = fp8 && ctx->fp8_split ? fp8_weight_mode(L.cin) : 0;
    const int nch = L.cin_p / (fp8 ? 32 : 16);
    const int ncc = wm == 1 ? 2 * nch : wm == 2 ? 2 * nch - 1 : nch;
    const float* w = ctx->d_master + L.woff;
    const float* b = ctx->d_master + L.boff;
    // the last layer of a tensor-core context with 64 input and 16 output channels
    // runs with folded horizontal taps (fewer, wider MMAs; see issue_item)
    L.xfold = l == c.n_layers - 1 && L.cin_p == 64 && L.cout_p == 16 && L.groups == 1 &&
              (c.conv_ks == 5 || c.conv_ks == 3);
    // tap blocks of 12 channels when the layer has at most 12 outputs (the
    // 2M = 12 logits): 5 x 12 = 60 -> 64 columns per output row instead of 80
    L.xf_cr = L.xfold ? (L.cout <= 12 ? 12 : 16) : 0;
    if (L.xfold) WSKPN_CUDA_TRY(cudaMemsetAsync(L.wtc, 0, L.wtc_bytes, st), ctx->err);
    if (fp8) {
        wscale_kernel<<<L.cout_p, 128, 0, st>>>(w, L.cin, L.cout, c.conv_ks, L.cout_p, L.wscale);
        WSKPN_CUDA_TRY(cudaGetLastError(), ctx->err);
    }
    pack_tc_kernel<<<148, 256, 0, st>>>(w, b, L.cin, L.cout, c.conv_ks, L.cout_p, L.groups, ncc, fp8, wm, L.xf_cr,
                                        L.wscale, ctx->act_scale[l], static_cast<uint8_t*>(L.wtc), L.ep_scale,
                                        L.ep_bias);
    WSKPN_CUDA_TRY(cudaGetLastError(), ctx->err);
    return WSKPN_OK;
}

template <int KS, int COUT_P, int NCC_IN, int NCC_W, bool FP8, int WM, bool XF, int EPI = 0, bool PIN = false>
static wskpn_status launch_tc_t(const CUtensorMap& map, const TcArgs& a, size_t smem, int grid, cudaStream_t st,
                                std::string& err) {
    auto kern = conv_tc_kernel<KS, COUT_P, NCC_IN, NCC_W, FP8, XF ? xf_rows_per_tile(KS, COUT_P) : tc::rows_per_tile(COUT_P),
                               WM, XF, EPI, PIN>;
    WSKPN_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), err);
    // programmatic dependent launch: set-up overlaps the previous kernel's
    // tail; the TMA producer waits for that kernel before reading activations
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(PIN ? tc::THREADS_PIN : tc::THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    WSKPN_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, map, a), err);
    return WSKPN_OK;
}

using TcLaunch = wskpn_status (*)(const CUtensorMap&, const TcArgs&, size_t, int, cudaStream_t, std::string&);

// The kernel instantiation for a layer shape: KS, output channels of one
// group, input chunks per row (hi/lo included), weight-image chunks,
// precision, e4m3 weight mode, folded taps.  nullptr when none is built.
static TcLaunch select_tc_kernel(int KS, int cg, int ncc_in, int ncc_w, bool fp8, int wm, bool xf, bool gm = false,
                                 bool rb = false, bool pin = false) {
    TcLaunch launch = nullptr;
    // the first layer assembling its own input (BF16 hi/lo, 10 -> 32)
    if (pin) {
        if (!xf && !gm && !rb && !fp8 && wm == 0 && cg == 32 && ncc_in == 2 && ncc_w == 1) {
            if (KS == 5) launch = launch_tc_t<5, 32, 2, 1, false, 0, false, 0, true>;
            if (KS == 3) launch = launch_tc_t<3, 32, 2, 1, false, 0, false, 0, true>;
        }
        if (!xf && !gm && !rb && fp8 && wm == 2 && cg == 32 && ncc_in == 2 && ncc_w == 1) {
            if (KS == 5) launch = launch_tc_t<5, 32, 2, 1, true, 2, false, 0, true>;
            if (KS == 3) launch = launch_tc_t<3, 32, 2, 1, true, 2, false, 0, true>;
        }
        return launch;
    }
#define WSKPN_TC_CASE(ks_, n_, nin_, nw_, f8_, wm_)                                                    \
    if (!launch && !xf && !gm && !rb && KS == ks_ && cg == n_ && ncc_in == nin_ && ncc_w == nw_ && fp8 == f8_ && wm == wm_) \
        launch = launch_tc_t<ks_, n_, nin_, nw_, f8_, wm_, false>;
#define WSKPN_TC_GM(ks_, n_, nin_, nw_)                                                                    \
    if (!launch && gm && !xf && !fp8 && KS == ks_ && cg == n_ && ncc_in == nin_ && ncc_w == nw_)             \
        launch = launch_tc_t<ks_, n_, nin_, nw_, false, 0, false, 1>;
#define WSKPN_TC_RB(ks_, n_, nin_, nw_)                                                                    \
    if (!launch && rb && !gm && !xf && !fp8 && KS == ks_ && cg == n_ && ncc_in == nin_ && ncc_w == nw_)      \
        launch = launch_tc_t<ks_, n_, nin_, nw_, false, 0, false, 2>;
    // the last layer 64 -> 12 or 16 with folded horizontal taps (tap blocks
    // of cg = 12 or 16 channels), BF16 (hi/lo activations, or single BF16
    // values when the split is tuned off) and e4m3 (hi/lo: three products per
    // chunk, or single-term)
#define WSKPN_TC_XF(n_)                                                                                          \
    if (xf && !gm && !rb && !fp8 && cg == n_ && KS == 5 && ncc_in == 8 && ncc_w == 4) launch = launch_tc_t<5, n_, 8, 4, false, 0, true>; \
    if (xf && !gm && !rb && !fp8 && cg == n_ && KS == 3 && ncc_in == 8 && ncc_w == 4) launch = launch_tc_t<3, n_, 8, 4, false, 0, true>; \
    if (xf && !gm && !rb && !fp8 && cg == n_ && KS == 5 && ncc_in == 4 && ncc_w == 4) launch = launch_tc_t<5, n_, 4, 4, false, 0, true>; \
    if (xf && !gm && !rb && !fp8 && cg == n_ && KS == 3 && ncc_in == 4 && ncc_w == 4) launch = launch_tc_t<3, n_, 4, 4, false, 0, true>; \
    if (xf && !gm && !rb && fp8 && cg == n_ && KS == 5 && wm == 1 && ncc_in == 4 && ncc_w == 4) launch = launch_tc_t<5, n_, 4, 4, true, 1, true>; \
    if (xf && !gm && !rb && fp8 && cg == n_ && KS == 3 && wm == 1 && ncc_in == 4 && ncc_w == 4) launch = launch_tc_t<3, n_, 4, 4, true, 1, true>; \
    if (xf && !gm && !rb && fp8 && cg == n_ && KS == 5 && wm == 0 && ncc_in == 2 && ncc_w == 2) launch = launch_tc_t<5, n_, 2, 2, true, 0, true>; \
    if (xf && !gm && !rb && fp8 && cg == n_ && KS == 3 && wm == 0 && ncc_in == 2 && ncc_w == 2) launch = launch_tc_t<3, n_, 2, 2, true, 0, true>;
    WSKPN_TC_XF(16) WSKPN_TC_XF(12)
#undef WSKPN_TC_XF
#define WSKPN_TC_BF16(ks_)                                                                                 \
    WSKPN_TC_CASE(ks_, 32, 1, 1, false, 0) WSKPN_TC_CASE(ks_, 32, 2, 1, false, 0)                          \
    WSKPN_TC_CASE(ks_, 48, 2, 2, false, 0) WSKPN_TC_CASE(ks_, 48, 4, 2, false, 0)                          \
    WSKPN_TC_CASE(ks_, 64, 3, 3, false, 0) WSKPN_TC_CASE(ks_, 64, 6, 3, false, 0)                          \
    WSKPN_TC_CASE(ks_, 16, 4, 4, false, 0) WSKPN_TC_CASE(ks_, 16, 8, 4, false, 0)                          \
    WSKPN_TC_CASE(ks_, 32, 4, 4, false, 0) WSKPN_TC_CASE(ks_, 32, 8, 4, false, 0)
// e4m3: single-term (widths 10-32-48-64-12 and 64-64), and hi/lo pairs of
// activations and weights (10 and 48 input channels with a trailing half
// chunk; 5x5 64-64 layers as two 32-channel output groups)
#define WSKPN_TC_FP8(ks_)                                                                                  \
    WSKPN_TC_CASE(ks_, 32, 1, 1, true, 0) WSKPN_TC_CASE(ks_, 48, 1, 1, true, 0)                            \
    WSKPN_TC_CASE(ks_, 64, 2, 2, true, 0) WSKPN_TC_CASE(ks_, 16, 2, 2, true, 0)                            \
    WSKPN_TC_CASE(ks_, 32, 2, 1, true, 2) WSKPN_TC_CASE(ks_, 48, 2, 2, true, 1)                            \
    WSKPN_TC_CASE(ks_, 64, 4, 3, true, 2) WSKPN_TC_CASE(ks_, 16, 4, 4, true, 1)                            \
    WSKPN_TC_CASE(ks_, 32, 4, 4, true, 1) WSKPN_TC_CASE(ks_, 64, 4, 4, true, 1)
// input gradients of the training step (BF16 gradients, weights transposed
// and flipped, the ReLU mask and bias sums in the epilogue): 12 -> 64,
// 64 -> 48, 48 -> 32, and 64 -> 64 as two 32-channel groups
#define WSKPN_TC_DGRAD(ks_)                                                                                \
    WSKPN_TC_GM(ks_, 64, 1, 1) WSKPN_TC_GM(ks_, 48, 4, 4) WSKPN_TC_GM(ks_, 32, 3, 3) WSKPN_TC_GM(ks_, 32, 4, 4)
// the training forward's ReLU layers with positive-channel bits (hi/lo
// activations): 10 -> 32, 32 -> 48, 48 -> 64 and 64 -> 64 as two 32-channel
// groups
#define WSKPN_TC_RELU_BITS(ks_) \
    WSKPN_TC_RB(ks_, 32, 2, 1) WSKPN_TC_RB(ks_, 48, 4, 2) WSKPN_TC_RB(ks_, 64, 6, 3) WSKPN_TC_RB(ks_, 32, 8, 4)
// the multi-resolution U-Net (3x3, hi/lo activations): 32-32, 48-48, 64-64,
// 112-48, 80-32 and the heads 48-5, 32-5
#define WSKPN_TC_UNET                                                                                      \
    WSKPN_TC_CASE(3, 32, 4, 2, false, 0) WSKPN_TC_CASE(3, 48, 6, 3, false, 0)                              \
    WSKPN_TC_CASE(3, 64, 8, 4, false, 0) WSKPN_TC_CASE(3, 48, 14, 7, false, 0)                             \
    WSKPN_TC_CASE(3, 32, 10, 5, false, 0) WSKPN_TC_CASE(3, 16, 6, 3, false, 0)                             \
    WSKPN_TC_CASE(3, 16, 4, 2, false, 0)
    WSKPN_TC_BF16(5) WSKPN_TC_BF16(3) WSKPN_TC_FP8(5) WSKPN_TC_FP8(3) WSKPN_TC_UNET
    WSKPN_TC_DGRAD(5) WSKPN_TC_DGRAD(3) WSKPN_TC_RELU_BITS(5) WSKPN_TC_RELU_BITS(3)
#undef WSKPN_TC_DGRAD
#undef WSKPN_TC_GM
#undef WSKPN_TC_RB
#undef WSKPN_TC_RELU_BITS
#undef WSKPN_TC_UNET
#undef WSKPN_TC_FP8
#undef WSKPN_TC_BF16
#undef WSKPN_TC_CASE
    return launch;
}

// One conv layer on the tensor cores, independent of a context.
// in: NHWC [B][H][W][cin_p x (split_in ? 2 : 1)] (BF16 or e4m3); out: NHWC
// with out_cp channels per stored pixel (x 2 when split_out), this layer's
// channels starting at out_c0, or (last) planar FP32 [B][cout][H][W].
struct TcRun {
    const Layer* L;
    int KS;
    bool fp8;
    int split_in, split_out;
    int last, relu;
    int out_cp, out_c0;
    int zero_pad;  // write storage channels past the layer's own (up to out_cp) as zeros
    int dup_src = -1, dup_dst = -1;  // e4m3 hi/lo trailing half chunk of the next layer (TcArgs)
    float out_qscale;
    unsigned int* status;
    int device;
    uint64_t wait_ns = MBAR_WAIT_NS;
    int probe = 0;
    const uint32_t* gbits = nullptr;  // input gradient: ReLU mask and bias sums in the epilogue (TcArgs)
    float* bias_part = nullptr;
    uint32_t* relu_bits = nullptr;    // ReLU layer: positive-channel bits of the output (TcArgs)
    int* grid_out = nullptr;      // receives the grid size (bias_part holds 4 rows per CTA)
    // the first layer assembling its input from these B FP32 frames (the
    // PIN kernels) instead of reading a stored input; in is then unused
    const wskpn_frame* frames = nullptr;
    PrepConst prep{};
    float in_qscale = 1.f;  // e4m3 input: 1 / its activation scale
};

static wskpn_status tc_run(const TcRun& r, const void* in, void* out, int B, int H, int W, cudaStream_t st,
                           std::string& err) {
    const Layer& L = *r.L;
    const bool fp8 = r.fp8;
    const int KS = r.KS;
    const int eb = fp8 ? 1 : 2;
    const int ch = fp8 ? 32 : 16;
    const bool pin = r.frames != nullptr;
    const int split = r.split_in;                   // hi/lo activations (BF16 or e4m3)
    const int wm = fp8 && split ? fp8_weight_mode(L.cin) : 0;  // e4m3 hi/lo weights with hi/lo activations
    const int cin_row = L.cin_p * (split ? 2 : 1);  // stored channels per input pixel
    const int ncc_in = L.cin_p / ch * (split ? 2 : 1);
    const int ncc_w = wm == 1 ? ncc_in : wm == 2 ? ncc_in - 1 : L.cin_p / ch;  // weight-image chunks
    const int cpb = chunks_per_box(ncc_in);
    CUtensorMap map;
    std::memset(&map, 0, sizeof(map));  // unused by the PIN kernels
    if (pin) {
        if (!split || r.last || !r.relu || r.gbits || r.relu_bits || L.xfold) {
            err = "conv_tc: input assembly in the first layer needs a ReLU layer with hi/lo input";
            return WSKPN_EINVAL;
        }
    } else {
        PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder(err);
        if (!encode) return WSKPN_EUNSUPPORTED;
        cuuint64_t gdim[4] = {(cuuint64_t)cin_row, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
        cuuint64_t gstr[3] = {(cuuint64_t)cin_row * eb, (cuuint64_t)W * cin_row * eb,
                              (cuuint64_t)H * W * cin_row * eb};
        cuuint32_t box[4] = {(cuuint32_t)(ch * cpb), (cuuint32_t)(tc::BM + KS - 1), 1, 1};
        cuuint32_t estr[4] = {1, 1, 1, 1};
        CUresult cr = encode(&map, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4,
                             const_cast<void*>(in), gdim, gstr, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                             cpb == 4 ? CU_TENSOR_MAP_SWIZZLE_128B
                                      : (cpb == 2 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B),
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (cr != CUDA_SUCCESS) {
            err = "cuTensorMapEncodeTiled failed (" + std::to_string((int)cr) + ")";
            return WSKPN_ECUDA;
        }
    }
    const int G = L.groups, cg0 = L.cout_p / G;
    const bool xf = L.xfold != 0;  // folded horizontal taps (the image was packed for them)
    // the kernel's channel parameter: channels per tap block when folded
    const int cg = xf ? L.xf_cr : cg0;
    const size_t group_bytes = L.wtc_bytes / G;
    TcArgs a{};
    a.wbytes = (uint32_t)(xf ? tc_wimg_bytes(KS, cg, ncc_w, cg) : group_bytes);
    a.out = out;
    a.B = B;
    a.H = H;
    a.W = W;
    a.cout = L.cout;
    a.out_cp = r.out_cp;
    a.last = r.last;
    a.relu = r.relu;
    a.split_out = r.split_out && !r.last;
    a.out_qscale = r.out_qscale;
    // boxes of 128 + KS - 1 rows of cpb x 32 B, each 1024-byte aligned (128B-swizzle atom)
    a.box_stride = (uint32_t)(((tc::BM + KS - 1) * tc::ROWB * cpb + 1023) / 1024 * 1024);
    a.row_bytes = tc_row_bytes(KS, ncc_in);
    if (xf && !(r.last && cg0 == 16)) {
        err = "conv_tc: folded-tap weights outside the last layer";
        return WSKPN_EINVAL;
    }
    const bool gm0 = r.gbits != nullptr, rb0 = r.relu_bits != nullptr;
    // the kernel's epilogue staging (its STG): as the kernel decides it
    const size_t stg =
        !xf && !gm0 && !rb0 && tc_stg_fits(KS, cg, ncc_in, ncc_w, fp8) ? tc_stg_bytes(cg, fp8) : 0;
    const size_t fixed = tc_fixed_bytes(KS, cg, ncc_w, xf ? cg : 0) + (xf ? tc_xf_bytes(KS) : 0) + stg;
    a.stage_bytes = tc_rows_per_item(KS, cg, ncc_in, ncc_w, stg, xf ? cg : 0) * a.row_bytes;  // the kernel's own RPI
    if (fixed + 2 * a.stage_bytes > tc::SMEM_MAX) {
        err = "conv_tc: layer weights and two input stages do not fit in shared memory";
        return WSKPN_EUNSUPPORTED;
    }
    const int stages = (int)((tc::SMEM_MAX - fixed) / a.stage_bytes);
    a.stages = stages < 6 ? stages : 6;
    // at least ~120 KB so that exactly one CTA (and one TMEM allocation) lives on an SM
    size_t smem = fixed + (size_t)a.stages * a.stage_bytes;
    if (smem < 120 * 1024) smem = 120 * 1024;
    a.tiles_x = cdiv(W, xf ? tc::BM - (KS - 1) : tc::BM);
    a.tiles_y = cdiv(H, xf ? xf_rows_per_tile(KS, cg) : tc::rows_per_tile(cg));
    a.ntiles = a.tiles_x * a.tiles_y * B;
    a.status = r.status;
    a.wait_ns = r.wait_ns;
    a.probe = r.probe;
    a.gbits = r.gbits;
    a.bias_part = r.bias_part;
    a.relu_bits = r.relu_bits;
    int nsm = 148;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, r.device);
    const int grid = a.ntiles < nsm ? a.ntiles : nsm;
    if (r.grid_out) *r.grid_out = grid;
    const bool gm = r.gbits != nullptr;
    if (r.relu_bits && (fp8 || xf || r.last || !r.relu || r.out_cp > 64 || r.out_c0 % 32 || (G > 1 && cg != 32))) {
        err = "conv_tc: ReLU bits need a BF16 ReLU layer of at most 64 channels in 32-channel groups";
        return WSKPN_EINVAL;
    }
    if (gm && (fp8 || xf || r.split_in || r.split_out || r.last || r.relu || !r.bias_part)) {
        err = "conv_tc: the gradient mask needs a single-BF16 input-gradient layer";
        return WSKPN_EINVAL;
    }
    const TcLaunch launch =
        select_tc_kernel(KS, cg, ncc_in, ncc_w, fp8, wm, xf, gm, r.relu_bits != nullptr, pin);
    if (!launch) {
        err = pin ? "conv_tc: no input-assembling kernel for this first layer (BF16 hi/lo 10 -> 32 is built)"
                  : "conv_tc: no kernel for this (KS, padded Cin, padded Cout, precision); widths 10-32-48-64-2M, "
                    "64-64 and the multi-resolution U-Net are built";
        return WSKPN_EUNSUPPORTED;
    }
    // PIN kernels take the frame pointers as a parameter table: at most
    // WSKPN_MAX_BATCH frames per launch
    const size_t out_pix_bytes = (size_t)r.out_cp * (fp8 ? 1 : 2) * (a.split_out ? 2 : 1);
    const int bstep = pin ? WSKPN_MAX_BATCH : B;
    for (int b0 = 0; b0 < B; b0 += bstep) {
        int gridc = grid;
        if (pin) {
            const int nb = B - b0 < bstep ? B - b0 : bstep;
            a.B = nb;
            a.ntiles = a.tiles_x * a.tiles_y * nb;
            gridc = a.ntiles < nsm ? a.ntiles : nsm;
            a.out = static_cast<uint8_t*>(out) + (size_t)b0 * H * W * out_pix_bytes;
            for (int j = 0; j < nb; ++j) {
                a.frames.r.p[j] = r.frames[b0 + j].radiance;
                a.frames.a.p[j] = r.frames[b0 + j].albedo;
                a.frames.n.p[j] = r.frames[b0 + j].normal;
                a.frames.d.p[j] = r.frames[b0 + j].depth;
            }
            a.prep = r.prep;
            a.in_qscale = r.in_qscale;
        }
        for (int g = 0; g < G; ++g) {  // each group reads the whole input and writes its channels
            a.wimg = static_cast<const uint8_t*>(L.wtc) + g * group_bytes;
            a.ep_scale = L.ep_scale + g * cg;
            a.ep_bias = L.ep_bias + g * cg;
            a.out_c0 = r.out_c0 + g * cg;
            const int end = r.out_c0 + L.cout_p;
            a.zero_c0 = end;
            a.zero_n = r.zero_pad && g == G - 1 && r.out_cp > end ? r.out_cp - end : 0;
            a.dup_src = r.dup_src;
            a.dup_dst = r.dup_dst;
            const wskpn_status s = launch(map, a, smem, gridc, st, err);
            if (s) return s;
        }
    }
    return WSKPN_OK;
}

int tc_split_of(const wskpn_ctx* ctx, int l) {
    return ctx->tc_split && ((ctx->tc_split_layers >> l) & 1u) ? 1 : 0;
}
bool tc_split_all(const wskpn_ctx* ctx) {
    for (int l = 0; l < ctx->cfg.n_layers; ++l)
        if (!tc_split_of(ctx, l)) return false;
    return true;
}

// One layer of a context's ImportanceNet (relu_bits: see TcArgs; BF16 only).
static wskpn_status conv_tc(wskpn_ctx* ctx, int l, const void* in, void* out, int B, int H, int W, cudaStream_t st,
                            uint32_t* relu_bits = nullptr, const wskpn_frame* frames = nullptr) {
    const wskpn_config& c = ctx->cfg;
    const bool fp8 = c.prec == WSKPN_FP8;
    TcRun r{};
    r.L = &ctx->layers[l];
    r.KS = c.conv_ks;
    r.fp8 = fp8;
    if (fp8) {
        r.split_in = r.split_out = ctx->fp8_split;
    } else {
        r.split_in = tc_split_of(ctx, l);
        r.split_out = l + 1 < c.n_layers ? tc_split_of(ctx, l + 1) : 0;
    }
    r.last = l == c.n_layers - 1;
    r.relu = !r.last;
    r.out_cp = r.last ? ctx->layers[l].cout_p : ctx->layers[l + 1].cin_p;  // stored channels per pixel
    r.zero_pad = 1;
    if (fp8 && ctx->fp8_split && !r.last && fp8_weight_mode(ctx->layers[l + 1].cin) == 2) {
        r.dup_src = ctx->layers[l + 1].cin / 32 * 32;  // the next layer's trailing half chunk
        r.dup_dst = r.dup_src + 16;
    }
    r.out_c0 = 0;
    r.out_qscale = fp8 && !r.last ? 1.f / ctx->act_scale[l + 1] : 1.f;
    r.status = ctx->d_status;
    r.device = ctx->device;
    r.wait_ns = ctx->wait_ns;
    r.probe = ctx->wait_probe;
    ctx->wait_probe = 0;  // the test hook applies to one launch
    r.relu_bits = relu_bits;
    if (frames) {  // the first layer assembles its input (same constants as the assembly kernel)
        r.frames = frames;
        r.prep.inv_gamma = (float)(1.0 / (double)c.gamma);
        r.prep.dnear = c.depth_near;
        r.prep.dscale = (float)(1.0 / ((double)c.depth_far - (double)c.depth_near));
        if (fp8) r.in_qscale = 1.f / ctx->act_scale[0];
    }
    return tc_run(r, in, out, B, H, W, st, ctx->err);
}

// The context's first layer can assemble its own input (hi/lo input pairs,
// BF16 or e4m3, and a kernel built for the layer's shape).
bool tc_fused_prep_supported(const wskpn_ctx* ctx) {
    const wskpn_config& c = ctx->cfg;
    if (c.n_layers < 2) return false;
    const Layer& L = ctx->layers[0];
    if (L.xfold || L.groups != 1) return false;
    if (c.prec == WSKPN_BF16) {
        if (!tc_split_of(ctx, 0)) return false;
        return select_tc_kernel(c.conv_ks, L.cout_p, 2 * (L.cin_p / 16), L.cin_p / 16, false, 0, false, false,
                                false, true) != nullptr;
    }
    if (c.prec == WSKPN_FP8) {
        if (!ctx->fp8_split || fp8_weight_mode(L.cin) != 2) return false;
        const int ncc_in = 2 * (L.cin_p / 32);
        return select_tc_kernel(c.conv_ks, L.cout_p, ncc_in, ncc_in - 1, true, 2, false, false, false, true) !=
               nullptr;
    }
    return false;
}

bool tc_relu_bits_supported(const wskpn_ctx* ctx, int l) {
    const Layer& L = ctx->layers[l];
    if (ctx->cfg.prec != WSKPN_BF16 || L.xfold || L.cout_p > 64 || (L.groups > 1 && L.cout_p / L.groups != 32))
        return false;
    const int ncc = L.cin_p / 16;
    return select_tc_kernel(ctx->cfg.conv_ks, L.cout_p / L.groups, 2 * ncc, ncc, false, 0, false, false, true) != nullptr;
}

wskpn_status tc_conv_layer(wskpn_ctx* ctx, int l, const void* in, void* out, int B, int H, int W, cudaStream_t st) {
    return conv_tc(ctx, l, in, out, B, H, W, st);
}

// A BF16 layer (hi/lo activations) outside a context: weight image, groups,
// epilogue bias; w [cout][cin][KS][KS] and b [cout] on the device.
wskpn_status tc_layer_create(Layer& L, int KS, const float* w, const float* b, cudaStream_t st, std::string& err) {
    L.cin_p = chan_pad(L.cin, false);
    L.cout_p = (L.cout + 15) / 16 * 16;
    if (L.cout_p > 64) {
        err = "tensor-core path supports at most 64 output channels per layer";
        return WSKPN_EUNSUPPORTED;
    }
    wskpn_status s = tc_layer_alloc(L, KS, false, false, err);
    if (s) return s;
    L.xfold = 0;
    pack_tc_kernel<<<148, 256, 0, st>>>(w, b, L.cin, L.cout, KS, L.cout_p, L.groups, L.cin_p / 16, 0, 0, 0, L.wscale, 1.f,
                                        static_cast<uint8_t*>(L.wtc), L.ep_scale, L.ep_bias);
    WSKPN_CUDA_TRY(cudaGetLastError(), err);
    return WSKPN_OK;
}

// Input gradient of a layer y = b + W * x (KS x KS cross-correlation, zero
// padding KS / 2): dL/dx[c](q) = sum_{o,t} W[o][c][t] dL/dy[o](q - t + pad),
// itself a KS x KS cross-correlation of dL/dy with cin and cout exchanged,
// every kernel flipped and no bias: wt[c][o][t] = w[o][c][KS*KS - 1 - t].
__global__ void transpose_flip_kernel(const float* __restrict__ w, int Cin, int Cout, int KK, float* __restrict__ wt) {
    const int n = Cin * Cout * KK;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int t = i % KK, o = (i / KK) % Cout, c = i / (KK * Cout);
        wt[i] = w[((size_t)o * Cin + c) * KK + (KK - 1 - t)];
    }
}

// The tensor-core layer (single BF16 values in and out) of the input gradient of a
// forward layer with cin -> cout channels: Lt.cin = cout, Lt.cout = cin.
// EUNSUPPORTED when no kernel is built for its shape (the caller then takes
// the FP32 path).
wskpn_status tc_dgrad_layer_alloc(Layer& Lt, int KS, int cin, int cout, std::string& err) {
    Lt.cin = cout;
    Lt.cout = cin;
    Lt.cin_p = chan_pad(Lt.cin, false);
    Lt.cout_p = (Lt.cout + 15) / 16 * 16;
    Lt.xfold = 0;
    if (Lt.cout_p > 64) {
        err = "tensor-core input gradient: at most 64 channels";
        return WSKPN_EUNSUPPORTED;
    }
    const wskpn_status s = tc_layer_alloc(Lt, KS, false, false, err);
    if (s) return s;
    const int ncc = Lt.cin_p / 16;
    if (!select_tc_kernel(KS, Lt.cout_p / Lt.groups, ncc, ncc, false, 0, false, true)) {
        err = "tensor-core input gradient: no kernel for this layer shape";
        return WSKPN_EUNSUPPORTED;
    }
    return WSKPN_OK;
}

// Packs Lt's weight image from the forward layer's FP32 weights w (OIHW
// [cout][cin][KS][KS] of the forward layer); wt: scratch of
// cin * cout * KS * KS floats; zero_bias: Lt.cout_p zeros.
wskpn_status tc_dgrad_layer_pack(Layer& Lt, int KS, const float* w, float* wt, const float* zero_bias,
                                 cudaStream_t st, std::string& err) {
    transpose_flip_kernel<<<148, 256, 0, st>>>(w, Lt.cout, Lt.cin, KS * KS, wt);
    WSKPN_CUDA_TRY(cudaGetLastError(), err);
    pack_tc_kernel<<<148, 256, 0, st>>>(wt, zero_bias, Lt.cin, Lt.cout, KS, Lt.cout_p, Lt.groups, Lt.cin_p / 16, 0, 0,
                                        0, Lt.wscale, 1.f, static_cast<uint8_t*>(Lt.wtc), Lt.ep_scale, Lt.ep_bias);
    WSKPN_CUDA_TRY(cudaGetLastError(), err);
    return WSKPN_OK;
}

void tc_layer_free(Layer& L) {
    cudaFree(L.wtc);
    cudaFree(L.ep_scale);
    cudaFree(L.ep_bias);
    cudaFree(L.wscale);
    L.wtc = nullptr;
    L.ep_scale = L.ep_bias = L.wscale = nullptr;
}

wskpn_status tc_layer_run(const Layer& L, int KS, const void* in, void* out, int out_cp, int out_c0, int last,
                          int relu, int B, int H, int W, unsigned int* status, int device, cudaStream_t st,
                          std::string& err) {
    TcRun r{};
    r.L = &L;
    r.KS = KS;
    r.fp8 = false;
    r.split_in = r.split_out = 1;
    r.last = last;
    r.relu = relu;
    r.out_cp = out_cp;
    r.out_c0 = out_c0;
    r.out_qscale = 1.f;
    r.status = status;
    r.device = device;
    return tc_run(r, in, out, B, H, W, st, err);
}

// tc_layer_run of a first layer that assembles its input from one frame's
// FP32 buffers (Sec. 5.1; the input-assembling kernel, BF16 hi/lo).
wskpn_status tc_layer_run_pin(const Layer& L, int KS, const wskpn_frame* frame, float gamma, float dnear, float dfar,
                              void* out, int out_cp, int relu, int H, int W, unsigned int* status, int device,
                              cudaStream_t st, std::string& err) {
    TcRun r{};
    r.L = &L;
    r.KS = KS;
    r.fp8 = false;
    r.split_in = r.split_out = 1;
    r.last = 0;
    r.relu = relu;
    r.out_cp = out_cp;
    r.out_c0 = 0;
    r.out_qscale = 1.f;
    r.status = status;
    r.device = device;
    r.frames = frame;
    r.prep.inv_gamma = (float)(1.0 / (double)gamma);
    r.prep.dnear = dnear;
    r.prep.dscale = (float)(1.0 / ((double)dfar - (double)dnear));
    return tc_run(r, nullptr, out, 1, H, W, st, err);
}

wskpn_status tc_dgrad_run(const Layer& Lt, int KS, const void* g, void* gx, const uint32_t* x_bits, float* bias_part,
                          int* nparts, int B, int H, int W, unsigned int* status, int device, cudaStream_t st,
                          std::string& err) {
    TcRun r{};
    r.L = &Lt;
    r.KS = KS;
    r.fp8 = false;
    r.split_in = r.split_out = 0;  // gradients as single BF16 values
    r.last = 0;
    r.relu = 0;
    r.out_cp = Lt.cout_p;
    r.out_c0 = 0;
    r.out_qscale = 1.f;
    r.status = status;
    r.device = device;
    r.gbits = x_bits;
    r.bias_part = bias_part;
    int grid = 0;
    r.grid_out = &grid;
    const wskpn_status s = tc_run(r, g, gx, B, H, W, st, err);
    *nparts = 4 * grid;
    return s;
}

wskpn_status launch_prep(const wskpn_frame* frames, int B, int H, int W, float gamma, float dnear, float dfar,
                         void* const* out, int layout, cudaStream_t st, std::string& err);

wskpn_status launch_prep_fp8(const wskpn_frame* frames, int B, int H, int W, float gamma, float dnear, float dfar,
                             void* const* out, float act_scale, int hilo, cudaStream_t st, std::string& err);

static wskpn_status tc_logits_fp8(wskpn_ctx* ctx, const wskpn_frame* frames, int B, int H, int W, float* z,
                                  cudaStream_t st) {
    const wskpn_config& c = ctx->cfg;
    if (!ctx->fp8_calibrated) {
        ctx->err = "FP8 context is not calibrated: call wskpn_calibrate first";
        return WSKPN_EUNSUPPORTED;
    }
    const size_t HW = (size_t)H * W;
    uint8_t* A = static_cast<uint8_t*>(ctx->d_tcA);
    uint8_t* Bf = static_cast<uint8_t*>(ctx->d_tcB);
    std::vector<void*> x0(B);
    const int split = ctx->fp8_split;
    for (int b = 0; b < B; ++b) x0[b] = A + (size_t)b * ctx->layers[0].cin_p * (split ? 2 : 1) * HW;
    // the first layer assembles its input tiles itself unless tuned off
    const bool fused = ctx->fused_prep && tc_fused_prep_supported(ctx);
    wskpn_status s = WSKPN_OK;
    if (!fused) {
        s = launch_prep_fp8(frames, B, H, W, c.gamma, c.depth_near, c.depth_far, x0.data(), ctx->act_scale[0],
                            split, st, ctx->err);
        if (s) return s;
    }
    prof_mark(ctx, 1, st);
    for (int l = 0; l < c.n_layers; ++l) {
        const void* in = l % 2 == 0 ? (const void*)A : (const void*)Bf;
        void* out = l == c.n_layers - 1 ? (void*)z : ((l + 1) % 2 == 0 ? (void*)A : (void*)Bf);
        s = conv_tc(ctx, l, in, out, B, H, W, st, nullptr, l == 0 && fused ? frames : nullptr);
        if (s) return s;
        prof_mark(ctx, 2 + l, st);
    }
    return WSKPN_OK;
}

wskpn_status tc_logits(wskpn_ctx* ctx, const wskpn_frame* frames, int B, int H, int W, float* z, cudaStream_t st) {
    const wskpn_config& c = ctx->cfg;
    if (c.prec == WSKPN_FP8) return tc_logits_fp8(ctx, frames, B, H, W, z, st);
    const size_t HW = (size_t)H * W;
    uint8_t* A = static_cast<uint8_t*>(ctx->d_tcA);
    uint8_t* Bf = static_cast<uint8_t*>(ctx->d_tcB);
    std::vector<void*> x0(B);
    const int split = tc_split_of(ctx, 0);
    const size_t x0_bytes = (size_t)ctx->layers[0].cin_p * 2 * (split ? 2 : 1) * HW;
    for (int b = 0; b < B; ++b) x0[b] = A + (size_t)b * x0_bytes;
    // the first layer assembles its input tiles itself (Sec. 5.1 inside its
    // producer) unless tuned off; otherwise the assembly kernel stores them
    const bool fused = ctx->fused_prep && tc_fused_prep_supported(ctx);
    wskpn_status s = WSKPN_OK;
    if (!fused) {
        s = launch_prep(frames, B, H, W, c.gamma, c.depth_near, c.depth_far, x0.data(), split ? 2 : 1, st,
                        ctx->err);
        if (s) return s;
    }
    prof_mark(ctx, 1, st);
    for (int l = 0; l < c.n_layers; ++l) {
        const void* in = l % 2 == 0 ? (const void*)A : (const void*)Bf;
        void* out = l == c.n_layers - 1 ? (void*)z : ((l + 1) % 2 == 0 ? (void*)A : (void*)Bf);
        s = conv_tc(ctx, l, in, out, B, H, W, st, nullptr, l == 0 && fused ? frames : nullptr);
        if (s) return s;
        prof_mark(ctx, 2 + l, st);
    }
    return WSKPN_OK;
}

// BF16 hi/lo NHWC [B][HW][hi(cp) | lo(cp)] -> planar FP32 out[b] [C][HW], x = hi + lo.
__global__ void hilo_to_planar_kernel(const __nv_bfloat16* __restrict__ in, int cp, int C, size_t HW, int B,
                                      PtrBatch<float*> out) {
    const size_t n = (size_t)B * C * HW;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t p = i % HW;
        const int c = (int)((i / HW) % C), b = (int)(i / (HW * C));
        const __nv_bfloat16* px = in + ((size_t)b * HW + p) * 2 * cp;
        out.p[b][(size_t)c * HW + p] = __bfloat162float(px[c]) + __bfloat162float(px[cp + c]);
    }
}

// The activations x_1 .. x_{L-1} of a BF16 context recomputed on the tensor
// cores exactly as its forward computes them (hi/lo activations), returned
// as planar FP32 acts[l - 1][b] [C_l][H][W] for the gradient kernels.
wskpn_status tc_recompute_acts(wskpn_ctx* ctx, const wskpn_frame* frames, int B, int H, int W,
                               const std::vector<std::vector<float*>>& acts, cudaStream_t st) {
    const wskpn_config& c = ctx->cfg;
    if (c.prec != WSKPN_BF16 || B > WSKPN_MAX_BATCH) {
        ctx->err = "tc_recompute_acts: BF16 contexts only, at most 16 frames";
        return WSKPN_EUNSUPPORTED;
    }
    const size_t HW = (size_t)H * W;
    uint8_t* A = static_cast<uint8_t*>(ctx->d_tcA);
    uint8_t* Bf = static_cast<uint8_t*>(ctx->d_tcB);
    const int split = tc_split_all(ctx) ? 1 : 0;
    std::vector<void*> x0(B);
    const size_t x0_bytes = (size_t)ctx->layers[0].cin_p * 2 * (split ? 2 : 1) * HW;
    for (int b = 0; b < B; ++b) x0[b] = A + (size_t)b * x0_bytes;
    wskpn_status s = launch_prep(frames, B, H, W, c.gamma, c.depth_near, c.depth_far, x0.data(), split ? 2 : 1, st,
                                 ctx->err);
    for (int l = 0; !s && l + 1 < c.n_layers; ++l) {
        const void* in = l % 2 == 0 ? (const void*)A : (const void*)Bf;
        void* out = (l + 1) % 2 == 0 ? (void*)A : (void*)Bf;
        s = conv_tc(ctx, l, in, out, B, H, W, st);
        if (s) break;
        if (!split) {
            ctx->err = "tc_recompute_acts: needs hi/lo activations";
            return WSKPN_EUNSUPPORTED;
        }
        PtrBatch<float*> o{};
        for (int b = 0; b < B; ++b) o.p[b] = acts[l][b];
        const Layer& L = ctx->layers[l];
        hilo_to_planar_kernel<<<148 * 8, 256, 0, st>>>(static_cast<const __nv_bfloat16*>(out), L.cout_p, L.cout, HW,
                                                       B, o);
        WSKPN_CUDA_TRY(cudaGetLastError(), ctx->err);
    }
    return s;
}

// The layer inputs x_0 .. x_{L-1} of a BF16 context (hi/lo activations)
// recomputed on the tensor cores exactly as its forward computes them, kept
// channels-last: xs[l] = NHWC [B][H][W][hi(cin_p) | lo(cin_p)] of layer l.
wskpn_status tc_recompute_nhwc(wskpn_ctx* ctx, const wskpn_frame* frames, int B, int H, int W,
                               const std::vector<void*>& xs, cudaStream_t st, const std::vector<uint32_t*>* bits) {
    const wskpn_config& c = ctx->cfg;
    if (c.prec != WSKPN_BF16 || !tc_split_all(ctx) || B > WSKPN_MAX_BATCH) {
        ctx->err = "tc_recompute_nhwc: BF16 contexts with hi/lo activations only, at most 16 frames";
        return WSKPN_EUNSUPPORTED;
    }
    const size_t HW = (size_t)H * W;
    std::vector<void*> x0(B);
    const size_t x0_bytes = (size_t)ctx->layers[0].cin_p * 2 * 2 * HW;
    for (int b = 0; b < B; ++b) x0[b] = static_cast<uint8_t*>(xs[0]) + (size_t)b * x0_bytes;
    wskpn_status s = launch_prep(frames, B, H, W, c.gamma, c.depth_near, c.depth_far, x0.data(), 2, st, ctx->err);
    for (int l = 0; !s && l + 1 < c.n_layers; ++l)
        s = conv_tc(ctx, l, xs[l], xs[l + 1], B, H, W, st, bits ? (*bits)[l + 1] : nullptr);
    return s;
}

// max over n non-negative floats (ReLU outputs, [0,1] inputs) by their bit patterns
__global__ void amax_nonneg_kernel(const float* __restrict__ x, size_t n, unsigned int* __restrict__ out) {
    unsigned int m = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        m = max(m, __float_as_uint(fmaxf(x[i], 0.f)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

wskpn_status launch_conv_simt(const float* const* in, float* const* out, int B, int H, int W, int Cin, int Cout,
                              int KS, const float* w_packed, const float* bias_padded, int relu, cudaStream_t st,
                              std::string& err);

}  // namespace wskpn

using namespace wskpn;

extern "C" wskpn_status wskpn_calibrate(wskpn_ctx* ctx, const wskpn_frame* frames, int batch, int h, int w,
                                        float margin, void* stream) {
    if (!ctx) return WSKPN_EINVAL;
    const wskpn_config& c = ctx->cfg;
    if (c.prec != WSKPN_FP8) {
        ctx->err = "wskpn_calibrate: only FP8 contexts have activation scales";
        return WSKPN_EINVAL;
    }
    if (!frames || batch < 1 || batch > WSKPN_MAX_BATCH || h < 1 || w < 1 || !(margin >= 1.f)) {
        ctx->err = "wskpn_calibrate: invalid argument";
        return WSKPN_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t HW = (size_t)h * w;
    int maxw = 0;
    for (int l = 0; l < c.n_layers; ++l) maxw = maxw > c.widths[l] ? maxw : c.widths[l];
    float* buf[2] = {nullptr, nullptr};
    unsigned int* d_amax = nullptr;
    auto cleanup = [&]() {
        cudaFree(buf[0]);
        cudaFree(buf[1]);
        cudaFree(d_amax);
    };
    if (cudaMalloc(&buf[0], (size_t)batch * maxw * HW * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&buf[1], (size_t)batch * maxw * HW * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&d_amax, WSKPN_MAX_LAYERS * sizeof(unsigned int)) != cudaSuccess) {
        cleanup();
        ctx->err = "wskpn_calibrate: temporary allocation failed";
        return WSKPN_ENOMEM;
    }
    wskpn_status s = WSKPN_OK;
    cudaMemsetAsync(d_amax, 0, WSKPN_MAX_LAYERS * sizeof(unsigned int), st);
    std::vector<void*> x0(batch);
    for (int b = 0; b < batch; ++b) x0[b] = buf[0] + (size_t)b * c.widths[0] * HW;
    s = launch_prep(frames, batch, h, w, c.gamma, c.depth_near, c.depth_far, x0.data(), 0, st, ctx->err);
    if (!s) s = ctx_simt_weights(ctx, st);
    std::vector<const float*> in(batch);
    std::vector<float*> out(batch);
    for (int l = 0; l < c.n_layers && !s; ++l) {
        amax_nonneg_kernel<<<148, 256, 0, st>>>(buf[l % 2], (size_t)batch * c.widths[l] * HW, d_amax + l);
        if (l == c.n_layers - 1) break;
        for (int b = 0; b < batch; ++b) {
            in[b] = buf[l % 2] + (size_t)b * c.widths[l] * HW;
            out[b] = buf[(l + 1) % 2] + (size_t)b * c.widths[l + 1] * HW;
        }
        const Layer& L = ctx->layers[l];
        s = launch_conv_simt(in.data(), out.data(), batch, h, w, L.cin, L.cout, c.conv_ks, L.w32, L.b32, 1, st,
                             ctx->err);
    }
    unsigned int h_amax[WSKPN_MAX_LAYERS] = {};
    if (!s && (cudaMemcpyAsync(h_amax, d_amax, sizeof(h_amax), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
               cudaStreamSynchronize(st) != cudaSuccess)) {
        ctx->err = "wskpn_calibrate: CUDA error";
        s = WSKPN_ECUDA;
    }
    cleanup();
    if (s) return s;
    for (int l = 0; l < c.n_layers; ++l) {
        float m;
        std::memcpy(&m, &h_amax[l], sizeof(m));
        ctx->act_scale[l] = m > 0.f ? m * margin / 448.f : 1.f;
    }
    ctx->fp8_calibrated = true;
    return ctx_repack(ctx, st);
}
