// Tensor-core path of the ImportanceNet convolutions (Sec. 4.1) on sm_103a:
// implicit-GEMM KSxKS conv + bias (+ ReLU) with tcgen05.mma, operands staged
// by TMA, FP32 accumulators in tensor memory.
//
// GEMM view of one tile: M = 128 consecutive pixels of an image row (TMEM
// lanes), N = padded output channels, K = KS*KS taps x input channels,
// consumed 32 bytes (16 BF16 or 32 e4m3 channels) at a time.  A CTA owns
// R = 4 output rows x 128 pixels and keeps 4 accumulators (one per output
// row) in TMEM, double-buffered across tiles so the epilogue of one tile
// overlaps the MMAs of the next.  Each input row is fetched once per tile
// and channel chunk and serves every (dy, dx) tap that reads it:
//   mode 0: one TMA box of 128 + KS - 1 pixels; the KS horizontal taps use
//           the same box through operand descriptors shifted by dx rows;
//   mode 1: KS TMA boxes of 128 pixels, one per horizontal tap.
// The weights of the layer stay resident in shared memory for the whole
// persistent kernel (pre-swizzled image, one bulk copy per CTA).
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
#include <cuda_fp8.h>

#include <mutex>
#include <vector>

#include "ctx.h"

namespace wskpn {

namespace tc {
constexpr int BM = 128;            // pixels per tile row = MMA M = TMEM lanes
constexpr int R = 4;               // output rows per tile
constexpr int THREADS = 192;
constexpr int ROWB = 32;           // bytes of one pixel row of one K chunk
constexpr uint32_t SMEM_MAX = 232448;
constexpr uint64_t WAIT_NS = 2000000000ull;
constexpr unsigned ST_TIMEOUT_PRODUCER = 1u, ST_TIMEOUT_MMA = 2u, ST_TIMEOUT_EPILOGUE = 4u;
}  // namespace tc

struct TcArgs {
    const void* wimg;        // shared-memory image of the layer's weights
    uint32_t wbytes;
    const float* ep_scale;   // [COUT_P] multiplier of the accumulator
    const float* ep_bias;    // [COUT_P]
    void* out;               // NHWC [B][H][W][COUT_P] activations, or planar FP32 [B][cout][H][W]
    int B, H, W;
    int ncc;                 // K chunks per tap
    int cout;                // real output channels
    int relu, last;
    float out_qscale;        // FP8 activations: 1 / scale of the output activation
    int mode;                // see file comment
    int desc_base_offset;    // fill the descriptor's base-offset field from the start address
    int stages;
    uint32_t stage_bytes;
    int tiles_x, tiles_y, ntiles;
    unsigned int* status;
};

// ------------------------------------------------------------- primitives
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t a, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait: false when the limit expired or another role aborted.
__device__ __noinline__ bool mbar_wait(uint32_t a, uint32_t parity, const volatile int* abort_flag) {
    if (mbar_try_wait(a, parity)) return true;
    const uint64_t t0 = gtimer();
    while (true) {
#pragma unroll 1
        for (int i = 0; i < 32; ++i)
            if (mbar_try_wait(a, parity)) return true;
        if (*abort_flag) return false;
        if (gtimer() - t0 > tc::WAIT_NS) return false;
    }
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(mbar)
        : "memory");
}
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// K-major operand, 32-byte swizzle: rows of 32 bytes, 8-row groups 256 B apart.
__device__ __forceinline__ uint64_t sdesc_sw32(uint32_t saddr, int base_offset_mode) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;              // leading byte offset (unused for this layout)
    d |= (uint64_t)(256 >> 4) << 32;     // stride byte offset: 8 rows x 32 B
    d |= (uint64_t)1 << 46;              // descriptor version for tcgen05
    if (base_offset_mode) d |= (uint64_t)((saddr >> 7) & 7u) << 49;
    d |= (uint64_t)6 << 61;              // 32-byte swizzle
    return d;
}
template <bool FP8>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if constexpr (FP8) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc)
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

template <int COUT_P>
__host__ __device__ constexpr uint32_t tmem_cols() {
    return 2 * tc::R * COUT_P <= 32 ? 32 : 2 * tc::R * COUT_P <= 64 ? 64 : 2 * tc::R * COUT_P <= 128 ? 128
           : 2 * tc::R * COUT_P <= 256 ? 256 : 512;
}

// ----------------------------------------------------------------- kernel
template <int KS, int COUT_P, bool FP8>
__global__ void __launch_bounds__(tc::THREADS, 1)
    conv_tc_kernel(const __grid_constant__ CUtensorMap tmap, const TcArgs a) {
    constexpr int PAD = KS / 2;
    constexpr int CH = FP8 ? 32 : 16;  // channels per K chunk
    constexpr uint32_t NCOL = tmem_cols<COUT_P>();
    static_assert(COUT_P % 16 == 0 && COUT_P >= 16 && COUT_P <= 256, "MMA N");
    static_assert(2 * tc::R * COUT_P <= 512, "TMEM columns");
    constexpr uint32_t IDESC = (1u << 4) | (FP8 ? 0u : ((1u << 7) | (1u << 10))) |
                               ((uint32_t)(COUT_P >> 3) << 17) | ((uint32_t)(tc::BM >> 4) << 24);

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
    volatile uint32_t* tmem_holder = reinterpret_cast<volatile uint32_t*>(fin + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(fin + 1) + 1;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(smem_u32(&accf[i]), 1);
            mbar_init(smem_u32(&acce[i]), 4);
        }
        mbar_init(smem_u32(wbar), 1);
        mbar_init(smem_u32(fin), 1);
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

    const int rows_in = tc::R + KS - 1;
    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            const uint32_t wb = smem_u32(wbar);
            mbar_expect_tx(wb, a.wbytes);
            for (uint32_t off = 0; off < a.wbytes; off += 32768u) {
                const uint32_t n = a.wbytes - off < 32768u ? a.wbytes - off : 32768u;
                bulk_load(smem_u32(sW + off), static_cast<const uint8_t*>(a.wimg) + off, n, wb);
            }
            uint32_t it = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x) {
                const int tx = t % a.tiles_x, ty = (t / a.tiles_x) % a.tiles_y, b = t / (a.tiles_x * a.tiles_y);
                const int x0 = tx * tc::BM, y0 = ty * tc::R;
                for (int ri = 0; ri < rows_in && ok; ++ri)
                    for (int cc = 0; cc < a.ncc; ++cc, ++it) {
                        const int s = it % S;
                        const uint32_t ph = (it / S) & 1u;
                        if (!mbar_wait(smem_u32(&empty[s]), ph ^ 1u, abort_flag)) {
                            ok = false;
                            break;
                        }
                        const uint32_t fb = smem_u32(&full[s]);
                        const uint32_t dst = smem_u32(sA + (size_t)s * a.stage_bytes);
                        if (a.mode == 0) {
                            mbar_expect_tx(fb, (tc::BM + KS - 1) * tc::ROWB);
                            tma_load_4d(dst, &tmap, cc * CH, x0 - PAD, y0 - PAD + ri, b, fb);
                        } else {
                            mbar_expect_tx(fb, KS * tc::BM * tc::ROWB);
                            for (int dx = 0; dx < KS; ++dx)
                                tma_load_4d(dst + dx * tc::BM * tc::ROWB, &tmap, cc * CH, x0 - PAD + dx,
                                            y0 - PAD + ri, b, fb);
                        }
                    }
            }
            if (!ok) {
                atomicOr(a.status, tc::ST_TIMEOUT_PRODUCER);
                *abort_flag = 1;
            }
            // Drain: every issued stage's load must have landed before exit.
            const uint32_t n_in_flight = it < (uint32_t)S ? it : (uint32_t)S;
            for (uint32_t k = 0; k < n_in_flight; ++k) {
                const uint32_t j = it - 1 - k;
                mbar_wait(smem_u32(&full[j % S]), (j / S) & 1u, abort_flag);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            bool ok = mbar_wait(smem_u32(wbar), 0, abort_flag);
            const uint32_t wbase = smem_u32(sW);
            uint32_t it = 0;
            int lt = 0;
            for (int t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x, ++lt) {
                const int buf = lt & 1;
                if (!mbar_wait(smem_u32(&acce[buf]), ((lt >> 1) & 1) ^ 1, abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t dbase = tmem + (uint32_t)(buf * tc::R * COUT_P);
                for (int ri = 0; ri < rows_in && ok; ++ri)
                    for (int cc = 0; cc < a.ncc; ++cc, ++it) {
                        const int s = it % S;
                        if (!mbar_wait(smem_u32(&full[s]), (it / S) & 1u, abort_flag)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t abase = smem_u32(sA + (size_t)s * a.stage_bytes);
#pragma unroll
                        for (int dy = 0; dy < KS; ++dy) {
                            const int ro = ri - dy;
                            if (ro < 0 || ro >= tc::R) continue;
#pragma unroll
                            for (int dx = 0; dx < KS; ++dx) {
                                const uint32_t aaddr =
                                    a.mode == 0 ? abase + dx * tc::ROWB : abase + dx * tc::BM * tc::ROWB;
                                const uint32_t baddr =
                                    wbase + (uint32_t)(((dy * KS + dx) * a.ncc + cc) * COUT_P * tc::ROWB);
                                mma<FP8>(dbase + (uint32_t)(ro * COUT_P), sdesc_sw32(aaddr, a.desc_base_offset),
                                         sdesc_sw32(baddr, 0), IDESC, (dy | cc | dx) != 0);
                            }
                        }
                        mma_commit(smem_u32(&empty[s]));  // frees the stage when these MMAs finish
                    }
                if (ok) mma_commit(smem_u32(&accf[buf]));
            }
            if (!ok) {
                atomicOr(a.status, tc::ST_TIMEOUT_MMA);
                *abort_flag = 1;
            }
            // Every issued MMA must complete before TMEM is released.
            mma_commit(smem_u32(fin));
            mbar_wait(smem_u32(fin), 0, abort_flag);
        }
    } else {
        // ------------------------------------------------ epilogue warps 2..5
        const int q = warp & 3;  // TMEM lane quarter this warp may access
        const int p = q * 32 + lane;
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        int lt = 0;
        for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++lt) {
            const int buf = lt & 1;
            int ok = 1;
            if (lane == 0) ok = mbar_wait(smem_u32(&accf[buf]), (lt >> 1) & 1, abort_flag);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) {
                if (lane == 0) {
                    atomicOr(a.status, tc::ST_TIMEOUT_EPILOGUE);
                    *abort_flag = 1;
                }
                break;
            }
            tc_fence_after();
            const int tx = t % a.tiles_x, ty = (t / a.tiles_x) % a.tiles_y, b = t / (a.tiles_x * a.tiles_y);
            const int x = tx * tc::BM + p;
#pragma unroll 1
            for (int r = 0; r < tc::R; ++r) {
                const int y = ty * tc::R + r;
                const bool valid = x < a.W && y < a.H;
                const uint32_t col = (uint32_t)(buf * tc::R * COUT_P + r * COUT_P);
#pragma unroll
                for (int c16 = 0; c16 < COUT_P / 16; ++c16) {
                    float v[16];
                    tmem_ld16(tmem + lane_base + col + c16 * 16, v);
                    if (!valid) continue;
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int o = c16 * 16 + j;
                        v[j] = fmaf(v[j], a.ep_scale[o], a.ep_bias[o]);
                        if (a.relu) v[j] = fmaxf(v[j], 0.f);
                    }
                    const size_t pix = ((size_t)b * a.H + y) * a.W + x;
                    if (a.last) {
                        float* z = static_cast<float*>(a.out);
                        const size_t HW = (size_t)a.H * a.W;
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const int o = c16 * 16 + j;
                            if (o < a.cout) z[((size_t)b * a.cout + o) * HW + (size_t)y * a.W + x] = v[j];
                        }
                    } else if constexpr (FP8) {
                        uint32_t w[4];
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const __nv_fp8x2_storage_t lo = __nv_cvt_float2_to_fp8x2(
                                make_float2(v[4 * j] * a.out_qscale, v[4 * j + 1] * a.out_qscale), __NV_SATFINITE,
                                __NV_E4M3);
                            const __nv_fp8x2_storage_t hi = __nv_cvt_float2_to_fp8x2(
                                make_float2(v[4 * j + 2] * a.out_qscale, v[4 * j + 3] * a.out_qscale),
                                __NV_SATFINITE, __NV_E4M3);
                            w[j] = (uint32_t)lo | ((uint32_t)hi << 16);
                        }
                        uint4* dst = reinterpret_cast<uint4*>(static_cast<uint8_t*>(a.out) + pix * COUT_P + c16 * 16);
                        *dst = make_uint4(w[0], w[1], w[2], w[3]);
                    } else {
                        __nv_bfloat162 h2[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) h2[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                        uint4* dst = reinterpret_cast<uint4*>(static_cast<uint8_t*>(a.out) + (pix * COUT_P + c16 * 16) * 2);
                        const uint4* src = reinterpret_cast<const uint4*>(h2);
                        dst[0] = src[0];
                        dst[1] = src[1];
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&acce[buf]));
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
static PFN_cuTensorMapEncodeTiled_v12000 get_encode(std::string& err) {
    static std::mutex mu;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !p) {
            err = "cuTensorMapEncodeTiled is not available from the driver";
            return nullptr;
        }
        fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

static int chan_pad(int c, bool fp8) { return fp8 ? (c + 31) / 32 * 32 : (c + 15) / 16 * 16; }
static int cout_pad(const wskpn_config& c, int l) {
    const bool fp8 = c.prec == WSKPN_FP8;
    return l == c.n_layers - 1 ? (c.widths[l + 1] + 15) / 16 * 16 : chan_pad(c.widths[l + 1], fp8);
}

size_t tc_act_bytes_per_pixel(const wskpn_config& c, int which) {
    const bool fp8 = c.prec == WSKPN_FP8;
    size_t m = 0;
    for (int l = 0; l < c.n_layers; ++l)
        if (l % 2 == which) {
            const size_t b = (size_t)chan_pad(c.widths[l], fp8) * (fp8 ? 1 : 2);
            m = b > m ? b : m;
        }
    return m;
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
    const int ncc = L.cin_p / (fp8 ? 32 : 16);
    L.wtc_bytes = (size_t)c.conv_ks * c.conv_ks * ncc * L.cout_p * tc::ROWB;
    WSKPN_CUDA_TRY(cudaMalloc(&L.wtc, L.wtc_bytes), ctx->err);
    WSKPN_CUDA_TRY(cudaMalloc(&L.ep_scale, L.cout_p * sizeof(float)), ctx->err);
    WSKPN_CUDA_TRY(cudaMalloc(&L.ep_bias, L.cout_p * sizeof(float)), ctx->err);
    WSKPN_CUDA_TRY(cudaMalloc(&L.wscale, L.cout_p * sizeof(float)), ctx->err);
    return WSKPN_OK;
}

// Builds the shared-memory image of a layer's B operand: chunk (tap, cc)
// holds COUT_P rows of 32 bytes (K-major), 32-byte swizzled like the TMA
// writes A: byte o of a chunk goes to o ^ (((o >> 7) & 1) << 4).
__global__ void pack_tc_kernel(const float* __restrict__ w, const float* __restrict__ bias, int Cin, int Cout,
                               int KS, int cout_p, int ncc, int fp8, const float* __restrict__ wscale,
                               float act_in_scale, uint8_t* __restrict__ img, float* __restrict__ ep_scale,
                               float* __restrict__ ep_bias) {
    const int ch = fp8 ? 32 : 16;
    const int n_el = KS * KS * ncc * cout_p * ch;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_el; i += gridDim.x * blockDim.x) {
        const int k = i % ch;
        const int n = (i / ch) % cout_p;
        const int chunk = i / (ch * cout_p);
        const int cc = chunk % ncc, t = chunk / ncc;
        const int cin = cc * ch + k;
        const float v = (n < Cout && cin < Cin) ? w[((size_t)n * Cin + cin) * KS * KS + t] : 0.f;
        const uint32_t o = (uint32_t)(n * 32 + k * (fp8 ? 1 : 2));
        const uint32_t phys = (uint32_t)chunk * cout_p * 32 + (o ^ (((o >> 7) & 1u) << 4));
        if (fp8) {
            img[phys] = (uint8_t)__nv_cvt_float_to_fp8(v / wscale[n], __NV_SATFINITE, __NV_E4M3);
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
    const int ncc = L.cin_p / (fp8 ? 32 : 16);
    const float* w = ctx->d_master + L.woff;
    const float* b = ctx->d_master + L.boff;
    if (fp8) {
        wscale_kernel<<<L.cout_p, 128, 0, st>>>(w, L.cin, L.cout, c.conv_ks, L.cout_p, L.wscale);
        WSKPN_CUDA_TRY(cudaGetLastError(), ctx->err);
    }
    pack_tc_kernel<<<148, 256, 0, st>>>(w, b, L.cin, L.cout, c.conv_ks, L.cout_p, ncc, fp8, L.wscale,
                                        ctx->act_scale[l], static_cast<uint8_t*>(L.wtc), L.ep_scale, L.ep_bias);
    WSKPN_CUDA_TRY(cudaGetLastError(), ctx->err);
    return WSKPN_OK;
}

template <int KS, int COUT_P, bool FP8>
static wskpn_status launch_tc_t(const CUtensorMap& map, const TcArgs& a, size_t smem, int grid, cudaStream_t st,
                                std::string& err) {
    WSKPN_CUDA_TRY(cudaFuncSetAttribute(conv_tc_kernel<KS, COUT_P, FP8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem),
                   err);
    conv_tc_kernel<KS, COUT_P, FP8><<<grid, tc::THREADS, smem, st>>>(map, a);
    WSKPN_CUDA_TRY(cudaGetLastError(), err);
    return WSKPN_OK;
}

// One conv layer on the tensor cores.  in: NHWC [B][H][W][cin_p] (BF16 or
// e4m3); out: NHWC [B][H][W][cout_p] or (last) planar FP32 [B][cout][H][W].
static wskpn_status conv_tc(wskpn_ctx* ctx, int l, const void* in, void* out, int B, int H, int W, cudaStream_t st) {
    const wskpn_config& c = ctx->cfg;
    const Layer& L = ctx->layers[l];
    const bool fp8 = c.prec == WSKPN_FP8;
    const int KS = c.conv_ks;
    const int eb = fp8 ? 1 : 2;
    const int ch = fp8 ? 32 : 16;
    PFN_cuTensorMapEncodeTiled_v12000 encode = get_encode(ctx->err);
    if (!encode) return WSKPN_EUNSUPPORTED;
    const int mode = ctx->tc_mode;
    CUtensorMap map;
    cuuint64_t gdim[4] = {(cuuint64_t)L.cin_p, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
    cuuint64_t gstr[3] = {(cuuint64_t)L.cin_p * eb, (cuuint64_t)W * L.cin_p * eb, (cuuint64_t)H * W * L.cin_p * eb};
    cuuint32_t box[4] = {(cuuint32_t)ch, (cuuint32_t)(mode == 0 ? tc::BM + KS - 1 : tc::BM), 1, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult cr = encode(&map, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4,
                         const_cast<void*>(in), gdim, gstr, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) {
        ctx->err = "cuTensorMapEncodeTiled failed (" + std::to_string((int)cr) + ")";
        return WSKPN_ECUDA;
    }
    TcArgs a{};
    a.wimg = L.wtc;
    a.wbytes = (uint32_t)L.wtc_bytes;
    a.ep_scale = L.ep_scale;
    a.ep_bias = L.ep_bias;
    a.out = out;
    a.B = B;
    a.H = H;
    a.W = W;
    a.ncc = L.cin_p / ch;
    a.cout = L.cout;
    a.last = l == c.n_layers - 1;
    a.relu = !a.last;
    a.out_qscale = fp8 && !a.last ? 1.f / ctx->act_scale[l + 1] : 1.f;
    a.mode = mode;
    a.desc_base_offset = ctx->tc_desc_base_offset;
    a.stage_bytes = mode == 0 ? (uint32_t)(((tc::BM + KS - 1) * tc::ROWB + 1023) / 1024 * 1024)
                              : (uint32_t)(KS * tc::BM * tc::ROWB);
    const size_t fixed = 1024 + ((L.wtc_bytes + 1023) / 1024 * 1024) + 256;
    if (fixed + 2 * a.stage_bytes > tc::SMEM_MAX) {
        ctx->err = "conv_tc: layer weights do not fit in shared memory";
        return WSKPN_EUNSUPPORTED;
    }
    int stages = (int)((tc::SMEM_MAX - fixed) / a.stage_bytes);
    const int max_stages = mode == 0 ? 8 : 4;
    a.stages = stages < max_stages ? stages : max_stages;
    // at least ~120 KB so that exactly one CTA (and one TMEM allocation) lives on an SM
    size_t smem = fixed + (size_t)a.stages * a.stage_bytes;
    if (smem < 120 * 1024) smem = 120 * 1024;
    a.tiles_x = cdiv(W, tc::BM);
    a.tiles_y = cdiv(H, tc::R);
    a.ntiles = a.tiles_x * a.tiles_y * B;
    a.status = ctx->d_status;
    int nsm = 148;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device);
    const int grid = a.ntiles < nsm ? a.ntiles : nsm;
#define WSKPN_TC_CASE(ks_, n_, f8_)                                                   \
    if (KS == ks_ && L.cout_p == n_ && fp8 == f8_)                                    \
        return launch_tc_t<ks_, n_, f8_>(map, a, smem, grid, st, ctx->err);
    WSKPN_TC_CASE(5, 16, false) WSKPN_TC_CASE(5, 32, false) WSKPN_TC_CASE(5, 48, false) WSKPN_TC_CASE(5, 64, false)
    WSKPN_TC_CASE(3, 16, false) WSKPN_TC_CASE(3, 32, false) WSKPN_TC_CASE(3, 48, false) WSKPN_TC_CASE(3, 64, false)
    WSKPN_TC_CASE(5, 16, true) WSKPN_TC_CASE(5, 32, true) WSKPN_TC_CASE(5, 64, true)
    WSKPN_TC_CASE(3, 16, true) WSKPN_TC_CASE(3, 32, true) WSKPN_TC_CASE(3, 64, true)
#undef WSKPN_TC_CASE
    ctx->err = "conv_tc: unsupported (KS, padded Cout, precision)";
    return WSKPN_EUNSUPPORTED;
}

wskpn_status launch_prep(const wskpn_frame* frames, int B, int H, int W, float gamma, float dnear, float dfar,
                         void* const* out, int layout, cudaStream_t st, std::string& err);

wskpn_status tc_logits(wskpn_ctx* ctx, const wskpn_frame* frames, int B, int H, int W, float* z, cudaStream_t st) {
    const wskpn_config& c = ctx->cfg;
    if (c.prec == WSKPN_FP8) {
        ctx->err = "FP8 convolutions are not enabled in this build";
        return WSKPN_EUNSUPPORTED;
    }
    const size_t HW = (size_t)H * W;
    uint8_t* A = static_cast<uint8_t*>(ctx->d_tcA);
    uint8_t* Bf = static_cast<uint8_t*>(ctx->d_tcB);
    std::vector<void*> x0(B);
    const size_t x0_bytes = (size_t)ctx->layers[0].cin_p * 2 * HW;
    for (int b = 0; b < B; ++b) x0[b] = A + (size_t)b * x0_bytes;
    wskpn_status s = launch_prep(frames, B, H, W, c.gamma, c.depth_near, c.depth_far, x0.data(), 1, st, ctx->err);
    if (s) return s;
    prof_mark(ctx, 1, st);
    for (int l = 0; l < c.n_layers; ++l) {
        const void* in = l % 2 == 0 ? (const void*)A : (const void*)Bf;
        void* out = l == c.n_layers - 1 ? (void*)z : ((l + 1) % 2 == 0 ? (void*)A : (void*)Bf);
        s = conv_tc(ctx, l, in, out, B, H, W, st);
        if (s) return s;
        prof_mark(ctx, 2 + l, st);
    }
    return WSKPN_OK;
}

}  // namespace wskpn
