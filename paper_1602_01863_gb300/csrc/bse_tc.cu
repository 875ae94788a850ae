// K_c apply on the 5th-generation tensor cores (Eq. matmul2 in BF16 with FP32
// accumulation).
//
// R = K_c Q with K_c stored as BF16 planes Kr, Ki [Nc][ldk] and Q packed as a
// split-BF16 operand B [16][ldk]: rows (Re hi, Im hi, Re lo, Im lo) x chains.
// Two accumulators per tile, D_r = Kr B^T and D_i = Ki B^T (128 x 16 FP32 each,
// in TMEM), give R_re = D_r[Re] - D_i[Im] and R_im = D_r[Im] + D_i[Re] with the
// hi and lo halves summed, so the Q operand carries ~16 mantissa bits while
// K_c carries BF16's 8.
//
// Schedule: each row tile's k-blocks are cut into chunks of a few k-blocks;
// the CTAs (at most one per SM) take chunks from a global counter, so a CTA
// that starts late (the apply can run beside the near field and pick up SMs
// as that kernel's last wave leaves them) simply takes fewer.  Each chunk's
// two accumulators (double-buffered in TMEM) go to its own slot of a partial
// buffer.  Each quarter of a row tile (32 rows) has its own counter: the
// epilogue warp that writes the quarter's rows of the tile's last chunk sums
// them over the tile's chunks in chunk order (deterministic, whichever CTAs
// computed them) and writes those rows of R.  The last CTA to finish resets
// the counters.
// Pipeline depth and chunk length are picked per K_c shape by timing
// (`tune`).
//
// Warp roles (192 threads): warp 0 TMA producer, warp 1 MMA issuer and TMEM
// owner, warps 2-5 epilogue (TMEM lanes 32 (w % 4) .. + 31).  Every mbarrier
// wait is bounded (by the context's wait limit, default ~2 s); on expiry the
// kernel raises bit 0 of the context status word, drains its copies and MMAs
// (waits bounded by the default), frees TMEM and returns.
#include <cuda.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "bse_internal.cuh"

namespace {

constexpr int BM = 128;          // rows per tile (MMA M)
constexpr int BK = 64;           // BF16 elements per k-block (128 bytes: one swizzle row)
constexpr int BN = 16;           // MMA N: split-BF16 Q columns
constexpr int A_TILE_BYTES = BM * BK * 2;                  // 16 KB
constexpr int B_TILE_BYTES = BN * BK * 2;                  // 2 KB
constexpr int STAGE_BYTES = 2 * A_TILE_BYTES + B_TILE_BYTES;
constexpr int TC_THREADS = 192;
constexpr int ACC_COLS = 32;     // D_r (16) + D_i (16) per accumulator buffer
constexpr int TMEM_COLS = 64;    // two accumulator buffers
constexpr long long WAIT_CYCLES = 4000000000LL;   // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: true when the phase completed, false (and status raised) on
// expiry after `limit` clock cycles.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* status, long long limit = WAIT_CYCLES) {
    const long long t0 = clock64();
    while (!mbar_try(bar, parity)) {
        if (clock64() - t0 > limit) {
            atomicOr(status, 1);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
        ::"r"(dst), "l"((uint64_t)map), "r"(bar), "r"(x), "r"(y)
        : "memory");
}

// Shared-memory matrix descriptor, K-major, 128-byte swizzle, 8-row atoms 1024 B apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;                    // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;          // stride byte offset between 8-row atoms
    d |= (uint64_t)1 << 46;                    // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;                    // SWIZZLE_128B
    return d;
}

// Instruction descriptor: kind::f16, A = B = BF16, D = F32, K-major A and B, M = 128, N = 16.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(d_tmem), "l"(a), "l"(b), "r"(IDESC), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Scheduling constants of one tensor-core K_c apply: the row tiles' k-blocks
// are cut into chunks of chunk_kb k-blocks (the last chunk of a row may be
// shorter); CTAs take chunks from a global counter in order.
struct TcSched {
    int kb_row;       // k-blocks per row tile (ldk / BK)
    int chunk_kb;     // k-blocks per chunk
    int chunks_row;   // chunks per row tile
    int total;        // chunks of all row tiles
    int Nc, nchains;
};

// Counters (ints, zero between launches): [0] next chunk, [1] CTAs finished,
// [2 + 4 tile + q] chunks of that row tile whose rows 32 q .. 32 q + 31 (the
// rows of epilogue warp q) are written.
template <int STAGES>
__global__ void __launch_bounds__(TC_THREADS, 1) k_tc_apply(const __grid_constant__ CUtensorMap map_kr,
                                                           const __grid_constant__ CUtensorMap map_ki,
                                                           const __grid_constant__ CUtensorMap map_b, const TcSched sc,
                                                           float* __restrict__ part, int* __restrict__ ctr,
                                                           float2* __restrict__ R, int* __restrict__ status,
                                                           long long wait_cycles) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t bar_full[STAGES], bar_empty[STAGES], bar_acc_full[2], bar_acc_empty[2], bar_cid[2], bar_drain;
    __shared__ int stage_meta[STAGES];   // chunk * 4 + first k-block (1) + last k-block (2); -1: no further chunk
    __shared__ int acc_meta[2];          // chunk held by an accumulator buffer; -1: no further chunk
    __shared__ uint32_t tmem_base_sh;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(smem_u32(&bar_full[s]), 1);
            mbar_init(smem_u32(&bar_empty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&bar_acc_full[b]), 1);
            mbar_init(smem_u32(&bar_acc_empty[b]), 128);
            mbar_init(smem_u32(&bar_cid[b]), 1);
        }
        mbar_init(smem_u32(&bar_drain), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem_base = tmem_base_sh;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------------------------------------------- TMA producer
            long long it = 0;
            bool ok = true;
            int c = atomicAdd(&ctr[0], 1);
            while (ok && c < sc.total) {
                const int cn = atomicAdd(&ctr[0], 1);            // the next chunk, taken while this one streams
                const int tile = c / sc.chunks_row, j = c - tile * sc.chunks_row;
                const int kb0 = j * sc.chunk_kb, kb1 = min(kb0 + sc.chunk_kb, sc.kb_row);
                for (int kb = kb0; kb < kb1; ++kb, ++it) {
                    const int s = (int)(it % STAGES);
                    if (it >= STAGES &&
                        !(ok = mbar_wait(smem_u32(&bar_empty[s]), (uint32_t)(((it / STAGES) - 1) & 1), status, wait_cycles)))
                        break;
                    stage_meta[s] = c * 4 + (kb == kb0 ? 1 : 0) + (kb + 1 == kb1 ? 2 : 0);
                    unsigned char* st = smem + (size_t)s * STAGE_BYTES;
                    const uint32_t fb = smem_u32(&bar_full[s]);
                    mbar_arrive_expect_tx(fb, STAGE_BYTES);
                    tma_load_2d(smem_u32(st), &map_kr, fb, kb * BK, tile * BM);
                    tma_load_2d(smem_u32(st + A_TILE_BYTES), &map_ki, fb, kb * BK, tile * BM);
                    tma_load_2d(smem_u32(st + 2 * A_TILE_BYTES), &map_b, fb, kb * BK, 0);
                }
                c = cn;
            }
            if (ok) {                                            // end marker for the issuer
                const int s = (int)(it % STAGES);
                if (it < STAGES || mbar_wait(smem_u32(&bar_empty[s]), (uint32_t)(((it / STAGES) - 1) & 1), status, wait_cycles)) {
                    stage_meta[s] = -1;
                    mbar_arrive(smem_u32(&bar_full[s]));
                    ++it;
                }
            }
            // drain: the copies of the last (up to STAGES) stages land before exit
            for (long long q = (it > STAGES ? it - STAGES : 0); q < it; ++q)
                mbar_wait(smem_u32(&bar_full[q % STAGES]), (uint32_t)((q / STAGES) & 1), status);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ----------------------------------------------------- MMA issuer
            int seg = 0;
            for (long long it = 0;; ++it) {
                const int s = (int)(it % STAGES);
                if (!mbar_wait(smem_u32(&bar_full[s]), (uint32_t)((it / STAGES) & 1), status, wait_cycles)) break;
                const int meta = *reinterpret_cast<volatile int*>(&stage_meta[s]);
                if (meta < 0) break;
                const bool first = (meta & 1) != 0, last = (meta & 2) != 0;
                const int ab = seg & 1;
                if (first && seg >= 2 &&
                    !mbar_wait(smem_u32(&bar_acc_empty[ab]), (uint32_t)(((seg >> 1) - 1) & 1), status, wait_cycles))
                    break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t st = smem_u32(smem + (size_t)s * STAGE_BYTES);
                const uint64_t dr = smem_desc(st), di = smem_desc(st + A_TILE_BYTES), db = smem_desc(st + 2 * A_TILE_BYTES);
                const uint32_t d_re = tmem_base + ab * ACC_COLS, d_im = d_re + BN;
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk) {
                    const uint32_t acc = (first && kk == 0) ? 0u : 1u;
                    mma_bf16(d_re, dr + 2 * kk, db + 2 * kk, acc);      // +32 bytes per K=16 step
                    mma_bf16(d_im, di + 2 * kk, db + 2 * kk, acc);
                }
                mma_commit(smem_u32(&bar_empty[s]));
                if (last) {
                    acc_meta[ab] = meta >> 2;
                    mma_commit(smem_u32(&bar_acc_full[ab]));
                    mbar_arrive(smem_u32(&bar_cid[ab]));        // publishes acc_meta to the epilogue
                    ++seg;
                }
            }
            // no further chunk (also after a wait gave up): tell the epilogue
            const int ab = seg & 1;
            if (seg < 2 || mbar_wait(smem_u32(&bar_acc_empty[ab]), (uint32_t)(((seg >> 1) - 1) & 1), status, wait_cycles)) {
                acc_meta[ab] = -1;
                mbar_arrive(smem_u32(&bar_cid[ab]));
            }
            mma_commit(smem_u32(&bar_drain));
            mbar_wait(smem_u32(&bar_drain), 0, status);
        }
    } else {
        // ---------------------------------------------------------- epilogue
        // Each chunk's accumulators go to part[chunk] (128 rows x 32 FP32).  For
        // each quarter of a row tile (the 32 rows one epilogue warp owns), the
        // warp that writes the tile's last chunk of those rows sums them over the
        // tile's chunks in chunk order (deterministic, whichever CTAs computed
        // them) and writes R = (D_r[Re] - D_i[Im], D_r[Im] + D_i[Re]) with the
        // hi and lo halves summed.
        const int quarter = warp & 3;
        const int row = quarter * 32 + lane;
        for (int j = 0;; ++j) {
            const int ab = j & 1;
            bool ok = mbar_wait(smem_u32(&bar_cid[ab]), (uint32_t)((j >> 1) & 1), status, wait_cycles);
            if (!__all_sync(0xffffffffu, ok)) break;
            const int chunk = *reinterpret_cast<volatile int*>(&acc_meta[ab]);
            if (chunk < 0) break;
            ok = mbar_wait(smem_u32(&bar_acc_full[ab]), (uint32_t)((j >> 1) & 1), status, wait_cycles);
            if (!__all_sync(0xffffffffu, ok)) break;       // warp-uniform: tcgen05.ld is warp-collective
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            float v[32];
            tmem_ld32(tmem_base + ((uint32_t)(quarter * 32) << 16) + ab * ACC_COLS, v);
            float4* dst = reinterpret_cast<float4*>(part + ((size_t)chunk * BM + row) * 32);
#pragma unroll
            for (int i = 0; i < 8; ++i) dst[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(smem_u32(&bar_acc_empty[ab]));
            __threadfence();
            __syncwarp();
            // this warp's 32 rows of the tile: the warp that writes them for the
            // tile's last chunk sums them over the tile's chunks
            const int tile = chunk / sc.chunks_row, cq = 2 + 4 * tile + quarter;
            int done = 0;
            if (lane == 0) done = atomicAdd(&ctr[cq], 1) == sc.chunks_row - 1;
            done = __shfl_sync(0xffffffffu, done, 0);
            if (!done) continue;
            __threadfence();
            {
                const int i = tile * BM + row;
                float acc[32];
#pragma unroll
                for (int k = 0; k < 32; ++k) acc[k] = 0.f;
                for (int cc = tile * sc.chunks_row; cc < (tile + 1) * sc.chunks_row; ++cc) {
                    const float4* src = reinterpret_cast<const float4*>(part + ((size_t)cc * BM + row) * 32);
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const float4 w = __ldcg(src + k);
                        acc[4 * k] += w.x; acc[4 * k + 1] += w.y; acc[4 * k + 2] += w.z; acc[4 * k + 3] += w.w;
                    }
                }
                if (i < sc.Nc) {
                    const float* Dr = acc;          // columns 0..15: Kr B^T
                    const float* Di = acc + 16;     // columns 16..31: Ki B^T
                    const int p = sc.nchains;
                    for (int ch = 0; ch < p; ++ch) {
                        const float re = (Dr[ch] + Dr[2 * p + ch]) - (Di[p + ch] + Di[3 * p + ch]);
                        const float im = (Dr[p + ch] + Dr[3 * p + ch]) + (Di[ch] + Di[2 * p + ch]);
                        R[(size_t)ch * sc.Nc + i] = make_float2(re, im);
                    }
                }
            }
            if (lane == 0) ctr[cq] = 0;                      // ready for the next launch
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS));
    if (threadIdx.x == 0) {
        // the last CTA of the launch resets the counters (every tile counter too
        // when a wait gave up and some tiles never completed)
        __threadfence();
        if (atomicAdd(&ctr[1], 1) == (int)gridDim.x - 1) {
            if (*reinterpret_cast<volatile int*>(status) & 1)
                for (int t2 = 0; t2 < 4 * (sc.total / sc.chunks_row); ++t2) ctr[2 + t2] = 0;
            ctr[0] = 0;
            ctr[1] = 0;
            __threadfence();
        }
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode(bse_ctx* ctx) {
    static EncodeTiledFn fn = nullptr;
    if (fn) return fn;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p) {
        ctx->err = "cuTensorMapEncodeTiled is not available from the driver";
        return nullptr;
    }
    fn = reinterpret_cast<EncodeTiledFn>(p);
    return fn;
}

// Tensor map of a row-major BF16 matrix [rows][ldk] with a (64 x box_rows) box.
int make_map(bse_ctx* ctx, CUtensorMap* m, const void* base, int ldk, int rows, int box_rows) {
    EncodeTiledFn enc = get_encode(ctx);
    if (!enc) return BSE_ERR_UNSUPPORTED;
    if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || (ldk * 2) % 16 != 0) {
        ctx->err = "tensor map base or stride not 16-byte aligned";
        return BSE_ERR_ARG;
    }
    const cuuint64_t dims[2] = {(cuuint64_t)ldk, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ldk * 2};
    const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        ctx->err = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
        return BSE_ERR_CUDA;
    }
    return BSE_OK;
}

// Launch shape of the tensor-core apply: pipeline depth, chunk length and CTA
// count, and where the counters sit behind the chunk partials.
struct TcPlan {
    int stages = 5, ctas = 0;
    TcSched sc{};
    size_t part_bytes = 0;   // chunk partials: total x 128 x 32 FP32
    size_t ctr_off = 0;      // byte offset of the counters (2 + 4 x row tiles ints)
    size_t bytes = 0;        // partials + counters
};

size_t tc_smem(int stages) { return (size_t)stages * STAGE_BYTES + 1024; }

TcPlan plan_for(int Nc, int ldk, int stages, int chunk_kb, int sm_count) {
    TcPlan p;
    p.stages = stages;
    p.sc.kb_row = ldk / BK;
    p.sc.chunk_kb = std::max(1, std::min(chunk_kb, p.sc.kb_row));
    p.sc.chunks_row = (p.sc.kb_row + p.sc.chunk_kb - 1) / p.sc.chunk_kb;
    const int tiles = (Nc + BM - 1) / BM;
    p.sc.total = tiles * p.sc.chunks_row;
    p.sc.Nc = Nc;
    p.sc.nchains = 1;
    p.ctas = std::max(1, std::min(std::max(sm_count, 1), p.sc.total));
    p.part_bytes = sizeof(float) * (size_t)p.sc.total * BM * 32;
    p.ctr_off = (p.part_bytes + 255) / 256 * 256;
    p.bytes = p.ctr_off + sizeof(int) * (size_t)(2 + 4 * tiles);
    return p;
}

struct TcState {
    CUtensorMap map_kr, map_ki, map_b;
    TcPlan plan;
};

bool g_attr_set[7] = {};

int set_smem_attr(bse_ctx* ctx, int stages) {
    if (g_attr_set[stages]) return BSE_OK;
    cudaError_t e = cudaSuccess;
    switch (stages) {
        case 4: e = cudaFuncSetAttribute(k_tc_apply<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem(4)); break;
        case 5: e = cudaFuncSetAttribute(k_tc_apply<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem(5)); break;
        case 6: e = cudaFuncSetAttribute(k_tc_apply<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem(6)); break;
        default: ctx->err = "unsupported tensor-core pipeline depth"; return BSE_ERR_ARG;
    }
    if (e != cudaSuccess) {
        ctx->err = std::string("k_tc_apply shared memory attribute: ") + cudaGetErrorString(e);
        return BSE_ERR_CUDA;
    }
    g_attr_set[stages] = true;
    return BSE_OK;
}

// One launch; `prio` != 0 sets the launch's scheduling priority to `prio_value`
// (the apply then yields SMs to higher-priority kernels that run beside it).
cudaError_t launch_tc(const TcState& st, const TcPlan& p, const CUtensorMap& map_b, void* part_ctr, float2* R,
                      int nchains, int* status, long long wait, cudaStream_t stream, bool prio, int prio_value) {
    TcSched sc = p.sc;
    sc.nchains = nchains;
    float* part = static_cast<float*>(part_ctr);
    int* ctr = reinterpret_cast<int*>(static_cast<unsigned char*>(part_ctr) + p.ctr_off);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(p.ctas);
    cfg.blockDim = dim3(TC_THREADS);
    cfg.dynamicSmemBytes = tc_smem(p.stages);
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributePriority;
    attr[0].val.priority = prio_value;
    cfg.attrs = prio ? attr : nullptr;
    cfg.numAttrs = prio ? 1 : 0;
    switch (p.stages) {
        case 4: return cudaLaunchKernelEx(&cfg, k_tc_apply<4>, st.map_kr, st.map_ki, map_b, sc, part, ctr, R, status, wait);
        case 5: return cudaLaunchKernelEx(&cfg, k_tc_apply<5>, st.map_kr, st.map_ki, map_b, sc, part, ctr, R, status, wait);
        default: return cudaLaunchKernelEx(&cfg, k_tc_apply<6>, st.map_kr, st.map_ki, map_b, sc, part, ctr, R, status, wait);
    }
}

}  // namespace

namespace {

struct TcChoice { int stages, chunk_kb; };
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, TcChoice> g_tuned;     // (N_c, ldk, SM count) -> launch shape

// Autotuner of the tensor-core apply's launch shape: times every (pipeline
// depth, chunk length) candidate on the handle's own K_c with CUDA events
// (3 warm-up + 10 timed launches each) and keeps the fastest; the choice is
// cached per (N_c, ldk, SM count) for the process.
TcChoice tune(bse_ctx* ctx, bse_interp* s, TcState& st) {
    const bse_coarse* c = s->co;
    const auto key = std::make_tuple(c->Nc, c->ldk, ctx->sm_count);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) return it->second;
    }
    const int kb_row = c->ldk / BK;
    std::vector<TcChoice> cand;
    for (int stages : {4, 5, 6})
        for (int ck : {8, 16, 32, 64}) {
            const int ckc = std::min(ck, kb_row);
            bool dup = false;
            for (const TcChoice& x : cand) dup = dup || (x.stages == stages && x.chunk_kb == ckc);
            if (!dup) cand.push_back({stages, ckc});
        }
    size_t bytes = 0;
    for (const TcChoice& x : cand) bytes = std::max(bytes, plan_for(c->Nc, c->ldk, x.stages, x.chunk_kb, ctx->sm_count).bytes);
    TcChoice best = {5, std::min(16, kb_row)};
    void* d_buf = nullptr;
    if (bse_alloc(ctx, &d_buf, bytes, "autotune partials") != BSE_OK) { cudaGetLastError(); return best; }
    cudaMemset(d_buf, 0, bytes);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_ms = 1e30f;
    for (const TcChoice& x : cand) {
        if (set_smem_attr(ctx, x.stages) != BSE_OK) continue;
        const TcPlan p = plan_for(c->Nc, c->ldk, x.stages, x.chunk_kb, ctx->sm_count);
        // the counters sit behind this candidate's partials: start them at zero
        cudaMemsetAsync(static_cast<unsigned char*>(d_buf) + p.ctr_off, 0, p.bytes - p.ctr_off, ctx->stream);
        bool ok = true;
        for (int r = 0; r < 3 && ok; ++r)
            ok = launch_tc(st, p, st.map_b, d_buf, (float2*)s->d_R, 1, ctx->d_status, WAIT_CYCLES, ctx->stream, false, 0) == cudaSuccess;
        cudaEventRecord(e0, ctx->stream);
        const int reps = 10;
        for (int r = 0; r < reps && ok; ++r)
            ok = launch_tc(st, p, st.map_b, d_buf, (float2*)s->d_R, 1, ctx->d_status, WAIT_CYCLES, ctx->stream, false, 0) == cudaSuccess;
        cudaEventRecord(e1, ctx->stream);
        float ms = 0.f;
        if (ok && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
            ms / reps < best_ms) {
            best_ms = ms / reps;
            best = x;
        }
    }
    cudaStreamSynchronize(ctx->stream);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(d_buf);
    cudaGetLastError();
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tuned[key] = best;
    return best;
}

}  // namespace

int bse_tc_prepare(bse_ctx* ctx, bse_interp* s) {
    const bse_coarse* c = s->co;
    int rc;
    if ((rc = bse_alloc(ctx, (void**)&s->d_Bop, sizeof(__nv_bfloat16) * BN * (size_t)c->ldk, "split-BF16 operand")) != BSE_OK)
        return rc;
    BSE_CUDA_TRY(ctx, cudaMemset(s->d_Bop, 0, sizeof(__nv_bfloat16) * BN * (size_t)c->ldk));
    TcState* st = new TcState();
    if ((rc = make_map(ctx, &st->map_kr, c->d_kr, c->ldk, c->Nc, BM)) != BSE_OK ||
        (rc = make_map(ctx, &st->map_ki, c->d_ki, c->ldk, c->Nc, BM)) != BSE_OK ||
        (rc = make_map(ctx, &st->map_b, s->d_Bop, c->ldk, BN, BN)) != BSE_OK) {
        delete st;
        return rc;
    }
    const TcChoice ch = tune(ctx, s, *st);
    if ((rc = set_smem_attr(ctx, ch.stages)) != BSE_OK) { delete st; return rc; }
    st->plan = plan_for(c->Nc, c->ldk, ch.stages, ch.chunk_kb, ctx->sm_count);
    const TcPlan& p = st->plan;
    if ((rc = bse_alloc(ctx, (void**)&s->d_part, p.bytes, "chunk partials")) != BSE_OK) {
        delete st;
        return rc;
    }
    BSE_CUDA_TRY(ctx, cudaMemset(s->d_part, 0, p.bytes));
    s->tc_ctas = p.ctas;
    s->tc_kblocks = p.sc.chunk_kb;
    s->tc_stages = p.stages;
    s->tc_state = st;
    return BSE_OK;
}

void bse_tc_release(bse_interp* s) {
    if (!s || !s->tc_state) return;
    delete reinterpret_cast<TcState*>(s->tc_state);
    s->tc_state = nullptr;
}

int bse_tc_apply(bse_ctx* ctx, bse_interp* s, int nchains, cudaStream_t stream, bool prio, int prio_value) {
    const TcState* st = reinterpret_cast<const TcState*>(s->tc_state);
    BSE_CUDA_TRY(ctx, launch_tc(*st, st->plan, st->map_b, s->d_part, (float2*)s->d_R, nchains, ctx->d_status,
                                ctx->wait_cycles > 0 ? ctx->wait_cycles : WAIT_CYCLES, stream, prio, prio_value));
    return BSE_OK;
}

// Bytes of the chunk partials and counters one tensor-core K_c apply uses.
size_t bse_tc_part_bytes(const bse_interp* s) {
    return reinterpret_cast<const TcState*>(s->tc_state)->plan.bytes;
}

// Tensor-core K_c apply with a caller-supplied operand buffer `bop` [16][ldk]
// (zeroed by the caller where unused), partials + counters `part`
// (bse_tc_part_bytes) and output R: the counters are cleared on the stream and
// a tensor map for `bop` is encoded on the stack; nothing is allocated.
int bse_tc_apply_scratch(bse_ctx* ctx, const bse_interp* s, int nchains, __nv_bfloat16* bop, float* part, void* R) {
    const bse_coarse* c = s->co;
    const TcState* st = reinterpret_cast<const TcState*>(s->tc_state);
    const TcPlan& p = st->plan;
    CUtensorMap map_b;
    int rc = make_map(ctx, &map_b, bop, c->ldk, BN, BN);
    if (rc != BSE_OK) return rc;
    BSE_CUDA_TRY(ctx, cudaMemsetAsync(reinterpret_cast<unsigned char*>(part) + p.ctr_off, 0, p.bytes - p.ctr_off, ctx->stream));
    BSE_CUDA_TRY(ctx, launch_tc(*st, p, map_b, part, (float2*)R, nchains, ctx->d_status,
                                ctx->wait_cycles > 0 ? ctx->wait_cycles : WAIT_CYCLES, ctx->stream, false, 0));
    return BSE_OK;
}
