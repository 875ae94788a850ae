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
// Schedule: the Nc/128 row tiles x ldk/64 k-blocks form one sequence of
// k-blocks; CTA g of G (one per SM) streams the contiguous range
// [g T / G, (g + 1) T / G), so every SM moves the same number of K_c bytes.
// A CTA's range touches at most a few row tiles; each touched tile yields one
// partial accumulator ("segment") written to scratch, and k_tc_reduce sums the
// segments of each tile in CTA order (deterministic).
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
constexpr int STAGES = 5;
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

__global__ void __launch_bounds__(TC_THREADS, 1) k_tc_apply(const __grid_constant__ CUtensorMap map_kr,
                                                           const __grid_constant__ CUtensorMap map_ki,
                                                           const __grid_constant__ CUtensorMap map_b, int kblocks_per_row,
                                                           long long total_blocks, int seg_max,
                                                           float* __restrict__ part, int* __restrict__ status,
                                                           long long wait_cycles) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t bar_full[STAGES], bar_empty[STAGES], bar_acc_full[2], bar_acc_empty[2], bar_drain;
    __shared__ uint32_t tmem_base_sh;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int G = gridDim.x, g = blockIdx.x;
    const long long q0 = (long long)g * total_blocks / G, q1 = (long long)(g + 1) * total_blocks / G;
    const int KB = kblocks_per_row;
    const int nseg = (q1 > q0) ? (int)((q1 - 1) / KB - q0 / KB + 1) : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(smem_u32(&bar_full[s]), 1);
            mbar_init(smem_u32(&bar_empty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&bar_acc_full[b]), 1);
            mbar_init(smem_u32(&bar_acc_empty[b]), 128);
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
            for (long long q = q0; q < q1 && ok; ++q, ++it) {
                const int s = (int)(it % STAGES);
                if (it >= STAGES) ok = mbar_wait(smem_u32(&bar_empty[s]), (uint32_t)(((it / STAGES) - 1) & 1), status, wait_cycles);
                if (!ok) break;
                const int tile = (int)(q / KB), kb = (int)(q % KB);
                unsigned char* st = smem + (size_t)s * STAGE_BYTES;
                const uint32_t fb = smem_u32(&bar_full[s]);
                mbar_arrive_expect_tx(fb, STAGE_BYTES);
                tma_load_2d(smem_u32(st), &map_kr, fb, kb * BK, tile * BM);
                tma_load_2d(smem_u32(st + A_TILE_BYTES), &map_ki, fb, kb * BK, tile * BM);
                tma_load_2d(smem_u32(st + 2 * A_TILE_BYTES), &map_b, fb, kb * BK, 0);
            }
            // drain: the last (up to STAGES) issued stages must have landed before exit
            const long long issued = it;
            for (long long j = (issued > STAGES ? issued - STAGES : 0); j < issued; ++j)
                mbar_wait(smem_u32(&bar_full[j % STAGES]), (uint32_t)((j / STAGES) & 1), status);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ----------------------------------------------------- MMA issuer
            long long it = 0;
            int seg = 0;
            bool ok = true;
            for (long long q = q0; q < q1 && ok; ++q, ++it) {
                const bool first = (q == q0) || (q % KB == 0);
                const bool last = (q + 1 == q1) || ((q + 1) % KB == 0);
                const int ab = seg & 1;
                if (first && seg >= 2) {
                    ok = mbar_wait(smem_u32(&bar_acc_empty[ab]), (uint32_t)(((seg >> 1) - 1) & 1), status, wait_cycles);
                    if (!ok) break;
                }
                const int s = (int)(it % STAGES);
                ok = mbar_wait(smem_u32(&bar_full[s]), (uint32_t)((it / STAGES) & 1), status, wait_cycles);
                if (!ok) break;
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
                    mma_commit(smem_u32(&bar_acc_full[ab]));
                    ++seg;
                }
            }
            mma_commit(smem_u32(&bar_drain));
            mbar_wait(smem_u32(&bar_drain), 0, status);
        }
    } else {
        // ---------------------------------------------------------- epilogue
        const int quarter = warp & 3;
        const int row = quarter * 32 + lane;
        for (int j = 0; j < nseg; ++j) {
            const int ab = j & 1;
            const bool ok = mbar_wait(smem_u32(&bar_acc_full[ab]), (uint32_t)((j >> 1) & 1), status, wait_cycles);
            if (!__all_sync(0xffffffffu, ok)) break;       // warp-uniform: tcgen05.ld is warp-collective
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            float v[32];
            tmem_ld32(tmem_base + ((uint32_t)(quarter * 32) << 16) + ab * ACC_COLS, v);
            float4* dst = reinterpret_cast<float4*>(part + (((size_t)g * seg_max + j) * BM + row) * 32);
#pragma unroll
            for (int i = 0; i < 8; ++i) dst[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(smem_u32(&bar_acc_empty[ab]));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS));
}

// Sum the segments of each row tile (CTA order) and combine the split
// accumulators into complex R [chain][Nc] (FP32).
__global__ void k_tc_reduce(const float* __restrict__ part, const int* __restrict__ tile_cta, const long long* __restrict__ cta_q0,
                            int kblocks_per_row, int seg_max, int Nc, int nchains, float2* __restrict__ R) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Nc) return;
    const int tile = i / BM, r = i % BM;
    const int g_lo = tile_cta[2 * tile], g_hi = tile_cta[2 * tile + 1];
    float acc[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) acc[c] = 0.f;
    for (int g = g_lo; g <= g_hi; ++g) {
        const int j = tile - (int)(cta_q0[g] / kblocks_per_row);
        const float4* src = reinterpret_cast<const float4*>(part + (((size_t)g * seg_max + j) * BM + r) * 32);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float4 v = src[q];
            acc[4 * q] += v.x; acc[4 * q + 1] += v.y; acc[4 * q + 2] += v.z; acc[4 * q + 3] += v.w;
        }
    }
    const float* Dr = acc;          // columns 0..15: Kr B^T
    const float* Di = acc + 16;     // columns 16..31: Ki B^T
    const int p = nchains;
    for (int c = 0; c < p; ++c) {
        const float re = (Dr[c] + Dr[2 * p + c]) - (Di[p + c] + Di[3 * p + c]);
        const float im = (Dr[p + c] + Dr[3 * p + c]) + (Di[c] + Di[2 * p + c]);
        R[(size_t)c * Nc + i] = make_float2(re, im);
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

struct TcPlan {
    int kblocks_per_row = 0, tiles = 0, ctas = 0, seg_max = 0;
    long long total = 0;
    std::vector<long long> q0;      // [ctas + 1]
    std::vector<int> tile_cta;      // [2 * tiles]
};

TcPlan plan_for(int Nc, int ldk, int sm_count) {
    TcPlan p;
    p.kblocks_per_row = ldk / BK;
    p.tiles = (Nc + BM - 1) / BM;
    p.total = (long long)p.tiles * p.kblocks_per_row;
    p.ctas = (int)std::min<long long>(std::max(sm_count, 1), p.total);
    p.q0.resize(p.ctas + 1);
    for (int g = 0; g <= p.ctas; ++g) p.q0[g] = (long long)g * p.total / p.ctas;
    p.seg_max = 0;
    for (int g = 0; g < p.ctas; ++g) {
        const long long a = p.q0[g], b = p.q0[g + 1];
        const int nseg = (b > a) ? (int)((b - 1) / p.kblocks_per_row - a / p.kblocks_per_row + 1) : 0;
        p.seg_max = std::max(p.seg_max, nseg);
    }
    p.tile_cta.resize(2 * p.tiles);
    for (int t = 0; t < p.tiles; ++t) {
        const long long lo = (long long)t * p.kblocks_per_row, hi = lo + p.kblocks_per_row - 1;
        int glo = -1, ghi = -1;
        for (int g = 0; g < p.ctas; ++g) {
            if (p.q0[g + 1] > lo && p.q0[g] <= hi) {
                if (glo < 0) glo = g;
                ghi = g;
            }
        }
        p.tile_cta[2 * t] = glo;
        p.tile_cta[2 * t + 1] = ghi;
    }
    return p;
}

struct TcState {
    CUtensorMap map_kr, map_ki, map_b;
    TcPlan plan;
    int* d_tile_cta = nullptr;
    long long* d_q0 = nullptr;
};

}  // namespace

namespace {

std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, int> g_tuned_ctas;     // (N_c, ldk, SM count) -> CTA count

// Autotuner for the persistent split of the k-block sequence: times the
// tensor-core apply (+ reduce) for a few CTA counts on the handle's own K_c
// with CUDA events and keeps the fastest; the choice is cached per shape.
int tune_ctas(bse_ctx* ctx, bse_interp* s, const CUtensorMap& mkr, const CUtensorMap& mki, const CUtensorMap& mb) {
    const bse_coarse* c = s->co;
    const auto key = std::make_tuple(c->Nc, c->ldk, ctx->sm_count);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tuned_ctas.find(key);
        if (it != g_tuned_ctas.end()) return it->second;
    }
    const int sm = std::max(ctx->sm_count, 1);
    const long long total = (long long)((c->Nc + BM - 1) / BM) * (c->ldk / BK);
    std::vector<int> cand;
    for (int d : {1, 2, 4, 8}) {
        const int g = (int)std::min<long long>(std::max(sm / d, 1), total);
        if (std::find(cand.begin(), cand.end(), g) == cand.end()) cand.push_back(g);
    }
    const int g34 = (int)std::min<long long>(std::max(3 * sm / 4, 1), total);
    if (std::find(cand.begin(), cand.end(), g34) == cand.end()) cand.push_back(g34);
    size_t part_bytes = 0;
    for (int g : cand) {
        const TcPlan p = plan_for(c->Nc, c->ldk, g);
        part_bytes = std::max(part_bytes, sizeof(float) * (size_t)p.ctas * p.seg_max * BM * 32);
    }
    float* d_part = nullptr;
    if (bse_alloc(ctx, (void**)&d_part, part_bytes, "autotune partials") != BSE_OK) return sm;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best = cand[0];
    float best_ms = 1e30f;
    for (int g : cand) {
        const TcPlan p = plan_for(c->Nc, c->ldk, g);
        int* d_tc = nullptr;
        long long* d_q = nullptr;
        if (bse_alloc(ctx, (void**)&d_tc, sizeof(int) * p.tile_cta.size(), "autotune tables") != BSE_OK) continue;
        if (bse_alloc(ctx, (void**)&d_q, sizeof(long long) * p.q0.size(), "autotune tables") != BSE_OK) { cudaFree(d_tc); continue; }
        cudaMemcpy(d_tc, p.tile_cta.data(), sizeof(int) * p.tile_cta.size(), cudaMemcpyHostToDevice);
        cudaMemcpy(d_q, p.q0.data(), sizeof(long long) * p.q0.size(), cudaMemcpyHostToDevice);
        auto launch = [&]() {
            k_tc_apply<<<p.ctas, TC_THREADS, STAGES * STAGE_BYTES + 1024, ctx->stream>>>(
                mkr, mki, mb, p.kblocks_per_row, p.total, p.seg_max, d_part, ctx->d_status, WAIT_CYCLES);
            k_tc_reduce<<<(c->Nc + 127) / 128, 128, 0, ctx->stream>>>(d_part, d_tc, d_q, p.kblocks_per_row, p.seg_max,
                                                                     c->Nc, 1, (float2*)s->d_R);
        };
        for (int r = 0; r < 3; ++r) launch();
        cudaEventRecord(e0, ctx->stream);
        const int reps = 10;
        for (int r = 0; r < reps; ++r) launch();
        cudaEventRecord(e1, ctx->stream);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms / reps < best_ms) {
            best_ms = ms / reps;
            best = g;
        }
        cudaFree(d_tc);
        cudaFree(d_q);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(d_part);
    cudaGetLastError();
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tuned_ctas[key] = best;
    return best;
}

}  // namespace

int bse_tc_prepare(bse_ctx* ctx, bse_interp* s) {
    const bse_coarse* c = s->co;
    int rc;
    if ((rc = bse_alloc(ctx, (void**)&s->d_Bop, sizeof(__nv_bfloat16) * BN * (size_t)c->ldk, "split-BF16 operand")) != BSE_OK)
        return rc;
    BSE_CUDA_TRY(ctx, cudaMemset(s->d_Bop, 0, sizeof(__nv_bfloat16) * BN * (size_t)c->ldk));
    static bool attr_set = false;
    if (!attr_set) {
        BSE_CUDA_TRY(ctx, cudaFuncSetAttribute(k_tc_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, STAGES * STAGE_BYTES + 1024));
        attr_set = true;
    }
    TcState* st = new TcState();
    if ((rc = make_map(ctx, &st->map_kr, c->d_kr, c->ldk, c->Nc, BM)) != BSE_OK ||
        (rc = make_map(ctx, &st->map_ki, c->d_ki, c->ldk, c->Nc, BM)) != BSE_OK ||
        (rc = make_map(ctx, &st->map_b, s->d_Bop, c->ldk, BN, BN)) != BSE_OK) {
        delete st;
        return rc;
    }
    const int ctas = tune_ctas(ctx, s, st->map_kr, st->map_ki, st->map_b);
    st->plan = plan_for(c->Nc, c->ldk, ctas);
    const TcPlan& p = st->plan;
    if ((rc = bse_alloc(ctx, (void**)&s->d_part, sizeof(float) * (size_t)p.ctas * p.seg_max * BM * 32, "tile partials")) != BSE_OK ||
        (rc = bse_alloc(ctx, (void**)&st->d_tile_cta, sizeof(int) * p.tile_cta.size(), "tile schedule")) != BSE_OK ||
        (rc = bse_alloc(ctx, (void**)&st->d_q0, sizeof(long long) * p.q0.size(), "cta schedule")) != BSE_OK) {
        cudaFree(st->d_tile_cta); cudaFree(st->d_q0);
        delete st;
        return rc;
    }
    BSE_CUDA_TRY(ctx, cudaMemcpy(st->d_tile_cta, p.tile_cta.data(), sizeof(int) * p.tile_cta.size(), cudaMemcpyHostToDevice));
    BSE_CUDA_TRY(ctx, cudaMemcpy(st->d_q0, p.q0.data(), sizeof(long long) * p.q0.size(), cudaMemcpyHostToDevice));
    s->tc_ctas = p.ctas;
    s->tc_kblocks = p.kblocks_per_row;
    s->tc_state = st;
    return BSE_OK;
}

void bse_tc_release(bse_interp* s) {
    if (!s || !s->tc_state) return;
    TcState* st = reinterpret_cast<TcState*>(s->tc_state);
    cudaFree(st->d_tile_cta);
    cudaFree(st->d_q0);
    delete st;
    s->tc_state = nullptr;
}

int bse_tc_apply(bse_ctx* ctx, bse_interp* s, int nchains) {
    const bse_coarse* c = s->co;
    const TcState* st = reinterpret_cast<const TcState*>(s->tc_state);
    const TcPlan& p = st->plan;
    k_tc_apply<<<p.ctas, TC_THREADS, STAGES * STAGE_BYTES + 1024, ctx->stream>>>(
        st->map_kr, st->map_ki, st->map_b, p.kblocks_per_row, p.total, p.seg_max, s->d_part, ctx->d_status,
        ctx->wait_cycles > 0 ? ctx->wait_cycles : WAIT_CYCLES);
    k_tc_reduce<<<(c->Nc + 127) / 128, 128, 0, ctx->stream>>>(s->d_part, st->d_tile_cta, st->d_q0, p.kblocks_per_row,
                                                             p.seg_max, c->Nc, nchains, (float2*)s->d_R);
    return BSE_OK;
}

// Bytes of the tile partials one tensor-core K_c apply writes.
size_t bse_tc_part_bytes(const bse_interp* s) {
    const TcState* st = reinterpret_cast<const TcState*>(s->tc_state);
    return sizeof(float) * (size_t)st->plan.ctas * st->plan.seg_max * BM * 32;
}

// Tensor-core K_c apply with a caller-supplied operand buffer `bop` [16][ldk]
// (zeroed by the caller where unused), tile partials `part` and output R: a
// tensor map for `bop` is encoded on the stack; nothing is allocated.
int bse_tc_apply_scratch(bse_ctx* ctx, const bse_interp* s, int nchains, __nv_bfloat16* bop, float* part, void* R) {
    const bse_coarse* c = s->co;
    const TcState* st = reinterpret_cast<const TcState*>(s->tc_state);
    const TcPlan& p = st->plan;
    CUtensorMap map_b;
    int rc = make_map(ctx, &map_b, bop, c->ldk, BN, BN);
    if (rc != BSE_OK) return rc;
    k_tc_apply<<<p.ctas, TC_THREADS, STAGES * STAGE_BYTES + 1024, ctx->stream>>>(
        st->map_kr, st->map_ki, map_b, p.kblocks_per_row, p.total, p.seg_max, part, ctx->d_status,
        ctx->wait_cycles > 0 ? ctx->wait_cycles : WAIT_CYCLES);
    k_tc_reduce<<<(c->Nc + 127) / 128, 128, 0, ctx->stream>>>(part, st->d_tile_cta, st->d_q0, p.kblocks_per_row,
                                                             p.seg_max, c->Nc, nchains, (float2*)R);
    return BSE_OK;
}
