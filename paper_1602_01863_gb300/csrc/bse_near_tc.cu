// Method 3 near field on the tensor cores, as two chained GEMMs per coarse cell.
//
// For one coarse cell C, one Lanczos step and every chain, the correction in
// coarse-basis form is
//   u(k, l) = sum_s A(k~_l, k~_s) [y1(k, s) - h_head(q_c(l, s)) z(k, s)],
//   y1(k, s) = sum_{k' near k, k' in slot s} h_head(q_d(k, k')) x(k'),   z(k, s) = sum x(k'),
// A = alpha O^v (x) O^c the Kronecker head block of Eq. diverg, s over the
// source slots, k over the N_div targets of C.
// Stage 1 (per slot): y1 and z are a product of the slot's near pattern S_s
// (rows (y1|z, target), columns = the slot's source rows; entries h_head(q_d)
// or 1) with the gathered source rows X_s.  S_s is the same for every cell
// (translation invariance of the near pattern), so set-up writes it once as
// TF32 images of 32-row K-blocks; the kernel gathers X_s (all chains, columns
// (chain, e, re|im)) transposed into shared memory and issues
//   D1 [128 = (y1|z, target)] x [32 * chains] += S_s[., K-block] * X_s[K-block]^T.
// Stage 2 (per slot): D1 is read back from TMEM into the B operand
//   B_s[(chain, k), (Y|Z, e', re|im)]  = y1(k, s), z(k, s)
// and, with the real form
//   Ahat_s[(l,e,.), (Y,e',.)] = [[Re c, -Im c], [Im c, Re c]],  c = A(k~_l, k~_s)[e][e'],
//   Ahat_s[(l,e,.), (Z,e',.)] = the same for -h_head(q_c(l, s)) c,
// formed in shared memory from the per-cell head factors,
//   D2 [256 = (l, e, re|im)] x [64 * chains] += Ahat_s [256 x 64] * B_s^T.
// tcgen05.mma kind::tf32 (10-bit mantissa, FP32 range: y1 and h_head z nearly
// cancel in u, which BF16 would not resolve), FP32 accumulators in TMEM.
//
// Warp roles (768 threads, one CTA per coarse cell):
//   warps 4-7      MMA issuer (warp 4, lane 0, also TMEM owner) and D1 -> B
//                  converters (TMEM lane quarters 0-3); after each slot the four
//                  warps convert D1 and meet at a named barrier, after which the
//                  issuer goes on.  Waits use the blocking mbarrier test: a
//                  spinning issuer measurably slowed the other warps
//   warps 8-15     stage-1 producers: the S image by one bulk copy, the X rows by
//                  4-byte cp.async gathers laid out so that a warp's 32 stores
//                  hit 32 distinct banks; each warp keeps the whole ring in
//                  flight and signals a stage once its copies have landed
//   warps 0-3, 16-23  Ahat writers (per slot, in two 128-row halves), with the
//                  slot's head factors staged one slot ahead
// The stage-2 MMAs of slot i - 1 are issued between the stage-1 K-blocks of slot
// i, so the tensor pipe works on one while the producers refill the ring; D1 and
// B are single-buffered (TMEM holds D2, 2 x 64 x chains columns, and D1,
// 32 x chains), Ahat is released half by half.
// Constraints: t <= 16, N_div <= 64, FP32 vectors, <= 3 chains per launch.
// Every wait is bounded; on expiry the kernel raises bit 1 of the status word,
// every role leaves its loop, the MMAs and copies in flight are drained and
// TMEM is freed.
#include <cuda.h>

#include <algorithm>
#include <functional>

#include "bse_internal.cuh"

namespace {

constexpr int NT_M = 256;                    // rows (corner l, transition e, re|im), 8 * 16 * 2
constexpr int NT_N = 64;                     // targets of the cell (padded)
constexpr int NT_KB = 32;                    // source rows per stage-1 K-block
constexpr int NT_STAGES = 3;                 // stage-1 ring depth
constexpr int S_BYTES = 128 * NT_KB * 4;     // one S image K-block: 16 KB
constexpr int A_KB = NT_M * 128;             // one 32-element K-block of A: 32 KB
constexpr int A_BYTES = 2 * A_KB;            // 64 KB per slot
constexpr int NT_THREADS = 768;
constexpr int NT_TMEM_COLS = 512;
constexpr int W_C0 = 4, W_CN = 4;            // MMA issuer (warp 4, lane 0) + converters (warp % 4 = TMEM lane quarter)
constexpr int W_P0 = 8, W_PN = 8;            // producers: warp W_P0 + p stages rows 4p .. 4p + 3
constexpr int W_A1 = 16;                     // Ahat writers: warps 0-3 and 16-23
constexpr int W_AN = W_C0 + (NT_THREADS / 32 - W_A1);
constexpr int NT_A = 32 * W_AN;              // Ahat writer threads
constexpr int NT_AMAX = 3;                   // items per writer thread and slot (8 t ceil(t / 2) <= 1024)
static_assert(NT_A * NT_AMAX >= 1024, "Ahat items per slot");
constexpr long long NT_WAIT_CYCLES = 400000000LL;   // ~0.2 s; a whole launch takes well under 10 ms

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(su32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
// every group but the newest NT_STAGES - 1 landed (the K-block NT_STAGES - 1 behind the newest)
__device__ __forceinline__ void cp_async_wait_lag() { asm volatile("cp.async.wait_group %0;" ::"n"(NT_STAGES - 1) : "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ uint32_t f2tf32(float v) {
    uint32_t u;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(v));
    return u;
}

// Byte offset of 32-bit element (row r, column k) of a K-major operand stored as
// K-blocks of 32 elements (128-byte rows), each block `rows` x 128 B with the
// 128-byte swizzle: 8-row atoms of 1024 B, 16-byte chunks XORed by r % 8.
__host__ __device__ __forceinline__ uint32_t sw128(int r, int k, int rows) {
    const int kb = k >> 5, kk = k & 31;
    return (uint32_t)(kb * rows * 128 + (r >> 3) * 1024 + (r & 7) * 128 + ((((kk >> 2) ^ (r & 7)) & 7) << 4) + ((kk & 3) << 2));
}

__device__ __forceinline__ void bar_init(uint32_t b, uint32_t c) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(b), "r"(c) : "memory");
}
__device__ __forceinline__ void bar_arrive(uint32_t b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(b) : "memory");
}
__device__ __forceinline__ void bar_arrive_tx(uint32_t b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool bar_try(uint32_t b, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(b), "r"(parity) : "memory");
    return ok != 0;
}
// Non-blocking test of a phase.
__device__ __forceinline__ bool bar_test(uint32_t b, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(b), "r"(parity) : "memory");
    return ok != 0;
}
// Bounded wait: false when another role gave up (abort flag) or the clock
// budget ran out (raises status bit 1 and the abort flag).
__device__ __forceinline__ bool bar_wait(uint32_t b, uint32_t parity, int* status, volatile int* abort_flag) {
    const long long t0 = clock64();
    while (!bar_try(b, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > NT_WAIT_CYCLES) {
            atomicOr(status, 2);
            *abort_flag = 1;
            return false;
        }
    }
    return true;
}
// Wait that ignores the abort flag (drain paths: copies and MMAs in flight always finish).
__device__ __forceinline__ void bar_drain(uint32_t b, uint32_t parity, int* status) {
    const long long t0 = clock64();
    while (!bar_try(b, parity)) {
        if (clock64() - t0 > NT_WAIT_CYCLES) { atomicOr(status, 2); return; }
    }
}
__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}
__device__ __forceinline__ uint64_t desc_sw128(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// kind::tf32, A = B = TF32, D = F32, both K-major, M = 128, N as given
__host__ __device__ constexpr uint32_t idesc_tf32(int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                 ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void commit(uint32_t b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(b) : "memory");
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

__device__ __forceinline__ void writers_sync() { asm volatile("bar.sync 1, %0;" ::"n"(NT_A) : "memory"); }
__device__ __forceinline__ void converters_sync() { asm volatile("bar.sync 2, %0;" ::"n"(32 * W_CN) : "memory"); }
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(su32(dst)), "l"(src) : "memory");
}

// Shared-memory bytes of one head-factor buffer: Hv, Hc of the 8 target corners
// for one slot, then h_head(q_c) of the 8 corners.
__host__ __device__ __forceinline__ int hb_bytes(int nv, int nc) {
    return ((8 * (nv * nv + nc * nc) * 8 + 32) + 15) & ~15;
}

// Pack four values rounded to TF32 into one 16-byte chunk.
__device__ __forceinline__ uint4 pack_tf32(float a, float b, float c, float d) {
    return make_uint4(f2tf32(a), f2tf32(b), f2tf32(c), f2tf32(d));
}

// Shared-memory layout (bytes from the 1024-aligned base) for `nch` chains.
struct NtLayout {
    int N1, N2, b_off, ring_off, stage_bytes, tab_off;
    __host__ __device__ NtLayout(int nch) {
        N1 = 32 * nch;
        N2 = 64 * nch;
        b_off = A_BYTES;                                  // Ahat: [2 K-blocks][256 rows][128 B]
        ring_off = b_off + 2 * N2 * 128;                  // B: [2 K-blocks (Y, Z)][N2 rows][128 B]
        stage_bytes = S_BYTES + N1 * 128;                 // ring stage: S K-block | X K-block
        tab_off = ring_off + NT_STAGES * stage_bytes;     // head-factor buffers [2], then slot tables
    }
};

// Slot table entry {slot, first K-block, K-blocks, source rows} and per-K-block
// info (slot ordinal | K-block in slot << 16) are staged in shared memory.
__global__ void __launch_bounds__(NT_THREADS, 1) k_near_tc(
    const float* __restrict__ X, const int* __restrict__ rows, const int4* __restrict__ slots,
    const int* __restrict__ rowstart, const int* __restrict__ kinfo, int nsl, int nkg, int nrows,
    const unsigned char* __restrict__ Simg, const float2* __restrict__ Hv, const float2* __restrict__ Hc,
    const float* __restrict__ hc, int n, int nd, int nv, int nc, int nb1, int smin, int ns1, int rmin, int nr1,
    int nch, float2* __restrict__ U, int* __restrict__ status) {
    // an earlier launch on this context gave up a wait: skip (the host reports BSE_ERR_TIMEOUT)
    if (*reinterpret_cast<volatile int*>(status) & 2) return;
    extern __shared__ unsigned char raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t bar_full[NT_STAGES], bar_sfull[NT_STAGES], bar_empty[NT_STAGES];
    __shared__ uint64_t bar_d1_full, bar_a_full[2], bar_a_free[2], bar_d2;
    __shared__ uint32_t tmem_sh;
    __shared__ int abort_sh;
    volatile int* abort_flag = &abort_sh;
    const int t = nv * nc, Ndiv = nd * nd * nd, nslot = ns1 * ns1 * ns1, nrel = nr1 * nr1 * nr1;
    const int nk = n * n * n * Ndiv, th = (t + 1) >> 1;
    // D2 rows (l, e, re|im) = 2 (l t + e) + re|im; the second 128-row half holds
    // anything only when 16 t > 128
    const int nmh = (16 * t > 128) ? 2 : 1;
    const NtLayout lay(nch);
    const int N1 = lay.N1, N2 = lay.N2;
    const int cell = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char* A2 = sm;
    unsigned char* B2 = sm + lay.b_off;
    unsigned char* ring = sm + lay.ring_off;
    const int hbb = hb_bytes(nv, nc);
    unsigned char* hbuf = sm + lay.tab_off;                     // [2][hbb]  head factors, slot parity
    int4* s_sl = reinterpret_cast<int4*>(hbuf + 2 * hbb);       // [nsl]
    int* s_rs = reinterpret_cast<int*>(s_sl + nsl);             // [nsl]
    int* s_ki = s_rs + nsl;                                     // [nkg]
    int* scell = s_ki + nkg;                                    // [nslot][8] source cells
    unsigned short* s_rows = reinterpret_cast<unsigned short*>(scell + nslot * 8);   // [nrows] js | corner << 8
    const Int3 ci = unflat3(cell, n);
    for (int i = tid; i < nsl; i += NT_THREADS) { s_sl[i] = slots[i]; s_rs[i] = rowstart[i]; }
    for (int i = tid; i < nkg; i += NT_THREADS) s_ki[i] = kinfo[i];
    for (int i = tid; i < nrows; i += NT_THREADS) {
        const int code = rows[i];
        s_rows[i] = (unsigned short)((code & 0xFF) | ((code >> 16) << 8));
    }
    for (int i = tid; i < nslot * 8; i += NT_THREADS) {
        const int s = i >> 3, l = i & 7;
        const Int3 so = unflat3(s, ns1);
        scell[i] = flat3(ci.a + so.a + smin - ((l >> 2) & 1), ci.b + so.b + smin - ((l >> 1) & 1),
                         ci.c + so.c + smin - (l & 1), n);
    }
    // zero the operands once: padding rows / columns stay zero for the whole kernel
    for (int i = tid; i < lay.tab_off / 16; i += NT_THREADS) reinterpret_cast<uint4*>(sm)[i] = make_uint4(0, 0, 0, 0);
    fence_async_smem();
    if (tid == 0) {
        for (int q = 0; q < NT_STAGES; ++q) {
            bar_init(su32(&bar_full[q]), W_PN);                // one arrival per producer warp
            bar_init(su32(&bar_sfull[q]), 1);
            bar_init(su32(&bar_empty[q]), 1);
        }
        bar_init(su32(&bar_d1_full), 1);
        for (int h = 0; h < 2; ++h) {
            bar_init(su32(&bar_a_full[h]), W_AN);
            bar_init(su32(&bar_a_free[h]), 1);
        }
        bar_init(su32(&bar_d2), 1);
        abort_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == W_C0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_sh)), "r"(NT_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_sh, tD1 = tmem + (uint32_t)(2 * N2);

    if (warp >= W_C0 && warp < W_P0) {
        // ---------------------------------------- MMA issuer and D1 -> B converters
        const int quarter = warp & 3;
        const int L = quarter * 32 + lane, yz = L >> 6, j = L & 63;
        unsigned char* dst = B2 + yz * (N2 * 128);
        const uint32_t id1 = idesc_tf32(N1), id2 = idesc_tf32(N2);
        const uint32_t a0 = su32(A2), b0 = su32(B2);
        const int n2mma = 8 * nmh;                               // stage-2 MMAs per slot: (half, Y|Z, k-step)
        bool ok = true;
        int kg = 0;
        for (int i = 0; i <= nsl; ++i) {
            if (warp == W_C0) {
                if (lane == 0 && ok) {
                    // phase i: stage 1 of slot i (i < nsl) with stage 2 of slot i - 1 (i > 0) spread between its K-blocks
                    const int nkb = (i < nsl) ? s_sl[i].z : 0;
                    int s2 = 0;                                  // next stage-2 MMA
                    // stage-2 MMAs up to `upto` (waiting for a half's Ahat when it is not ready)
                    auto issue_s2 = [&](int upto, bool force) {
                        (void)force;
                        while (ok && s2 < upto) {
                            const int mh = s2 >> 3, yzb = (s2 >> 2) & 1, kk = s2 & 3;
                            if ((s2 & 7) == 0) {
                                const uint32_t ab = su32(&bar_a_full[mh]), par = (uint32_t)((i - 1) & 1);
                                ok = bar_wait(ab, par, status, abort_flag);
                                if (!ok) return;
                                tc_fence_after();
                            }
                            mma(tmem + (uint32_t)(mh * N2), desc_sw128(a0 + yzb * A_KB + mh * (A_KB / 2) + kk * 32),
                                desc_sw128(b0 + yzb * N2 * 128 + kk * 32), id2, (i > 1 || yzb > 0 || kk > 0) ? 1u : 0u);
                            ++s2;
                            if ((s2 & 7) == 0) commit(su32(&bar_a_free[mh]));
                        }
                    };
                    for (int kb = 0; kb < nkb && ok; ++kb, ++kg) {
                        const int q = kg % NT_STAGES;
                        const uint32_t par = (uint32_t)((kg / NT_STAGES) & 1);
                        ok = bar_wait(su32(&bar_full[q]), par, status, abort_flag) &&
                             bar_wait(su32(&bar_sfull[q]), par, status, abort_flag);
                        if (!ok) break;
                        fence_async_smem();                      // the producers' cp.async writes, for the async proxy
                        tc_fence_after();
                        const uint32_t sa = su32(ring + q * lay.stage_bytes), sb = sa + S_BYTES;
#pragma unroll
                        for (int kk = 0; kk < NT_KB / 8; ++kk)
                            mma(tD1, desc_sw128(sa + kk * 32), desc_sw128(sb + kk * 32), id1, (kb > 0 || kk > 0) ? 1u : 0u);
                        commit(su32(&bar_empty[q]));
                        if (i > 0) issue_s2(n2mma * (kb + 1) / (nkb + 1), false);
                    }
                    if (i > 0) issue_s2(n2mma, true);
                    if (ok && i < nsl) commit(su32(&bar_d1_full));   // S1(i) and S2(i - 1) done: D1 full, B and Ahat free
                }
                __syncwarp();
                ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            }
            if (i == nsl) break;
            // convert D1(i) into B; the four warps meet at a named barrier every slot
            bool got = ok && bar_wait(su32(&bar_d1_full), (uint32_t)(i & 1), status, abort_flag);
            got = __all_sync(0xffffffffu, got);
            if (got) {
                tc_fence_after();
                for (int ch = 0; ch < nch; ++ch) {
                    float v[32];
                    tmem_ld32(tD1 + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(ch * 32), v);
#pragma unroll
                    for (int c = 0; c < 8; ++c)
                        *reinterpret_cast<uint4*>(dst + sw128(ch * 64 + j, 4 * c, N2)) =
                            pack_tf32(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
                }
                fence_async_smem();
            }
            ok = ok && got;
            tc_fence_before();
            converters_sync();                                   // D1 read, B(i) written
            tc_fence_after();
        }
        if (warp == W_C0 && lane == 0) {
            commit(su32(&bar_d2));
            bar_drain(su32(&bar_d2), 0, status);                 // every MMA finished (also on the abort path)
        }
        __syncwarp();
    } else if (warp >= W_P0 && warp < W_A1) {
        // -------------------------------------------------- stage-1 producers
        // Lane (row rr, float octet): each warp instruction copies 8 floats of
        // 4 source rows; the octet is rotated by the row so that the 4 rows read
        // different 32-byte chunks (distinct L1 banks), and the shared-memory
        // destinations of the 32 lanes fall in 32 distinct banks.  Each warp
        // keeps up to NT_STAGES K-blocks in flight: after issuing K-block kg it
        // waits for its own copies of K-block kg - (NT_STAGES - 1) and signals
        // that stage with one arrival per warp.
        const int p = warp - W_P0;
        const int rr = p * 4 + (lane & 3), n0 = lane >> 2, twot = 2 * t;
        const size_t chs = (size_t)nk * 8 * t * 2;             // floats per chain of X
        bool ok = true;
        int issued = 0;
        for (int kg = 0; kg < nkg; ++kg) {
            const int q = kg % NT_STAGES;
            if (kg >= NT_STAGES) ok = bar_wait(su32(&bar_empty[q]), (uint32_t)(((kg / NT_STAGES) - 1) & 1), status, abort_flag);
            if (!__all_sync(0xffffffffu, ok)) { ok = false; break; }
            const int i = s_ki[kg] & 0xFFFF, kb = s_ki[kg] >> 16;
            const int4 si = s_sl[i];
            const int r = kb * NT_KB + rr;
            const int code = r < si.w ? (int)s_rows[s_rs[i] + r] : -1;
            unsigned char* Sq = ring + q * lay.stage_bytes;
            unsigned char* Bq = Sq + S_BYTES;
            if (p == 0 && lane == 0) {
                const uint32_t sb = su32(&bar_sfull[q]);
                bar_arrive_tx(sb, S_BYTES);
                bulk_copy(su32(Sq), Simg + (size_t)(si.y + kb) * S_BYTES, S_BYTES, sb);
            }
            if (code >= 0) {
                const int js = code & 0xFF, l = code >> 8;
                const float* src = X + (((size_t)scell[si.x * 8 + l] * Ndiv + js) * 8 + l) * t * 2;
                for (int ch = 0; ch < nch; ++ch)
#pragma unroll
                    for (int fo = 0; fo < 4; ++fo) {
                        const int nn = (((fo + lane) & 3) << 3) + n0;
                        if (nn < twot) cp_async4(Bq + sw128(ch * 32 + nn, rr, N1), src + ch * chs + nn);
                    }
            }
            cp_async_commit();
            ++issued;
            if (kg >= NT_STAGES - 1) {
                cp_async_wait_lag();                             // this thread's copies of K-block kg - (NT_STAGES - 1) landed
                fence_async_smem();
                __syncwarp();
                if (lane == 0) bar_arrive(su32(&bar_full[(kg - (NT_STAGES - 1)) % NT_STAGES]));
            }
        }
        cp_async_wait0();
        fence_async_smem();
        __syncwarp();
        if (ok && lane == 0)                                     // the last NT_STAGES - 1 K-blocks
            for (int j = std::max(0, issued - (NT_STAGES - 1)); j < issued; ++j) bar_arrive(su32(&bar_full[j % NT_STAGES]));
        if (p == 0 && lane == 0)                                 // bulk copies in flight must land before exit
            for (int j = std::max(0, issued - NT_STAGES); j < issued; ++j)
                bar_drain(su32(&bar_sfull[j % NT_STAGES]), (uint32_t)((j / NT_STAGES) & 1), status);
    } else {
        // ------------------------------------------------------ Ahat writers
        // Items (l, e, pair of e') are fixed per thread: decode them once.  The
        // slot's head factors are staged one slot ahead by cp.async into
        // hbuf[slot parity]; the writers never leave the loop early (named
        // barriers), they skip the work once a wait gave up.
        const int ta = (warp < W_C0 ? warp : warp - W_A1 + W_C0) * 32 + lane;
        const int nvv = nv * nv, ncc = nc * nc, nitem = 8 * t * th, per = nvv + ncc + 1;
        int d0[NT_AMAX], d1[NT_AMAX], d2[NT_AMAX];
#pragma unroll
        for (int k = 0; k < NT_AMAX; ++k) {
            const int it = ta + k * NT_A;
            d0[k] = d1[k] = d2[k] = -1;
            if (it < nitem) {
                const int l = it / (t * th), e = (it / th) % t, qp = it % th;
                const int n1 = e / nc, n2 = e % nc, ep0 = 2 * qp, ep1 = 2 * qp + 1, has1 = ep1 < t;
                const int e1 = has1 ? ep1 : ep0;
                const int hv0 = l * nvv + n1 * nv + ep0 / nc, hv1 = l * nvv + n1 * nv + e1 / nc;
                const int hm0 = l * ncc + n2 * nc + ep0 % nc, hm1 = l * ncc + n2 * nc + e1 % nc;
                const int row = (l * t + e) * 2;
                d0[k] = hv0 | (hv1 << 9) | (hm0 << 18);
                d1[k] = hm1 | (((int)sw128(row, 4 * qp, NT_M) >> 4) << 9) | (l << 21) | (has1 << 24) | (((l * t + e) >= 64) << 25);
                d2[k] = (int)sw128(row + 1, 4 * qp, NT_M) >> 4;
            }
        }
        auto prefetch = [&](int i) {
            const Int3 so = unflat3(s_sl[i].x, ns1);
            const int oa = so.a + smin - rmin, ob = so.b + smin - rmin, oc = so.c + smin - rmin;
            float2* hvS = reinterpret_cast<float2*>(hbuf + (i & 1) * hbb);
            float2* hmS = hvS + 8 * nvv;
            float* hcS = reinterpret_cast<float*>(hmS + 8 * ncc);
            for (int j = ta; j < 8 * per; j += NT_A) {
                const int l = j / per, w = j - l * per;
                const int l1 = (l >> 2) & 1, l2 = (l >> 1) & 1, l3 = l & 1;
                const int kt = flat3(ci.a + l1, ci.b + l2, ci.c + l3, n);
                const int r = ((oa - l1) * nr1 + (ob - l2)) * nr1 + (oc - l3);
                if (w < nvv) cp_async8(hvS + l * nvv + w, Hv + ((size_t)kt * nrel + r) * nvv + w);
                else if (w < nvv + ncc) cp_async8(hmS + l * ncc + (w - nvv), Hc + ((size_t)kt * nrel + r) * ncc + (w - nvv));
                else cp_async4(hcS + l, hc + r);
            }
        };
        bool ok = true;
        prefetch(0);
        cp_async_commit();
        for (int i = 0; i < nsl; ++i) {
            writers_sync();                                      // every writer is done with slot i - 1's buffer
            if (i + 1 < nsl) prefetch(i + 1);
            cp_async_commit();
            cp_async_wait1();                                    // this thread's copies for slot i landed
            writers_sync();                                      // everyone's copies for slot i landed
            const float2* hvS = reinterpret_cast<const float2*>(hbuf + (i & 1) * hbb);
            const float2* hmS = hvS + 8 * nvv;
            const float* hcS = reinterpret_cast<const float*>(hmS + 8 * ncc);
            for (int mh = 0; mh < nmh; ++mh) {
                if (ok && i > 0) ok = bar_wait(su32(&bar_a_free[mh]), (uint32_t)((i - 1) & 1), status, abort_flag);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) continue;
#pragma unroll
                for (int k = 0; k < NT_AMAX; ++k) {
                    if (d0[k] < 0 || ((d1[k] >> 25) & 1) != mh) continue;
                    const int l = (d1[k] >> 21) & 7;
                    const float2 c0 = cmul(hvS[d0[k] & 511], hmS[(d0[k] >> 18) & 511]);
                    const float2 c1 = ((d1[k] >> 24) & 1) ? cmul(hvS[(d0[k] >> 9) & 511], hmS[d1[k] & 511])
                                                          : make_float2(0.f, 0.f);
                    const float mhc = -hcS[l];
                    const uint32_t o0 = (uint32_t)(((d1[k] >> 9) & 4095) << 4), o1 = (uint32_t)(d2[k] << 4);
                    *reinterpret_cast<uint4*>(A2 + o0) = pack_tf32(c0.x, -c0.y, c1.x, -c1.y);
                    *reinterpret_cast<uint4*>(A2 + o1) = pack_tf32(c0.y, c0.x, c1.y, c1.x);
                    *reinterpret_cast<uint4*>(A2 + A_KB + o0) = pack_tf32(mhc * c0.x, -mhc * c0.y, mhc * c1.x, -mhc * c1.y);
                    *reinterpret_cast<uint4*>(A2 + A_KB + o1) = pack_tf32(mhc * c0.y, mhc * c0.x, mhc * c1.y, mhc * c1.x);
                }
                fence_async_smem();
                __syncwarp();
                if (lane == 0) bar_arrive(su32(&bar_a_full[mh]));
            }
        }
        cp_async_wait0();
    }

    // ------------------------------------------------------------- epilogue
    const bool done = bar_wait(su32(&bar_d2), 0, status, abort_flag);
    if (__all_sync(0xffffffffu, done) && !*abort_flag) {
        tc_fence_after();
        // warp w reads TMEM lanes 32 (w % 4).. of items (half, 32-column chunk) w / 4, w / 4 + 6, ...
        const int quarter = warp & 3, cg = warp >> 2, nchunk = N2 / 32;
        for (int item = cg; item < nmh * nchunk; item += NT_THREADS / 128) {
            const int mh = item / nchunk, c = item % nchunk, ch = c >> 1, j0 = (c & 1) * 32;
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(mh * N2 + c * 32), v);
            const int row = mh * 128 + quarter * 32 + lane;
            const int pair = row >> 1, ri = row & 1;
            const int l = pair / t, e = pair % t;
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
                const float other = __shfl_xor_sync(0xffffffffu, v[jj], 1);
                const int j = j0 + jj;
                if (ri == 0 && l < 8 && j < Ndiv && interp_active(j, l, nd, nb1))
                    U[(((size_t)ch * nk + (size_t)cell * Ndiv + j) * 8 + l) * t + e] = make_float2(v[jj], other);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == W_C0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NT_TMEM_COLS));
    }
}

// S images: entry {K-block, target, row in K-block, near-offset index}; the
// y1 row of the target gets h_head, the z row 1 (images zeroed beforehand).
__global__ void k_near_pattern(const int4* __restrict__ ent, int nent, const float* __restrict__ hd,
                               unsigned char* __restrict__ img) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nent) return;
    const int4 e = ent[i];
    unsigned char* b = img + (size_t)e.x * S_BYTES;
    *reinterpret_cast<uint32_t*>(b + sw128(e.y, e.z, 128)) = f2tf32(hd[e.w]);
    *reinterpret_cast<uint32_t*>(b + sw128(64 + e.y, e.z, 128)) = f2tf32(1.0f);
}

size_t near_tc_smem(int nv, int nc, int nch, int nsl, int nkg, int nslot, int nrows) {
    const NtLayout lay(nch);
    return 1024 + (size_t)lay.tab_off + 2 * (size_t)hb_bytes(nv, nc) + 20 * (size_t)nsl + 4 * (size_t)nkg +
           32 * (size_t)nslot + 2 * (size_t)nrows;
}

}  // namespace

// Decide whether the tensor-core near field serves this handle (FP32 M3 with
// t <= 16 and N_div <= 64), and build its per-slot source rows and pattern
// images from the per-(target, slot) near lists (needs the near head values).
int bse_near_tc_prepare(bse_ctx* ctx, bse_interp* s, const std::vector<std::vector<NearEntry>>& per_slot) {
    s->nf_tc = 0;
    if (s->vec_prec != BSE_PREC_F32 || s->t > 16 || s->Ndiv > NT_N || s->scheme != BSE_SCHEME_M3) return BSE_OK;
    const int Ndiv = s->Ndiv, nslot = s->nslot;
    std::vector<int4> slots, pent;
    std::vector<int> rows, rowstart, kinfo, loc((size_t)Ndiv * 8, -1);
    int kstart = 0;
    for (int sl = 0; sl < nslot; ++sl) {
        std::vector<int> used;
        for (int j = 0; j < Ndiv; ++j)
            for (const NearEntry& en : per_slot[(size_t)j * nslot + sl]) used.push_back(en.js_src * 8 + en.l_src);
        if (used.empty()) continue;                             // nothing of this slot reaches the cell
        std::sort(used.begin(), used.end());
        used.erase(std::unique(used.begin(), used.end()), used.end());
        const int R = (int)used.size(), nkb = (R + NT_KB - 1) / NT_KB, ord = (int)slots.size();
        for (int r = 0; r < R; ++r) loc[used[r]] = r;
        for (int j = 0; j < Ndiv; ++j)
            for (const NearEntry& en : per_slot[(size_t)j * nslot + sl]) {
                const int r = loc[en.js_src * 8 + en.l_src];
                pent.push_back(make_int4(kstart + r / NT_KB, j, r % NT_KB, en.near_idx));
            }
        slots.push_back(make_int4(sl, kstart, nkb, R));
        rowstart.push_back((int)rows.size());
        for (int r = 0; r < R; ++r) rows.push_back((used[r] / 8) | ((used[r] % 8) << 16));
        for (int kb = 0; kb < nkb; ++kb) kinfo.push_back(ord | (kb << 16));
        kstart += nkb;
    }
    if (slots.empty() || slots.size() >= 65536) return BSE_OK;
    int maxsm = 0;
    cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
    const size_t smem = near_tc_smem(s->nv, s->nc, 3, (int)slots.size(), (int)kinfo.size(), nslot, (int)rows.size());
    if (smem > (size_t)maxsm) return BSE_OK;
    auto upload = [&](void** dst, const void* src, size_t bytes, const char* what) -> int {
        int rc = bse_alloc(ctx, dst, bytes, what);
        if (rc != BSE_OK) return rc;
        BSE_CUDA_TRY(ctx, cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
        return BSE_OK;
    };
    int rc;
    int4* d_pent = nullptr;
    if ((rc = upload((void**)&s->d_tc_rows, rows.data(), sizeof(int) * rows.size(), "near rows")) != BSE_OK) return rc;
    if ((rc = upload((void**)&s->d_tc_slots, slots.data(), sizeof(int4) * slots.size(), "near slots")) != BSE_OK) return rc;
    if ((rc = upload((void**)&s->d_tc_rowstart, rowstart.data(), sizeof(int) * rowstart.size(), "near row starts")) != BSE_OK) return rc;
    if ((rc = upload((void**)&s->d_tc_kinfo, kinfo.data(), sizeof(int) * kinfo.size(), "near K-blocks")) != BSE_OK) return rc;
    if ((rc = bse_alloc(ctx, (void**)&s->d_tc_simg, (size_t)kstart * S_BYTES, "near pattern images")) != BSE_OK) return rc;
    if ((rc = upload((void**)&d_pent, pent.data(), sizeof(int4) * pent.size(), "near pattern entries")) != BSE_OK) return rc;
    BSE_CUDA_TRY(ctx, cudaMemsetAsync(s->d_tc_simg, 0, (size_t)kstart * S_BYTES, ctx->stream));
    k_near_pattern<<<(int)((pent.size() + 255) / 256), 256, 0, ctx->stream>>>(d_pent, (int)pent.size(),
                                                                               (const float*)s->d_hd, s->d_tc_simg);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(d_pent);
    if (e != cudaSuccess) {
        ctx->err = std::string("near pattern images: ") + cudaGetErrorString(e);
        return BSE_ERR_CUDA;
    }
    s->nf_tc_nsl = (int)slots.size();
    s->nf_tc_nkg = (int)kinfo.size();
    s->nf_tc_nrows = (int)rows.size();
    s->nf_tc = 1;
    return BSE_OK;
}

int bse_near_tc_launch(bse_ctx* ctx, const bse_interp* s, int nchains, const void* X, void* U) {
    // at most three chains per launch (TMEM: 160 columns per chain)
    for (int c0 = 0; c0 < nchains; c0 += 3) {
        const int nch = std::min(3, nchains - c0);
        const size_t smem = near_tc_smem(s->nv, s->nc, nch, s->nf_tc_nsl, s->nf_tc_nkg, s->nslot, s->nf_tc_nrows);
        // handles of different sizes share the kernel's attribute: only ever raise it
        cudaFuncAttributes fa;
        BSE_CUDA_TRY(ctx, cudaFuncGetAttributes(&fa, k_near_tc));
        if ((size_t)fa.maxDynamicSharedSizeBytes < smem)
            BSE_CUDA_TRY(ctx, cudaFuncSetAttribute(k_near_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        const size_t off = (size_t)c0 * s->nk * 8 * s->t;
        k_near_tc<<<s->co->nkc, NT_THREADS, smem, ctx->stream>>>(
            (const float*)((const float2*)X + off), s->d_tc_rows, s->d_tc_slots, s->d_tc_rowstart, s->d_tc_kinfo,
            s->nf_tc_nsl, s->nf_tc_nkg, s->nf_tc_nrows, s->d_tc_simg, (const float2*)s->d_Hv, (const float2*)s->d_Hc,
            (const float*)s->d_hc, s->n, s->nd, s->nv, s->nc, s->nb1, s->smin, s->ns1, s->rmin, s->nr1, nch,
            (float2*)U + off, ctx->d_status);
    }
    return BSE_OK;
}
