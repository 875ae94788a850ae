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
// (chain, e, re|im)) transposed into shared memory with cp.async and issues
//   D1 [128 = (y1|z, target)] x [32 * chains] += S_s[., K-block] * X_s[K-block]^T
// through a three-stage ring.
// Stage 2 (per slot): D1 is read back from TMEM into the B operand
//   B_s[(chain, k), (Y|Z, e', re|im)]  = y1(k, s), z(k, s)
// and, with the real form
//   Ahat_s[(l,e,.), (Y,e',.)] = [[Re c, -Im c], [Im c, Re c]],  c = A(k~_l, k~_s)[e][e'],
//   Ahat_s[(l,e,.), (Z,e',.)] = the same for -h_head(q_c(l, s)) c,
// formed in shared memory from the per-cell head factors,
//   D2 [256 = (l, e, re|im)] x [64 * chains] += Ahat_s [256 x 64] * B_s^T.
// tcgen05.mma kind::tf32 (10-bit mantissa, FP32 range: y1 and h_head z nearly
// cancel in u, which BF16 would not resolve), FP32 accumulators in TMEM.
// Constraints: t <= 16, N_div <= 64, FP32 vectors, <= 3 chains per launch.
// Every wait is bounded.
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
constexpr int NT_THREADS = 512;
constexpr int NT_TMEM_COLS = 512;
constexpr long long NT_WAIT_CYCLES = 4000000000LL;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(su32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(su32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(su32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ uint32_t f2tf32(float v) {
    uint32_t u;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(v));
    return u;
}
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

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
__device__ __forceinline__ bool bar_try(uint32_t b, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(b), "r"(parity) : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool bar_wait(uint32_t b, uint32_t parity, int* status) {
    const long long t0 = clock64();
    while (!bar_try(b, parity)) {
        if (clock64() - t0 > NT_WAIT_CYCLES) {
            atomicOr(status, 2);
            return false;
        }
    }
    return true;
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

// Pack four values rounded to TF32 into one 16-byte chunk.
__device__ __forceinline__ uint4 pack_tf32(float a, float b, float c, float d) {
    uint4 u;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u.x) : "f"(a));
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u.y) : "f"(b));
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u.z) : "f"(c));
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u.w) : "f"(d));
    return u;
}

// Shared-memory bytes of one head-factor buffer: Hv, Hc of the 8 target corners
// for one slot, then h_head(q_c) of the 8 corners.
__host__ __device__ __forceinline__ int hb_bytes(int nv, int nc) {
    return ((8 * (nv * nv + nc * nc) * 8 + 32) + 15) & ~15;
}

// Slot table entry {slot, first K-block, K-blocks, source rows} and per-K-block
// info (slot ordinal | K-block in slot << 16) are staged in shared memory.
__global__ void __launch_bounds__(NT_THREADS, 1) k_near_tc(
    const float* __restrict__ X, const int* __restrict__ rows, const int4* __restrict__ slots,
    const int* __restrict__ rowstart, const int* __restrict__ kinfo, int nsl, int nkg,
    const unsigned char* __restrict__ Simg, const float2* __restrict__ Hv, const float2* __restrict__ Hc,
    const float* __restrict__ hc, int n, int nd, int nv, int nc, int nb1, int smin, int ns1, int rmin, int nr1,
    int nch, float2* __restrict__ U, int* __restrict__ status) {
    extern __shared__ unsigned char raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t bar_s[NT_STAGES], bar_d1, bar_mma2, bar_drain;
    __shared__ uint32_t tmem_sh;
    __shared__ int abort_flag;
    const int t = nv * nc, Ndiv = nd * nd * nd, nslot = ns1 * ns1 * ns1, nrel = nr1 * nr1 * nr1;
    const int nk = n * n * n * Ndiv, th = (t + 1) >> 1, hbb = hb_bytes(nv, nc), nitem = 8 * t * th;
    const int N1 = 32 * nch, N2 = 64 * nch, stage_bytes = S_BYTES + N1 * 128;
    const int cell = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char* A2 = sm;                                     // [A_BYTES]   Ahat_s
    unsigned char* B2 = sm + A_BYTES;                           // [2][N2 x 128 B]  B_s, Y and Z K-blocks
    unsigned char* ring = B2 + 2 * N2 * 128;                    // [NT_STAGES][S K-block | X K-block]
    unsigned char* hbuf = ring + NT_STAGES * stage_bytes;       // [2][hbb]
    int4* aidx = reinterpret_cast<int4*>(hbuf + 2 * hbb);       // [nitem] A-tile item tables
    int4* s_sl = aidx + nitem;                                  // [nsl]
    int* s_rs = reinterpret_cast<int*>(s_sl + nsl);             // [nsl]
    int* s_ki = s_rs + nsl;                                     // [nkg]
    int* scell = s_ki + nkg;                                    // [nslot][8] source cells
    const Int3 ci = unflat3(cell, n);
    for (int i = tid; i < nsl; i += NT_THREADS) { s_sl[i] = slots[i]; s_rs[i] = rowstart[i]; }
    for (int i = tid; i < nkg; i += NT_THREADS) s_ki[i] = kinfo[i];
    for (int i = tid; i < nslot * 8; i += NT_THREADS) {
        const int s = i >> 3, l = i & 7;
        const Int3 so = unflat3(s, ns1);
        scell[i] = flat3(ci.a + so.a + smin - ((l >> 2) & 1), ci.b + so.b + smin - ((l >> 1) & 1),
                         ci.c + so.c + smin - (l & 1), n);
    }
    // A-tile items: {Hv offsets of e'0 | e'1 << 16, Hc offsets likewise, chunk offsets of the re | im rows,
    // corner | (e'1 exists) << 8}
    for (int it = tid; it < nitem; it += NT_THREADS) {
        const int l = it / (t * th), e = (it / th) % t, qp = it % th;
        const int n1 = e / nc, n2 = e % nc, ep0 = 2 * qp, ep1 = 2 * qp + 1, has1 = ep1 < t;
        const int e1 = has1 ? ep1 : ep0;
        const int row = (l * t + e) * 2, kq = 4 * qp;
        aidx[it] = make_int4((l * nv * nv + n1 * nv + ep0 / nc) | ((l * nv * nv + n1 * nv + e1 / nc) << 16),
                             (l * nc * nc + n2 * nc + ep0 % nc) | ((l * nc * nc + n2 * nc + e1 % nc) << 16),
                             (int)sw128(row, kq, NT_M) | ((int)sw128(row + 1, kq, NT_M) << 16), l | (has1 << 8));
    }
    // zero the operands once: padding rows / columns stay zero for the whole kernel
    for (int i = tid; i < (int)((ring + NT_STAGES * stage_bytes - sm) / 16); i += NT_THREADS)
        reinterpret_cast<uint4*>(sm)[i] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        for (int q = 0; q < NT_STAGES; ++q) bar_init(su32(&bar_s[q]), 1);
        bar_init(su32(&bar_d1), 1);
        bar_init(su32(&bar_mma2), 1);
        bar_init(su32(&bar_drain), 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_sh)), "r"(NT_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_sh, tD1 = tmem + (uint32_t)(2 * N2);

    // stage-1 gather map: warp w stages rows w and w + 16 of a K-block, lane = (e, re|im)
    const int twot = 2 * t;
    int rc[2];                                                  // row codes of the next K-block to stage
    auto load_codes = [&](int kg) {
        const int i = s_ki[kg] & 0xFFFF, kb = s_ki[kg] >> 16;
        const int R = s_sl[i].w;
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
            const int r = kb * NT_KB + warp + 16 * rr;
            rc[rr] = r < R ? __ldg(rows + s_rs[i] + r) : -1;
        }
    };
    auto prefetch = [&](int kg) {
        const int i = s_ki[kg] & 0xFFFF, kb = s_ki[kg] >> 16, q = kg % NT_STAGES;
        const int4 si = s_sl[i];
        const int s = si.x;
        unsigned char* Sq = ring + q * stage_bytes;
        unsigned char* Bq = Sq + S_BYTES;
        const unsigned char* src = Simg + (size_t)(si.y + kb) * S_BYTES;
        for (int c = tid; c < S_BYTES / 16; c += NT_THREADS) cp_async16(Sq + 16 * c, src + 16 * c);
        if (lane < twot) {
#pragma unroll
            for (int rr = 0; rr < 2; ++rr) {
                if (rc[rr] < 0) continue;
                const int js = rc[rr] & 0xFFFF, l = rc[rr] >> 16, kk = warp + 16 * rr;
                const size_t rowsrc = (((size_t)scell[s * 8 + l] * Ndiv + js) * 8 + l) * t;
                for (int ch = 0; ch < nch; ++ch)
                    cp_async4(Bq + sw128(ch * 32 + lane, kk, N1), X + ((size_t)ch * nk * 8 * t + rowsrc) * 2 + lane);
            }
        }
        if (kb == 0) {                                          // first K-block of a slot: its head factors
            const Int3 so = unflat3(s, ns1);
            const int oa = so.a + smin, ob = so.b + smin, oc = so.c + smin;
            float2* hvS = reinterpret_cast<float2*>(hbuf + (i & 1) * hbb);
            float2* hmS = hvS + 8 * nv * nv;
            float* hcS = reinterpret_cast<float*>(hmS + 8 * nc * nc);
            const int nvv = nv * nv, ncc = nc * nc, per = nvv + ncc + 1;
            for (int j = tid; j < 8 * per; j += NT_THREADS) {
                const int l = j / per, w = j - l * per;
                const int l1 = (l >> 2) & 1, l2 = (l >> 1) & 1, l3 = l & 1;
                const int kt = flat3(ci.a + l1, ci.b + l2, ci.c + l3, n);
                const int r = ((oa - l1 - rmin) * nr1 + (ob - l2 - rmin)) * nr1 + (oc - l3 - rmin);
                if (w < nvv) cp_async8(hvS + l * nvv + w, Hv + ((size_t)kt * nrel + r) * nvv + w);
                else if (w < nvv + ncc) cp_async8(hmS + l * ncc + (w - nvv), Hc + ((size_t)kt * nrel + r) * ncc + (w - nvv));
                else cp_async4(hcS + l, hc + r);
            }
        }
    };

    const uint32_t id1 = idesc_tf32(N1), id2 = idesc_tf32(N2);
    load_codes(0);
    prefetch(0);
    cp_async_commit();
    if (nkg > 1) load_codes(1);
    for (int kg = 0; kg < nkg; ++kg) {
        const int i = s_ki[kg] & 0xFFFF, kb = s_ki[kg] >> 16, q = kg % NT_STAGES;
        const int4 si = s_sl[i];
        // the stage of K-block kg + 1 was read by the MMAs of K-block kg + 1 - NT_STAGES
        if (kg + 1 < nkg) {
            if (kg + 1 >= NT_STAGES) {
                const int qn = (kg + 1) % NT_STAGES, use = (kg + 1 - NT_STAGES) / NT_STAGES;
                if (!bar_wait(su32(&bar_s[qn]), (uint32_t)(use & 1), status)) abort_flag = 1;
            }
            prefetch(kg + 1);
            if (kg + 2 < nkg) load_codes(kg + 2);
        }
        cp_async_commit();
        cp_async_wait1();                                       // this thread's copies of K-block kg landed
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (abort_flag) break;
        // stage 1: D1 (+)= S_s[., K-block] * X[K-block]^T
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sa = su32(ring + q * stage_bytes), sb = sa + S_BYTES;
#pragma unroll
            for (int kk = 0; kk < NT_KB / 8; ++kk)
                mma(tD1, desc_sw128(sa + kk * 32), desc_sw128(sb + kk * 32), id1, (kb > 0 || kk > 0) ? 1u : 0u);
            commit(su32(&bar_s[q]));
        }
        if (kb == si.z - 1) {
            // slot end: Ahat_s, then D1 complete -> B_s -> stage 2.  Ahat and B_s are
            // rewritten here: the previous slot's stage-2 MMAs must be done.
            if (tid == 0) {
                commit(su32(&bar_d1));
                if (i > 0 && !bar_wait(su32(&bar_mma2), (uint32_t)((i - 1) & 1), status)) abort_flag = 1;
            }
            __syncthreads();
            if (abort_flag) break;
            {
                // Ahat_s: item (l, e, pair of e') writes one 16-byte chunk to four rows
                const float2* hvS = reinterpret_cast<const float2*>(hbuf + (i & 1) * hbb);
                const float2* hmS = hvS + 8 * nv * nv;
                const float* hcS = reinterpret_cast<const float*>(hmS + 8 * nc * nc);
                for (int it = tid; it < nitem; it += NT_THREADS) {
                    const int4 ix = aidx[it];
                    const float2 c0 = cmul(hvS[ix.x & 0xFFFF], hmS[ix.y & 0xFFFF]);
                    float2 c1 = cmul(hvS[ix.x >> 16], hmS[ix.y >> 16]);
                    if (!(ix.w >> 8)) c1 = make_float2(0.f, 0.f);
                    const float mh = -hcS[ix.w & 0xFF];
                    const int o0 = ix.z & 0xFFFF, o1 = (ix.z >> 16) & 0xFFFF;
                    *reinterpret_cast<uint4*>(A2 + o0) = pack_tf32(c0.x, -c0.y, c1.x, -c1.y);
                    *reinterpret_cast<uint4*>(A2 + o1) = pack_tf32(c0.y, c0.x, c1.y, c1.x);
                    *reinterpret_cast<uint4*>(A2 + A_KB + o0) = pack_tf32(mh * c0.x, -mh * c0.y, mh * c1.x, -mh * c1.y);
                    *reinterpret_cast<uint4*>(A2 + A_KB + o1) = pack_tf32(mh * c0.y, mh * c0.x, mh * c1.y, mh * c1.x);
                }
            }
            if (tid == 0 && !bar_wait(su32(&bar_d1), (uint32_t)(i & 1), status)) abort_flag = 1;
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (abort_flag) break;
            if (warp < 4) {
                const int L = warp * 32 + lane, yz = L >> 6, j = L & 63;
                for (int ch = 0; ch < nch; ++ch) {
                    float v[32];
                    tmem_ld32(tD1 + ((uint32_t)(warp * 32) << 16) + (uint32_t)(ch * 32), v);
                    unsigned char* dst = B2 + yz * (N2 * 128);
#pragma unroll
                    for (int c = 0; c < 8; ++c)
                        *reinterpret_cast<uint4*>(dst + sw128(ch * 64 + j, 4 * c, N2)) =
                            pack_tf32(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t a0 = su32(A2), b0 = su32(B2);
#pragma unroll
                for (int mh = 0; mh < 2; ++mh)
#pragma unroll
                    for (int kb2 = 0; kb2 < 2; ++kb2)
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)
                            mma(tmem + (uint32_t)(mh * N2), desc_sw128(a0 + kb2 * A_KB + mh * (A_KB / 2) + kk * 32),
                                desc_sw128(b0 + kb2 * N2 * 128 + kk * 32), id2, (i > 0 || kb2 > 0 || kk > 0) ? 1u : 0u);
                commit(su32(&bar_mma2));
            }
        }
    }
    cp_async_wait0();
    // all MMAs done before reading TMEM (and before freeing it on any path)
    if (tid == 0) {
        commit(su32(&bar_drain));
        if (!bar_wait(su32(&bar_drain), 0, status)) abort_flag = 1;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!abort_flag) {
        // epilogue: warp w reads TMEM lanes 32 (w % 4).. of items (half, 32-column chunk) w / 4, w / 4 + 4, ...
        const int quarter = warp & 3, cg = warp >> 2, nchunk = N2 / 32;
        for (int item = cg; item < 2 * nchunk; item += 4) {
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
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NT_TMEM_COLS));
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

size_t near_tc_smem(int nv, int nc, int nch, int nsl, int nkg, int nslot) {
    const int t = nv * nc, th = (t + 1) / 2;
    return 1024 + A_BYTES + (size_t)2 * 64 * nch * 128 + (size_t)NT_STAGES * (S_BYTES + 32 * nch * 128) +
           2 * (size_t)hb_bytes(nv, nc) + 16 * (size_t)(8 * t * th) + 20 * (size_t)nsl + 4 * (size_t)nkg +
           32 * (size_t)nslot;
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
    const size_t smem = near_tc_smem(s->nv, s->nc, 3, (int)slots.size(), (int)kinfo.size(), nslot);
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
    s->nf_tc = 1;
    return BSE_OK;
}

int bse_near_tc_launch(bse_ctx* ctx, const bse_interp* s, int nchains, const void* X, void* U) {
    // at most three chains per launch (TMEM: 160 columns per chain)
    for (int c0 = 0; c0 < nchains; c0 += 3) {
        const int nch = std::min(3, nchains - c0);
        const size_t smem = near_tc_smem(s->nv, s->nc, nch, s->nf_tc_nsl, s->nf_tc_nkg, s->nslot);
        // handles of different sizes share the kernel's attribute: only ever raise it
        cudaFuncAttributes fa;
        BSE_CUDA_TRY(ctx, cudaFuncGetAttributes(&fa, k_near_tc));
        if ((size_t)fa.maxDynamicSharedSizeBytes < smem)
            BSE_CUDA_TRY(ctx, cudaFuncSetAttribute(k_near_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        const size_t off = (size_t)c0 * s->nk * 8 * s->t;
        k_near_tc<<<s->co->nkc, NT_THREADS, smem, ctx->stream>>>(
            (const float*)((const float2*)X + off), s->d_tc_rows, s->d_tc_slots, s->d_tc_rowstart, s->d_tc_kinfo,
            s->nf_tc_nsl, s->nf_tc_nkg, s->d_tc_simg, (const float2*)s->d_Hv, (const float2*)s->d_Hc,
            (const float*)s->d_hc, s->n, s->nd, s->nv, s->nc, s->nb1, s->smin, s->ns1, s->rmin, s->nr1, nch,
            (float2*)U + off, ctx->d_status);
    }
    return BSE_OK;
}
