// Method 3 near field with the head contraction on the tensor cores.
//
// For one coarse cell C and one Lanczos step, the correction in coarse-basis
// form is
//   u(k, l) = sum_s A(k~_l, k~_s) [y1(k, s) - h_head(q_c(l, s)) z(k, s)],
// A = alpha O^v (x) O^c the Kronecker head block of Eq. diverg, s over the
// source slots, k over the N_div targets of C.  In real form this is a GEMM
//   D [(l, e, re|im) = 256] x [k = 64] = sum_s  Ahat_s [256 x 64] * B_s [64 x 64]^T
// with, per slot, K = (y1 | z, e', re|im) = 64 and
//   Ahat_s[(l,e,.), (Y,e',.)] = [[Re c, -Im c], [Im c, Re c]],  c = A(k~_l, k~_s)[e][e'],
//   Ahat_s[(l,e,.), (Z,e',.)] = the same for -h_head(q_c(l, s)) c,
//   B_s[k, (Y|Z, e', re|im)]  = y1(k, s), z(k, s).
// Each slot's Ahat is formed in shared memory from the per-cell head factors
// (a few KB, L2-resident), so no image of it is kept in HBM; y1, z are formed
// on the CUDA cores exactly as in the CUDA-core kernels.  Operands are TF32
// (10-bit mantissa, FP32 range) rather than BF16 because y1 and h_head z
// nearly cancel in u.  tcgen05.mma kind::tf32, M = 128 (two halves of the 256
// rows), N = 64, K = 8, FP32 accumulators in TMEM (two per chain).  Shared
// memory per operand: two K-blocks of 32 elements (Y block, Z block), each
// 128-byte rows with the 128-byte swizzle.
// The source rows a slot references and its contribution lists are the same
// for every cell (translation invariance of the near pattern), so set-up
// compacts them per slot and cuts each slot into units of at most NT_RCAP
// source rows and NT_ECAP contributions.  A unit's record (its schedule and
// contribution list) and source rows are staged in shared memory; within a
// unit the targets are split into segments of about equal length assigned
// longest-first to thread groups (a group = one target, four transitions per
// thread), and a target split over several segments is summed from shared-
// memory partials in a fixed order, so results are deterministic.
// Pipeline over steps g = (unit, chain): while step g is formed, cp.async
// brings step g + 1's record, source rows and (at a slot change) head factors
// into the other half of a double buffer; B ping-pongs between two buffers so
// the MMAs of step g run under the forming of step g + 1.  Every unit of a
// slot is one more K = 64 block against the same Ahat, so Ahat is rebuilt
// only when the slot changes.
// Constraints: t <= 16, N_div <= 64, FP32 vectors, <= 4 chains.  Every wait is bounded.
#include <cuda.h>

#include <algorithm>
#include <functional>

#include "bse_internal.cuh"

namespace {

constexpr int NT_M = 256;                    // rows (corner l, transition e, re|im), 8 * 16 * 2
constexpr int NT_N = 64;                     // targets of the cell
constexpr int A_KB = NT_M * 128;             // one 32-element K-block of A: 32 KB
constexpr int B_KB = NT_N * 128;             // one K-block of B: 8 KB
constexpr int A_BYTES = 2 * A_KB;            // 64 KB per slot
constexpr int B_BYTES = 2 * B_KB;            // 16 KB per unit
constexpr int NT_THREADS = 512;
constexpr int NT_RCAP = 128;                 // source rows per unit
constexpr int NT_ECAP = 2048;                // contributions per unit
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
// kind::tf32, A = B = TF32, D = F32, both K-major, M = 128, N = 64
constexpr uint32_t NT_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NT_N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                 ::"r"(d), "l"(a), "l"(b), "r"(NT_IDESC), "r"(acc));
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

// Packed FP32x2 arithmetic on (re, im) pairs held in 64-bit registers.
__device__ __forceinline__ uint64_t pack2(float a, float b) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 unpack2(uint64_t v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ void fma2(uint64_t& d, uint64_t a, uint64_t b) {
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(a), "l"(b));
}
__device__ __forceinline__ void add2(uint64_t& d, uint64_t b) { asm("add.rn.f32x2 %0, %0, %1;" : "+l"(d) : "l"(b)); }

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

// y1 and z of one target for this thread's transitions 2qd, 2qd+1 (y[0..1])
// and 2(qd+tq), 2(qd+tq)+1 (y[2..3]): one 16-byte chunk per operand block
// each; transitions at or beyond t are written as zero.
__device__ __forceinline__ void store_b_row(unsigned char* Bt, int j, int qd, int tq, int t, const uint64_t* y,
                                            const uint64_t* z) {
    float2 yv[4], zv[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int e = 2 * qd + (k >> 1) * 2 * tq + (k & 1);
        yv[k] = e < t ? unpack2(y[k]) : make_float2(0.f, 0.f);
        zv[k] = e < t ? unpack2(z[k]) : make_float2(0.f, 0.f);
    }
    const int c0 = 4 * qd, c1 = 4 * qd + 4 * tq;
    *reinterpret_cast<uint4*>(Bt + sw128(j, c0, NT_N)) = pack_tf32(yv[0].x, yv[0].y, yv[1].x, yv[1].y);
    *reinterpret_cast<uint4*>(Bt + sw128(j, c1, NT_N)) = pack_tf32(yv[2].x, yv[2].y, yv[3].x, yv[3].y);
    *reinterpret_cast<uint4*>(Bt + sw128(j, 32 + c0, NT_N)) = pack_tf32(zv[0].x, zv[0].y, zv[1].x, zv[1].y);
    *reinterpret_cast<uint4*>(Bt + sw128(j, 32 + c1, NT_N)) = pack_tf32(zv[2].x, zv[2].y, zv[3].x, zv[3].y);
}

// Record layout (ints, every section 16-byte aligned):
//   [0..3] rows, contributions, segments, split targets of the unit
//   [4 ..) segment starts per group (groups + 1, padded to 4)
//   then segments {q0, q1, target, partial or -1}, split targets {target, first partial, count, 0},
//   contributions (row byte offset in the staged rows | near-offset index << 16, padded to 4).
__host__ __device__ __forceinline__ int rec_seg_off(int G) { return 4 + ((G + 1 + 3) & ~3); }

__global__ void __launch_bounds__(NT_THREADS, 1) k_near_tc(
    const float2* __restrict__ X, const int* __restrict__ rows, const int2* __restrict__ urow,
    const int* __restrict__ rec, const int2* __restrict__ urec, const int2* __restrict__ uinfo, int nunits,
    const float* __restrict__ hd, int n_near, const float2* __restrict__ Hv, const float2* __restrict__ Hc,
    const float* __restrict__ hc, int n, int nd, int nv, int nc, int nb1, int smin, int ns1, int rmin, int nr1,
    int nchains, int rec_max, int npart, float2* __restrict__ U, int* __restrict__ status) {
    extern __shared__ unsigned char raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t bar_b[2], bar_mma, bar_drain;
    __shared__ uint32_t tmem_sh;
    __shared__ int abort_flag;
    const int t = nv * nc, Ndiv = nd * nd * nd, nslot = ns1 * ns1 * ns1, nrel = nr1 * nr1 * nr1;
    const int nk = n * n * n * Ndiv, th = (t + 1) >> 1, tq = (t + 3) >> 2, tpe = 4 * tq, hbb = hb_bytes(nv, nc);
    const int nitem = 8 * t * th;                               // A-tile items (corner, e, pair of e')
    const int G = NT_THREADS / tq, seg_off = rec_seg_off(G);
    const int cell = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char* Abuf = sm;                                   // [A_BYTES]
    unsigned char* Bbuf = sm + A_BYTES;                         // [2][B_BYTES]
    float2* Xb = reinterpret_cast<float2*>(Bbuf + 2 * B_BYTES); // [2][NT_RCAP][tpe]
    uint4* P = reinterpret_cast<uint4*>(Xb + 2 * (size_t)NT_RCAP * tpe);    // [npart][tq][4]
    int* recb = reinterpret_cast<int*>(P + (size_t)npart * tq * 4);         // [2][rec_max]
    unsigned char* hbuf = reinterpret_cast<unsigned char*>(recb + 2 * (size_t)rec_max);   // [2][hbb]
    int4* aidx = reinterpret_cast<int4*>(hbuf + 2 * hbb);       // [nitem] A-tile item tables
    int2* s_urow = reinterpret_cast<int2*>(aidx + nitem);       // [nunits]
    int2* s_urec = s_urow + nunits;                             // [nunits]
    int2* s_uinf = s_urec + nunits;                             // [nunits]
    float* hds = reinterpret_cast<float*>(s_uinf + nunits);     // [n_near]
    int* scell = reinterpret_cast<int*>(hds + n_near);          // [nslot][8] source cells
    const Int3 ci = unflat3(cell, n);
    for (int i = tid; i < n_near; i += NT_THREADS) hds[i] = hd[i];
    for (int i = tid; i < nunits; i += NT_THREADS) { s_urow[i] = urow[i]; s_urec[i] = urec[i]; s_uinf[i] = uinfo[i]; }
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
    // zero both operands once: padding rows / columns stay zero for the whole kernel
    for (int i = tid; i < (A_BYTES + 2 * B_BYTES) / 16; i += NT_THREADS)
        reinterpret_cast<uint4*>(sm)[i] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        bar_init(su32(&bar_b[0]), 1);
        bar_init(su32(&bar_b[1]), 1);
        bar_init(su32(&bar_mma), 1);
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
    const uint32_t tmem = tmem_sh;

    // staging map: a row is t float2, copied as t / 2 16-byte chunks (t even) or t 8-byte ones;
    // this thread copies rows my_r + k rpp (k < 4 covers NT_RCAP rows for every t <= 16)
    const bool even = (t & 1) == 0;
    const int cpr = even ? t / 2 : t, rpp = NT_THREADS / cpr, my_r = tid / cpr, my_c = tid - my_r * cpr;
    const int NG = nunits * nchains;
    int rc[4];                                                  // row codes of the next step to stage
    auto load_codes = [&](int g) {
        const int2 ur = s_urow[g / nchains];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int r = my_r + k * rpp;
            rc[k] = (my_r < rpp && r < ur.y) ? __ldg(rows + ur.x + r) : -1;
        }
    };
    auto prefetch = [&](int g) {
        const int u = g / nchains, ch = g - u * nchains, hf = g & 1;
        const int2 rr = s_urec[u], inf = s_uinf[u];
        const int s = inf.x;
        int* rb = recb + (size_t)hf * rec_max;
        for (int i = tid; i < (rr.y >> 2); i += NT_THREADS) cp_async16(rb + 4 * i, rec + rr.x + 4 * i);
        const float2* Xc = X + (size_t)ch * nk * 8 * t;
        float2* xb = Xb + (size_t)hf * NT_RCAP * tpe;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (rc[k] < 0) continue;
            const int r = my_r + k * rpp, js = rc[k] & 0xFFFF, l = rc[k] >> 16;
            const float2* src = Xc + (((size_t)scell[s * 8 + l] * Ndiv + js) * 8 + l) * t;
            if (even) cp_async16(xb + r * tpe + 2 * my_c, src + 2 * my_c);
            else cp_async8(xb + r * tpe + my_c, src + my_c);
        }
        if (ch == 0 && ((inf.y >> 16) & 1)) {                   // first unit of a slot: its head factors
            const Int3 so = unflat3(s, ns1);
            const int oa = so.a + smin, ob = so.b + smin, oc = so.c + smin;
            float2* hvS = reinterpret_cast<float2*>(hbuf + (inf.y & 1) * hbb);
            float2* hmS = hvS + 8 * nv * nv;
            float* hcS = reinterpret_cast<float*>(hmS + 8 * nc * nc);
            const int nvv = nv * nv, ncc = nc * nc, per = nvv + ncc + 1;
            for (int i = tid; i < 8 * per; i += NT_THREADS) {
                const int l = i / per, w = i - l * per;
                const int l1 = (l >> 2) & 1, l2 = (l >> 1) & 1, l3 = l & 1;
                const int kt = flat3(ci.a + l1, ci.b + l2, ci.c + l3, n);
                const int r = ((oa - l1 - rmin) * nr1 + (ob - l2 - rmin)) * nr1 + (oc - l3 - rmin);
                if (w < nvv) cp_async8(hvS + l * nvv + w, Hv + ((size_t)kt * nrel + r) * nvv + w);
                else if (w < nvv + ncc) cp_async8(hmS + l * ncc + (w - nvv), Hc + ((size_t)kt * nrel + r) * ncc + (w - nvv));
                else cp_async4(hcS + l, hc + r);
            }
        }
    };

    const int my_g = tid / tq, my_qd = tid - my_g * tq, par = my_g & 1;
    const int ca = my_qd + tq * par, cb = my_qd + tq * (1 - par);   // chunks read first / second (bank stagger)
    load_codes(0);
    prefetch(0);
    cp_async_commit();
    if (NG > 1) load_codes(1);
    for (int g = 0; g < NG; ++g) {
        const int u = g / nchains, ch = g - u * nchains, bb = g & 1;
        const int2 inf = s_uinf[u];
        const int ord = inf.y & 0xFFFF, first = (inf.y >> 16) & 1, last = (inf.y >> 17) & 1;
        if (g + 1 < NG) {
            prefetch(g + 1);
            if (g + 2 < NG) load_codes(g + 2);
        }
        cp_async_commit();
        cp_async_wait1();                                       // this thread's copies of step g landed
        if (tid == 0) {
            bool ok = true;
            // B buffer bb was read by the MMAs of step g - 2
            if (g >= 2) ok = bar_wait(su32(&bar_b[bb]), (uint32_t)(((g - 2) >> 1) & 1), status);
            // A is rewritten at a slot change: every MMA of the previous slot must be done
            if (ok && ch == 0 && first && ord > 0) ok = bar_wait(su32(&bar_mma), (uint32_t)((ord - 1) & 1), status);
            if (!ok) abort_flag = 1;
        }
        __syncthreads();
        if (abort_flag) break;
        if (ch == 0 && first) {
            // Ahat_s: item (l, e, pair of e') writes one 16-byte chunk to four rows
            const float2* hvS = reinterpret_cast<const float2*>(hbuf + (ord & 1) * hbb);
            const float2* hmS = hvS + 8 * nv * nv;
            const float* hcS = reinterpret_cast<const float*>(hmS + 8 * nc * nc);
            for (int it = tid; it < nitem; it += NT_THREADS) {
                const int4 ix = aidx[it];
                const float2 c0 = cmul(hvS[ix.x & 0xFFFF], hmS[ix.y & 0xFFFF]);
                float2 c1 = cmul(hvS[ix.x >> 16], hmS[ix.y >> 16]);
                if (!(ix.w >> 8)) c1 = make_float2(0.f, 0.f);
                const float mh = -hcS[ix.w & 0xFF];
                const int o0 = ix.z & 0xFFFF, o1 = (ix.z >> 16) & 0xFFFF;
                *reinterpret_cast<uint4*>(Abuf + o0) = pack_tf32(c0.x, -c0.y, c1.x, -c1.y);
                *reinterpret_cast<uint4*>(Abuf + o1) = pack_tf32(c0.y, c0.x, c1.y, c1.x);
                *reinterpret_cast<uint4*>(Abuf + A_KB + o0) = pack_tf32(mh * c0.x, -mh * c0.y, mh * c1.x, -mh * c1.y);
                *reinterpret_cast<uint4*>(Abuf + A_KB + o1) = pack_tf32(mh * c0.y, mh * c0.x, mh * c1.y, mh * c1.x);
            }
        }
        // y1, z of this chain by the unit's balanced schedule: group my_g runs its segments
        const int* rb = recb + (size_t)bb * rec_max;
        const int nseg = rb[2], nfix = rb[3];
        const int4* segs = reinterpret_cast<const int4*>(rb + seg_off);
        const int4* fixes = segs + nseg;
        const int* ent = reinterpret_cast<const int*>(fixes + nfix);
        const unsigned char* xa = reinterpret_cast<const unsigned char*>(Xb + (size_t)bb * NT_RCAP * tpe) + 16 * ca;
        const unsigned char* xbq = reinterpret_cast<const unsigned char*>(Xb + (size_t)bb * NT_RCAP * tpe) + 16 * cb;
        unsigned char* Bt = Bbuf + (size_t)bb * B_BYTES;
        if (my_g < G) {
            const int i1 = rb[4 + my_g + 1];
            for (int i = rb[4 + my_g]; i < i1; ++i) {
                const int4 sg = segs[i];
                uint64_t y[4] = {0, 0, 0, 0}, z[4] = {0, 0, 0, 0};
                int q = sg.x;
                for (; q + 2 <= sg.y; q += 2) {
                    const int ea = ent[q], eb = ent[q + 1];
                    const ulonglong2 a0 = *reinterpret_cast<const ulonglong2*>(xa + (ea & 0xFFFF));
                    const ulonglong2 a1 = *reinterpret_cast<const ulonglong2*>(xbq + (ea & 0xFFFF));
                    const ulonglong2 b0 = *reinterpret_cast<const ulonglong2*>(xa + (eb & 0xFFFF));
                    const ulonglong2 b1 = *reinterpret_cast<const ulonglong2*>(xbq + (eb & 0xFFFF));
                    const float ha = hds[ea >> 16], hb = hds[eb >> 16];
                    const uint64_t hha = pack2(ha, ha), hhb = pack2(hb, hb);
                    fma2(y[0], hha, a0.x); fma2(y[1], hha, a0.y); fma2(y[2], hha, a1.x); fma2(y[3], hha, a1.y);
                    add2(z[0], a0.x); add2(z[1], a0.y); add2(z[2], a1.x); add2(z[3], a1.y);
                    fma2(y[0], hhb, b0.x); fma2(y[1], hhb, b0.y); fma2(y[2], hhb, b1.x); fma2(y[3], hhb, b1.y);
                    add2(z[0], b0.x); add2(z[1], b0.y); add2(z[2], b1.x); add2(z[3], b1.y);
                }
                if (q < sg.y) {
                    const int ea = ent[q];
                    const ulonglong2 a0 = *reinterpret_cast<const ulonglong2*>(xa + (ea & 0xFFFF));
                    const ulonglong2 a1 = *reinterpret_cast<const ulonglong2*>(xbq + (ea & 0xFFFF));
                    const float ha = hds[ea >> 16];
                    const uint64_t hha = pack2(ha, ha);
                    fma2(y[0], hha, a0.x); fma2(y[1], hha, a0.y); fma2(y[2], hha, a1.x); fma2(y[3], hha, a1.y);
                    add2(z[0], a0.x); add2(z[1], a0.y); add2(z[2], a1.x); add2(z[3], a1.y);
                }
                if (par) {                                      // back to (chunk qd, chunk qd + tq) order
                    uint64_t tmp;
                    tmp = y[0]; y[0] = y[2]; y[2] = tmp; tmp = y[1]; y[1] = y[3]; y[3] = tmp;
                    tmp = z[0]; z[0] = z[2]; z[2] = tmp; tmp = z[1]; z[1] = z[3]; z[3] = tmp;
                }
                if (sg.w < 0) {
                    store_b_row(Bt, sg.z, my_qd, tq, t, y, z);
                } else {
                    uint4* pp = P + ((size_t)sg.w * tq + my_qd) * 4;
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        pp[k] = make_uint4((uint32_t)y[2 * k], (uint32_t)(y[2 * k] >> 32), (uint32_t)y[2 * k + 1],
                                           (uint32_t)(y[2 * k + 1] >> 32));
                        pp[2 + k] = make_uint4((uint32_t)z[2 * k], (uint32_t)(z[2 * k] >> 32), (uint32_t)z[2 * k + 1],
                                               (uint32_t)(z[2 * k + 1] >> 32));
                    }
                }
            }
        }
        if (nfix > 0) {
            __syncthreads();                                    // partials complete
            if (my_g < G) {
                for (int f = my_g; f < nfix; f += G) {
                    const int4 fx = fixes[f];
                    uint64_t y[4] = {0, 0, 0, 0}, z[4] = {0, 0, 0, 0};
                    for (int p = fx.y; p < fx.y + fx.z; ++p) {
                        const uint4* pp = P + ((size_t)p * tq + my_qd) * 4;
#pragma unroll
                        for (int k = 0; k < 2; ++k) {
                            const uint4 a = pp[k], b = pp[2 + k];
                            add2(y[2 * k], (uint64_t)a.x | ((uint64_t)a.y << 32));
                            add2(y[2 * k + 1], (uint64_t)a.z | ((uint64_t)a.w << 32));
                            add2(z[2 * k], (uint64_t)b.x | ((uint64_t)b.y << 32));
                            add2(z[2 * k + 1], (uint64_t)b.z | ((uint64_t)b.w << 32));
                        }
                    }
                    store_b_row(Bt, fx.x, my_qd, tq, t, y, z);
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();                                        // operands complete; staged buffers bb free again
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = su32(Abuf), b0 = su32(Bt);
#pragma unroll
            for (int mh = 0; mh < 2; ++mh) {
                const uint32_t d = tmem + (uint32_t)((ch * 2 + mh) * NT_N);
#pragma unroll
                for (int kb = 0; kb < 2; ++kb)
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        mma(d, desc_sw128(a0 + kb * A_KB + mh * (A_KB / 2) + kk * 32),
                            desc_sw128(b0 + kb * B_KB + kk * 32), (u == 0 && kb == 0 && kk == 0) ? 0u : 1u);
            }
            commit(su32(&bar_b[bb]));
            if (last && ch == nchains - 1) commit(su32(&bar_mma));
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
        // epilogue: 4 groups of 4 warps; group g reads accumulators c = g, g + 4, ... (c = 2 ch + mh)
        const int g = warp >> 2, q = warp & 3;
        for (int c = g; c < 2 * nchains; c += 4) {
            const int ch = c >> 1, mh = c & 1;
            const int row = mh * 128 + q * 32 + lane;
            float v[64];
            const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(c * NT_N);
            tmem_ld32(ta, v);
            tmem_ld32(ta + 32, v + 32);
            const int pair = row >> 1, ri = row & 1;
            const int l = pair / t, e = pair % t;
#pragma unroll
            for (int k = 0; k < NT_N; ++k) {
                const float other = __shfl_xor_sync(0xffffffffu, v[k], 1);
                if (ri == 0 && l < 8 && k < Ndiv && interp_active(k, l, nd, nb1))
                    U[(((size_t)ch * nk + (size_t)cell * Ndiv + k) * 8 + l) * t + e] = make_float2(v[k], other);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NT_TMEM_COLS));
}

}  // namespace

// Decide whether the tensor-core near field serves this handle (FP32 M3 with
// t <= 16 and N_div <= 64), build its unit records from the cell-batched lists
// (pairs: js | corner << 16; clist: pair index | near index << 16 in
// [N_div][nslot] order) and size its shared memory.
int bse_near_tc_prepare(bse_ctx* ctx, bse_interp* s, const std::vector<int>& pairs, const std::vector<int>& clist,
                        const std::vector<int>& cstart) {
    s->nf_tc = 0;
    if (s->vec_prec != BSE_PREC_F32 || s->t > 16 || s->Ndiv > NT_N || s->scheme != BSE_SCHEME_M3 || s->npairs >= 65536)
        return BSE_OK;                                          // not applicable: other kernels serve it
    const int Ndiv = s->Ndiv, nslot = s->nslot, t = s->t;
    const int th = (t + 1) / 2, tq = (t + 3) / 4, tpe = 4 * tq, G = NT_THREADS / tq, nitem = 8 * t * th;
    const int seg_off = rec_seg_off(G);
    int maxsm = 0;
    cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
    struct Unit { int slot, ord, first, last; std::vector<int> rows; std::vector<std::vector<int>> ent; };
    std::vector<Unit> units;
    std::vector<int> loc(pairs.size(), -1);
    int ord = 0;
    for (int sl = 0; sl < nslot; ++sl) {
        // contributions of the slot per target, and per source pair
        std::vector<std::vector<int>> per_j(Ndiv);
        std::vector<int> used, uses(pairs.size(), 0);
        for (int j = 0; j < Ndiv; ++j)
            for (int q = cstart[(size_t)j * (nslot + 1) + sl]; q < cstart[(size_t)j * (nslot + 1) + sl + 1]; ++q) {
                per_j[j].push_back(clist[q]);
                if (uses[clist[q] & 0xFFFF]++ == 0) used.push_back(clist[q] & 0xFFFF);
            }
        if (used.empty()) continue;                             // nothing of this slot reaches the cell
        std::sort(used.begin(), used.end());
        // cut the slot's source rows into units within the row and contribution caps
        const size_t u0 = units.size();
        size_t i = 0;
        while (i < used.size()) {
            Unit un;
            un.slot = sl; un.ord = ord; un.first = (units.size() == u0); un.last = 0;
            long long ecount = 0;
            while (i < used.size() && (int)un.rows.size() < NT_RCAP && (un.rows.empty() || ecount + uses[used[i]] <= NT_ECAP)) {
                loc[used[i]] = (int)un.rows.size();
                un.rows.push_back(used[i]);
                ecount += uses[used[i]];
                ++i;
            }
            un.ent.assign(Ndiv, {});
            for (int j = 0; j < Ndiv; ++j)
                for (int e : per_j[j]) {
                    const int p = e & 0xFFFF;
                    if (loc[p] >= 0 && loc[p] < (int)un.rows.size() && un.rows[loc[p]] == p)
                        un.ent[j].push_back((loc[p] * tpe * 8) | (e & ~0xFFFF));
                }
            units.push_back(std::move(un));
        }
        units.back().last = 1;
        ++ord;
    }
    if (units.empty() || (size_t)NT_RCAP * tpe * 8 >= 65536) return BSE_OK;
    // records: the schedule of each unit
    std::vector<int> rec, rows;
    std::vector<int2> urow, urec, uinfo;
    int rec_max = 0, npart_max = 0;
    const size_t fixed_wo_rec = 1024 + A_BYTES + 2 * (size_t)B_BYTES + 2 * sizeof(float2) * (size_t)NT_RCAP * tpe +
                                2 * (size_t)hb_bytes(s->nv, s->nc) + 16 * (size_t)nitem + 24 * units.size() +
                                sizeof(float) * (size_t)s->n_near + sizeof(int) * 8 * (size_t)nslot;
    // room for partials, assuming records up to the caps
    const size_t rec_cap_bytes = 4 * ((size_t)seg_off + 4 * (G + Ndiv) + 4 * Ndiv + NT_ECAP + 4);
    if (fixed_wo_rec + 2 * rec_cap_bytes + 64 * (size_t)tq > (size_t)maxsm) return BSE_OK;
    const int npart_cap = (int)(((size_t)maxsm - fixed_wo_rec - 2 * rec_cap_bytes) / (64 * (size_t)tq));
    for (const Unit& un : units) {
        std::vector<int> q0(Ndiv), cnt(Ndiv), ent;
        long long total = 0;
        for (int j = 0; j < Ndiv; ++j) {
            q0[j] = (int)ent.size();
            ent.insert(ent.end(), un.ent[j].begin(), un.ent[j].end());
            cnt[j] = (int)un.ent[j].size();
            total += cnt[j];
        }
        // segment length E: search upward from an equal share per group for the
        // schedule of least estimated time (entries + 2 per segment on the busiest
        // group, plus the fix-up pass when targets are split), within the partials' room
        auto build = [&](long long E, std::vector<int4>& out, int& np, long long& cost) -> bool {
            out.clear();
            np = 0;
            int max_ns = 0;
            for (int j = 0; j < Ndiv; ++j) {
                const int ns = cnt[j] == 0 ? 1 : (int)((cnt[j] + E - 1) / E);
                if (ns == 1) {
                    out.push_back(make_int4(q0[j], q0[j] + cnt[j], j, -1));
                } else {
                    for (int k = 0; k < ns; ++k) {
                        const int a = q0[j] + (int)((long long)cnt[j] * k / ns), b = q0[j] + (int)((long long)cnt[j] * (k + 1) / ns);
                        out.push_back(make_int4(a, b, j, np + k));
                    }
                    np += ns;
                    max_ns = std::max(max_ns, ns);
                }
            }
            if (np > npart_cap) return false;
            std::vector<int> lens(out.size());
            for (size_t i = 0; i < out.size(); ++i) lens[i] = out[i].y - out[i].x;
            std::sort(lens.begin(), lens.end(), std::greater<int>());
            std::vector<long long> load(G, 0);
            for (int L : lens) {
                int best = 0;
                for (int g = 1; g < G; ++g)
                    if (load[g] < load[best]) best = g;
                load[best] += L + 2;
            }
            cost = *std::max_element(load.begin(), load.end()) + (np ? 8 + 2 * max_ns : 0);
            return true;
        };
        std::vector<int4> segs, trial;
        int npart = 0;
        {
            long long best_cost = -1, bestE = 0;
            const int maxc = std::max(1, *std::max_element(cnt.begin(), cnt.end()));
            for (long long E = std::max<long long>(1, (total + G - 1) / G);; E += std::max<long long>(1, E / 4)) {
                int np;
                long long cost;
                if (build(E, trial, np, cost) && (best_cost < 0 || cost < best_cost)) { best_cost = cost; bestE = E; }
                if (E >= maxc) break;
            }
            long long cost;
            build(bestE, segs, npart, cost);                    // E = max count always fits: no partials
        }
        npart_max = std::max(npart_max, npart);
        std::vector<int4> fixes;                                // split targets: consecutive partials
        for (size_t i = 0; i < segs.size();) {
            size_t k = i;
            while (k < segs.size() && segs[k].z == segs[i].z) ++k;
            if (segs[i].w >= 0) fixes.push_back(make_int4(segs[i].z, segs[i].w, (int)(k - i), 0));
            i = k;
        }
        // longest first onto the least-loaded group (the same cost model)
        std::vector<int> order(segs.size());
        for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
        std::stable_sort(order.begin(), order.end(),
                         [&](int a, int b) { return segs[a].y - segs[a].x > segs[b].y - segs[b].x; });
        std::vector<long long> load(G, 0);
        std::vector<std::vector<int>> gl(G);
        for (int i : order) {
            int best = 0;
            for (int g = 1; g < G; ++g)
                if (load[g] < load[best]) best = g;
            load[best] += segs[i].y - segs[i].x + 2;
            gl[best].push_back(i);
        }
        // the record
        const size_t base = rec.size();
        rec.resize(base + seg_off, 0);
        rec[base + 0] = (int)un.rows.size();
        rec[base + 1] = (int)total;
        rec[base + 2] = (int)segs.size();
        rec[base + 3] = (int)fixes.size();
        int sidx = 0;
        for (int g = 0; g < G; ++g) {
            rec[base + 4 + g] = sidx;
            for (int i : gl[g]) {
                rec.push_back(segs[i].x); rec.push_back(segs[i].y); rec.push_back(segs[i].z); rec.push_back(segs[i].w);
                ++sidx;
            }
        }
        rec[base + 4 + G] = sidx;
        for (const int4& f : fixes) { rec.push_back(f.x); rec.push_back(f.y); rec.push_back(f.z); rec.push_back(f.w); }
        rec.insert(rec.end(), ent.begin(), ent.end());
        while (rec.size() % 4) rec.push_back(0);
        const int len = (int)(rec.size() - base);
        rec_max = std::max(rec_max, len);
        urec.push_back(make_int2((int)base, len));
        urow.push_back(make_int2((int)rows.size(), (int)un.rows.size()));
        for (int p : un.rows) rows.push_back(pairs[p]);
        uinfo.push_back(make_int2(un.slot, un.ord | (un.first << 16) | (un.last << 17)));
    }
    const size_t smem = fixed_wo_rec + 2 * sizeof(int) * (size_t)rec_max + 64 * (size_t)tq * std::max(npart_max, 1);
    if (smem > (size_t)maxsm) return BSE_OK;
    auto upload = [&](void** dst, const void* src, size_t bytes, const char* what) -> int {
        int rc = bse_alloc(ctx, dst, bytes, what);
        if (rc != BSE_OK) return rc;
        BSE_CUDA_TRY(ctx, cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
        return BSE_OK;
    };
    int rc;
    if ((rc = upload((void**)&s->d_tc_rows, rows.data(), sizeof(int) * rows.size(), "near rows")) != BSE_OK) return rc;
    if ((rc = upload((void**)&s->d_tc_urow, urow.data(), sizeof(int2) * urow.size(), "near unit rows")) != BSE_OK) return rc;
    if ((rc = upload((void**)&s->d_tc_rec, rec.data(), sizeof(int) * rec.size(), "near unit records")) != BSE_OK) return rc;
    if ((rc = upload((void**)&s->d_tc_urec, urec.data(), sizeof(int2) * urec.size(), "near record index")) != BSE_OK) return rc;
    if ((rc = upload((void**)&s->d_tc_uinfo, uinfo.data(), sizeof(int2) * uinfo.size(), "near unit info")) != BSE_OK) return rc;
    s->nf_tc_units = (int)units.size();
    s->nf_tc_rec_max = rec_max;
    s->nf_tc_npart = std::max(npart_max, 1);
    s->nf_tc_smem = smem;
    s->nf_tc = 1;
    return BSE_OK;
}

int bse_near_tc_launch(bse_ctx* ctx, const bse_interp* s, int nchains, const void* X, void* U) {
    // handles of different sizes share the kernel's attribute: only ever raise it
    cudaFuncAttributes fa;
    BSE_CUDA_TRY(ctx, cudaFuncGetAttributes(&fa, k_near_tc));
    if ((size_t)fa.maxDynamicSharedSizeBytes < s->nf_tc_smem)
        BSE_CUDA_TRY(ctx, cudaFuncSetAttribute(k_near_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s->nf_tc_smem));
    k_near_tc<<<s->co->nkc, NT_THREADS, s->nf_tc_smem, ctx->stream>>>(
        (const float2*)X, s->d_tc_rows, s->d_tc_urow, s->d_tc_rec, s->d_tc_urec, s->d_tc_uinfo, s->nf_tc_units,
        (const float*)s->d_hd, s->n_near, (const float2*)s->d_Hv, (const float2*)s->d_Hc, (const float*)s->d_hc, s->n,
        s->nd, s->nv, s->nc, s->nb1, s->smin, s->ns1, s->rmin, s->nr1, nchains, s->nf_tc_rec_max, s->nf_tc_npart,
        (float2*)U, ctx->d_status);
    return BSE_OK;
}
