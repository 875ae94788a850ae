// bse_apply_h_noalloc: one application of the interpolated H that allocates no
// device memory.
//
// Who needs it: callers that must not call cudaMalloc during their work, for
// example a host framework that owns all device memory through its own pool
// (a cudaMalloc behind its back can fail or fragment it), or a real-time
// loop in which cudaMalloc's implicit device-wide synchronisation is not
// allowed.  bse_apply_h takes its per-call scratch from the handle, which
// bse_interp_setup allocated; this variant takes it from the file-scope
// array below instead, so after set-up nothing is allocated on any path.
//
// The array is a static __device__ object of the library's device module: a
// device holds BSE_NOALLOC_SCRATCH_BYTES of it from the moment that module is
// loaded on it until the process exits.  With CUDA's lazy module loading the
// module loads on first use, and that load allocates; so bse_ctx_create calls
// bse_noalloc_prepare, which looks up the array's device address
// (cudaGetSymbolAddress, which loads the module) once per device, with that
// device current, at set-up.  In host code the array's name is only a
// host-side stand-in for the device object; the address found here is what
// the kernels get.  Create the context before any stream capture.
// Every call shares the one array, which keeps the previous call's contents:
// the buffers that must start at zero are cleared on each call, and calls
// that overlap on the GPU (two streams, or two host threads) race on it.
#include <mutex>

#include "bse_internal.cuh"

#define BSE_NOALLOC_SCRATCH_BYTES (32u << 20)   // 32 MiB
#define BSE_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) unsigned char g_noalloc_scratch[BSE_NOALLOC_SCRATCH_BYTES];

namespace {

void* g_scratch_addr[BSE_NOALLOC_MAX_DEVICES] = {};
std::mutex g_scratch_mu;

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

int bse_noalloc_prepare(bse_ctx* ctx) {
    if (ctx->device < 0 || ctx->device >= BSE_NOALLOC_MAX_DEVICES) return BSE_OK;   // the entry point refuses it
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (g_scratch_addr[ctx->device]) return BSE_OK;
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        ctx->err = std::string("cudaGetSymbolAddress of the static scratch failed: ") + cudaGetErrorString(e);
        return BSE_ERR_CUDA;
    }
    g_scratch_addr[ctx->device] = p;
    return BSE_OK;
}

extern "C" int bse_apply_h_noalloc(bse_ctx* ctx, bse_interp* s, int nvec, const void* x, void* y) {
    if (!ctx || !s || !x || !y) return BSE_ERR_ARG;
    if (nvec < 1 || nvec > BSE_MAX_CHAINS) {
        ctx->err = "nvec must be in 1..4";
        return BSE_ERR_ARG;
    }
    if (ctx->device < 0 || ctx->device >= BSE_NOALLOC_MAX_DEVICES) {
        ctx->err = "device index above the no-allocation table";
        return BSE_ERR_UNSUPPORTED;
    }
    if (s->learned) {
        ctx->err = "the learned correction is not available without allocation (use bse_apply_h)";
        return BSE_ERR_UNSUPPORTED;
    }
    if (cudaSetDevice(ctx->device) != cudaSuccess) return BSE_ERR_CUDA;
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        base = g_scratch_addr[ctx->device];           // looked up by bse_ctx_create
    }
    if (!base) {
        ctx->err = "the static scratch of this device was not set up (bse_ctx_create)";
        return BSE_ERR_CUDA;
    }
    // Carve the per-call buffers (each 256-byte aligned) out of the array.
    const bse_coarse* c = s->co;
    const size_t vsz = (s->vec_prec == BSE_PREC_F64) ? sizeof(double2) : sizeof(float2);
    const bool m3 = s->scheme == BSE_SCHEME_M3;
    const bool bf16 = c->kc_prec == BSE_PREC_BF16;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += align256(bytes);
        return o;
    };
    const size_t oQ = take(vsz * nvec * c->Nc);
    const size_t oR = take(vsz * nvec * c->Nc);
    const size_t oX = m3 ? take(vsz * nvec * (size_t)s->nk * 8 * s->t) : 0;
    const size_t oU = m3 ? take(vsz * nvec * (size_t)s->nk * 8 * s->t) : 0;
    const size_t oD = take(sizeof(double2) * nvec * BSE_MAX_VEC_BLOCKS);
    const size_t oB = bf16 ? take(sizeof(__nv_bfloat16) * 16 * (size_t)c->ldk) : 0;
    const size_t oP = bf16 ? take(bse_tc_part_bytes(s)) : 0;
    if (off > BSE_NOALLOC_SCRATCH_BYTES) {
        ctx->err = "bse_apply_h_noalloc needs " + std::to_string(off) + " bytes of scratch; the static array holds " +
                   std::to_string((size_t)BSE_NOALLOC_SCRATCH_BYTES) + " (use bse_apply_h)";
        return BSE_ERR_UNSUPPORTED;
    }
    unsigned char* b = static_cast<unsigned char*>(base);
    ApplyScratch sc;
    sc.Q = b + oQ;
    sc.R = b + oR;
    sc.X = m3 ? b + oX : nullptr;
    sc.U = m3 ? b + oU : nullptr;
    sc.dot = reinterpret_cast<double2*>(b + oD);
    sc.bop = bf16 ? reinterpret_cast<__nv_bfloat16*>(b + oB) : nullptr;
    sc.part = bf16 ? reinterpret_cast<float*>(b + oP) : nullptr;
    int rc = bse_apply_scratch(ctx, s, nvec, x, y, sc);
    if (rc != BSE_OK) return rc;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        ctx->err = std::string("apply H (no allocation): ") + cudaGetErrorString(e);
        return BSE_ERR_CUDA;
    }
    int status = 0;
    BSE_CUDA_TRY(ctx, cudaMemcpy(&status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (status) {
        cudaMemset(ctx->d_status, 0, sizeof(int));
        ctx->err = bse_timeout_message(status);
        return BSE_ERR_TIMEOUT;
    }
    return BSE_OK;
}
