// extern "C" entry points of the library (see include/bse.h for the contract).
#include <cmath>
#include <cstring>
#include <atomic>
#include <new>

#include "bse_internal.cuh"

namespace {

bool finite_arr(const double* p, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

int set_arg_error(bse_ctx* ctx, const char* msg) {
    if (ctx) ctx->err = msg;
    return BSE_ERR_ARG;
}

template <typename P>
int upload(bse_ctx* ctx, P** dst, const double* src, size_t ndouble, const char* what) {
    int rc = bse_alloc(ctx, (void**)dst, sizeof(double) * ndouble, what);
    if (rc != BSE_OK) return rc;
    BSE_CUDA_TRY(ctx, cudaMemcpy(*dst, src, sizeof(double) * ndouble, cudaMemcpyHostToDevice));
    return BSE_OK;
}

void free_coarse(bse_coarse* c) {
    if (!c) return;
    cudaFree(c->d_offsets); cudaFree(c->d_gen_v); cudaFree(c->d_gen_c); cudaFree(c->d_mu);
    cudaFree(c->d_dip); cudaFree(c->d_Uv); cudaFree(c->d_Uc); cudaFree(c->d_kc);
    delete c;
}

void free_interp(bse_interp* s) {
    if (!s) return;
    bse_release_run_state(s);
    void* ptrs[] = {s->d_dE, s->d_Dv, s->d_Dc, s->d_P, s->d_list, s->d_list_start, s->d_hd, s->d_Hv, s->d_Hc,
                    s->d_hc, s->d_Q, s->d_R, s->d_X, s->d_U, s->d_Bop, s->d_part, s->d_vec[0],
                    s->d_vec[1], s->d_vec[2], s->d_part_dot, s->d_part_nrm, s->d_a, s->d_aim, s->d_b, s->d_stop,
                    s->d_basis, s->d_cgs_part, s->d_cgs_h, s->d_pairs, s->d_clist, s->d_cstart,
                    s->d_lker, s->d_lgrid, s->d_tw_fwd, s->d_tc_rows, s->d_tc_slots,
                    s->d_tc_kinfo, s->d_tc_simg, s->d_tc_aimg, s->d_xscale, s->d_xscale_gen, s->d_H2};
    for (void* p : ptrs) cudaFree(p);
    bse_tc_release(s);
    delete s;
}

}  // namespace

long long bse_next_serial() {
    static std::atomic<long long> counter{0};
    return ++counter;
}

extern "C" {

int bse_version(void) { return 10100; }

int bse_ctx_create(bse_ctx** out, int device, void* cuda_stream) {
    if (!out) return BSE_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return BSE_ERR_CUDA;
    }
    if (device < 0 || device >= ndev) return BSE_ERR_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return BSE_ERR_CUDA;
    bse_ctx* ctx = new (std::nothrow) bse_ctx();
    if (!ctx) return BSE_ERR_OOM;
    ctx->device = device;
    ctx->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    if (!ctx->stream) {
        // A stream of our own (blocking: ordered with the legacy default stream),
        // so that the step loop can be captured in a CUDA graph.
        if (cudaStreamCreate(&ctx->stream) != cudaSuccess) {
            delete ctx;
            return BSE_ERR_CUDA;
        }
        ctx->own_stream = true;
    }
    cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (bse_alloc(ctx, (void**)&ctx->d_status, sizeof(int), "status word") != BSE_OK) {
        delete ctx;
        return BSE_ERR_OOM;
    }
    cudaMemset(ctx->d_status, 0, sizeof(int));
    ctx->serial = bse_next_serial();
    // Load the library's device module and look up the no-allocation scratch
    // here, at set-up, so that bse_apply_h_noalloc never triggers the lazy
    // module load (and its allocation) itself.
    if (bse_noalloc_prepare(ctx) != BSE_OK || bse_prepare_aux(ctx) != BSE_OK) {
        bse_release_ctx_state(ctx);
        cudaFree(ctx->d_status);
        if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
        delete ctx;
        return BSE_ERR_CUDA;
    }
    *out = ctx;
    return BSE_OK;
}

void bse_ctx_destroy(bse_ctx* ctx) {
    if (!ctx) return;
    bse_release_ctx_state(ctx);
    cudaFree(ctx->d_status);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

const char* bse_last_error(const bse_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int bse_build_coarse(bse_ctx* ctx, const bse_model* m, int n_coarse, int kc_prec, const void* user_kc,
                     bse_coarse** out) {
    if (!ctx || !out) return BSE_ERR_ARG;
    *out = nullptr;
    if (!m) return set_arg_error(ctx, "model is NULL");
    if (m->nv < 1 || m->nv > BSE_MAX_BANDS || m->nc < 1 || m->nc > BSE_MAX_BANDS)
        return set_arg_error(ctx, "nv and nc must be in 1..8");
    if (n_coarse < 1 || n_coarse > 64) return set_arg_error(ctx, "n_coarse must be in 1..64");
    if (kc_prec != BSE_PREC_F64 && kc_prec != BSE_PREC_F32 && kc_prec != BSE_PREC_BF16)
        return set_arg_error(ctx, "unknown K_c precision");
    if (m->direct_shells != 27 && m->direct_shells != 1) return set_arg_error(ctx, "direct_shells must be 27 or 1");
    const double sc[] = {m->eps_inf, m->kappa, m->e_k, m->e_gap, m->band_width, m->h0};
    if (!finite_arr(sc, 6) || m->eps_inf == 0.0) return set_arg_error(ctx, "non-finite model constant or eps_inf = 0");
    if (!m->offsets || !m->gen_v || !m->gen_c || !m->mu || !m->dip) return set_arg_error(ctx, "model array is NULL");
    const int nv = m->nv, nc = m->nc;
    if (!finite_arr(m->offsets, nv * nc) || !finite_arr(m->gen_v, 12 * nv * nv) || !finite_arr(m->gen_c, 12 * nc * nc) ||
        !finite_arr(m->mu, 2 * 7 * 26 * nv * nc) || !finite_arr(m->dip, 2 * 7 * 3 * nv * nc))
        return set_arg_error(ctx, "non-finite model array entry");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return BSE_ERR_CUDA;
    bse_coarse* c = new (std::nothrow) bse_coarse();
    if (!c) return BSE_ERR_OOM;
    c->n = n_coarse; c->nv = nv; c->nc = nc; c->t = nv * nc;
    c->nkc = n_coarse * n_coarse * n_coarse;
    const long long Nc = (long long)c->t * c->nkc;
    if (Nc > (1 << 20)) { free_coarse(c); ctx->err = "coarse dimension above 2^20"; return BSE_ERR_UNSUPPORTED; }
    c->Nc = (int)Nc;
    c->kc_prec = kc_prec;
    c->ldk = (int)((Nc + 63) / 64 * 64);
    c->eps_inf = m->eps_inf; c->kappa = m->kappa; c->e_k = m->e_k; c->e_gap = m->e_gap;
    c->band_width = m->band_width; c->h0 = m->h0; c->direct_shells = m->direct_shells;
    c->h_const = m->h_const ? 1 : 0; c->exchange_on = m->exchange_on ? 1 : 0;
    c->alpha = -(m->e_k / c->nkc) * 4.0 * 3.14159265358979323846 / m->eps_inf;
    int rc;
    if ((rc = upload(ctx, &c->d_offsets, m->offsets, nv * nc, "offsets")) != BSE_OK ||
        (rc = upload(ctx, &c->d_gen_v, m->gen_v, 12 * nv * nv, "gen_v")) != BSE_OK ||
        (rc = upload(ctx, &c->d_gen_c, m->gen_c, 12 * nc * nc, "gen_c")) != BSE_OK ||
        (rc = upload(ctx, &c->d_mu, m->mu, 2 * 7 * 26 * nv * nc, "mu")) != BSE_OK ||
        (rc = upload(ctx, &c->d_dip, m->dip, 2 * 7 * 3 * nv * nc, "dip")) != BSE_OK ||
        (rc = bse_setup_coarse_device(ctx, c, user_kc)) != BSE_OK) {
        free_coarse(c);
        return rc;
    }
    *out = c;
    return BSE_OK;
}

int bse_coarse_get_kc(bse_ctx* ctx, const bse_coarse* c, double* host_kc) {
    if (!ctx || !c || !host_kc) return BSE_ERR_ARG;
    const size_t Nc = c->Nc;
    if (c->kc_prec == BSE_PREC_F64) {
        BSE_CUDA_TRY(ctx, cudaMemcpy(host_kc, c->d_kc, sizeof(double2) * Nc * Nc, cudaMemcpyDeviceToHost));
        return BSE_OK;
    }
    if (c->kc_prec == BSE_PREC_F32) {
        std::vector<float2> tmp(Nc * Nc);
        BSE_CUDA_TRY(ctx, cudaMemcpy(tmp.data(), c->d_kc, sizeof(float2) * Nc * Nc, cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < Nc * Nc; ++i) { host_kc[2 * i] = tmp[i].x; host_kc[2 * i + 1] = tmp[i].y; }
        return BSE_OK;
    }
    std::vector<__nv_bfloat16> re(Nc * c->ldk), im(Nc * c->ldk);
    BSE_CUDA_TRY(ctx, cudaMemcpy(re.data(), c->d_kr, sizeof(__nv_bfloat16) * Nc * c->ldk, cudaMemcpyDeviceToHost));
    BSE_CUDA_TRY(ctx, cudaMemcpy(im.data(), c->d_ki, sizeof(__nv_bfloat16) * Nc * c->ldk, cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < Nc; ++i)
        for (size_t j = 0; j < Nc; ++j) {
            host_kc[2 * (i * Nc + j)] = (double)__bfloat162float(re[i * c->ldk + j]);
            host_kc[2 * (i * Nc + j) + 1] = (double)__bfloat162float(im[i * c->ldk + j]);
        }
    return BSE_OK;
}

void bse_free_coarse(bse_coarse* c) { free_coarse(c); }

int bse_interp_setup(bse_ctx* ctx, const bse_coarse* c, int n_div, int scheme, double width_w, int vec_prec,
                     const bse_dense_inputs* dense, bse_interp** out) {
    if (!ctx || !out) return BSE_ERR_ARG;
    *out = nullptr;
    if (!c) return set_arg_error(ctx, "coarse handle is NULL");
    if (n_div < 1 || n_div > 16) return set_arg_error(ctx, "n_div must be in 1..16");
    const int base = scheme & ~(BSE_NB1 | BSE_NF_CUDA_CORES);
    if (base != BSE_SCHEME_M1 && base != BSE_SCHEME_M2 && base != BSE_SCHEME_M3) return set_arg_error(ctx, "unknown scheme");
    if (vec_prec != BSE_PREC_F64 && vec_prec != BSE_PREC_F32) return set_arg_error(ctx, "vec_prec must be F64 or F32");
    if ((c->kc_prec == BSE_PREC_F64) != (vec_prec == BSE_PREC_F64)) {
        ctx->err = "supported (K_c, vector) precisions: (F64, F64), (F32, F32), (BF16, F32)";
        return BSE_ERR_UNSUPPORTED;
    }
    if (base == BSE_SCHEME_M3) {
        if (!std::isfinite(width_w) || width_w < 0.0 || 2.0 * width_w >= (double)c->n)
            return set_arg_error(ctx, "M3 width must satisfy 0 <= w < n/2 (near region inside half the zone)");
        if (c->h_const) return set_arg_error(ctx, "M3 needs the Yukawa direct term (h_const = 0)");
    }
    if (base == BSE_SCHEME_M2) {
        if (c->h_const) return set_arg_error(ctx, "M2 needs the Yukawa direct term (h_const = 0)");
        if (c->kc_prec != BSE_PREC_F64 || vec_prec != BSE_PREC_F64) {
            ctx->err = "M2 (stored dense H) is built for complex128 K_c and vectors";
            return BSE_ERR_UNSUPPORTED;
        }
        const long long Nd = (long long)c->nkc * n_div * n_div * n_div * c->t;
        if (Nd > 16384) {
            ctx->err = "M2 stores the dense H: N must be <= 16384";
            return BSE_ERR_UNSUPPORTED;
        }
    }
    const long long nk = (long long)c->nkc * n_div * n_div * n_div;
    if (nk * c->t > (1LL << 31) - 1) { ctx->err = "dense dimension above 2^31"; return BSE_ERR_UNSUPPORTED; }
    if (dense) {
        const size_t N = (size_t)nk * c->t;
        if ((dense->dE && !finite_arr(dense->dE, N)) || (dense->P && !finite_arr(dense->P, 6 * N)) ||
            (dense->Dv && !finite_arr(dense->Dv, 16 * (size_t)nk * c->nv * c->nv)) ||
            (dense->Dc && !finite_arr(dense->Dc, 16 * (size_t)nk * c->nc * c->nc)))
            return set_arg_error(ctx, "non-finite entry in the dense inputs");
    }
    if (cudaSetDevice(ctx->device) != cudaSuccess) return BSE_ERR_CUDA;
    bse_interp* s = new (std::nothrow) bse_interp();
    if (!s) return BSE_ERR_OOM;
    s->co = c; s->n = c->n; s->nd = n_div; s->Ndiv = n_div * n_div * n_div; s->nk = (int)nk;
    s->nv = c->nv; s->nc = c->nc; s->t = c->t; s->N = (int)(nk * c->t);
    s->scheme = base; s->nb1 = (scheme & BSE_NB1) ? 1 : 0; s->vec_prec = vec_prec; s->width = width_w;
    s->nf_force_cuda_cores = (scheme & BSE_NF_CUDA_CORES) ? 1 : 0;
    s->serial = bse_next_serial();
    int rc = bse_setup_interp_device(ctx, s, dense);
    if (rc != BSE_OK) { free_interp(s); return rc; }
    *out = s;
    return BSE_OK;
}

void bse_free_interp(bse_interp* s) { free_interp(s); }

int bse_interp_info(const bse_interp* s, long long* info) {
    if (!s || !info) return BSE_ERR_ARG;
    info[0] = s->N; info[1] = s->nk; info[2] = s->co->Nc; info[3] = s->t;
    info[4] = s->n; info[5] = s->nd; info[6] = s->n_near; info[7] = s->vec_prec;
    return BSE_OK;
}

int bse_interp_kc_plan(const bse_interp* s, int* plan) {
    if (!s || !plan) return BSE_ERR_ARG;
    if (!s->tc_state) return BSE_ERR_UNSUPPORTED;
    plan[0] = s->tc_stages; plan[1] = s->tc_kblocks; plan[2] = s->tc_ctas;
    return BSE_OK;
}

int bse_dipoles(bse_ctx* ctx, bse_interp* s, int npol, const double* pol_dirs, void* p_out, double* pnorm2) {
    if (!ctx || !s || !pol_dirs || !p_out || !pnorm2) return BSE_ERR_ARG;
    if (npol < 1 || npol > BSE_MAX_CHAINS) return set_arg_error(ctx, "npol must be in 1..4");
    if (!finite_arr(pol_dirs, 3 * npol)) return set_arg_error(ctx, "non-finite direction");
    return bse_make_dipoles(ctx, s, npol, pol_dirs, p_out, pnorm2);
}

int bse_apply_h(bse_ctx* ctx, bse_interp* s, int nvec, const void* x, void* y) {
    if (!ctx || !s || !x || !y) return BSE_ERR_ARG;
    if (nvec < 1 || nvec > BSE_MAX_CHAINS) return set_arg_error(ctx, "nvec must be in 1..4");
    return bse_apply_once(ctx, s, nvec, x, y, false);
}

int bse_haydock_run(bse_ctx* ctx, bse_interp* const* sys, int nsys, const int* npol, const double* pol_dirs,
                    int nsteps, int flags, double* a, double* b, double* pnorm2, int* steps_done) {
    if (!ctx || !sys || !npol || !pol_dirs || !a || !b || !pnorm2 || !steps_done) return BSE_ERR_ARG;
    if (nsys < 1) return set_arg_error(ctx, "nsys must be >= 1");
    if (nsteps < 1 || nsteps > 100000) return set_arg_error(ctx, "nsteps must be in 1..100000");
    if (flags & ~(BSE_REORTH_CGS2 | BSE_USE_GRAPH | BSE_PROFILE | BSE_STOP_CONVERGED))
        return set_arg_error(ctx, "unknown flag");
    if ((flags & BSE_STOP_CONVERGED) && !ctx->stop_set)
        return set_arg_error(ctx, "BSE_STOP_CONVERGED needs a rule (bse_set_stop_rule)");
    int total = 0;
    for (int i = 0; i < nsys; ++i) {
        if (!sys[i]) return set_arg_error(ctx, "system handle is NULL");
        if (npol[i] < 1 || npol[i] > BSE_MAX_CHAINS) return set_arg_error(ctx, "npol must be in 1..4");
        total += npol[i];
    }
    if (!finite_arr(pol_dirs, 3 * (size_t)total)) return set_arg_error(ctx, "non-finite direction");
    for (int i = 0; i < nsys; ++i)
        for (int j = 0; j < i; ++j)
            if (sys[i] == sys[j]) return set_arg_error(ctx, "a system handle appears twice (each owns its scratch)");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return BSE_ERR_CUDA;
    if (nsys > 1 && (flags & BSE_USE_GRAPH) && !(flags & BSE_PROFILE))
        return bse_run_batch(ctx, sys, nsys, npol, pol_dirs, nsteps, flags, a, b, pnorm2, steps_done);
    int worst = BSE_OK, off = 0;
    for (int i = 0; i < nsys; ++i) {
        int rc = bse_run_chains(ctx, sys[i], npol[i], pol_dirs + 3 * off, nsteps, flags, a + (size_t)off * nsteps,
                                b + (size_t)off * (nsteps + 1), pnorm2 + off, steps_done + off);
        if (rc < 0) return rc;
        if (rc > 0) worst = rc;
        off += npol[i];
    }
    return worst;
}

int bse_set_stop_rule(bse_ctx* ctx, double tol, int check_every, double s_eps, double eta, int nw,
                      const double* omega) {
    if (!ctx || !omega) return BSE_ERR_ARG;
    const double sc[] = {tol, s_eps, eta};
    if (!finite_arr(sc, 3) || tol <= 0.0 || eta <= 0.0 || check_every < 1 || nw < 1 || !finite_arr(omega, nw))
        return set_arg_error(ctx, "stop rule needs tol > 0, check_every >= 1, eta > 0, nw >= 1, finite numbers");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return BSE_ERR_CUDA;
    if (nw > ctx->stop_nw) {
        cudaFree(ctx->d_stop_omega);
        ctx->d_stop_omega = nullptr;
        ctx->stop_nw = 0;
        int rc = bse_alloc(ctx, (void**)&ctx->d_stop_omega, sizeof(double) * nw, "stop-rule frequencies");
        if (rc != BSE_OK) return rc;
    }
    BSE_CUDA_TRY(ctx, cudaMemcpy(ctx->d_stop_omega, omega, sizeof(double) * nw, cudaMemcpyHostToDevice));
    ctx->stop_nw = nw;
    ctx->stop_tol = tol;
    ctx->stop_every = check_every;
    ctx->stop_seps = s_eps;
    ctx->stop_eta = eta;
    ctx->stop_set = 1;
    return BSE_OK;
}

int bse_ctx_set_wait_limit(bse_ctx* ctx, long long cycles) {
    if (!ctx) return BSE_ERR_ARG;
    if (cycles < 0) return set_arg_error(ctx, "wait limit must be >= 0 (0: default)");
    ctx->wait_cycles = cycles;
    return BSE_OK;
}

int bse_last_kernel_times(const bse_ctx* ctx, double* ms, long long* counts) {
    if (!ctx || !ms || !counts) return BSE_ERR_ARG;
    for (int k = 0; k < KC_COUNT; ++k) {
        counts[k] = ctx->kt_n[k];
        ms[k] = ctx->kt_n[k] ? ctx->kt_ms[k] / ctx->kt_n[k] : 0.0;
    }
    return BSE_OK;
}

int bse_spectrum(bse_ctx* ctx, int nchains, int nsteps, const int* steps_done, const double* a, const double* b,
                 const double* pnorm2, double prefactor, double eta, int nw, const double* omega, double* eps) {
    if (!ctx || !steps_done || !a || !b || !pnorm2 || !omega || !eps) return BSE_ERR_ARG;
    if (nchains < 1 || nsteps < 1 || nw < 1) return set_arg_error(ctx, "nchains, nsteps, nw must be >= 1");
    for (int c = 0; c < nchains; ++c)
        if (steps_done[c] < 0 || steps_done[c] > nsteps) return set_arg_error(ctx, "steps_done out of range");
    if (!std::isfinite(prefactor) || !std::isfinite(eta) || eta <= 0.0) return set_arg_error(ctx, "bad prefactor or eta");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return BSE_ERR_CUDA;
    return bse_cf_device(ctx, nchains, nsteps, steps_done, a, b, pnorm2, prefactor, eta, nw, omega, eps);
}

}  // extern "C"
