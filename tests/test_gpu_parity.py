"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances
  FP64 plain path: 1e-10 relative on Lanczos coefficients a_n, b_n (CGS2 in
  both implementations), 1e-12 on single H applications, 1e-13 on K_c.
  Mixed forms (BF16 / complex64 K_c, FP32 vectors, FP64 reductions):
  1e-3 max peak-normalised error on Im eps over the frequency window.
"""
import functools

import numpy as np
import pytest

from oracle import haydock as oh
from oracle import interp as oi
from oracle import model as om
from paper_1602_01863_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_01863_gb300 import bse
    torch.cuda.set_device(0)
    c = bse.Context(0, torch.cuda.current_stream().cuda_stream)
    yield c
    c.close()


@functools.lru_cache(maxsize=None)
def oracle_interp(seed, nv, nc, n, nd, scheme="8nb", width=1.0):
    return oi.Interp(synth.draw_model(seed, nv, nc), n, nd, scheme=scheme, width=width)


@functools.lru_cache(maxsize=None)
def oracle_H(seed, nv, nc, n, nd, method, scheme="8nb", width=1.0):
    return oracle_interp(seed, nv, nc, n, nd, scheme, width).H_dense(method)


def gpu_system(ctx, seed, nv, nc, n, nd, method="m1", scheme="8nb", width=1.0, kc_prec=0, vec_prec=0, extra=0):
    from paper_1602_01863_gb300 import bse
    m = synth.draw_model(seed, nv, nc)
    co = ctx.bse_build_coarse(m, n, kc_prec)
    sch = (bse.SCHEME_M3 if method == "m3" else bse.SCHEME_M1) | (bse.NB1 if scheme == "1nb" else 0) | extra
    it = ctx.bse_interp_setup(co, nd, sch, width, vec_prec)
    return co, it


def apply_gpu(ctx, it, x: np.ndarray) -> np.ndarray:
    dt = torch.complex128 if it.vec_prec == 0 else torch.complex64
    xs = torch.from_numpy(np.ascontiguousarray(x)).to(dt).cuda()
    ys = torch.empty_like(xs)
    ctx.bse_apply_h(it, x.shape[0], xs.data_ptr(), ys.data_ptr())
    torch.cuda.synchronize()
    return ys.cpu().numpy().astype(np.complex128)


# ------------------------------------------------------------------- K_c
@pytest.mark.parametrize("n,nv,nc", [(2, 2, 3), (3, 3, 3), (4, 3, 3), (3, 1, 5)])
def test_kc_matches_oracle(ctx, n, nv, nc):
    m = synth.draw_model(5, nv, nc)
    co = ctx.bse_build_coarse(m, n, 0)
    K = co.get_kc()
    Kref = om.kernel_matrix(om.GridModel(m, om.coarse_coords(n), n))
    assert np.abs(K - Kref).max() <= 1e-13 * np.abs(Kref).max()
    co.free()


def test_kc_bf16_and_c64_are_roundings_of_oracle(ctx):
    m = synth.draw_model(6, 3, 3)
    Kref = om.kernel_matrix(om.GridModel(m, om.coarse_coords(4), 4))
    for prec, rel in ((2, 2.0 ** -8), (1, 2.0 ** -23)):
        co = ctx.bse_build_coarse(m, 4, prec)
        K = co.get_kc()
        floor = 1e-15 * np.abs(Kref).max()          # entries that are rounding noise (~1e-21) in both
        for part in (np.real, np.imag):
            err = np.abs(part(K) - part(Kref))
            assert np.all(err <= rel * np.abs(part(Kref)) + floor)
        off = ~np.eye(K.shape[0], dtype=bool)
        assert np.abs(K - K.conj().T)[off].max() == 0.0     # rounding keeps K_c exactly Hermitian off the diagonal
        assert np.abs(np.diag(K).imag).max() <= floor       # the diagonal is real up to noise
        co.free()


# --------------------------------------------------------- single apply
@pytest.mark.parametrize("case", [
    dict(seed=1, nv=3, nc=3, n=4, nd=2, method="m1"),
    dict(seed=1, nv=3, nc=3, n=4, nd=2, method="m3"),
    dict(seed=2, nv=2, nc=3, n=3, nd=3, method="m3"),
    dict(seed=3, nv=2, nc=2, n=4, nd=2, method="m3", scheme="1nb"),
    dict(seed=4, nv=1, nc=2, n=5, nd=1, method="m1"),
])
def test_apply_h_f64_matches_oracle(ctx, case):
    scheme = case.get("scheme", "8nb")
    co, it = gpu_system(ctx, case["seed"], case["nv"], case["nc"], case["n"], case["nd"], case["method"], scheme)
    H = oracle_H(case["seed"], case["nv"], case["nc"], case["n"], case["nd"], case["method"], scheme)
    x = synth.random_vectors(7, (3, it.N))
    y = apply_gpu(ctx, it, x)
    yr = (H @ x.T).T
    assert np.abs(y - yr).max() <= 1e-12 * np.abs(yr).max()
    it.free()
    co.free()


@pytest.mark.parametrize("nv,nc,method", [(4, 4, "m3"), (4, 6, "m3"), (3, 3, "m3"), (2, 3, "m3"), (4, 4, "m1")])
def test_apply_h_fp32_matches_oracle(ctx, nv, nc, method):
    """FP32 vectors with complex64 K_c (staged kernels for 3x3, 4x4
    and 4x6 bands, generic ones otherwise, CUDA-core near field), 3 chains:
    FP32-level agreement."""
    from paper_1602_01863_gb300 import bse
    co, it = gpu_system(ctx, 13, nv, nc, 3, 2, method, kc_prec=1, vec_prec=1, extra=bse.NF_CUDA_CORES)
    H = oracle_H(13, nv, nc, 3, 2, method)
    x = synth.random_vectors(9, (3, it.N)).astype(np.complex64).astype(np.complex128)
    y = apply_gpu(ctx, it, x)
    yr = (H @ x.T).T
    assert np.abs(y - yr).max() <= 2e-5 * np.abs(yr).max()
    it.free()
    co.free()


@pytest.mark.parametrize("nv,nc,n,nd", [(4, 4, 4, 4), (3, 3, 4, 2), (2, 3, 3, 3)])
def test_tensor_core_near_field(ctx, nv, nc, n, nd):
    """M3 near field on tcgen05 (TF32 head blocks and y1, z; FP32 accumulation)
    against the oracle on sampled rows and against the CUDA-core kernel.
    Bar: TF32 operand rounding (2^-11 relative) amplified by the partial
    cancellation of y1 against h_head z, a few parts in 1e3 of |near field|."""
    from paper_1602_01863_gb300 import bse
    co, it = gpu_system(ctx, 21, nv, nc, n, nd, "m3", kc_prec=1, vec_prec=1)
    co2, it2 = gpu_system(ctx, 21, nv, nc, n, nd, "m3", kc_prec=1, vec_prec=1, extra=bse.NF_CUDA_CORES)
    x = synth.random_vectors(4, (2, it.N)).astype(np.complex64).astype(np.complex128)
    y = apply_gpu(ctx, it, x)
    y2 = apply_gpu(ctx, it2, x)
    I = oi.Interp(synth.draw_model(21, nv, nc), n, nd, width=1.0, build_dense_kc=False)
    rows = np.array([0, 3, it.Nk // 2, it.Nk - 1])
    for v in range(2):
        ref_m1 = I.apply_m1_rows(x[v], rows)
        nf = I.near_field_rows(x[v], rows)
        got = y[v].reshape(I.Nk, I.t)[rows]
        err = np.abs(got - (ref_m1 + nf)).max() / np.abs(nf).max()
        print(f"tensor-core near field, relative error {err:.3e}")
        assert err <= 5e-3
    near2 = y2 - y
    assert np.abs(near2).max() <= 2e-3 * np.abs(y2).max()
    it.free(); co.free(); it2.free(); co2.free()


# ----------------------------------------------------------- Haydock FP64
@pytest.mark.parametrize("method", ["m1", "m3"])
def test_haydock_fp64_matches_oracle(ctx, method):
    """The small configuration: coarse 4^3, 3v x 3c, n_div 2 (N = 4608), 100 steps, CGS2."""
    from paper_1602_01863_gb300 import bse
    co, it = gpu_system(ctx, 1, 3, 3, 4, 2, method)
    e = np.array([[1.0, 0.0, 0.0]])
    a, b, pn2, st, rc = ctx.bse_haydock_run([it], [1], e, 100, bse.REORTH_CGS2)
    I = oracle_interp(1, 3, 3, 4, 2)
    H = oracle_H(1, 3, 3, 4, 2, method)
    ra, rb, rpn2, _ = oh.haydock(lambda v: H @ v, I.dipole(e[0]), 100, "cgs2")
    assert rc == 0 and st[0] == 100
    assert abs(pn2[0] - rpn2) <= 1e-13 * rpn2
    assert np.max(np.abs(a[0] - ra) / np.abs(ra)) < 1e-10
    assert np.max(np.abs(b[0, 1:] - rb[1:]) / np.abs(rb[1:])) < 1e-10
    # graph-captured loop gives bitwise the same coefficients
    a2, b2, _, _, _ = ctx.bse_haydock_run([it], [1], e, 100, bse.REORTH_CGS2 | bse.USE_GRAPH)
    assert np.array_equal(a, a2) and np.array_equal(b, b2)
    # the device continued fraction equals the oracle's
    w = synth.frequency_grid(1000)
    eps = ctx.bse_spectrum(a, b, pn2, st, 1.0 / I.Nk, 0.1, w)
    ref = oh.epsilon(ra, rb, rpn2, 1.0 / I.Nk, 0.1, w)
    assert np.abs(eps[0] - ref).max() <= 1e-10 * np.abs(ref.imag).max()
    it.free()
    co.free()


def test_haydock_three_chains_and_plain_recursion(ctx):
    """p = 3 polarisations share one H; no reorthogonalisation (the paper's
    recursion) compared on the first 30 coefficients, where plain Lanczos is
    still orthogonal to working precision."""
    from paper_1602_01863_gb300 import bse
    co, it = gpu_system(ctx, 9, 2, 3, 3, 2, "m3")
    I = oracle_interp(9, 2, 3, 3, 2)
    H = oracle_H(9, 2, 3, 3, 2, "m3")
    dirs = np.eye(3)
    a, b, pn2, st, rc = ctx.bse_haydock_run([it], [3], dirs, 30, 0)
    for ch in range(3):
        ra, rb, rpn2, _ = oh.haydock(lambda v: H @ v, I.dipole(dirs[ch]), 30, "none")
        assert np.max(np.abs(a[ch] - ra) / np.abs(ra)) < 1e-10
        assert np.max(np.abs(b[ch, 1:] - rb[1:]) / np.abs(rb[1:])) < 1e-10
    it.free()
    co.free()


def test_breakdown_stops_chain(ctx):
    """N = 8 (coarse 2^3, n_div 1, 1v x 1c): the Krylov space is exhausted
    after at most 8 steps; the chain stops and reports it."""
    from paper_1602_01863_gb300 import bse
    co, it = gpu_system(ctx, 12, 1, 1, 2, 1, "m1")
    a, b, pn2, st, rc = ctx.bse_haydock_run([it], [1], np.array([[1.0, 0, 0]]), 12, bse.REORTH_CGS2)
    assert rc == bse.BSE_WARN_BREAKDOWN and st[0] <= 8
    H = oracle_H(12, 1, 1, 2, 1, "m1")
    I = oracle_interp(12, 1, 1, 2, 1)
    ra, rb, rpn2, _ = oh.haydock(lambda v: H @ v, I.dipole([1, 0, 0]), 12, "cgs2")
    k = min(st[0], len(ra))
    assert np.allclose(a[0, :k], ra[:k], rtol=1e-10)
    it.free()
    co.free()


# -------------------------------------------------------------- mixed forms
@pytest.mark.parametrize("kc_prec", [2, 1])
@pytest.mark.parametrize("method", ["m1", "m3"])
def test_mixed_spectrum_small(ctx, kc_prec, method):
    """BF16 (tensor cores) and complex64 K_c with FP32 vectors at the small
    configuration: Im eps within 1e-3 of the FP64 oracle."""
    co, it = gpu_system(ctx, 1, 3, 3, 4, 2, method, kc_prec=kc_prec, vec_prec=1)
    e = np.array([[1.0, 0.0, 0.0]])
    a, b, pn2, st, rc = ctx.bse_haydock_run([it], [1], e, 100, 0)
    I = oracle_interp(1, 3, 3, 4, 2)
    H = oracle_H(1, 3, 3, 4, 2, method)
    w = synth.frequency_grid(1000)
    ref = oh.epsilon_brute(H, I.dipole(e[0]), 1.0 / I.Nk, 0.1, w)
    eps = ctx.bse_spectrum(a, b, pn2, st, 1.0 / I.Nk, 0.1, w)
    assert oh.spectrum_error(eps[0].imag, ref.imag) < 1e-3
    it.free()
    co.free()


def test_mixed_apply_h_ragged_tiles(ctx):
    """Tensor-core apply with N_c = 1944 (15 full 128-row tiles + a ragged one)
    and 3 chains: relative error of y = H x against the oracle at the BF16 level."""
    co, it = gpu_system(ctx, 8, 3, 3, 6, 1, "m1", kc_prec=2, vec_prec=1)
    I = oi.Interp(synth.draw_model(8, 3, 3), 6, 1)
    x = synth.random_vectors(3, (3, it.N))
    y = apply_gpu(ctx, it, x)
    yr = np.stack([I.apply_m1(v) for v in x])
    rel = np.linalg.norm(y - yr) / np.linalg.norm(yr - I.dE[None] * x)
    assert rel < 4e-3, rel
    it.free()
    co.free()


# ------------------------------------------------------------------ errors
def test_argument_errors(ctx):
    from paper_1602_01863_gb300 import bse
    m = synth.draw_model(0, 2, 2)
    co = ctx.bse_build_coarse(m, 4, 0)
    with pytest.raises(bse.BseError) as e:
        ctx.bse_interp_setup(co, 0)
    assert e.value.code == bse.BSE_ERR_ARG
    with pytest.raises(bse.BseError) as e:
        ctx.bse_interp_setup(co, 2, bse.SCHEME_M3, 2.0)              # w >= n/2
    assert e.value.code == bse.BSE_ERR_ARG
    with pytest.raises(bse.BseError) as e:
        ctx.bse_interp_setup(co, 2, bse.SCHEME_M1, 1.0, bse.PREC_F32)   # F64 K_c with F32 vectors
    assert e.value.code == bse.BSE_ERR_UNSUPPORTED
    bad = synth.draw_model(0, 2, 2)
    bad.mu[0, 0, 0, 0] = np.nan
    with pytest.raises(bse.BseError) as e:
        ctx.bse_build_coarse(bad, 2, 0)
    assert e.value.code == bse.BSE_ERR_ARG
    co.free()
