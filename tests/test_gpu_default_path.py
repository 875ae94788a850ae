"""Parity of the default mixed path: BF16 / complex64 K_c, FP32 vectors and the
tensor-core Method-3 near field (FP16 operands with power-of-two scales: 10
explicit mantissa bits, as TF32), i.e. what the benchmark times.

Bars
  * Spectrum (Sec. 5.1 accuracy measure, peak-normalised Im eps): 1e-3 against
    the FP64 plain path, which is itself pinned to the FP64 oracle at 1e-10
    (a_n, b_n) and 1e-11 (sampled full-size rows).
  * Near field alone: TF32 keeps 10 explicit mantissa bits (unit roundoff
    2^-11 ~ 4.9e-4).  The head blocks are applied to y1 and z separately and
    y1 - h_head(q_c) z cancels to about a tenth of |y1|, so the rounding of
    y1, z and of the head blocks is amplified about tenfold: a few parts in
    1e3 of |near field|.  The bar is 5e-3 of max |near field| of each row.
  * Whole vector: FP32 arithmetic elsewhere (2e-5 of max |H x|) plus the TF32
    near-field term above.
"""
import numpy as np
import pytest

from oracle import haydock as oh
from oracle import interp as oi
from paper_1602_01863_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NF_BAR = 5e-3


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_01863_gb300 import bse
    torch.cuda.set_device(0)
    c = bse.Context(0, torch.cuda.current_stream().cuda_stream)
    yield c
    c.close()


def _apply(ctx, it, x):
    xs = torch.from_numpy(np.ascontiguousarray(x)).to(torch.complex64).cuda()
    ys = torch.empty_like(xs)
    ctx.bse_apply_h(it, x.shape[0], xs.data_ptr(), ys.data_ptr())
    torch.cuda.synchronize()
    return ys.cpu().numpy().astype(np.complex128)


def _system(ctx, model, n, nd, scheme, kc_prec):
    from paper_1602_01863_gb300 import bse
    co = ctx.bse_build_coarse(model, n, kc_prec)
    it = ctx.bse_interp_setup(co, nd, scheme, 1.0, bse.PREC_F32)
    return co, it


@pytest.mark.parametrize("nv,nc,n,nd", [(4, 4, 3, 2), (3, 3, 3, 2), (2, 3, 3, 3)])
def test_whole_vector_default_near_field(ctx, nv, nc, n, nd):
    """y = H x over the whole vector with the default (tensor-core) near field,
    against the oracle's dense Method-3 matrix."""
    from paper_1602_01863_gb300 import bse
    m = synth.draw_model(41, nv, nc)
    co, it = _system(ctx, m, n, nd, bse.SCHEME_M3, bse.PREC_F32)
    I = oi.Interp(m, n, nd, width=1.0)
    H3, H1 = I.H_dense("m3"), I.H_dense("m1")
    x = synth.random_vectors(5, (3, it.N)).astype(np.complex64).astype(np.complex128)
    y = _apply(ctx, it, x)
    yr = (H3 @ x.T).T
    nf = ((H3 - H1) @ x.T).T
    err = np.abs(y - yr).max()
    bar = 2e-5 * np.abs(yr).max() + NF_BAR * np.abs(nf).max()
    print(f"whole vector: err {err:.3e}, bar {bar:.3e}, |nf| {np.abs(nf).max():.3e}, |Hx| {np.abs(yr).max():.3e}")
    assert err <= bar
    it.free()
    co.free()


def _cell_rows(nd, Nk, cell):
    return np.arange(cell * nd ** 3, (cell + 1) * nd ** 3)


def test_near_field_rows_every_subpoint_and_wrap(ctx):
    """The tensor-core near field on 128 dense rows: all 64 sub-points of the
    first coarse cell (every sub-point class; its near partners wrap around
    the zone) and all 64 of the last cell (wrapping the other way), coarse 4^3,
    4v x 4c, n_div 4.  GPU near field = H^{M3} x - H^{M1} x with complex64 K_c
    (the M1 parts are the same kernels); oracle = the pair-by-pair correction."""
    from paper_1602_01863_gb300 import bse
    m = synth.draw_model(43, 4, 4)
    n, nd = 4, 4
    co3, it3 = _system(ctx, m, n, nd, bse.SCHEME_M3, bse.PREC_F32)
    co1, it1 = _system(ctx, m, n, nd, bse.SCHEME_M1, bse.PREC_F32)
    x = synth.random_vectors(6, (3, it3.N)).astype(np.complex64).astype(np.complex128)
    nf_gpu = _apply(ctx, it3, x) - _apply(ctx, it1, x)
    I = oi.Interp(m, n, nd, width=1.0, build_dense_kc=False)
    rows = np.concatenate([_cell_rows(nd, I.Nk, 0), _cell_rows(nd, I.Nk, n ** 3 - 1)])
    worst = 0.0
    for v in (0, 2):
        ref = I.near_field_rows(x[v], rows)
        got = nf_gpu[v].reshape(I.Nk, I.t)[rows]
        per_row = np.abs(got - ref).max(axis=1) / np.abs(ref).max(axis=1)
        worst = max(worst, float(per_row.max()))
    print(f"near field, worst per-row error / max |near field| of the row: {worst:.3e}")
    assert worst <= NF_BAR
    for it, co in ((it3, co3), (it1, co1)):
        it.free()
        co.free()


@pytest.mark.slow
def test_single_system_default_path_spectrum(ctx):
    """Coarse 8^3, 4v x 4c, n_div 4 (N = 524288), 3 polarisations, 300 steps:
    the default mixed path (BF16 K_c on tcgen05, tensor-core near field, FP32
    vectors, FP64 reductions) against the FP64 plain path on the same device,
    peak-normalised Im eps per chain within 1e-3."""
    from paper_1602_01863_gb300 import bse
    s = synth.single_system()
    w = synth.frequency_grid(1000)
    pref = synth.S_EPS / s.nk_dense
    spectra = {}
    for kc, vec in ((bse.PREC_BF16, bse.PREC_F32), (bse.PREC_F64, bse.PREC_F64)):
        co = ctx.bse_build_coarse(s.model, s.n_coarse, kc)
        it = ctx.bse_interp_setup(co, s.n_div, bse.SCHEME_M3, 1.0, vec)
        a, b, pn2, st, rc = ctx.bse_haydock_run([it], [3], s.pol_dirs, 300, bse.USE_GRAPH)
        assert rc == 0 and np.all(st == 300)
        spectra[kc] = (ctx.bse_spectrum(a, b, pn2, st, pref, synth.ETA, w), a, b)
        it.free()
        co.free()
    mixed, a_m, b_m = spectra[bse.PREC_BF16]
    plain, a_p, b_p = spectra[bse.PREC_F64]
    errs = [oh.spectrum_error(mixed[c].imag, plain[c].imag) for c in range(3)]
    print("Im eps error per chain (mixed vs FP64):", ", ".join(f"{e:.2e}" for e in errs))
    # the first coefficients, before rounding differences are amplified by the recursion
    print("a_1..a_10 max relative difference:", float(np.max(np.abs(a_m[:, :10] - a_p[:, :10]) / np.abs(a_p[:, :10]))))
    assert max(errs) <= 1e-3
    assert np.all(np.abs(a_m[:, :10] - a_p[:, :10]) <= 1e-3 * np.abs(a_p[:, :10]))


def test_concurrent_kc_apply_matches_serial_schedule(ctx):
    """With the tensor-core near field the K_c apply runs beside it (auxiliary
    stream, lowest scheduling priority) and its CTAs take chunks of K_c from a
    counter; the tile sums run in chunk order, so the Haydock coefficients of
    the graph run, the eager run and the profiled run (kernels one after
    another) are equal bit for bit.  The autotuned launch shape is reported."""
    from paper_1602_01863_gb300 import bse
    m = synth.draw_model(31, 4, 4)
    co, it = _system(ctx, m, 6, 4, bse.SCHEME_M3, bse.PREC_BF16)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    stages, chunk, ctas = it.kc_plan()
    assert stages in (4, 5, 6) and 1 <= chunk <= 64 and 1 <= ctas <= sms
    dirs = np.eye(3)
    runs = [ctx.bse_haydock_run([it], [3], dirs, 40, f) for f in (bse.USE_GRAPH, 0, bse.PROFILE, bse.USE_GRAPH)]
    for a, b, pn2, sd, _ in runs[1:]:
        assert np.array_equal(a, runs[0][0]) and np.array_equal(b, runs[0][1])
    assert np.all(np.isfinite(runs[0][0])) and np.all(runs[0][1][:, 1:] > 0)
    it.free()
    co.free()
