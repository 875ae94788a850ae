"""Full-size parity on sampled outputs.

At the benchmark's sizes the oracle cannot form H, so one application
y = H x of the GPU path is compared with the oracle at a few sampled dense
points (K_c rows of their corners built on demand, the M3 near field pair by
pair).  Tolerances: FP64 plain path 1e-11 relative to max |y - dE x|; BF16
K_c paths 5e-3 (BF16 rounding of K_c, FP32 vectors).
"""
import numpy as np
import pytest

from oracle import interp as oi
from oracle import learned as ol
from paper_1602_01863_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

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


def _apply(ctx, it, x):
    dt = torch.complex128 if it.vec_prec == 0 else torch.complex64
    xs = torch.from_numpy(np.ascontiguousarray(x)).to(dt).cuda()
    ys = torch.empty_like(xs)
    ctx.bse_apply_h(it, x.shape[0], xs.data_ptr(), ys.data_ptr())
    torch.cuda.synchronize()
    return ys.cpu().numpy().astype(np.complex128)


def _check_rows(I, x, y, rows, m3, tol):
    ref = I.apply_m1_rows(x, rows)
    if m3:
        ref = ref + I.near_field_rows(x, rows)
    got = y.reshape(I.Nk, I.t)[rows]
    dex = (I.dE * x).reshape(I.Nk, I.t)[rows]
    assert np.abs(got - ref).max() <= tol * np.abs(ref - dex).max()


@pytest.mark.parametrize("kc_prec,vec_prec,tol", [(2, 1, 5e-3), (0, 0, 1e-11)])
def test_single_system_size_m3(ctx, kc_prec, vec_prec, tol):
    """Coarse 8^3, 4v x 4c, n_div 4 (N = 524288), Method 3, w = 1."""
    s = synth.single_system()
    co = ctx.bse_build_coarse(s.model, s.n_coarse, kc_prec)
    it = ctx.bse_interp_setup(co, s.n_div, 1, 1.0, vec_prec)
    x = synth.random_vectors(31, (1, it.N))
    y = _apply(ctx, it, x)[0]
    I = oi.Interp(s.model, s.n_coarse, s.n_div, width=1.0, build_dense_kc=False)
    rows = np.array([0, 4097, 17000, it.Nk - 1])
    _check_rows(I, x[0], y, rows, True, tol)
    it.free()
    co.free()


def test_largest_size_m1_m3_rows_and_trained_learned_run(ctx):
    """Coarse 12^3, 4v x 6c, n_div 4 (N = 2654208):
    * BF16 K_c (41472^2 = 6.9 GB), FP32 vectors: sampled rows of one M1
      application against the oracle (5e-3 of the kernel part);
    * the Method-3 near field at t = 24 (CUDA-core kernel) in FP64 (complex128
      K_c, 27.5 GB): H^{M3} x - H^{M1} x against the oracle's pair-by-pair
      correction on rows that include the zone wrap, 1e-8 of the row's near
      field.  (At this size the correction is ~4e-6 of |H x|, so an FP32
      difference of two applications would be dominated by FP32 rounding.)
    * the learned correction with a network trained on the method's pairs
      (4v x 6c, coarse 4^3, n_div 4), 500 steps x 3 chains: finite, positive b,
      Im eps >= 0, training loss halved."""
    import bench
    from paper_1602_01863_gb300 import bse
    s = synth.largest_system()
    I = oi.Interp(s.model, s.n_coarse, s.n_div, build_dense_kc=False)
    x = synth.random_vectors(32, (1, I.N))
    co64 = ctx.bse_build_coarse(s.model, s.n_coarse, bse.PREC_F64)
    it1 = ctx.bse_interp_setup(co64, s.n_div, bse.SCHEME_M1, 1.0, bse.PREC_F64)
    it3 = ctx.bse_interp_setup(co64, s.n_div, bse.SCHEME_M3, 1.0, bse.PREC_F64)
    nf_rows = np.array([0, 1, 63, 70000, I.Nk - 1])
    nf = (_apply(ctx, it3, x)[0] - _apply(ctx, it1, x)[0]).reshape(I.Nk, I.t)[nf_rows]
    ref = I.near_field_rows(x[0], nf_rows)
    per_row = np.abs(nf - ref).max(axis=1) / np.abs(ref).max(axis=1)
    print("largest system: FP64 near-field per-row error", per_row)
    assert per_row.max() <= 1e-8
    it1.free()
    it3.free()
    co64.free()
    co = ctx.bse_build_coarse(s.model, s.n_coarse, bse.PREC_BF16)
    it = ctx.bse_interp_setup(co, s.n_div, bse.SCHEME_M1, 1.0, bse.PREC_F32)
    y = _apply(ctx, it, x)[0]
    _check_rows(I, x[0], y, np.array([3, 50000, it.Nk - 5]), False, 5e-3)
    mlp, first, last = bench.train_network(ctx, bse, synth, 4, 6, blocks=256, steps=1500)
    assert last < 0.5 * first
    ctx.bse_interp_set_learned(it, mlp, 8)
    a, b, pn2, st, rc = ctx.bse_haydock_run([it], [3], s.pol_dirs, 500, bse.USE_GRAPH)
    assert rc == 0 and np.all(st == 500)
    assert np.all(np.isfinite(a)) and np.all(b[:, 1:] > 0)
    eps = ctx.bse_spectrum(a, b, pn2, st, 1.0 / it.Nk, 0.1, synth.frequency_grid(2000))
    assert np.all(eps.imag > -1e-9 * np.abs(eps.imag).max())
    mlp.free()
    it.free()
    co.free()


def test_fp32_near_field_at_t24(ctx):
    """The FP32 CUDA-core near field at t = 24 (4v x 6c), n_div 4, coarse 4^3:
    H^{M3} x - H^{M1} x on rows of the first and last cells against the oracle.
    Bar: 5e-3 of the row's near field plus FP32 rounding of the two
    applications (3e-7 of max |H x| of the row)."""
    from paper_1602_01863_gb300 import bse
    m = synth.draw_model(33, 4, 6)
    co = ctx.bse_build_coarse(m, 4, bse.PREC_F32)
    it1 = ctx.bse_interp_setup(co, 4, bse.SCHEME_M1, 1.0, bse.PREC_F32)
    it3 = ctx.bse_interp_setup(co, 4, bse.SCHEME_M3, 1.0, bse.PREC_F32)
    x = synth.random_vectors(34, (1, it1.N)).astype(np.complex64).astype(np.complex128)
    y1 = _apply(ctx, it1, x)[0]
    y3 = _apply(ctx, it3, x)[0]
    I = oi.Interp(m, 4, 4, width=1.0, build_dense_kc=False)
    rows = np.concatenate([np.arange(0, 64, 7), np.arange(I.Nk - 64, I.Nk, 9)])
    nf = (y3 - y1).reshape(I.Nk, I.t)[rows]
    ref = I.near_field_rows(x[0], rows)
    ymax = np.abs(y3.reshape(I.Nk, I.t)[rows]).max(axis=1)
    err = np.abs(nf - ref).max(axis=1)
    bar = 5e-3 * np.abs(ref).max(axis=1) + 3e-7 * ymax
    print("t = 24 FP32 near field: worst error / bar", float((err / bar).max()))
    assert np.all(err <= bar)
    it1.free()
    it3.free()
    co.free()
