"""Batched Haydock runs: many uneven systems in one CUDA graph launch.

The batch must give exactly (bitwise) what the systems give one by one; a
member is also checked against the FP64 oracle, and the full 24-system
uneven batch (grids 4^3-8^3, n_div 2-4, bands 2x2-6x6, 72 chains) is checked
by properties that hold at any size.
"""
import numpy as np
import pytest

from oracle import haydock as oh
from oracle import interp as oi
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


MEMBERS = [  # seed, nv, nc, n, n_div, scheme, kc_prec, vec_prec, npol
    (101, 2, 3, 4, 2, 1, 2, 1, 3),
    (102, 3, 2, 3, 3, 0, 2, 1, 1),
    (103, 4, 4, 4, 2, 1, 1, 1, 2),
    (104, 2, 2, 5, 2, 1, 0, 0, 3),
]


def _build(ctx, members):
    handles = []
    for seed, nv, nc, n, nd, scheme, kc, vec, npol in members:
        co = ctx.bse_build_coarse(synth.draw_model(seed, nv, nc), n, kc)
        it = ctx.bse_interp_setup(co, nd, scheme, 1.0, vec)
        handles.append((co, it, npol))
    return handles


def test_batched_graph_equals_individual_runs(ctx):
    from paper_1602_01863_gb300 import bse
    hs = _build(ctx, MEMBERS)
    dirs = np.concatenate([np.eye(3)[:npol] for _, _, npol in hs])
    m = 40
    a, b, pn2, st, rc = ctx.bse_haydock_run([h[1] for h in hs], [h[2] for h in hs], dirs, m, bse.USE_GRAPH)
    assert rc == 0
    off = 0
    for co, it, npol in hs:
        a1, b1, p1, s1, _ = ctx.bse_haydock_run([it], [npol], dirs[off:off + npol], m, 0)
        assert np.array_equal(a[off:off + npol], a1) and np.array_equal(b[off:off + npol], b1)
        assert np.array_equal(pn2[off:off + npol], p1) and np.array_equal(st[off:off + npol], s1)
        off += npol
    # the FP64 member against the oracle (plain recursion, first 30 steps)
    seed, nv, nc, n, nd = MEMBERS[3][:5]
    I = oi.Interp(synth.draw_model(seed, nv, nc), n, nd, width=1.0)
    H = I.H_dense("m3")
    o = sum(h[2] for h in hs[:3])
    for ch in range(3):
        ra, rb, rpn2, _ = oh.haydock(lambda v: H @ v, I.dipole(np.eye(3)[ch]), 30, "none")
        assert np.max(np.abs(a[o + ch, :30] - ra) / np.abs(ra)) < 1e-10
        assert np.max(np.abs(b[o + ch, 1:31] - rb[1:]) / np.abs(rb[1:])) < 1e-10
    for co, it, _ in hs:
        it.free()
        co.free()


def test_duplicate_handle_rejected(ctx):
    from paper_1602_01863_gb300 import bse
    hs = _build(ctx, MEMBERS[:1])
    it = hs[0][1]
    with pytest.raises(bse.BseError) as e:
        ctx.bse_haydock_run([it, it], [1, 1], np.eye(3)[:2], 5, bse.USE_GRAPH)
    assert e.value.code == bse.BSE_ERR_ARG
    it.free()
    hs[0][0].free()


@pytest.mark.slow
def test_uneven_batch_of_24_systems_properties(ctx):
    """The 24-system uneven batch (72 chains, M3, BF16 K_c) in one graph launch:
    finite coefficients, b > 0, a_i inside a generous window around the
    single-particle energies (1.1-3.4 eV), and Im eps >= 0 (all poles of the
    truncated fraction have positive weights).  Every system's coefficients
    equal its own one-system run bit for bit (the batch changes the schedule,
    not the arithmetic), and for the systems with N <= 41000 the mixed
    spectrum is within 1e-3 (peak-normalised Im eps) of the FP64 plain path,
    which the FP64 tests pin to the oracle."""
    from paper_1602_01863_gb300 import bse
    systems = synth.batched_systems()
    hs = []
    for s in systems:
        co = ctx.bse_build_coarse(s.model, s.n_coarse, bse.PREC_BF16)
        it = ctx.bse_interp_setup(co, s.n_div, bse.SCHEME_M3, 1.0, bse.PREC_F32)
        hs.append((co, it))
    dirs = np.concatenate([s.pol_dirs for s in systems])
    m = 60
    a, b, pn2, st, rc = ctx.bse_haydock_run([h[1] for h in hs], [3] * len(hs), dirs, m, bse.USE_GRAPH)
    assert rc in (0, bse.BSE_WARN_BREAKDOWN)
    assert np.all(np.isfinite(a)) and np.all(np.isfinite(b)) and np.all(pn2 > 0)
    w = synth.frequency_grid(500)
    off = 0
    for s in systems:
        for ch in range(3):
            k = st[off + ch]
            assert np.all(b[off + ch, 1:k + 1] > 0)
            assert np.all(a[off + ch, :k] > -2.0) and np.all(a[off + ch, :k] < 8.0)
            eps = ctx.bse_spectrum(a[off + ch:off + ch + 1], b[off + ch:off + ch + 1], pn2[off + ch:off + ch + 1],
                                   st[off + ch:off + ch + 1], 1.0 / s.nk_dense, 0.1, w)
            assert eps[0].imag.min() > -1e-9 * eps[0].imag.max()
        off += 3
    off = 0
    for s, (co, it) in zip(systems, hs):
        a1, b1, pn1, st1, _ = ctx.bse_haydock_run([it], [3], s.pol_dirs, m, bse.USE_GRAPH)
        assert np.array_equal(a1, a[off:off + 3]) and np.array_equal(b1, b[off:off + 3])
        if s.n_dense_dim <= 41000:
            co64 = ctx.bse_build_coarse(s.model, s.n_coarse, bse.PREC_F64)
            it64 = ctx.bse_interp_setup(co64, s.n_div, bse.SCHEME_M3, 1.0, bse.PREC_F64)
            a2, b2, pn2_, st2, _ = ctx.bse_haydock_run([it64], [3], s.pol_dirs, m, bse.USE_GRAPH)
            for ch in range(3):
                e1 = ctx.bse_spectrum(a1[ch:ch + 1], b1[ch:ch + 1], pn1[ch:ch + 1], st1[ch:ch + 1], 1.0 / s.nk_dense, 0.1, w)
                e2 = ctx.bse_spectrum(a2[ch:ch + 1], b2[ch:ch + 1], pn2_[ch:ch + 1], st2[ch:ch + 1], 1.0 / s.nk_dense, 0.1, w)
                assert np.max(np.abs(e1[0].imag - e2[0].imag)) <= 1e-3 * np.max(np.abs(e2[0].imag))
            it64.free()
            co64.free()
        off += 3
    for co, it in hs:
        it.free()
        co.free()
