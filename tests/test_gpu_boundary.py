"""The C ABI with caller-supplied inputs, the Sec. 5.1 stopping rule, and
cached step-loop graphs.

  * Caller inputs (Sec. 3 statement of the problem: K_c, d, Delta E, P): the
    library's model is one crystal (seed A) while K_c, the overlaps d, Delta E
    and P come from another (seed B) through bse_build_coarse(user_kc) and
    bse_interp_setup(dense).  The Haydock coefficients must then be the
    oracle's for crystal B alone (1e-10, FP64, CGS2), so no model table can
    have leaked in.
  * Stopping rule: the GPU stops each chain at the same step as the oracle's
    haydock_until_converged and its coefficients agree to 1e-10 up to there.
  * Graphs: a cached graph replays to the same coefficients, follows a change
    of step count, and a run that replays it allocates no device memory.
"""
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


def _rel(x, ref):
    return float(np.max(np.abs(x - ref) / np.abs(ref)))


def test_caller_supplied_kc_and_dense_tables(ctx):
    from paper_1602_01863_gb300 import bse
    n, nd, nv, nc = 3, 2, 2, 3
    mA = synth.draw_model(51, nv, nc)
    mB = synth.draw_model(52, nv, nc, eps_inf=8.0)
    IB = oi.Interp(mB, n, nd)
    kc = torch.from_numpy(np.ascontiguousarray(IB.Kc)).cuda()
    co = ctx.bse_build_coarse(mA, n, bse.PREC_F64, user_kc_ptr=kc.data_ptr())
    K = co.get_kc()
    assert np.array_equal(K, IB.Kc)
    dense = {"dE": IB.dE, "P": IB.dense.P.transpose(1, 0, 2, 3).reshape(3, -1), "Dv": IB.Dv, "Dc": IB.Dc}
    it = ctx.bse_interp_setup(co, nd, bse.SCHEME_M1, 1.0, bse.PREC_F64, dense=dense)
    e = np.array([[0.3, -0.5, 0.8]])
    a, b, pn2, st, rc = ctx.bse_haydock_run([it], [1], e, 60, bse.REORTH_CGS2)
    H = IB.H_dense("m1")
    ra, rb, rpn2, _ = oh.haydock(lambda v: H @ v, IB.dipole(e[0]), 60, "cgs2")
    assert rc == 0
    assert abs(pn2[0] - rpn2) <= 1e-13 * rpn2
    assert _rel(a[0], ra) < 1e-10 and _rel(b[0, 1:], rb[1:]) < 1e-10
    # the same K_c in BF16 storage is its rounding
    co2 = ctx.bse_build_coarse(mA, n, bse.PREC_BF16, user_kc_ptr=kc.data_ptr())
    K2 = co2.get_kc()
    assert np.all(np.abs(K2.real - IB.Kc.real) <= 2.0 ** -8 * np.abs(IB.Kc.real) + 1e-300)
    co2.free()
    it.free()
    co.free()


def test_dense_inputs_reject_non_finite(ctx):
    from paper_1602_01863_gb300 import bse
    m = synth.draw_model(53, 1, 2)
    co = ctx.bse_build_coarse(m, 2, bse.PREC_F64)
    N = 2 * 8 * 8
    dE = np.ones(N)
    dE[5] = np.inf
    with pytest.raises(bse.BseError) as err:
        ctx.bse_interp_setup(co, 2, bse.SCHEME_M1, 1.0, bse.PREC_F64, dense={"dE": dE})
    assert err.value.code == bse.BSE_ERR_ARG
    co.free()


@pytest.mark.parametrize("method,reorth", [("m3", True), ("m1", False)])
def test_stop_rule_matches_oracle(ctx, method, reorth):
    """Sec. 5.1 rule, check every 5 steps, 1 %, on coarse 4^3, 2v x 2c, n_div 2."""
    from paper_1602_01863_gb300 import bse
    m = synth.draw_model(54, 2, 2)
    I = oi.Interp(m, 4, 2, width=1.0)
    H = I.H_dense(method)
    w = synth.frequency_grid(600)
    every, tol = 5, 0.01
    ctx.bse_set_stop_rule(tol, every, synth.S_EPS, synth.ETA, w)
    co = ctx.bse_build_coarse(m, 4, bse.PREC_F64)
    it = ctx.bse_interp_setup(co, 2, bse.SCHEME_M3 if method == "m3" else bse.SCHEME_M1, 1.0, bse.PREC_F64)
    dirs = np.eye(3)
    flags = bse.STOP_CONVERGED | (bse.REORTH_CGS2 if reorth else 0)
    a, b, pn2, st, rc = ctx.bse_haydock_run([it], [3], dirs, 200, flags)
    assert rc == 0
    for ch in range(3):
        ra, rb, rpn2, _ = oh.haydock_until_converged(lambda v: H @ v, I.dipole(dirs[ch]), 200, every, tol,
                                                     synth.S_EPS / I.Nk, synth.ETA, w, "cgs2" if reorth else "none")
        k = len(ra)
        assert st[ch] == k, (ch, st[ch], k)
        assert _rel(a[ch, :k], ra) < 1e-10 and _rel(b[ch, 1:k + 1], rb[1:k + 1]) < 1e-10
        assert np.all(a[ch, k:] == 0.0)
    # the same systems in a batched graph stop at the same steps
    co2 = ctx.bse_build_coarse(synth.draw_model(55, 2, 3), 3, bse.PREC_F64)
    it2 = ctx.bse_interp_setup(co2, 2, bse.SCHEME_M1, 1.0, bse.PREC_F64)
    a2, b2, _, st2, _ = ctx.bse_haydock_run([it2], [2], dirs[:2], 200, flags)
    ab, bb, _, stb, rcb = ctx.bse_haydock_run([it, it2], [3, 2], np.concatenate([dirs, dirs[:2]]), 200,
                                              flags | bse.USE_GRAPH)
    assert rcb == 0
    assert np.array_equal(stb, np.concatenate([st, st2]))
    assert np.array_equal(ab[:3], a) and np.array_equal(ab[3:], a2)
    it.free(); co.free(); it2.free(); co2.free()


def test_graph_cache_replays_and_allocates_nothing(ctx):
    """A cached step-loop graph: the second run replays it (same coefficients
    bit for bit), a different step count recaptures it, the result equals the
    run without a graph, and replays allocate no device memory."""
    from paper_1602_01863_gb300 import bse
    m = synth.draw_model(56, 3, 3)
    co = ctx.bse_build_coarse(m, 4, bse.PREC_BF16)
    it = ctx.bse_interp_setup(co, 2, bse.SCHEME_M3, 1.0, bse.PREC_F32)
    dirs = np.eye(3)
    r0 = ctx.bse_haydock_run([it], [3], dirs, 40, 0)
    r1 = ctx.bse_haydock_run([it], [3], dirs, 40, bse.USE_GRAPH)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        r2 = ctx.bse_haydock_run([it], [3], dirs, 40, bse.USE_GRAPH)
        ctx.bse_spectrum(r2[0], r2[1], r2[2], r2[3], 1.0 / it.Nk, 0.1, synth.frequency_grid(1000))
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    for x, y, z in zip(r0[:4], r1[:4], r2[:4]):
        assert np.array_equal(x, y) and np.array_equal(y, z)
    r3 = ctx.bse_haydock_run([it], [3], dirs, 25, bse.USE_GRAPH)
    r4 = ctx.bse_haydock_run([it], [3], dirs, 25, 0)
    for x, y in zip(r3[:4], r4[:4]):
        assert np.array_equal(x, y)
    it.free()
    co.free()
