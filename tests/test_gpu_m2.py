"""Method 2 on the GPU (Sec. 4): the interpolated coefficients of Eq. diverg for
every pair, the head divided by the dense q, the whole Hamiltonian stored.

Parity with the oracle's dense K^{M2} (itself pinned: exact for the head-only
constant-mu model on every pair, equal to M3 on near pairs, explicit for
n_div = 1): 1e-12 on single applications, 1e-10 on the Haydock coefficients
(FP64, CGS2) at the small configuration."""
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


@pytest.mark.parametrize("nv,nc,n,nd,scheme", [(2, 3, 3, 2, "8nb"), (1, 2, 4, 3, "8nb"), (2, 2, 4, 2, "1nb")])
def test_m2_apply_matches_oracle(ctx, nv, nc, n, nd, scheme):
    from paper_1602_01863_gb300 import bse
    m = synth.draw_model(71, nv, nc)
    co = ctx.bse_build_coarse(m, n, bse.PREC_F64)
    it = ctx.bse_interp_setup(co, nd, bse.SCHEME_M2 | (bse.NB1 if scheme == "1nb" else 0), 1.0, bse.PREC_F64)
    H = oi.Interp(m, n, nd, scheme=scheme).H_dense("m2")
    x = synth.random_vectors(3, (3, it.N))
    xs = torch.from_numpy(x).cuda()
    ys = torch.empty_like(xs)
    ctx.bse_apply_h(it, 3, xs.data_ptr(), ys.data_ptr())
    y = ys.cpu().numpy()
    yr = (H @ x.T).T
    assert np.abs(y - yr).max() <= 1e-12 * np.abs(yr).max()
    it.free()
    co.free()


def test_m2_haydock_small_configuration(ctx):
    """Coarse 4^3, 3v x 3c, n_div 2 (N = 4608), 100 steps, CGS2, x polarisation."""
    from paper_1602_01863_gb300 import bse
    s = synth.small_system()
    co = ctx.bse_build_coarse(s.model, s.n_coarse, bse.PREC_F64)
    it = ctx.bse_interp_setup(co, s.n_div, bse.SCHEME_M2, 1.0, bse.PREC_F64)
    e = s.pol_dirs[:1]
    a, b, pn2, st, rc = ctx.bse_haydock_run([it], [1], e, 100, bse.REORTH_CGS2 | bse.USE_GRAPH)
    I = oi.Interp(s.model, s.n_coarse, s.n_div)
    H = I.H_dense("m2")
    ra, rb, rpn2, _ = oh.haydock(lambda v: H @ v, I.dipole(e[0]), 100, "cgs2")
    assert rc == 0 and st[0] == 100
    assert np.max(np.abs(a[0] - ra) / np.abs(ra)) < 1e-10
    assert np.max(np.abs(b[0, 1:] - rb[1:]) / np.abs(rb[1:])) < 1e-10
    it.free()
    co.free()


def test_m2_rejects_mixed_precision(ctx):
    from paper_1602_01863_gb300 import bse
    co = ctx.bse_build_coarse(synth.draw_model(72, 2, 2), 3, bse.PREC_F32)
    with pytest.raises(bse.BseError) as err:
        ctx.bse_interp_setup(co, 2, bse.SCHEME_M2, 1.0, bse.PREC_F32)
    assert err.value.code == bse.BSE_ERR_UNSUPPORTED
    co.free()
