"""Failure detection on the GPU without a fault: a bounded wait that runs out.

The tensor-core K_c apply waits on mbarriers for its TMA loads, its MMAs and
its epilogue, each wait bounded by a clock-cycle budget.  A testing aid
(bse_ctx_set_wait_limit) shortens that budget to one cycle, which no TMA load
meets: the kernel's first wait gives up, the kernel raises its status bit,
drains the copies and MMAs it has in flight under the default budget, frees
its tensor memory and returns.  The call must report BSE_ERR_TIMEOUT naming
the K_c apply, and with the default budget restored the same context must
give the normal result again, bit for bit, and run a Haydock recursion."""
import numpy as np
import pytest

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


def test_kc_apply_wait_gives_up_and_context_recovers(ctx):
    from paper_1602_01863_gb300 import bse
    m = synth.draw_model(61, 3, 3)
    co = ctx.bse_build_coarse(m, 6, bse.PREC_BF16)
    it = ctx.bse_interp_setup(co, 2, bse.SCHEME_M3, 1.0, bse.PREC_F32)
    x = torch.from_numpy(synth.random_vectors(4, (3, it.N)).astype(np.complex64)).cuda()
    y0 = torch.empty_like(x)
    ctx.bse_apply_h(it, 3, x.data_ptr(), y0.data_ptr())
    ref = y0.cpu().numpy()
    ctx.bse_ctx_set_wait_limit(1)
    y1 = torch.empty_like(x)
    with pytest.raises(bse.BseError) as err:
        ctx.bse_apply_h(it, 3, x.data_ptr(), y1.data_ptr())
    assert err.value.code == bse.BSE_ERR_TIMEOUT and "K_c apply" in str(err.value)
    with pytest.raises(bse.BseError) as err:                       # the same inside a Haydock run (graph)
        ctx.bse_haydock_run([it], [3], synth.POL3, 5, bse.USE_GRAPH)
    assert err.value.code == bse.BSE_ERR_TIMEOUT
    ctx.bse_ctx_set_wait_limit(0)
    y2 = torch.empty_like(x)
    ctx.bse_apply_h(it, 3, x.data_ptr(), y2.data_ptr())
    assert np.array_equal(y2.cpu().numpy(), ref)
    a, b, pn2, st, rc = ctx.bse_haydock_run([it], [3], synth.POL3, 20, bse.USE_GRAPH)
    a2, b2, _, _, _ = ctx.bse_haydock_run([it], [3], synth.POL3, 20, 0)
    assert rc == 0 and np.all(st == 20) and np.array_equal(a, a2) and np.all(np.isfinite(b))
    with pytest.raises(bse.BseError) as err:
        ctx.bse_ctx_set_wait_limit(-5)
    assert err.value.code == bse.BSE_ERR_ARG
    it.free()
    co.free()
