"""bse_apply_h_noalloc against bse_apply_h, through the C ABI.

bse_apply_h_noalloc is for callers that cannot call cudaMalloc once their
work is under way (for example a framework that hands all device memory out
of its own pool, or a loop where cudaMalloc's implicit synchronisation is
forbidden): it takes its scratch from a fixed 32 MiB device array inside the
library instead of the handle.  These tests check that it gives the same
y = H x as bse_apply_h on two calls in a row, with a call on another system in
between (the array keeps the previous call's contents, so this also checks that
stale data is cleared), that those calls change the device's free memory by
nothing, and that a size whose scratch does not fit is refused with a clear
error.

This file is collected last on purpose.
"""
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


def _run(ctx, it, x, noalloc):
    dt = torch.complex128 if it.vec_prec == 0 else torch.complex64
    xs = torch.from_numpy(np.ascontiguousarray(x)).to(dt).cuda()
    ys = torch.full_like(xs, complex(float("nan"), float("nan")))
    fn = ctx.bse_apply_h_noalloc if noalloc else ctx.bse_apply_h
    fn(it, x.shape[0], xs.data_ptr(), ys.data_ptr())
    torch.cuda.synchronize()
    return ys.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("case", [
    # FP64 plain path, Method 3 (near-field pieces in the static array), 2 vectors
    dict(seed=1, nv=3, nc=3, n=4, nd=2, scheme=1, kc=0, vec=0, nvec=2, rtol=1e-12),
    # mixed path: BF16 K_c on the tensor cores (operand + tile partials), ragged tiles, 3 vectors
    dict(seed=8, nv=3, nc=3, n=6, nd=1, scheme=0, kc=2, vec=1, nvec=3, rtol=1e-6),
    # the benchmark's path: BF16 K_c, FP32 vectors, Method 3 on the tensor-core
    # near field (the X / U pieces in the static array), 3 vectors
    dict(seed=9, nv=3, nc=3, n=4, nd=2, scheme=1, kc=2, vec=1, nvec=3, rtol=1e-5),
])
def test_noalloc_matches_apply_h_twice(ctx, case):
    m = synth.draw_model(case["seed"], case["nv"], case["nc"])
    co = ctx.bse_build_coarse(m, case["n"], case["kc"])
    it = ctx.bse_interp_setup(co, case["nd"], case["scheme"], 1.0, case["vec"])
    # a differently sized system whose no-allocation call fills the shared
    # array with other contents between the two calls under test
    mo = synth.draw_model(case["seed"] + 100, 2, 2)
    coo = ctx.bse_build_coarse(mo, 3, case["kc"])
    ito = ctx.bse_interp_setup(coo, 2, case["scheme"], 1.0, case["vec"])
    xo = synth.random_vectors(23, (2, ito.N))
    x1 = synth.random_vectors(21, (case["nvec"], it.N))
    x2 = synth.random_vectors(22, (case["nvec"], it.N))
    refs = [_run(ctx, it, x, noalloc=False) for x in (x1, x2)]
    _run(ctx, ito, xo, noalloc=True)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for x, ref in zip((x1, x2), refs):                    # two calls in a row, different inputs
        got = _run(ctx, it, x, noalloc=True)
        assert np.all(np.isfinite(got))
        assert np.abs(got - ref).max() <= case["rtol"] * np.abs(ref).max()
        _run(ctx, ito, xo, noalloc=True)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0         # nothing was allocated on the device
    ito.free()
    coo.free()
    it.free()
    co.free()


def test_noalloc_rejects_sizes_beyond_the_static_array(ctx):
    from paper_1602_01863_gb300 import bse
    m = synth.draw_model(3, 4, 4)
    co = ctx.bse_build_coarse(m, 6, bse.PREC_F64)
    it = ctx.bse_interp_setup(co, 3, bse.SCHEME_M3, 1.0, bse.PREC_F64)     # M3 pieces: ~95 MB for 4 vectors
    x = torch.zeros((4, it.N), dtype=torch.complex128, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(bse.BseError) as e:
        ctx.bse_apply_h_noalloc(it, 4, x.data_ptr(), y.data_ptr())
    assert e.value.code == bse.BSE_ERR_UNSUPPORTED and "static array" in str(e.value)
    it.free()
    co.free()
