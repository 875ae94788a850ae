"""Host-side checks of the C ABI: the library builds, loads and exports every
symbol include/bse.h declares; the binding refuses to run without it."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bse.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bse_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def built_lib():
    from paper_1602_01863_gb300 import build as b
    if not os.path.exists(b.LIB_PATH):
        b.build()
    return ctypes.CDLL(b.LIB_PATH)


def test_header_declares_the_paper_level_calls():
    names = declared_functions()
    for f in ("bse_build_coarse", "bse_interp_setup", "bse_haydock_run", "bse_spectrum"):
        assert f in names


def test_library_exports_every_declared_symbol(built_lib):
    for name in declared_functions():
        assert hasattr(built_lib, name), name


def test_binding_names_match_header():
    from paper_1602_01863_gb300 import bse
    assert sorted(bse.EXPORTED) == declared_functions()


def test_missing_library_fails_loudly(tmp_path):
    from paper_1602_01863_gb300 import bse
    saved = bse._lib
    bse._lib = None
    try:
        with pytest.raises(RuntimeError, match="not built"):
            bse.load(str(tmp_path / "nope.so"))
    finally:
        bse._lib = saved


def test_version_and_context_without_gpu(built_lib):
    """bse_version needs no device; bse_ctx_create reports BSE_ERR_CUDA (-3)
    when no CUDA device is visible instead of falling back to the CPU."""
    assert built_lib.bse_version() >= 10000
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    rc = built_lib.bse_ctx_create(ctypes.byref(h), 0, None)
    assert rc == -3 and not h.value


def test_model_struct_layout():
    from paper_1602_01863_gb300 import bse, synth
    m = synth.draw_model(0, 3, 2)
    s, keep = bse.model_struct(m)
    assert s.nv == 3 and s.nc == 2 and s.direct_shells == 27
    assert keep[3].size == 2 * 7 * 26 * 3 * 2 and keep[4].size == 2 * 7 * 3 * 3 * 2


def test_null_arguments_are_rejected_on_the_host(built_lib):
    """Corrupt arguments (NULL handles and outputs) come back as BSE_ERR_ARG
    (-1) from every entry point before any device call, so these checks run
    without a GPU."""
    lib = built_lib
    P, N = ctypes.c_void_p, None
    dummy = (ctypes.c_double * 8)()
    idummy = (ctypes.c_int * 8)()
    lldummy = (ctypes.c_longlong * 8)()
    calls = {
        "bse_ctx_create": lambda: lib.bse_ctx_create(N, 0, N),
        "bse_build_coarse": lambda: lib.bse_build_coarse(N, N, 4, 0, N, N),
        "bse_coarse_get_kc": lambda: lib.bse_coarse_get_kc(N, N, dummy),
        "bse_interp_setup": lambda: lib.bse_interp_setup(N, N, 2, 0, ctypes.c_double(1.0), 0, N, N),
        "bse_set_stop_rule": lambda: lib.bse_set_stop_rule(N, ctypes.c_double(0.01), 10, ctypes.c_double(1.0),
                                                           ctypes.c_double(0.1), 4, dummy),
        "bse_interp_info": lambda: lib.bse_interp_info(N, lldummy),
        "bse_interp_kc_plan": lambda: lib.bse_interp_kc_plan(N, idummy),
        "bse_ctx_set_wait_limit": lambda: lib.bse_ctx_set_wait_limit(N, ctypes.c_longlong(0)),
        "bse_dipoles": lambda: lib.bse_dipoles(N, N, 1, dummy, N, dummy),
        "bse_apply_h": lambda: lib.bse_apply_h(N, N, 1, N, N),
        "bse_apply_h_noalloc": lambda: lib.bse_apply_h_noalloc(N, N, 1, N, N),
        "bse_haydock_run": lambda: lib.bse_haydock_run(N, N, 1, idummy, dummy, 4, 0, dummy, dummy, dummy, idummy),
        "bse_last_kernel_times": lambda: lib.bse_last_kernel_times(N, dummy, lldummy),
        "bse_spectrum": lambda: lib.bse_spectrum(N, 1, 4, idummy, dummy, dummy, dummy, ctypes.c_double(1.0),
                                                 ctypes.c_double(0.1), 4, dummy, dummy),
    }
    for name, call in calls.items():
        assert call() == -1, name
