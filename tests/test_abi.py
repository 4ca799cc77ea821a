"""The C-ABI library loads and exports every symbol include/krpls.h declares
(no compute calls: runs without a GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "include", "krpls.h")


def declared_symbols():
    txt = open(HDR).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(krp_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def built_lib():
    from paper_2301_12584_gb300 import build as B
    if not os.path.exists(os.path.join(ROOT, "paper_2301_12584_gb300", "libkrpls.so")):
        B.build()
    return os.path.join(ROOT, "paper_2301_12584_gb300", "libkrpls.so")


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ["krp_create", "krp_destroy", "krp_set_factor", "krp_sample", "krp_gather", "krp_solve_dense",
              "krp_sptensor_create", "krp_solve_sparse", "krp_cp_als_sweep", "krp_sync_status"]:
        assert s in syms


def test_library_exports_every_declared_symbol(built_lib):
    out = subprocess.run(["nm", "-D", "--defined-only", built_lib], capture_output=True, text=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if l.strip())
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing


def test_binding_covers_every_symbol_and_loads(built_lib):
    from paper_2301_12584_gb300 import krpls
    L = krpls.lib()
    bound = {n for n, _, _ in krpls.SIGNATURES}
    assert set(declared_symbols()) <= bound
    for n in bound:
        assert hasattr(L, n)


def test_host_argument_checks_without_gpu(built_lib):
    """krp_create rejects bad arguments before touching the device."""
    import ctypes as C
    from paper_2301_12584_gb300 import krpls
    L = krpls.lib()
    h = C.c_void_p()
    I = (C.c_int64 * 3)(64, 64, 64)
    assert L.krp_create(C.byref(h), 3, I, 0, 0, 0, None) == krpls.KRP_EINVAL      # R = 0
    assert L.krp_create(C.byref(h), 3, I, 129, 0, 0, None) == krpls.KRP_EINVAL    # R > 128
    assert L.krp_create(C.byref(h), 0, I, 8, 0, 0, None) == krpls.KRP_EINVAL      # N = 0
    assert L.krp_create(C.byref(h), 3, I, 8, 100, 0, None) == krpls.KRP_EINVAL    # F > 4R
    assert L.krp_create(C.byref(h), 3, I, 8, 0, 7, None) == krpls.KRP_EINVAL      # precision
    assert L.krp_create(None, 3, I, 8, 0, 0, None) == krpls.KRP_EINVAL
    assert L.krp_create(C.byref(h), 17, (C.c_int64 * 17)(*([8] * 17)), 8, 0, 0, None) == krpls.KRP_EINVAL  # N > 16
    assert L.krp_create(C.byref(h), 3, (C.c_int64 * 3)(64, 0, 64), 8, 0, 0, None) == krpls.KRP_EINVAL    # I_k = 0
    assert L.krp_create(C.byref(h), 3, (C.c_int64 * 3)(64, 1 << 31, 64), 8, 0, 0, None) == krpls.KRP_EINVAL
    assert L.krp_create(C.byref(h), 3, None, 8, 0, 0, None) == krpls.KRP_EINVAL                          # I_host
    assert L.krp_create(C.byref(h), 3, I, 8, -1, 0, None) == krpls.KRP_EINVAL                            # F < 0
    assert h.value is None
    # other entry points reject a NULL handle or output before any device work
    assert L.krp_set_descent_form(None, 0) == krpls.KRP_EINVAL
    assert L.krp_sample(None, -1, 16, 1, 0, None, None, None, None) != krpls.KRP_OK
    assert L.krp_get_factor(None, 0, None, 0) == krpls.KRP_EINVAL
    assert b"R" in L.krp_last_error(None) or L.krp_last_error(None)
