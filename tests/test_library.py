"""Host-side checks of the C ABI library (no GPU needed): it builds, loads and exports
every symbol that include/s2w.h declares."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    hdr = open(os.path.join(ROOT, "include", "s2w.h")).read()
    return sorted(set(re.findall(r"^(?:s2w_status|const char\s*\*)\s+(s2w_[a-z_0-9]+)\s*\(", hdr, re.M)))


@pytest.fixture(scope="module")
def built_lib():
    from paper_2402_01282_gb300 import _build
    if not os.path.exists(_build.LIB):
        _build.build()
    import paper_2402_01282_gb300 as s2w
    return s2w.load()


def test_exports_every_declared_symbol(built_lib):
    import paper_2402_01282_gb300 as s2w
    declared = _declared_symbols()
    assert declared, "no declarations found"
    for name in declared:
        assert hasattr(built_lib, name), f"{name} missing from libs2w.so"
    assert sorted(s2w.EXPORTS) == declared


def test_version_string(built_lib):
    assert b"sm_103a" in built_lib.s2w_version()


def test_invalid_params_rejected_without_gpu(built_lib):
    """Parameter validation runs before any CUDA call."""
    import ctypes
    import paper_2402_01282_gb300 as s2w
    h = ctypes.c_void_p()
    for bad in [dict(L=1, N=1), dict(L=8, N=9), dict(L=8, N=2, lam=1.0), dict(L=8, N=2, spin=8),
                dict(L=8, N=2, batch=0), dict(L=8, N=2, reality=1, spin=1), dict(L=8, N=2, J0=99)]:
        kw = dict(L=8, N=2, J0=0, spin=0, reality=0, batch=1, precision=0, precompute=0, lam=2.0)
        kw.update(bad)
        p = s2w.Params(kw["L"], kw["N"], kw["J0"], kw["spin"], kw["reality"], kw["batch"],
                       kw["precision"], kw["precompute"], kw["lam"])
        st = built_lib.s2w_plan_create(ctypes.byref(p), None, ctypes.byref(h))
        assert st == 1, (bad, st)
        assert h.value is None
        assert built_lib.s2w_last_error()
    assert built_lib.s2w_plan_destroy(None) == 1
    assert built_lib.s2w_forward(None, None, None, None, None) == 1


def test_no_cpu_fallback_when_library_missing(tmp_path):
    import paper_2402_01282_gb300 as s2w
    saved = s2w._lib
    s2w._lib = None
    try:
        with pytest.raises(RuntimeError):
            s2w.load(str(tmp_path / "missing.so"))
    finally:
        s2w._lib = saved
