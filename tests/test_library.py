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
                dict(L=8, N=2, batch=0), dict(L=8, N=2, reality=1, spin=1), dict(L=8, N=2, J0=99),
                dict(L=8, N=2, sampling=2), dict(L=8, N=2, sampling=-1)]:
        kw = dict(L=8, N=2, J0=0, spin=0, reality=0, batch=1, precision=0, precompute=0, lam=2.0, sampling=0)
        kw.update(bad)
        p = s2w.Params(kw["L"], kw["N"], kw["J0"], kw["spin"], kw["reality"], kw["batch"],
                       kw["precision"], kw["precompute"], kw["lam"], kw["sampling"])
        st = built_lib.s2w_plan_create(ctypes.byref(p), None, ctypes.byref(h))
        assert st == 1, (bad, st)
        assert h.value is None
        assert built_lib.s2w_last_error()
    assert built_lib.s2w_plan_destroy(None) == 1
    assert built_lib.s2w_forward(None, None, None, None, None) == 1
    # the runtime queries on a NULL plan
    a, b, c = ctypes.c_int(7), ctypes.c_int(7), ctypes.c_int(7)
    assert built_lib.s2w_plan_launch_shapes(None, 0, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)) == 1
    assert built_lib.s2w_plan_dft_forms(None, 0, ctypes.byref(a), ctypes.byref(b)) == 1
    assert (a.value, b.value) == (7, 7)   # outputs untouched on error
    t, w = ctypes.c_int64(7), ctypes.c_int64(7)
    assert built_lib.s2w_plan_device_bytes(None, ctypes.byref(t), ctypes.byref(w)) == 1
    assert (t.value, w.value) == (7, 7)
    assert built_lib.s2w_plan_inject_timeout(None, 1) == 1
    assert built_lib.s2w_plan_set_dft_forms(None, 0, -1, -1) == 1
    assert built_lib.s2w_check(None) == 1
    # Driscoll-Healy above its supported band-limit: unsupported, still before any CUDA call
    p = s2w.Params(600, 2, 0, 0, 0, 1, 0, 0, 2.0, s2w.S2W_SAMPLING_DH)
    assert built_lib.s2w_plan_create(ctypes.byref(p), None, ctypes.byref(h)) == 5
    # the sliced tensor-core mode beyond K = 512 reduction terms (L > 512, or more than 512 rings)
    for L, smp in ((600, s2w.S2W_SAMPLING_MW), (300, s2w.S2W_SAMPLING_DH)):
        p = s2w.Params(L, 2, 0, 0, 0, 1, s2w.S2W_FP64_TC, 0, 2.0, smp)
        assert built_lib.s2w_plan_create(ctypes.byref(p), None, ctypes.byref(h)) == 5
    # an unknown precision mode
    p = s2w.Params(8, 2, 0, 0, 0, 1, 7, 0, 2.0, 0)
    assert built_lib.s2w_plan_create(ctypes.byref(p), None, ctypes.byref(h)) == 1


def test_param_structs_match_header(tmp_path):
    """The ctypes mirrors of the three parameter structs have the C layout (sizes and the
    offset of their last field), checked against a host program compiled from the header."""
    import ctypes
    import subprocess
    import paper_2402_01282_gb300 as s2w
    src = tmp_path / "layout.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "s2w.h"\n'
                   'int main(void) {\n'
                   '  printf("%zu %zu\\n", sizeof(s2w_params), offsetof(s2w_params, sampling));\n'
                   '  printf("%zu %zu\\n", sizeof(s2w_ball_params), offsetof(s2w_ball_params, sampling));\n'
                   '  printf("%zu %zu\\n", sizeof(s2w_ball_wav_params), offsetof(s2w_ball_wav_params, sampling));\n'
                   '  return 0;\n}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [tuple(int(v) for v in line.split()) for line in subprocess.run(
        [str(exe)], check=True, capture_output=True, text=True).stdout.split("\n") if line]
    for (size, off), cls in zip(got, [s2w.Params, s2w.BallParams, s2w.BallWavParams]):
        assert ctypes.sizeof(cls) == size, cls
        assert cls.sampling.offset == off, cls


def test_no_cpu_fallback_when_library_missing(tmp_path):
    import paper_2402_01282_gb300 as s2w
    saved = s2w._lib
    s2w._lib = None
    try:
        with pytest.raises(RuntimeError):
            s2w.load(str(tmp_path / "missing.so"))
    finally:
        s2w._lib = saved
