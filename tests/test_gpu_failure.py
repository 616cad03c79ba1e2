"""Failure detection on the GPU without a GPU fault: the two device-side statuses that
s2w_check reports.

* S2W_ETIMEOUT: s2w_plan_inject_timeout makes the first bounded mbarrier wait of every
  tensor-core contraction launch wait on a barrier that nothing completes; the wait runs out
  after its poll limit, the kernel records the status, lets its own copies in flight land, frees
  its tensor memory and returns.  The test checks the status, then that the same plan computes
  the right result once the hook is off (the context stayed usable).
* S2W_ENONFINITE: in S2W_FP64_TC the exponent pass that reads every value before the slicing
  records a NaN or Inf; a map with one NaN pixel must be reported, a clean map must not.

Nothing here traps, faults or hangs the GPU: every wait involved is bounded.
"""
import numpy as np
import pytest

import synth
from oracle import wavelet

pytestmark = pytest.mark.gpu
TOL = 1e-11


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max()


def _map(L, B, seed):
    from oracle import harmonic
    return np.stack([harmonic.sht_inverse(synth.flm_random(L, synth.rng_for(seed, b), reality=True), L).real
                     for b in range(B)])


def test_injected_timeout_reports_and_recovers(lib):
    import torch
    L, N, J0, B = 24, 3, 1, 2
    plan = lib.Plan(L, N, 2.0, J0, reality=True, batch=B, precision=lib.S2W_FP64_TC)
    f = _map(L, B, 610)
    fd = torch.from_numpy(f).cuda()
    wav, scal = plan.empty_wav(), plan.empty_scal()
    plan.inject_timeout(True)
    plan.forward(fd, wav, scal)
    with pytest.raises(lib.S2WError) as ei:
        plan.check()
    assert ei.value.status == 4, str(ei.value)          # S2W_ETIMEOUT
    plan.check()                                         # the word was cleared by the read
    plan.inject_timeout(False)
    plan.forward(fd, wav, scal)
    plan.check()
    W_ref, Wp_ref = wavelet.analysis(f[0], L, N, 2.0, J0, 0, True)
    for s, w in enumerate(W_ref):
        assert rel(plan.scale_view(wav, s)[0].cpu().numpy(), w) < TOL
    assert rel(scal[0].cpu().numpy(), Wp_ref) < TOL
    # the synthesis path (forward contractions) takes the same timeout path
    f2 = plan.empty_map()
    plan.inject_timeout(True)
    plan.inverse(wav, scal, f2)
    with pytest.raises(lib.S2WError) as ei:
        plan.check()
    assert ei.value.status == 4
    plan.inject_timeout(False)
    plan.inverse(wav, scal, f2)
    plan.check()
    assert rel(f2.cpu().numpy(), f) < TOL
    plan.close()


@pytest.mark.parametrize("value", [float("nan"), float("inf")])
def test_nonfinite_input_is_reported(lib, value):
    import torch
    L, N, J0, B = 32, 4, 1, 3
    plan = lib.Plan(L, N, 2.0, J0, reality=True, batch=B, precision=lib.S2W_FP64_TC)
    f = _map(L, B, 611)
    bad = f.copy()
    bad[1, 7, 13] = value
    wav, scal = plan.empty_wav(), plan.empty_scal()
    plan.forward(torch.from_numpy(bad).cuda(), wav, scal)
    with pytest.raises(lib.S2WError) as ei:
        plan.check()
    assert ei.value.status == 6, str(ei.value)          # S2W_ENONFINITE
    plan.forward(torch.from_numpy(f).cuda(), wav, scal)
    plan.check()                                         # a clean map reports nothing
    # a non-finite wavelet coefficient is caught on the synthesis side too
    wbad = wav.clone()
    wbad[2, wbad.shape[1] // 2] = value
    f2 = plan.empty_map()
    plan.inverse(wbad, scal, f2)
    with pytest.raises(lib.S2WError) as ei:
        plan.check()
    assert ei.value.status == 6
    plan.close()


@pytest.mark.parametrize("value", [float("nan"), float("inf")])
@pytest.mark.parametrize("mode", [1, 2])   # S2W_FP32_SPLIT, S2W_BF16
def test_reduced_modes_report_nonfinite_input(lib, mode, value):
    """The reduced modes run their SHT on the sliced float64-accurate kernels, whose exponent
    pass reads every input value: a non-finite pixel is reported, and a clean map is not.  A
    non-finite wavelet coefficient passes the reduced-precision scale as a non-finite value (the
    integer float64 <-> float32 conversions carry Inf and NaN over) and is reported by the
    exponent pass of the final inverse SHT."""
    import torch
    L, N, J0, B = 32, 4, 1, 2
    plan = lib.Plan(L, N, 2.0, J0, reality=True, batch=B, precision=mode)
    f = _map(L, B, 612)
    bad = f.copy()
    bad[1, 5, 9] = value
    wav, scal = plan.empty_wav(), plan.empty_scal()
    plan.forward(torch.from_numpy(bad).cuda(), wav, scal)
    with pytest.raises(lib.S2WError) as ei:
        plan.check()
    assert ei.value.status == 6, str(ei.value)
    plan.forward(torch.from_numpy(f).cuda(), wav, scal)
    plan.check()
    wbad = wav.clone()
    wbad[0, wbad.shape[1] - 5] = value   # the top wavelet scale of map 0
    f2 = plan.empty_map()
    plan.inverse(wbad, scal, f2)
    with pytest.raises(lib.S2WError) as ei:
        plan.check()
    assert ei.value.status == 6, str(ei.value)
    plan.inverse(wav, scal, f2)
    plan.check()
    plan.close()
