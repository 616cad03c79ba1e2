"""The azimuthal DFTs of S2W_FP64_TC in each of their forms, against the float64 oracle.

Form 2 is the prime-factor tensor-core kernel (kernels_dftp.cu: 2L-1 = n1 n2, the n2-point
stage an exact sliced GEMM, the n1-point stage and the gamma DFT in compensated float32), form 1
the direct tensor-core GEMM, form 0 the compensated SIMT kernels.  Each is forced through
s2w_plan_set_dft_forms and the transform compared element by element with the oracle at the
float64 tolerance (1e-11): the spin SHT (forward on arbitrary samples, which pins the exact MW
operator, and inverse), and the wavelet transform whose scales carry several jobs per ring.
Sizes span every factorisation the kernel takes (n1 = 1 at L <= 32, 5 x 51 at L = 128, 7 x 73 at
L = 256), a last pass that is only partly filled, real and complex maps and spins.
"""
import numpy as np
import pytest

import synth
from oracle import harmonic, wavelet

pytestmark = pytest.mark.gpu
TOL = 1e-11


def rel(a, b):
    d = np.abs(np.asarray(a) - np.asarray(b)).max()
    s = np.abs(np.asarray(b)).max()
    return d / s if s > 0 else d   # a scale whose filter vanishes on l < L is all zero


def to_dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def force(lib, plan, k, form):
    try:
        plan.set_dft_forms(k, form, form)
    except lib.S2WError as e:
        if e.status == 5:
            pytest.skip(f"form {form} has no tables for transform {k} at this size")
        raise


@pytest.mark.parametrize("form", [2, 1, 0])
@pytest.mark.parametrize("L,spin,real,B", [(2, 0, True, 1), (5, 0, True, 3), (16, 1, False, 2), (24, 0, True, 2),
                                           (32, 2, False, 1), (128, 0, True, 3), (256, 0, True, 2)])
def test_sht_forms(lib, L, spin, real, B, form):
    plan = lib.Plan(L, 2, 2.0, 0, spin=spin, reality=real, batch=B, precision=lib.S2W_FP64_TC)
    force(lib, plan, 0, form)
    assert plan.dft_forms(0) == (form, form)
    rng = synth.rng_for(620, L)
    f = synth.pixels_random((B, L, 2 * L - 1), rng, complex_=not real)
    flm = plan.empty_flm()
    plan.sht_forward(to_dev(f), flm)
    got = flm.cpu().numpy()
    for b in range(B):
        ref = harmonic.sht_forward(f[b], L, spin)
        assert rel(got[b], ref[:, L - 1:] if real else ref) < TOL, b
    a = np.stack([synth.flm_random(L, rng, spin=spin, reality=real) for _ in range(B)])
    fd = plan.empty_map()
    plan.sht_inverse(to_dev(a[:, :, L - 1:] if real else a), fd)
    got = fd.cpu().numpy()
    for b in range(B):
        ref = harmonic.sht_inverse(a[b], L, spin)
        assert rel(got[b], ref.real if real else ref) < TOL, b
    plan.check()
    plan.close()


@pytest.mark.parametrize("form", [2, 1])
@pytest.mark.parametrize("L,N,J0,spin,real,B", [(32, 4, 0, 0, True, 2), (17, 3, 1, 0, True, 3), (16, 2, 1, 2, False, 1)])
def test_wavelet_forms(lib, L, N, J0, spin, real, B, form):
    plan = lib.Plan(L, N, 2.0, J0, spin=spin, reality=real, batch=B, precision=lib.S2W_FP64_TC)
    for k in range(plan.nscales + 2):
        try:
            plan.set_dft_forms(k, form, form)
        except lib.S2WError:
            pass   # that transform keeps its default form
    rng = synth.rng_for(621, L)
    a = [synth.flm_random(L, rng, spin=spin, reality=real) for _ in range(B)]
    f = np.stack([harmonic.sht_inverse(x, L, spin) for x in a])
    f = f.real if real else f
    wav, scal, f2 = plan.empty_wav(), plan.empty_scal(), plan.empty_map()
    plan.forward(to_dev(f), wav, scal)
    plan.inverse(wav, scal, f2)
    plan.check()
    for b in range(B):
        W_ref, Wp_ref = wavelet.analysis(f[b], L, N, 2.0, J0, spin, real)
        for s, w in enumerate(W_ref):
            assert rel(plan.scale_view(wav, s)[b].cpu().numpy(), w) < TOL, (b, s)
        assert rel(scal[b].cpu().numpy(), Wp_ref) < TOL
    assert rel(f2.cpu().numpy(), f) < TOL
    plan.close()


def test_headline_scales_prime_factor(lib, oracle_256):
    """The L = 256, N = 8, J0 = 2 workload (16 real maps) with the prime-factor DFTs on every
    transform that has them (the default): every wavelet scale of map 0 and of map 15 against the
    oracle, and the round trip of all 16 maps."""
    f, W_ref, Wp_ref = oracle_256
    L, N, lam, J0, B = 256, 8, 2.0, 2, 16
    plan = lib.Plan(L, N, lam, J0, reality=True, batch=B, precision=lib.S2W_FP64_TC)
    forms = [plan.dft_forms(k) for k in range(plan.nscales + 2)]
    assert forms[0] == (2, 2) and forms[-1] == (2, 2), forms   # the SHT and the top scale at 7 x 73
    wav, scal, f2 = plan.empty_wav(), plan.empty_scal(), plan.empty_map()
    plan.forward(to_dev(f), wav, scal)
    plan.inverse(wav, scal, f2)
    plan.check()
    for s, w in enumerate(W_ref):
        assert rel(plan.scale_view(wav, s)[0].cpu().numpy(), w) < TOL, s
    assert rel(scal[0].cpu().numpy(), Wp_ref) < TOL
    W15, Wp15 = wavelet.analysis(f[15], L, N, lam, J0, 0, True)
    for s, w in enumerate(W15):
        assert rel(plan.scale_view(wav, s)[15].cpu().numpy(), w) < TOL, s
    assert rel(f2.cpu().numpy(), f) < TOL
    plan.close()
