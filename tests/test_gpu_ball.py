"""GPU parity of the ball transforms (Fourier-Laguerre radial transform, Eqs. 6-8, and the
spherical-Laguerre transform Z, Eqs. 9-11) against the float64 oracle."""
import numpy as np
import pytest

import synth
from oracle import harmonic, laguerre

pytestmark = pytest.mark.gpu
TOL = 1e-11
# S2W_FP64 (compensated SIMT radial maps), S2W_FP64_NATIVE, and the tensor-core modes, whose radial
# maps run as exact sliced GEMMs on the tensor cores (float64-accurate; the spin SHT is float64-
# accurate in every mode, so the whole transform is held to 1e-11 in all of them)
MODES = [0, 3, 4, 1, 2]


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max()


def to_dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("P,tau", [(8, 1.0), (33, 0.7), (128, 1.0), (150, 2.5)])
def test_nodes_and_weights(lib, P, tau):
    plan = lib.BallPlan(4, P, tau, batch=1)
    r, om = plan.nodes()
    r_ref, om_ref, _ = laguerre.quadrature(P, tau)
    assert np.abs(r - r_ref).max() / r_ref.max() < 1e-13
    assert np.abs(om / om_ref - 1).max() < 1e-12
    plan.close()


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("L,P,tau,B,real", [(8, 8, 1.0, 2, True), (17, 33, 0.7, 1, False), (5, 128, 1.0, 3, True)])
def test_radial_parity(lib, L, P, tau, B, real, mode):
    plan = lib.BallPlan(L, P, tau, reality=real, batch=B, precision=mode)
    rng = synth.rng_for(700, P)
    x = synth.pixels_random((B, P, L, plan.Mc), rng, complex_=True)
    out = plan.empty_coeffs()
    plan.laguerre_forward(to_dev(x), out)
    got = out.cpu().numpy()
    for b in range(B):
        assert rel(got[b], laguerre.radial_forward(x[b], P, tau)) < TOL
    plan.laguerre_inverse(to_dev(x), out)
    got = out.cpu().numpy()
    for b in range(B):
        assert rel(got[b], laguerre.radial_inverse(x[b], P, tau)) < TOL
    plan.close()


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("L,P,real,B", [(12, 10, True, 2), (9, 7, False, 1)])
def test_spherical_laguerre_parity(lib, L, P, real, B, mode):
    plan = lib.BallPlan(L, P, 1.0, reality=real, batch=B, precision=mode)
    flmp = [synth.flmp_random(L, P, synth.rng_for(701, b), reality=real) for b in range(B)]
    f = np.stack([laguerre.spherical_laguerre_inverse(x, L, P) for x in flmp])
    if real:
        f = f.real
    out = plan.empty_coeffs()
    plan.sl_forward(to_dev(f), out)
    got = out.cpu().numpy()
    for b in range(B):
        ref = laguerre.spherical_laguerre_forward(f[b], L, P)
        ref = ref[:, :, L - 1:] if real else ref
        assert rel(got[b], ref) < TOL
    pix = plan.empty_pixels()
    cin = np.stack([x[:, :, L - 1:] if real else x for x in flmp])
    plan.sl_inverse(to_dev(cin), pix)
    got = pix.cpu().numpy()
    for b in range(B):
        assert rel(got[b], f[b]) < TOL
    plan.close()


@pytest.mark.parametrize("mode", [0, 4])
def test_ball_full_size_128(lib, mode):
    """The L = P = 128 real ball field: Z^-1 then Z recovers f_lmp, and the radial step of one
    angular column block matches the oracle."""
    L, P = 128, 128
    plan = lib.BallPlan(L, P, 1.0, reality=True, batch=1, precision=mode)
    flmp = synth.flmp_random(L, P, synth.rng_for(5, 0), reality=True)[None, :, :, L - 1:]
    pix = plan.empty_pixels()
    plan.sl_inverse(to_dev(flmp), pix)
    out = plan.empty_coeffs()
    plan.sl_forward(pix, out)
    assert rel(out.cpu().numpy(), flmp) < TOL
    x = synth.pixels_random((1, P, L, plan.Mc), synth.rng_for(702, 0), complex_=True)
    plan.laguerre_forward(to_dev(x), out)
    got = out.cpu().numpy()[0][:, :8]
    assert rel(got, laguerre.radial_forward(x[0][:, :8], P, 1.0)) < TOL
    plan.close()
