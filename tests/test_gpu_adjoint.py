"""Adjoints on the GPU (s2w_forward_adjoint, s2w_inverse_adjoint; Sec. 4.3) against the oracle.

* Tiny band-limits, element by element against oracle.adjoint (the conjugate transposes of
  the oracle's analysis and synthesis matrices), every precision mode:
  max|x - x_ref| / max|x_ref| <= 1e-11 (the adjoints are float64-accurate in every mode).
* The L = 256, N = 8, J0 = 2 workload in the benchmark's launch configuration (16 maps):
  <gW, A f> = <A^H gW, f> with f and A f from the oracle, and, for band-limited maps x,
  <S^H y, A x> = <y, S A x> = <y, x> (exact reconstruction), each within 1e-11 of the
  Cauchy-Schwarz bound.
* The differentiation study (L = 512, N = 4, lambda = 2, J0 = 3, 8 real maps, loss
  sum_j mean |W^j|^2): the autograd gradient against central finite differences (h = 1e-6)
  of the loss evaluated with the library's analysis.
* Autograd at tiny L: the same loss's gradient against the oracle gradient 2 A^H W / n, and
  torch.autograd.gradcheck of both Functions.
"""
import functools

import numpy as np
import pytest

import synth
from oracle import adjoint, harmonic, wavelet

pytestmark = pytest.mark.gpu
TOL = 1e-11
MODES = [0, 3, 1, 2, 4]   # S2W_FP64, S2W_FP64_NATIVE, S2W_FP32_SPLIT, S2W_BF16, S2W_FP64_TC
CASES = [  # L, N, lam, J0, spin, real, B
    (8, 3, 2.0, 0, 0, True, 2),
    (8, 2, 2.0, 1, 2, False, 1),
    (7, 3, 1.7, 0, 0, True, 1),
    (6, 1, 2.0, 0, 0, True, 1),
    (5, 5, 2.0, 0, 1, False, 2),
]


def rel(a, b):
    d = np.abs(np.asarray(a) - np.asarray(b)).max()
    s = np.abs(np.asarray(b)).max()
    return d / s if s > 0 else d


def to_dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def inner(u, v):
    return float(np.real(np.vdot(np.asarray(u).ravel(), np.asarray(v).ravel())))


@functools.lru_cache(maxsize=None)
def matrices(L, N, lam, J0, spin, real):
    return (adjoint.analysis_matrix(L, N, lam, J0, spin, real),
            adjoint.synthesis_matrix(L, N, lam, J0, spin, real))


def split_wav(plan, wav_row):
    return [wav_row[plan.wav_offsets[s]:plan.wav_offsets[s + 1]].reshape(plan.scale_shape(s))
            for s in range(plan.nscales)]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("L,N,lam,J0,spin,real,B", CASES)
def test_forward_adjoint_parity(lib, L, N, lam, J0, spin, real, B, mode):
    plan = lib.Plan(L, N, lam, J0, spin=spin, reality=real, batch=B, precision=mode)
    A, _ = matrices(L, N, lam, J0, spin, real)
    rng = synth.rng_for(910, L)
    gw = synth.pixels_random((B, plan.wav_elems), rng, complex_=not real)
    gp = synth.pixels_random((B, plan.L_phi, 2 * plan.L_phi - 1), rng, complex_=not real)
    gf = plan.empty_map()
    plan.forward_adjoint(to_dev(gw), to_dev(gp), gf)
    plan.check()
    got = gf.cpu().numpy()
    for b in range(B):
        ref = adjoint.analysis_adjoint(split_wav(plan, gw[b]), gp[b], L, N, lam, J0, spin, real, matrix=A)
        assert rel(got[b], ref) < TOL, (b, rel(got[b], ref))


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("L,N,lam,J0,spin,real,B", CASES)
def test_inverse_adjoint_parity(lib, L, N, lam, J0, spin, real, B, mode):
    plan = lib.Plan(L, N, lam, J0, spin=spin, reality=real, batch=B, precision=mode)
    _, S = matrices(L, N, lam, J0, spin, real)
    rng = synth.rng_for(911, L)
    gf = synth.pixels_random((B, L, 2 * L - 1), rng, complex_=not real)
    gw, gp = plan.empty_wav(), plan.empty_scal()
    plan.inverse_adjoint(to_dev(gf), gw, gp)
    plan.check()
    gw, gp = gw.cpu().numpy(), gp.cpu().numpy()
    for b in range(B):
        ref_w, ref_p = adjoint.synthesis_adjoint(gf[b], L, N, lam, J0, spin, real, matrix=S)
        got_w = split_wav(plan, gw[b])
        for s in range(plan.nscales):
            assert rel(got_w[s], ref_w[s]) < TOL, (b, s)
        assert rel(gp[b], ref_p) < TOL


def test_adjoints_full_size_256(lib, oracle_256):
    """The benchmark workload: 16 real maps at L = 256, N = 8, lambda = 2, J0 = 2."""
    import torch
    f, W_ref, Wp_ref = oracle_256
    L, N, lam, J0, B = 256, 8, 2.0, 2, 16
    plan = lib.Plan(L, N, lam, J0, reality=True, batch=B, precision=0)
    rng = synth.rng_for(912, 0)
    gw = synth.pixels_random((B, plan.wav_elems), rng)
    gp = synth.pixels_random((B, plan.L_phi, 2 * plan.L_phi - 1), rng)
    gf = plan.empty_map()
    plan.forward_adjoint(to_dev(gw), to_dev(gp), gf)
    plan.check()
    gf0 = gf[0].cpu().numpy()
    lhs = sum(inner(g, w) for g, w in zip(split_wav(plan, gw[0]), W_ref)) + inner(gp[0], Wp_ref)
    bound = np.sqrt(np.sum(gw[0] ** 2) + np.sum(gp[0] ** 2)) * \
        np.sqrt(sum(np.sum(np.abs(w) ** 2) for w in W_ref) + np.sum(np.abs(Wp_ref) ** 2))
    assert abs(lhs - inner(gf0, f[0])) < TOL * bound
    # synthesis adjoint through exact reconstruction, every map of the batch
    x = torch.from_numpy(f).cuda()
    wav, scal = plan.empty_wav(), plan.empty_scal()
    plan.forward(x, wav, scal)
    y = synth.pixels_random((B, L, 2 * L - 1), rng)
    sw, sp = plan.empty_wav(), plan.empty_scal()
    plan.inverse_adjoint(to_dev(y), sw, sp)
    plan.check()
    lhs = (sw * wav).sum(dim=(1,)) + (sp * scal).sum(dim=(1, 2))
    rhs = (to_dev(y) * x).sum(dim=(1, 2))
    norms = torch.sqrt((sw ** 2).sum(1) + (sp ** 2).sum((1, 2))) * torch.sqrt((wav ** 2).sum(1) + (scal ** 2).sum((1, 2)))
    assert float(((lhs - rhs).abs() / norms).max()) < TOL


def test_loss_gradient_differentiation_study(lib):
    """L = 512, N = 4, lambda = 2, J0 = 3, 8 real maps; loss = sum_j mean |W^j|^2 (Sec. 4.3).

    The loss is quadratic in the pixels, so the central difference (L(f + h v) - L(f - h v)) / 2h
    equals the directional derivative for every h, and h can be chosen so that the loss's own
    rounding (relative ~1e-13, the transforms' float64 class) stays far below the difference:
    h = 0.5 along band-limited directions of the map's own size, h = 1e3 along single pixels (the
    difference grows like h, the rounding of L(f +- h e_p) like h^2 Q_pp, which balance near
    h^2 ~ L / Q_pp).  Both must agree with the adjoint's gradient to 1e-9.  The inner-product
    identity <A^H A v, v> = ||A v||^2 is checked to 1e-12 at the same size."""
    import torch
    from paper_2402_01282_gb300 import autograd
    L, N, lam, J0, B = 512, 4, 2.0, 3, 8
    plan = lib.Plan(L, N, lam, J0, reality=True, batch=B, precision=0)
    flm = np.stack([synth.flm_random(L, synth.rng_for(4, b), reality=True)[:, L - 1:] for b in range(B)])
    f = plan.empty_map()
    plan.sht_inverse(to_dev(flm), f)

    def loss_of(x):
        wav, _ = autograd.analysis(x, plan)
        return sum((plan.scale_view(wav, s) ** 2).mean(dim=(1, 2, 3)).sum() for s in range(plan.nscales))

    x = f.clone().requires_grad_(True)
    (grad,) = torch.autograd.grad(loss_of(x), x)
    with torch.no_grad():
        for k in range(3):   # seeded band-limited directions
            vl = np.stack([synth.flm_random(L, synth.rng_for(4, 100 + 8 * k + b), reality=True)[:, L - 1:]
                           for b in range(B)])
            v = plan.empty_map()
            plan.sht_inverse(to_dev(vl), v)
            fd = float(loss_of(f + 0.5 * v) - loss_of(f - 0.5 * v))
            an = float((grad * v).sum())
            assert abs(fd - an) <= 1e-9 * abs(an), (k, fd, an)
        rng = synth.rng_for(4, 200)
        pix = [(int(rng.integers(B)), int(rng.integers(L)), int(rng.integers(2 * L - 1))) for _ in range(32)]
        fdp, gp = [], []
        for (b, t, p) in pix:
            e = torch.zeros_like(f)
            e[b, t, p] = 1e3
            fdp.append(float(loss_of(f + e) - loss_of(f - e)) / 2e3)
            gp.append(float(grad[b, t, p]))
        err = max(abs(a - c) for a, c in zip(fdp, gp)) / max(abs(c) for c in gp)
        assert err <= 1e-9, err
        # <A^H (A v), v> = ||A v||^2
        v = to_dev(synth.pixels_random((B, L, 2 * L - 1), synth.rng_for(4, 302)))
        wav, scal = plan.empty_wav(), plan.empty_scal()
        plan.forward(v, wav, scal)
        g2 = plan.empty_map()
        plan.forward_adjoint(wav, scal, g2)
        lhs = float((g2 * v).sum())
        rhs = float((wav ** 2).sum() + (scal ** 2).sum())
        assert abs(lhs - rhs) <= 1e-12 * rhs, (lhs, rhs)
    plan.check()


@pytest.mark.parametrize("L,N,lam,J0,spin,real,B", CASES[:3])
def test_autograd_gradient_against_oracle(lib, L, N, lam, J0, spin, real, B):
    import torch
    from paper_2402_01282_gb300 import autograd
    plan = lib.Plan(L, N, lam, J0, spin=spin, reality=real, batch=B, precision=0)
    A, _ = matrices(L, N, lam, J0, spin, real)
    rng = synth.rng_for(913, L)
    f = synth.pixels_random((B, L, 2 * L - 1), rng, complex_=not real)
    x = to_dev(f).requires_grad_(True)
    wav, _ = autograd.analysis(x, plan)
    loss = sum((plan.scale_view(wav, s).abs() ** 2).mean(dim=(1, 2, 3)).sum() for s in range(plan.nscales))
    (grad,) = torch.autograd.grad(loss, x)
    grad = grad.cpu().numpy()
    for b in range(B):
        wavs, wphi = wavelet.analysis(f[b], L, N, lam, J0, spin, reality=real)
        ref = adjoint.analysis_adjoint([2.0 * w / w.size for w in wavs], np.zeros_like(wphi), L, N, lam, J0,
                                       spin, real, matrix=A)
        assert rel(grad[b], ref) < 1e-10


@pytest.mark.parametrize("spin,real", [(0, True), (2, False)])
def test_gradcheck(lib, spin, real):
    """The transforms are linear, so the numerical Jacobian is exact for any step; a large
    step (1e-2) keeps the forward transform's ~1e-13 rounding from being amplified by 1/eps."""
    import torch
    from paper_2402_01282_gb300 import autograd
    L, N = 5, 2
    plan = lib.Plan(L, N, 2.0, 0, spin=spin, reality=real, batch=1, precision=0)
    rng = synth.rng_for(914, L + spin)
    x = to_dev(synth.pixels_random((1, L, 2 * L - 1), rng, complex_=not real)).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda t: autograd.analysis(t, plan), (x,), eps=1e-2, atol=1e-9, rtol=1e-7)
    wav = to_dev(synth.pixels_random((1, plan.wav_elems), rng, complex_=not real)).requires_grad_(True)
    scal = to_dev(synth.pixels_random((1, plan.L_phi, 2 * plan.L_phi - 1), rng, complex_=not real)).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda a, b: autograd.synthesis(a, b, plan), (wav, scal), eps=1e-2, atol=1e-9,
                                    rtol=1e-7)
