"""Driscoll-Healy sampling on the GPU (sampling = S2W_SAMPLING_DH) against the oracle's DH
transforms (oracle.harmonic with samp="dh", the DH quadrature), element by element.

* Spin SHT and Wigner transforms both ways in the three float64 modes: forward transforms on
  arbitrary samples (the exact DH forward operator, not only its band-limited action), inverse
  transforms on band-limited coefficients; 1e-11.
* The wavelet transform (Algorithm 1) on DH grids: every wavelet map, the scaling map and the
  round trip; float64 modes at 1e-11, the reduced modes at their 1e-5 / 1e-3 targets.
* Adjoints at tiny band-limits against the conjugate transposes of the oracle's DH operators.
* The ball wavelet transform on DH angular grids at small sizes.
* The largest supported band-limit (L = 512, 1024 rings): SHT both ways on sampled maps.
* The L = 256, N = 8, J0 = 2 workload (16 real maps) on DH grids: map 0 against the oracle on
  every output and the round trip of all 16.
"""
import functools

import numpy as np
import pytest

import synth
from oracle import adjoint, ballwav, harmonic, laguerre, wavelet

pytestmark = pytest.mark.gpu
DH = 1
TOL = 1e-11
MODES = [(0, 0), (3, 0), (0, 1), (4, 0)]
REDUCED = {1: 1e-5, 2: 1e-3}


def rel(a, b):
    d = np.abs(np.asarray(a) - np.asarray(b)).max()
    s = np.abs(np.asarray(b)).max()
    return d / s if s > 0 else d


def to_dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def inner(u, v):
    return float(np.real(np.vdot(np.asarray(u).ravel(), np.asarray(v).ravel())))


def internal_flm(flm_full, L, real):
    return flm_full[:, L - 1:] if real else flm_full


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("L,spin,real,B", [(2, 0, True, 1), (8, 0, True, 3), (17, 0, False, 2), (33, 0, True, 2),
                                           (11, 2, False, 3), (64, 0, True, 1)])
def test_dh_sht_parity(lib, L, spin, real, B, mode):
    plan = lib.Plan(L, min(2, L), 2.0, 0, spin=spin, reality=real, batch=B, precision=mode[0], precompute=mode[1],
                    sampling=DH)
    assert plan.map_elems == 2 * L * (2 * L - 1)
    rng = synth.rng_for(940, L)
    f = synth.pixels_random((B, 2 * L, 2 * L - 1), rng, complex_=not real)
    flm_d = plan.empty_flm()
    plan.sht_forward(to_dev(f), flm_d)
    got = flm_d.cpu().numpy()
    for b in range(B):
        assert rel(got[b], internal_flm(harmonic.sht_forward(f[b], L, spin, samp="dh"), L, real)) < TOL
    flm = np.stack([synth.flm_random(L, rng, spin=spin, reality=real) for _ in range(B)])
    fd = plan.empty_map()
    plan.sht_inverse(to_dev(np.stack([internal_flm(x, L, real) for x in flm])), fd)
    got = fd.cpu().numpy()
    for b in range(B):
        ref = harmonic.sht_inverse(flm[b], L, spin, samp="dh")
        assert rel(got[b], ref.real if real else ref) < TOL
    plan.check()


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("L,N,real,B", [(33, 4, True, 2), (20, 3, False, 1), (9, 9, False, 2)])
def test_dh_wigner_parity(lib, L, N, real, B, mode):
    import torch
    plan = lib.Plan(L, N, 2.0, 0, reality=real, batch=B, precision=mode[0], precompute=mode[1], sampling=DH)
    rng = synth.rng_for(941, L)
    for s in range(plan.nscales):
        Lj, Nj = plan.Lj[s], plan.Nj[s]
        assert plan.scale_shape(s) == (2 * Nj - 1, 2 * Lj, 2 * Lj - 1)
        flmn = np.stack([synth.flmn_random(Lj, Nj, rng) for _ in range(B)])
        if real:
            for b in range(B):
                fr = harmonic.wigner_inverse(flmn[b], Lj, Nj, samp="dh").real
                flmn[b] = harmonic.wigner_forward(fr, Lj, Nj, samp="dh")
        cin = flmn[:, :, :, (Lj - 1 if real else 0):]
        fd = torch.empty((B, *plan.scale_shape(s)), dtype=plan.dtype, device="cuda")
        plan.wigner_inverse(s, to_dev(cin), fd)
        got = fd.cpu().numpy()
        for b in range(B):
            ref = harmonic.wigner_inverse(flmn[b], Lj, Nj, samp="dh")
            assert rel(got[b], ref.real if real else ref) < TOL
        pix = synth.pixels_random((B, *plan.scale_shape(s)), rng, complex_=not real)
        out = plan.empty_flmn(s)
        plan.wigner_forward(s, to_dev(pix), out)
        got = out.cpu().numpy()
        for b in range(B):
            ref = harmonic.wigner_forward(pix[b], Lj, Nj, samp="dh")[:, :, (Lj - 1 if real else 0):]
            assert rel(got[b], ref) < TOL
    plan.check()


def _dh_wavelet(lib, L, N, lam, J0, spin, real, B, cfg, mode):
    plan = lib.Plan(L, N, lam, J0, spin=spin, reality=real, batch=B, precision=mode[0], precompute=mode[1],
                    sampling=DH)
    flms = [synth.flm_random(L, synth.rng_for(cfg, b), spin=spin, reality=real) for b in range(B)]
    fs = [harmonic.sht_inverse(x, L, spin, samp="dh") for x in flms]
    f = np.stack([x.real for x in fs] if real else fs)
    wav, scal = plan.empty_wav(), plan.empty_scal()
    plan.forward(to_dev(f), wav, scal)
    f2 = plan.empty_map()
    plan.inverse(wav, scal, f2)
    plan.check()
    return plan, f, wav.cpu().numpy(), scal.cpu().numpy(), f2.cpu().numpy()


WAVELET_CASES = [  # L, N, lam, J0, spin, real, B, cfg
    (32, 4, 2.0, 0, 0, True, 1, 942),
    (16, 3, 2.0, 1, 2, False, 2, 943),
    (23, 5, 1.7, 1, 0, True, 3, 944),
]


@pytest.mark.parametrize("mode", MODES + [(1, 0), (2, 0)])
@pytest.mark.parametrize("L,N,lam,J0,spin,real,B,cfg", WAVELET_CASES)
def test_dh_wavelet_parity(lib, L, N, lam, J0, spin, real, B, cfg, mode):
    tol = REDUCED.get(mode[0], TOL)
    plan, f, wv, sc, f2 = _dh_wavelet(lib, L, N, lam, J0, spin, real, B, cfg, mode)
    for b in range(B):
        W_ref, Wp_ref = wavelet.analysis(f[b], L, N, lam, J0, spin, real, samp="dh")
        for s, w_ref in enumerate(W_ref):
            got = wv[b, plan.wav_offsets[s]:plan.wav_offsets[s + 1]].reshape(plan.scale_shape(s))
            assert rel(got, w_ref) < tol, (b, s)
        assert rel(sc[b], Wp_ref) < tol
        assert rel(f2[b], f[b]) < tol


@functools.lru_cache(maxsize=None)
def _matrices(L, N, lam, J0, spin, real):
    return (adjoint.analysis_matrix(L, N, lam, J0, spin, real, samp="dh"),
            adjoint.synthesis_matrix(L, N, lam, J0, spin, real, samp="dh"))


@pytest.mark.parametrize("mode", [0, 3, 1, 2, 4])
@pytest.mark.parametrize("L,N,lam,J0,spin,real,B", [(8, 3, 2.0, 0, 0, True, 2), (6, 2, 2.0, 1, 2, False, 1),
                                                    (7, 3, 1.7, 0, 0, True, 1)])
def test_dh_adjoints(lib, L, N, lam, J0, spin, real, B, mode):
    plan = lib.Plan(L, N, lam, J0, spin=spin, reality=real, batch=B, precision=mode, sampling=DH)
    A, S = _matrices(L, N, lam, J0, spin, real)
    rng = synth.rng_for(945, L)
    gw = synth.pixels_random((B, plan.wav_elems), rng, complex_=not real)
    gp = synth.pixels_random((B, plan.R_phi, 2 * plan.L_phi - 1), rng, complex_=not real)
    gf = plan.empty_map()
    plan.forward_adjoint(to_dev(gw), to_dev(gp), gf)
    x = synth.pixels_random((B, 2 * L, 2 * L - 1), rng, complex_=not real)
    sw, sp = plan.empty_wav(), plan.empty_scal()
    plan.inverse_adjoint(to_dev(x), sw, sp)
    plan.check()
    gf, sw, sp = gf.cpu().numpy(), sw.cpu().numpy(), sp.cpu().numpy()
    for b in range(B):
        wavs = [gw[b, plan.wav_offsets[s]:plan.wav_offsets[s + 1]].reshape(plan.scale_shape(s))
                for s in range(plan.nscales)]
        ref = adjoint.analysis_adjoint(wavs, gp[b], L, N, lam, J0, spin, real, matrix=A, samp="dh")
        assert rel(gf[b], ref) < TOL
        rw, rp = adjoint.synthesis_adjoint(x[b], L, N, lam, J0, spin, real, matrix=S, samp="dh")
        for s in range(plan.nscales):
            got = sw[b, plan.wav_offsets[s]:plan.wav_offsets[s + 1]].reshape(plan.scale_shape(s))
            assert rel(got, rw[s]) < TOL, (b, s)
        assert rel(sp[b], rp) < TOL


@pytest.mark.parametrize("mode", [(0, 0), (0, 1), (4, 0)])
def test_dh_ball_wavelet(lib, mode):
    L, N, P, nu, J0, J0r, B = 8, 2, 7, 2.0, 0, 0, 2
    plan = lib.BallWavPlan(L, N, P, 2.0, nu, J0, J0r, batch=B, precision=mode[0], precompute=mode[1], sampling=DH)
    f = []
    for b in range(B):
        flmp = synth.flmp_random(L, P, synth.rng_for(946, b), reality=True)
        f.append(laguerre.spherical_laguerre_inverse(flmp, L, P, samp="dh").real)
    f = np.stack(f)
    assert f.shape == (B, P, 2 * L, 2 * L - 1)
    wav, scal = plan.empty_wav(), plan.empty_field()
    plan.forward(to_dev(f), wav, scal)
    f2 = plan.empty_field()
    plan.inverse(wav, scal, f2)
    plan.check()
    got_s = scal.cpu().numpy()
    for b in range(B):
        wref, sref = ballwav.analysis(f[b], L, N, P, 2.0, nu, J0, J0r, samp="dh")
        assert rel(got_s[b], sref) < TOL
        for k, (j, jr) in enumerate(plan.scales):
            assert rel(plan.scale_view(wav, k)[b].cpu().numpy(), wref[(j, jr)]) < TOL, (b, j, jr)
    assert rel(f2.cpu().numpy(), f) < TOL


@pytest.mark.parametrize("mode", [(0, 0), (3, 0)])
def test_dh_max_bandlimit_sht(lib, mode):
    """L = 512 (1024 rings, one thread per ring in the forward contraction): two maps, SHT
    both ways; forward of arbitrary samples and inverse of band-limited coefficients, sampled
    rows against the oracle."""
    L, B = 512, 2
    plan = lib.Plan(L, 1, 2.0, 9, reality=True, batch=B, precision=mode[0], precompute=mode[1], sampling=DH)
    rng = synth.rng_for(947, 0)
    flm = np.stack([synth.flm_random(L, rng, reality=True) for _ in range(B)])
    fd = plan.empty_map()
    plan.sht_inverse(to_dev(np.stack([internal_flm(x, L, True) for x in flm])), fd)
    got = fd.cpu().numpy()
    ref = harmonic.sht_inverse(flm[1], L, 0, samp="dh").real
    assert rel(got[1], ref) < TOL
    pix = synth.pixels_random((B, 2 * L, 2 * L - 1), rng)
    out = plan.empty_flm()
    plan.sht_forward(to_dev(pix), out)
    plan.check()
    got = out.cpu().numpy()
    assert rel(got[0], harmonic.sht_forward(pix[0], L, 0, samp="dh")[:, L - 1:]) < TOL
    # round trip of the band-limited maps through the GPU alone
    plan.sht_forward(fd, out)
    plan.check()
    assert rel(out.cpu().numpy(), np.stack([internal_flm(x, L, True) for x in flm])) < TOL


@pytest.fixture(scope="module")
def oracle_dh_256():
    L, N, lam, J0, B = 256, 8, 2.0, 2, 16
    flms = [synth.flm_random(L, synth.rng_for(2, b), reality=True) for b in range(B)]
    f = np.stack([harmonic.sht_inverse(x, L, 0, samp="dh").real for x in flms])
    W_ref, Wp_ref = wavelet.analysis(f[0], L, N, lam, J0, 0, True, samp="dh")
    return f, W_ref, Wp_ref


@pytest.mark.parametrize("mode", MODES + [(1, 0), (2, 0)])
def test_dh_full_size_256(lib, oracle_dh_256, mode):
    L, N, lam, J0, B = 256, 8, 2.0, 2, 16
    tol = REDUCED.get(mode[0], TOL)
    f, W_ref, Wp_ref = oracle_dh_256
    plan = lib.Plan(L, N, lam, J0, reality=True, batch=B, precision=mode[0], precompute=mode[1], sampling=DH)
    wav, scal = plan.empty_wav(), plan.empty_scal()
    plan.forward(to_dev(f), wav, scal)
    f2 = plan.empty_map()
    plan.inverse(wav, scal, f2)
    plan.check()
    wv = wav[0].cpu().numpy()
    for s, w_ref in enumerate(W_ref):
        got = wv[plan.wav_offsets[s]:plan.wav_offsets[s + 1]].reshape(plan.scale_shape(s))
        assert rel(got, w_ref) < tol, (mode, s)
    assert rel(scal[0].cpu().numpy(), Wp_ref) < tol
    f2 = f2.cpu().numpy()
    for b in range(B):
        assert rel(f2[b], f[b]) < tol, (mode, b)
    plan.close()
