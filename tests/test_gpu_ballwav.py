"""Directional wavelet transform on the ball on the GPU (s2w_ball_forward / _inverse and their
adjoints) against oracle.ballwav.

* Small fields (several radial scales and a ragged non-dyadic nu): every wavelet block and the
  scaling coefficients element by element against the oracle's analysis; the synthesis of
  arbitrary (not band-limited) coefficients against the oracle's synthesis; 1e-11.
* Adjoints at small sizes through the inner-product identity with the oracle's transforms.
* The ball study's configuration (L = P = 128, N = 4, lambda = nu = 2, J0 = J0' = 0, one real
  field): a band-limited field built as a sum of separable terms K_{p_q}(r) g_q(w), whose
  spherical-Laguerre coefficients are known exactly, so sampled nodes of sampled scales have
  oracle values from a single Wigner transform each; plus the round trip and the adjoint
  identity over the whole field.
"""
import math

import numpy as np
import pytest

import synth
from oracle import ballwav, filters, harmonic, laguerre

pytestmark = pytest.mark.gpu
TOL = 1e-11


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def to_dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def inner(u, v):
    return float(np.real(np.vdot(np.asarray(u).ravel(), np.asarray(v).ravel())))


CASES = [  # L, N, P, nu, J0, J0r, B
    (8, 2, 8, 2.0, 0, 0, 1),
    (6, 3, 7, 1.7, 1, 0, 2),
    (9, 1, 5, 2.0, 0, 1, 1),
]


def fields(L, P, B, cfg):
    out = []
    for b in range(B):
        flmp = synth.flmp_random(L, P, synth.rng_for(cfg, b), reality=True)
        out.append(laguerre.spherical_laguerre_inverse(flmp, L, P).real)
    return np.stack(out)


# (precision, precompute) and the tolerance of the wavelet and scaling coefficients: float64
# accuracy (1e-11) in the float64 modes; the reduced modes' targets for S2W_FP32_SPLIT (1e-5) and
# S2W_BF16 (1e-3), whose radial maps run on the tensor cores float64-accurately and whose sphere
# contractions carry the reduced precision
BALL_MODES = [((0, 0), 1e-11), ((3, 0), 1e-11), ((0, 1), 1e-11), ((4, 0), 1e-11), ((1, 0), 1e-5), ((2, 0), 1e-3)]


@pytest.mark.parametrize("mode,tol", BALL_MODES)
@pytest.mark.parametrize("L,N,P,nu,J0,J0r,B", CASES)
def test_ball_analysis_parity(lib, L, N, P, nu, J0, J0r, B, mode, tol):
    TOL = tol
    plan = lib.BallWavPlan(L, N, P, 2.0, nu, J0, J0r, batch=B, precision=mode[0], precompute=mode[1])
    f = fields(L, P, B, 920)
    wav, scal = plan.empty_wav(), plan.empty_field()
    plan.forward(to_dev(f), wav, scal)
    plan.check()
    got_s = scal.cpu().numpy()
    for b in range(B):
        wref, sref = ballwav.analysis(f[b], L, N, P, 2.0, nu, J0, J0r)
        assert rel(got_s[b], sref) < TOL
        for k, (j, jr) in enumerate(plan.scales):
            got = plan.scale_view(wav, k)[b].cpu().numpy()
            assert rel(got, wref[(j, jr)]) < TOL, (b, j, jr)
    f2 = plan.empty_field()
    plan.inverse(wav, scal, f2)
    plan.check()
    assert rel(f2.cpu().numpy(), f) < TOL


@pytest.mark.parametrize("L,N,P,nu,J0,J0r,B", CASES[:2])
def test_ball_synthesis_arbitrary(lib, L, N, P, nu, J0, J0r, B):
    plan = lib.BallWavPlan(L, N, P, 2.0, nu, J0, J0r, batch=B)
    rng = synth.rng_for(921, L)
    wav = synth.pixels_random((plan.wav_elems,), rng)
    scal = synth.pixels_random((B, P, L, 2 * L - 1), rng)
    f = plan.empty_field()
    plan.inverse(to_dev(wav), to_dev(scal), f)
    plan.check()
    got = f.cpu().numpy()
    for b in range(B):
        wavs = {}
        for k, (j, jr) in enumerate(plan.scales):
            a, e = plan.wav_offsets[k], plan.wav_offsets[k + 1]
            wavs[(j, jr)] = wav[a:e].reshape(B, plan.Pj[k], 2 * plan.Nj[k] - 1, plan.Lj[k], 2 * plan.Lj[k] - 1)[b]
        ref = ballwav.synthesis(wavs, scal[b], L, N, P, 2.0, nu, J0, J0r)
        assert rel(got[b], ref) < TOL


@pytest.mark.parametrize("mode", [0, 4])   # the adjoints' radial maps: SIMT and tensor cores (transposed tables)
@pytest.mark.parametrize("L,N,P,nu,J0,J0r,B", CASES[:2])
def test_ball_adjoints(lib, L, N, P, nu, J0, J0r, B, mode):
    plan = lib.BallWavPlan(L, N, P, 2.0, nu, J0, J0r, batch=B, precision=mode)
    rng = synth.rng_for(922, L)
    x = synth.pixels_random((B, P, L, 2 * L - 1), rng)
    gw = synth.pixels_random((plan.wav_elems,), rng)
    gs = synth.pixels_random((B, P, L, 2 * L - 1), rng)
    gf = plan.empty_field()
    plan.forward_adjoint(to_dev(gw), to_dev(gs), gf)
    sw, ss = plan.empty_wav(), plan.empty_field()
    plan.inverse_adjoint(to_dev(x), sw, ss)
    plan.check()
    gf, sw, ss = gf.cpu().numpy(), sw.cpu().numpy(), ss.cpu().numpy()
    for b in range(B):
        wref, sref = ballwav.analysis(x[b], L, N, P, 2.0, nu, J0, J0r)
        lhs = inner(gs[b], sref)
        for k, (j, jr) in enumerate(plan.scales):
            a, e = plan.wav_offsets[k], plan.wav_offsets[k + 1]
            blk = gw[a:e].reshape(B, -1)[b]
            lhs += inner(blk, wref[(j, jr)])
        bound = np.linalg.norm(np.concatenate([gs[b].ravel()] + [gw[plan.wav_offsets[k]:plan.wav_offsets[k + 1]]
                                                                 .reshape(B, -1)[b] for k in range(plan.nscales)]))
        bound *= math.sqrt(np.sum(sref ** 2) + sum(np.sum(w ** 2) for w in wref.values()))
        assert abs(lhs - inner(gf[b], x[b])) < TOL * bound
        # synthesis side: <S^H x, (W, W^Phi)> = <x, S (W, W^Phi)>
        wavs = {}
        for k, (j, jr) in enumerate(plan.scales):
            a, e = plan.wav_offsets[k], plan.wav_offsets[k + 1]
            wavs[(j, jr)] = gw[a:e].reshape(B, plan.Pj[k], 2 * plan.Nj[k] - 1, plan.Lj[k], 2 * plan.Lj[k] - 1)[b]
        fs = ballwav.synthesis(wavs, gs[b], L, N, P, 2.0, nu, J0, J0r)
        lhs = inner(ss[b], gs[b])
        for k in range(plan.nscales):
            a, e = plan.wav_offsets[k], plan.wav_offsets[k + 1]
            lhs += inner(sw[a:e].reshape(B, -1)[b], gw[a:e].reshape(B, -1)[b])
        assert abs(lhs - inner(x[b], fs)) < TOL * np.linalg.norm(x[b]) * (np.linalg.norm(gw) + np.linalg.norm(gs)) * 10


@pytest.mark.parametrize("mode,tune", [(0, False), (4, False), (4, True)])   # S2W_FP64; S2W_FP64_TC (the
def test_ball_full_size_config(lib, mode, tune):                             # study's mode), also autotuned
    """L = P = 128, N = 4, lambda = nu = 2, J0 = J0' = 0, one real field."""
    import torch
    L, N, P, lam, nu = 128, 4, 128, 2.0, 2.0
    plan = lib.BallWavPlan(L, N, P, lam, nu, 0, 0, batch=1, precision=mode)
    if tune:
        plan.autotune()   # the sphere transforms' launch shapes and DFT forms, as the bench runs them
    _, _, K = laguerre.quadrature(P)
    pq = [1, 5, 37, 127]   # p = 1 reaches the lowest radial scale (kappa^0(1) = 1)
    a = [synth.flm_random(L, synth.rng_for(5, q), reality=True) for q in range(len(pq))]
    g = [harmonic.sht_inverse(x, L).real for x in a]
    f = np.zeros((1, P, L, 2 * L - 1))
    for q, p in enumerate(pq):
        f[0] += K[:, p][:, None, None] * g[q][None]
    wav, scal = plan.empty_wav(), plan.empty_field()
    fd = to_dev(f)
    plan.forward(fd, wav, scal)
    plan.check()
    # sampled oracle values: W^{jj'}(r'_i) = D^-1_j [(8 pi^2/(2l+1)) conj(Psi^j) sum_q kappa^{j'}(p_q) K_{p_q}(r'_i) a_q]
    sl = {}
    for k, (j, jr) in enumerate(plan.scales):
        sl[(j, jr)] = k
    for (j, jr, i) in [(7, 7, 3), (6, 5, 10), (4, 2, 7), (7, 0, 1)]:
        k = sl[(j, jr)]
        Lj, Nj, Pj = plan.Lj[k], plan.Nj[k], plan.Pj[k]
        _, _, Kj = laguerre.quadrature(Pj)
        kap = ballwav.radial_kappa(P, nu, jr)
        gl = np.zeros((L, 2 * L - 1), dtype=np.complex128)
        for q, p in enumerate(pq):
            if p < Pj:
                gl += kap[p] * Kj[i, p] * a[q]
        psi = filters.wavelet_filter(L, N, lam, j)
        coef = np.zeros((2 * Nj - 1, Lj, 2 * Lj - 1), dtype=np.complex128)
        s = slice(L - Lj, L + Lj - 1)
        for l in range(Lj):
            for n in range(-(Nj - 1), Nj):
                coef[n + Nj - 1, l] = (8 * math.pi ** 2 / (2 * l + 1)) * gl[l, s] * np.conj(psi[l, n + N - 1])
        ref = harmonic.wigner_inverse(coef, Lj, Nj).real
        got = plan.scale_view(wav, k)[0, i].cpu().numpy()
        assert rel(got, ref) < TOL, (j, jr, i, rel(got, ref))
    # round trip and the adjoint identity over the whole field
    f2 = plan.empty_field()
    plan.inverse(wav, scal, f2)
    plan.check()
    assert float((f2 - fd).abs().max() / fd.abs().max()) < TOL
    rng = synth.rng_for(923, 0)
    gw = to_dev(synth.pixels_random((plan.wav_elems,), rng))
    gs = to_dev(synth.pixels_random((1, P, L, 2 * L - 1), rng))
    gf = plan.empty_field()
    plan.forward_adjoint(gw, gs, gf)
    plan.check()
    lhs = float((gw * wav).sum() + (gs * scal).sum())
    rhs = float((gf * fd).sum())
    bound = float(torch.sqrt((gw ** 2).sum() + (gs ** 2).sum()) * torch.sqrt((wav ** 2).sum() + (scal ** 2).sum()))
    assert abs(lhs - rhs) < TOL * bound
