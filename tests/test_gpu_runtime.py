"""Runtime around the transforms on the GPU: the autotuner (s2w_plan_autotune) and the batch
executor (s2w_batch_*: several plans of mixed band-limit and spin replayed as one CUDA graph).

* After autotuning, the chosen shapes are among the candidates and the transforms still match
  the oracle element by element (1e-11).
* A mixed batch (band-limits, spins, real and complex maps, batch sizes) run as one graph gives
  every plan's wavelet coefficients within 1e-11 of the oracle and its round trip within 1e-11.
* The batching study's configuration (64 complex maps, L in {64, 128, 256, 512} x 16, spin 0 and
  2 alternating, N = 4, white coefficients) as one graph in the float64-accurate tensor-core
  mode: the round trip of every map within 1e-11, and one map of each band-limit against the
  oracle (every scale for L <= 256; at L = 512 the scaling map, every scale with L_j <= 256 and
  two rings of each scale at L_j = 512, through the oracle's single-ring inverse transform).
"""
import numpy as np
import pytest

import synth
from oracle import filters, harmonic, sampling, wavelet

pytestmark = pytest.mark.gpu
TOL = 1e-11


def rel(a, b):
    d = np.abs(np.asarray(a) - np.asarray(b)).max()
    s = np.abs(np.asarray(b)).max()
    return d / s if s > 0 else d


def to_dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def maps_for(L, spin, real, B, cfg, white=False):
    var = (lambda l: np.ones_like(l)) if white else synth.power_law
    flm = [synth.flm_random(L, synth.rng_for(cfg, b), spin=spin, reality=real, variance=var) for b in range(B)]
    f = np.stack([harmonic.sht_inverse(x, L, spin) for x in flm])
    return f.real.copy() if real else f


def check_against_oracle(plan, f, wav, L, N, lam, J0, spin, real, maps=None):
    w = wav.cpu().numpy()
    for b in (range(plan.batch) if maps is None else maps):
        W_ref, _ = wavelet.analysis(f[b], L, N, lam, J0, spin, real)
        for s in range(plan.nscales):
            got = w[b, plan.wav_offsets[s]:plan.wav_offsets[s + 1]].reshape(plan.scale_shape(s))
            assert rel(got, W_ref[s]) < TOL, (L, spin, b, s)


@pytest.mark.parametrize("precision", [0, 4])   # S2W_FP64, S2W_FP64_TC (DFT form chosen by timing)
def test_autotune_keeps_results(lib, precision):
    L, N, lam, J0, B = 24, 4, 2.0, 0, 3
    plan = lib.Plan(L, N, lam, J0, reality=True, batch=B, precision=precision)
    forms = [plan.dft_forms(k) for k in range(plan.nscales + 2)]
    # before autotuning: the prime-factor tensor-core DFTs wherever S2W_FP64_TC has their tables
    # (the SHT and every wavelet scale at L = 24: 2L_j - 1 <= 47 fits; the scaling function at
    # L_Phi = 1 has no factorisation and takes the direct tensor-core form), else SIMT
    if precision == 4:
        assert forms[0] == (2, 2) and all(f == (2, 2) for f in forms[2:]), forms
        assert forms[1] in ((1, 1), (2, 2)), forms
    else:
        assert all(f == (0, 0) for f in forms), forms
    plan.autotune()
    for k in range(plan.nscales + 2):
        th_f, th_i, mb = plan.launch_shapes(k)
        assert th_f in (128, 256, 384, 512) and th_i in (128, 256, 384, 512) and mb in (4, 8, 16)
        assert all(v in ((0, 1, 2) if precision == 4 else (0,)) for v in plan.dft_forms(k))
    f = maps_for(L, 0, True, B, 930)
    wav, scal, f2 = plan.empty_wav(), plan.empty_scal(), plan.empty_map()
    plan.forward(to_dev(f), wav, scal)
    plan.inverse(wav, scal, f2)
    plan.check()
    check_against_oracle(plan, f, wav, L, N, lam, J0, 0, True)
    assert rel(f2.cpu().numpy(), f) < TOL


def test_batch_mixed_plans(lib):
    specs = [(16, 3, 0, False, 2), (24, 3, 2, False, 1), (16, 2, 0, True, 3), (9, 4, 1, False, 2)]
    plans, fs, fd, wavs, scals, outs = [], [], [], [], [], []
    for (L, N, spin, real, B) in specs:
        p = lib.Plan(L, N, 2.0, 0, spin=spin, reality=real, batch=B)
        f = maps_for(L, spin, real, B, 931 + L + spin)
        plans.append(p)
        fs.append(f)
        fd.append(to_dev(f))
        wavs.append(p.empty_wav())
        scals.append(p.empty_scal())
        outs.append(p.empty_map())
    batch = lib.Batch(plans, fd, wavs, scals, outs, what=2)
    for _ in range(2):
        batch.launch()
    for p in plans:
        p.check()
    for (L, N, spin, real, B), p, f, w, o in zip(specs, plans, fs, wavs, outs):
        check_against_oracle(p, f, w, L, N, 2.0, 0, spin, real)
        assert rel(o.cpu().numpy(), f) < TOL
    batch.close()


def test_batching_study_config(lib):
    """64 complex maps, L in {64, 128, 256, 512} (16 each, spin 0 and 2 alternating), N = 4, in
    S2W_FP64_TC (the headline's precision): the DFT forms at these sizes are the prime-factor
    kernels (127 = 1 x 127, 255 = 3 x 85, 511 = 7 x 73) and the direct form at 1023."""
    plans, fd, wavs, scals, outs, checked = [], [], [], [], [], []
    for L in (64, 128, 256, 512):
        for spin in (0, 2):
            p = lib.Plan(L, 4, 2.0, 0, spin=spin, reality=False, batch=8, precision=lib.S2W_FP64_TC)
            flm = np.stack([synth.flm_random(L, synth.rng_for(3, 16 * L + 2 * b + spin // 2), spin=spin,
                                             variance=lambda l: np.ones_like(l)) for b in range(8)])
            x = p.empty_map()
            p.sht_inverse(to_dev(flm), x)   # timing-free input synthesis (band-limited maps)
            if spin == {64: 2, 128: 0, 256: 2, 512: 0}[L]:   # one map per band-limit
                f0 = harmonic.sht_inverse(flm[0], L, spin)   # the oracle's samples, shared by both sides
                x[0] = to_dev(f0)
                checked.append((len(plans), L, spin, f0))
            plans.append(p)
            fd.append(x)
            wavs.append(p.empty_wav())
            scals.append(p.empty_scal())
            outs.append(p.empty_map())
    batch = lib.Batch(plans, fd, wavs, scals, outs, what=2)
    batch.launch()
    for p in plans:
        p.check()
    for x, o in zip(fd, outs):
        assert float((o - x).abs().max() / x.abs().max()) < TOL
    for k, L, spin, f0 in checked:
        p, w, sc = plans[k], wavs[k][0].cpu().numpy(), scals[k][0].cpu().numpy()
        got = [w[p.wav_offsets[s]:p.wav_offsets[s + 1]].reshape(p.scale_shape(s)) for s in range(p.nscales)]
        if L <= 256:
            W_ref, Wp_ref = wavelet.analysis(f0, L, 4, 2.0, 0, spin, False)
            for s in range(p.nscales):
                assert rel(got[s], W_ref[s]) < TOL, (L, s)
            assert rel(sc.reshape(Wp_ref.shape), Wp_ref) < TOL, L
            continue
        flm = harmonic.sht_forward(f0, L, spin)
        LP = filters.scaling_bandlimit(L, 2.0, 0)
        Wp_ref = harmonic.sht_inverse(wavelet.scaling_coefficients(flm, L, 2.0, 0, spin), LP, 0)
        assert rel(sc.reshape(Wp_ref.shape), Wp_ref) < TOL
        for s, (j, Lj, Nj) in enumerate(filters.scale_bandlimits(L, 4, 2.0, 0)):
            assert (Lj, Nj) == (p.Lj[s], p.Nj[s])
            coef = wavelet.scale_coefficients(flm, L, 4, 2.0, j, Lj, Nj, spin)
            if Lj <= 256:
                assert rel(got[s], harmonic.wigner_inverse(coef, Lj, Nj)) < TOL, (L, s)
                continue
            th = sampling.thetas(Lj)
            rings = {t: harmonic.wigner_inverse_ring(coef, Lj, Nj, th[t]) for t in (3, 301)}
            scale = max(np.abs(r).max() for r in rings.values())
            for t, ring in rings.items():
                assert np.abs(got[s][:, t, :] - ring).max() < TOL * scale, (L, s, t)
    batch.close()
