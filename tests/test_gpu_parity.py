"""GPU parity of the CUDA path against the float64 oracle, element by element.

Inputs come from synth (seeded) and, for maps, from the oracle's inverse transforms;
nothing expected is computed on the GPU.  Tolerance: max|x - x_ref| / max|x_ref|
<= 1e-11 in float64 mode (the float64 target of the method's error budget).
"""
import numpy as np
import pytest

import synth
from oracle import filters, harmonic, wavelet

pytestmark = pytest.mark.gpu
TOL = 1e-11
MODES = [(0, 0), (3, 0), (0, 1), (4, 0)]   # (precision, precompute): S2W_FP64 on the fly,
                                           # S2W_FP64_NATIVE, S2W_FP64 with precomputed quadrature-folded
                                           # Wigner-d tables, S2W_FP64_TC (sliced tables, tensor cores)


def rel(a, b):
    d = np.abs(np.asarray(a) - np.asarray(b)).max()
    s = np.abs(np.asarray(b)).max()
    return d / s if s > 0 else d


def to_dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def internal_flm(flm_full, L, real):
    """Oracle [L, 2L-1] -> the library's [L, Mc] storage."""
    return flm_full[:, L - 1:] if real else flm_full


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("L,spin,real,B", [(2, 0, True, 1), (8, 0, True, 3), (17, 0, False, 2), (33, 0, True, 2),
                                           (16, 1, False, 1), (11, 2, False, 3), (64, 0, True, 1)])
def test_sht_parity(lib, L, spin, real, B, mode):
    plan = lib.Plan(L, min(2, L), 2.0, 0, spin=spin, reality=real, batch=B, precision=mode[0], precompute=mode[1])
    rng = synth.rng_for(500, L)
    # arbitrary samples: pins the exact MW forward operator, not only its band-limited action
    f = synth.pixels_random((B, L, 2 * L - 1), rng, complex_=not real)
    flm_d = plan.empty_flm()
    plan.sht_forward(to_dev(f), flm_d)
    got = flm_d.cpu().numpy()
    for b in range(B):
        ref = internal_flm(harmonic.sht_forward(f[b], L, spin), L, real)
        assert rel(got[b], ref) < TOL
    # inverse of band-limited coefficients
    flm = np.stack([synth.flm_random(L, rng, spin=spin, reality=real) for _ in range(B)])
    fd = plan.empty_map()
    plan.sht_inverse(to_dev(np.stack([internal_flm(x, L, real) for x in flm])), fd)
    got = fd.cpu().numpy()
    for b in range(B):
        ref = harmonic.sht_inverse(flm[b], L, spin)
        assert rel(got[b], ref.real if real else ref) < TOL
    plan.check()


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("L,N,real,B", [(33, 4, True, 2), (20, 3, False, 1), (9, 9, False, 2)])
def test_wigner_parity(lib, L, N, real, B, mode):
    plan = lib.Plan(L, N, 2.0, 0, reality=real, batch=B, precision=mode[0], precompute=mode[1])
    rng = synth.rng_for(501, L)
    for s in range(plan.nscales):
        Lj, Nj = plan.Lj[s], plan.Nj[s]
        flmn = np.stack([synth.flmn_random(Lj, Nj, rng) for _ in range(B)])
        if real:   # a real SO(3) function: F^l_{-m,-n} = (-1)^(m-n) conj F^l_mn
            for b in range(B):
                fr = harmonic.wigner_inverse(flmn[b], Lj, Nj).real
                flmn[b] = harmonic.wigner_forward(fr, Lj, Nj)
        Mcj = Lj if real else 2 * Lj - 1
        cin = flmn[:, :, :, (Lj - 1 if real else 0):]
        fd = lib_empty(plan, s)
        plan.wigner_inverse(s, to_dev(np.ascontiguousarray(cin)), fd)
        got = fd.cpu().numpy()
        for b in range(B):
            ref = harmonic.wigner_inverse(flmn[b], Lj, Nj)
            assert rel(got[b], ref.real if real else ref) < TOL
        # forward on arbitrary samples (complex plans) / real samples (real plans)
        pix = synth.pixels_random((B, *plan.scale_shape(s)), rng, complex_=not real)
        out = plan.empty_flmn(s)
        plan.wigner_forward(s, to_dev(pix), out)
        got = out.cpu().numpy()
        assert got.shape[-1] == Mcj
        for b in range(B):
            ref = harmonic.wigner_forward(pix[b], Lj, Nj)[:, :, (Lj - 1 if real else 0):]
            assert rel(got[b], ref) < TOL
    plan.check()


def lib_empty(plan, s):
    import torch
    return torch.empty((plan.batch, *plan.scale_shape(s)), dtype=plan.dtype, device="cuda")


def _wavelet_case(lib, L, N, lam, J0, spin, real, B, cfg, mode=(0, 0)):
    plan = lib.Plan(L, N, lam, J0, spin=spin, reality=real, batch=B, precision=mode[0], precompute=mode[1])
    flms = [synth.flm_random(L, synth.rng_for(cfg, b), spin=spin, reality=real) for b in range(B)]
    fs = [harmonic.sht_inverse(x, L, spin) for x in flms]
    if real:
        fs = [x.real for x in fs]
    f = np.stack(fs)
    wav, scal = plan.empty_wav(), plan.empty_scal()
    plan.forward(to_dev(f), wav, scal)
    f2 = plan.empty_map()
    plan.inverse(wav, scal, f2)
    plan.check()
    return plan, f, wav, scal, f2.cpu().numpy()


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("L,N,lam,J0,spin,real,B,cfg", [
    (32, 4, 2.0, 0, 0, True, 1, 1),          # the L=32, N=4 single-map workload
    (16, 3, 2.0, 1, 2, False, 2, 502),        # spin 2, complex
    (23, 5, 1.7, 1, 0, True, 3, 503),         # non-dyadic lambda, ragged sizes
    (10, 1, 2.0, 0, 0, True, 1, 504),         # axisymmetric N = 1
])
def test_wavelet_parity(lib, L, N, lam, J0, spin, real, B, cfg, mode):
    plan, f, wav, scal, f2 = _wavelet_case(lib, L, N, lam, J0, spin, real, B, cfg, mode)
    wv = wav.cpu().numpy()
    sc = scal.cpu().numpy()
    for b in range(B):
        W_ref, Wp_ref = wavelet.analysis(f[b], L, N, lam, J0, spin, real)
        for s, w_ref in enumerate(W_ref):
            got = wv[b, plan.wav_offsets[s]:plan.wav_offsets[s + 1]].reshape(plan.scale_shape(s))
            assert rel(got, w_ref) < TOL, (b, s)
        assert rel(sc[b], Wp_ref) < TOL
        # synthesis parity on the GPU's own coefficient layout (same inputs to both sides)
        ref_f = wavelet.synthesis(W_ref, Wp_ref, L, N, lam, J0, spin, real)
        assert rel(f2[b], ref_f) < TOL
        assert rel(f2[b], f[b]) < TOL          # exact reconstruction (Eq. 31)


def test_synthesis_on_arbitrary_coefficients(lib):
    """Synthesis is a fixed linear operator; check it on coefficients that are not the
    analysis of any signal (arbitrary samples on every scale)."""
    L, N, lam, J0 = 16, 3, 2.0, 1
    plan = lib.Plan(L, N, lam, J0, reality=True, batch=1)
    rng = synth.rng_for(505, 0)
    wav = synth.pixels_random((1, plan.wav_elems), rng)
    scal = synth.pixels_random((1, plan.L_phi, 2 * plan.L_phi - 1), rng)
    fd = plan.empty_map()
    plan.inverse(to_dev(wav), to_dev(scal), fd)
    W = [wav[0, plan.wav_offsets[s]:plan.wav_offsets[s + 1]].reshape(plan.scale_shape(s))
         for s in range(plan.nscales)]
    ref = wavelet.synthesis(W, scal[0], L, N, lam, J0, 0, True)
    assert rel(fd.cpu().numpy()[0], ref) < TOL


def test_full_size_256(lib, oracle_256):
    """The L=256, N=8, lambda=2, J0=2 workload of 16 real maps in the launch configuration the
    benchmark times, in both float64 modes: map 0 against the oracle on every output, and the
    round trip of all 16."""
    import torch
    L, N, lam, J0, B = 256, 8, 2.0, 2, 16
    f, W_ref, Wp_ref = oracle_256
    for mode in MODES:
        plan = lib.Plan(L, N, lam, J0, reality=True, batch=B, precision=mode[0], precompute=mode[1])
        wav, scal = plan.empty_wav(), plan.empty_scal()
        plan.forward(to_dev(f), wav, scal)
        f2 = plan.empty_map()
        plan.inverse(wav, scal, f2)
        plan.check()
        wv = wav[0].cpu().numpy()
        for s, w_ref in enumerate(W_ref):
            got = wv[plan.wav_offsets[s]:plan.wav_offsets[s + 1]].reshape(plan.scale_shape(s))
            assert rel(got, w_ref) < TOL, (mode, s)
        assert rel(scal[0].cpu().numpy(), Wp_ref) < TOL
        f2 = f2.cpu().numpy()
        for b in range(B):
            assert rel(f2[b], f[b]) < TOL, (mode, b)
        plan.close()


def test_full_size_steps_256(lib):
    """Per-step parity at L = 256, batch 16: SHT both ways and the Wigner transforms at the
    top scale (L_j = 256, N_j = 8), compared on map 0 and map 15."""
    import torch
    L, N, B = 256, 8, 16
    plan = lib.Plan(L, N, 2.0, 2, reality=True, batch=B)
    rng = synth.rng_for(506, 0)
    flm = np.stack([synth.flm_random(L, rng, reality=True) for _ in range(B)])
    fd = plan.empty_map()
    plan.sht_inverse(to_dev(np.ascontiguousarray(flm[:, :, L - 1:])), fd)
    got = fd.cpu().numpy()
    for b in (0, B - 1):
        assert rel(got[b], harmonic.sht_inverse(flm[b], L).real) < TOL
    pix = synth.pixels_random((B, L, 2 * L - 1), rng)
    out = plan.empty_flm()
    plan.sht_forward(to_dev(pix), out)
    got = out.cpu().numpy()
    for b in (0, B - 1):
        assert rel(got[b], harmonic.sht_forward(pix[b], L)[:, L - 1:]) < TOL
    s = plan.nscales - 1
    Lj, Nj = plan.Lj[s], plan.Nj[s]
    flmn = synth.flmn_random(Lj, Nj, rng)
    fr = harmonic.wigner_inverse(flmn, Lj, Nj).real
    flmn = harmonic.wigner_forward(fr, Lj, Nj)
    cin = np.ascontiguousarray(np.broadcast_to(flmn[:, :, Lj - 1:], (B, *flmn[:, :, Lj - 1:].shape)))
    wd = torch.empty((B, *plan.scale_shape(s)), dtype=torch.float64, device="cuda")
    plan.wigner_inverse(s, to_dev(cin), wd)
    assert rel(wd.cpu().numpy()[B - 1], fr) < TOL
    pix = synth.pixels_random((B, *plan.scale_shape(s)), rng)
    out = plan.empty_flmn(s)
    plan.wigner_forward(s, to_dev(pix), out)
    assert rel(out.cpu().numpy()[0], harmonic.wigner_forward(pix[0], Lj, Nj)[:, :, Lj - 1:]) < TOL
    plan.check()


@pytest.mark.parametrize("mode", [(0, 1), (4, 0)])
def test_dynamic_range_and_map_chunks(lib, mode):
    """20 maps (two 16-map chunks of the tensor-core operands) whose amplitudes span 30 orders
    of magnitude: every map's wavelet maps and round trip against the oracle relative to that
    map's own scale (the per-column exponents of the sliced operands)."""
    L, N, lam, J0, B = 24, 3, 2.0, 1, 20
    plan = lib.Plan(L, N, lam, J0, reality=True, batch=B, precision=mode[0], precompute=mode[1])
    amp = [10.0 ** (-15 + 30 * b / (B - 1)) for b in range(B)]
    flms = [amp[b] * synth.flm_random(L, synth.rng_for(507, b), reality=True) for b in range(B)]
    f = np.stack([harmonic.sht_inverse(x, L).real for x in flms])
    wav, scal = plan.empty_wav(), plan.empty_scal()
    plan.forward(to_dev(f), wav, scal)
    f2 = plan.empty_map()
    plan.inverse(wav, scal, f2)
    plan.check()
    wv, sc, f2 = wav.cpu().numpy(), scal.cpu().numpy(), f2.cpu().numpy()
    for b in (0, 7, 15, 16, 19):
        W_ref, Wp_ref = wavelet.analysis(f[b], L, N, lam, J0, 0, True)
        for s, w_ref in enumerate(W_ref):
            got = wv[b, plan.wav_offsets[s]:plan.wav_offsets[s + 1]].reshape(plan.scale_shape(s))
            assert rel(got, w_ref) < TOL, (b, s)
        assert rel(sc[b], Wp_ref) < TOL
    for b in range(B):
        assert rel(f2[b], f[b]) < TOL, b


def test_sliced_mode_largest_bandlimit(lib):
    """S2W_FP64_TC at L = 512 (K = 512 reduction terms, the largest the exact float32 sums of
    the sliced products allow): two maps, the SHT both ways on arbitrary samples and
    band-limited coefficients against the oracle, and the round trip on the GPU."""
    L, B = 512, 2
    plan = lib.Plan(L, 1, 2.0, 9, reality=True, batch=B, precision=4)
    rng = synth.rng_for(508, 0)
    flm = np.stack([synth.flm_random(L, rng, reality=True) for _ in range(B)])
    fd = plan.empty_map()
    plan.sht_inverse(to_dev(np.ascontiguousarray(flm[:, :, L - 1:])), fd)
    got = fd.cpu().numpy()
    assert rel(got[1], harmonic.sht_inverse(flm[1], L).real) < TOL
    pix = synth.pixels_random((B, L, 2 * L - 1), rng)
    out = plan.empty_flm()
    plan.sht_forward(to_dev(pix), out)
    plan.check()
    assert rel(out.cpu().numpy()[0], harmonic.sht_forward(pix[0], L)[:, L - 1:]) < TOL
    plan.sht_forward(fd, out)
    plan.check()
    assert rel(out.cpu().numpy(), flm[:, :, L - 1:]) < TOL
