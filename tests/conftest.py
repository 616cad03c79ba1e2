import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def lib():
    """The CUDA library through its Python binding; only for tests marked gpu."""
    import paper_2402_01282_gb300 as s2w
    s2w.load()
    return s2w


@pytest.fixture(scope="session")
def oracle_256():
    """The oracle's analysis of map 0 of the L=256, N=8, J0=2 workload (computed once)."""
    import numpy as np
    import synth
    from oracle import harmonic, wavelet
    L, N, lam, J0, B = 256, 8, 2.0, 2, 16
    flms = [synth.flm_random(L, synth.rng_for(2, b), reality=True) for b in range(B)]
    f = np.stack([harmonic.sht_inverse(x, L).real for x in flms])
    W_ref, Wp_ref = wavelet.analysis(f[0], L, N, lam, J0, 0, True)
    return f, W_ref, Wp_ref
