"""FP64 CPU oracle for the directional wavelet transform on the sphere and ball.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (``paper_2402_01282_gb300``) never imports it and
shares no code with it: the GPU library computes the same transforms by a
different algorithm (theta-space Wigner-d recursion and a sampled quadrature
matrix), while this oracle follows the Fourier-space route of McEwen-Wiaux
sampling: Wigner-d functions expanded as trigonometric polynomials in beta,
azimuthal and polar integrals done as direct DFT sums, and the colatitude
integral done exactly by convolving with the Fourier weights of sin(theta) on
[0, pi].  On Driscoll-Healy sampling the colatitude integral is instead the DH
quadrature (weights from the moment conditions), applied to the same Fourier-space
Wigner-d functions.

Everything is float64 / complex128, unblocked and unfused, so that each step can
be read against the paper:

* ``wigner``    Wigner-d functions as trigonometric polynomials (Sec. 2.2, Eq. 47).
* ``sampling``  McEwen-Wiaux grids on S^2 and SO(3) and the sin-weight integrals; the
                Driscoll-Healy grids and their colatitude weights.
* ``harmonic``  spin spherical-harmonic transform (Sec. 2.1, Eqs. 2-3) and Wigner
                transform (Sec. 2.2, Eqs. 4-5).
* ``filters``   scale-discretised tiling and dictionary (App. A, Eqs. A2-A10).
* ``wavelet``   Algorithm 1 (Sec. 4, Eqs. 40-42) with the multiresolution
                band-limits of Sec. 3.3 (Eq. 38).
* ``laguerre``  Fourier-Laguerre radial transform (Sec. 2.3, Eqs. 6-11).
* ``ballwav``   directional wavelet transform on the ball (Sec. 3.2, App. A.3-A.4) with the
                radial multiresolution of Sec. 3.3.
* ``adjoint``   adjoints of the analysis and synthesis operators (Sec. 4.3), by brute
                force: the conjugate transpose of the operator's matrix (tiny L only).

Parity pins for each function live in ``tests/test_oracle_*.py``.
"""
from . import sampling, wigner, harmonic, filters, wavelet, laguerre, adjoint, ballwav  # noqa: F401
