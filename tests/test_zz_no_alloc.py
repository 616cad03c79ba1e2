"""s2w_sht_inverse_static: the inverse SHT whose scratch is the library's fixed device array.

It exists for callers that cannot allocate device memory when they need a transform (a host
application that owns every device allocation, or code running during CUDA graph capture)
and cannot borrow the plan's workspace.  Checked here through the C ABI against
s2w_sht_inverse, on two calls in a row (the array keeps the previous call's contents), at
the 1e-11 tolerance of the other float64 tests, in every precision mode and on both samplings;
and the size limit, batch * R(L) * Mc <= 2^20 complex elements, is checked to reject cleanly.
This file is collected last so that a failure here does not hide other tests.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
TOL = 1e-11


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


# (L, spin, real, batch, precision mode, precompute, sampling): every precision mode (the static
# call always contracts by the on-the-fly recursion, whatever path s2w_sht_inverse takes), the
# precomputed-table mode, and Driscoll-Healy grids (2L rings, so the size limit is reached at half
# the L of MW)
CASES = [(32, 0, True, 3, 0, 0, 0), (17, 1, False, 2, 0, 0, 0), (33, 0, True, 2, 3, 0, 0),
         (256, 0, True, 16, 0, 0, 0), (64, 0, True, 4, 4, 0, 0), (256, 0, True, 16, 4, 0, 0),
         (40, 0, True, 2, 1, 0, 0), (24, 2, False, 2, 2, 0, 0), (48, 0, True, 3, 0, 1, 0),
         (20, 0, True, 2, 0, 0, 1), (19, 1, False, 2, 4, 0, 1), (181, 0, True, 16, 0, 0, 1)]


@pytest.mark.parametrize("L,spin,real,B,mode,pre,samp", CASES)
def test_static_scratch_matches_sht_inverse(lib, L, spin, real, B, mode, pre, samp):
    import torch
    plan = lib.Plan(L, 2, 2.0, 0, spin=spin, reality=real, batch=B, precision=mode, precompute=pre, sampling=samp)
    rng = synth.rng_for(600, L)
    flm = np.stack([synth.flm_random(L, rng, spin=spin, reality=real) for _ in range(B)])
    if real:
        flm = flm[:, :, L - 1:]
    flm_d = torch.from_numpy(np.ascontiguousarray(flm)).cuda()
    ref = plan.empty_map()
    plan.sht_inverse(flm_d, ref)
    ref = ref.cpu().numpy()
    for _ in range(2):
        out = plan.empty_map()
        out.fill_(float("nan") if real else complex(float("nan"), 0.0))
        plan.sht_inverse_static(flm_d, out)
        plan.check()
        assert rel(out.cpu().numpy(), ref) < TOL
    plan.close()


@pytest.mark.parametrize("L,B,samp", [(257, 16, 0), (182, 16, 1)])
def test_static_scratch_rejects_oversize(lib, L, B, samp):
    # batch * R(L) * Mc just above the 2^20 limit: 16 * 257 * 257 on MW, 16 * 364 * 182 on DH
    import torch
    plan = lib.Plan(L, 2, 2.0, 0, reality=True, batch=B, sampling=samp)
    flm = torch.zeros((B, L, plan.Mc), dtype=torch.complex128, device="cuda")
    out = plan.empty_map()
    with pytest.raises(lib.S2WError) as ei:
        plan.sht_inverse_static(flm, out)
    assert ei.value.status == 1 and "exceeds the fixed scratch" in str(ei.value)
    plan.check()
    plan.close()
