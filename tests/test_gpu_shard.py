"""The m-sharded spin SHT's stage calls on the GPU (s2w_sht_inverse_columns / _rings,
s2w_sht_forward_rings / _columns), against the float64 oracle.

One process and one GPU: R virtual ranks run one after another on a shared column buffer (what
the all-to-all of the driver assembles), so every stage call runs on exactly its rank's range
and nothing waits on another rank.  The composed result is compared element by element with the
oracle (1e-11) and with the whole-transform calls, in each precision mode (the stages always run
the float64-accurate on-the-fly kernels), on MW and DH grids, for real and spin maps.  The
driver itself (paper_2402_01282_gb300.shard) runs over a one-rank NCCL group."""
import numpy as np
import pytest

import synth
from oracle import harmonic

pytestmark = pytest.mark.gpu
TOL = 1e-11


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


def to_dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("mode", [0, 3, 4, 1])
@pytest.mark.parametrize("L,spin,real,sampling,B,R", [(16, 0, True, 0, 2, 3), (17, 2, False, 0, 1, 2),
                                                      (12, 1, False, 1, 2, 5), (9, 0, True, 1, 1, 4),
                                                      (64, 0, True, 0, 3, 7)])
def test_stages_compose_to_the_sht(lib, mode, L, spin, real, sampling, B, R):
    import torch
    plan = lib.Plan(L, 2, 2.0, 0, spin=spin, reality=real, batch=B, precision=mode, sampling=sampling)
    parts = [lib.shard_layout(L, spin, real, sampling, R, r) for r in range(R)]
    rng = synth.rng_for(940, L)
    a = np.stack([synth.flm_random(L, rng, spin=spin, reality=real) for _ in range(B)])
    flm = to_dev(a[:, :, L - 1:] if real else a)
    samp = "dh" if sampling else "mw"
    ref = np.stack([harmonic.sht_inverse(a[b], L, spin, samp) for b in range(B)])
    ref = ref.real if real else ref
    # inverse: every rank's columns, then every rank's rings
    G = plan.empty_cols()
    G.fill_(float("nan"))
    f = plan.empty_map()
    f.fill_(float("nan"))
    for c0, c1, _, _ in parts:
        plan.sht_inverse_columns(flm, G, c0, c1)
    for _, _, t0, t1 in parts:
        plan.sht_inverse_rings(G, f, t0, t1)
    got = f.cpu().numpy()
    assert rel(got, ref) < TOL
    whole = plan.empty_map()
    plan.sht_inverse(flm, whole)
    assert rel(got, whole.cpu().numpy()) < TOL
    # forward: every rank's rings, then every rank's columns
    G.fill_(float("nan"))
    out = plan.empty_flm()
    out.fill_(float("nan"))
    fd = to_dev(ref)
    for _, _, t0, t1 in parts:
        plan.sht_forward_rings(fd, G, t0, t1)
    for c0, c1, _, _ in parts:
        plan.sht_forward_columns(G, out, c0, c1)
    plan.check()
    got = out.cpu().numpy()
    assert rel(got, a[:, :, L - 1:] if real else a) < TOL
    plan.close()


def test_ranges_touch_nothing_else(lib):
    """A stage call writes only its range: columns outside [c0, c1) of cols, rings outside
    [t0, t1) of f and coefficients of other m keep their contents."""
    import torch
    L, B = 12, 2
    plan = lib.Plan(L, 2, 2.0, 0, spin=0, reality=False, batch=B, precision=0)
    rng = synth.rng_for(941, L)
    a = to_dev(np.stack([synth.flm_random(L, rng) for _ in range(B)]))
    G = plan.empty_cols()
    G.fill_(7.0)
    plan.sht_inverse_columns(a, G, 5, 9)
    keep = torch.ones_like(G, dtype=torch.bool)
    keep[:, :, 5:9] = False
    assert bool((G[keep] == 7.0).all()) and not bool((G[:, :, 5:9] == 7.0).any())
    f = plan.empty_map()
    f.fill_(3.0)
    plan.sht_inverse_rings(G, f, 2, 6)
    keep = torch.ones_like(f, dtype=torch.bool)
    keep[:, 2:6] = False
    assert bool((f[keep] == 3.0).all())
    G2 = plan.empty_cols()
    G2.fill_(5.0)
    plan.sht_forward_rings(f, G2, 1, 4)
    keep = torch.ones_like(G2, dtype=torch.bool)
    keep[:, 1:4] = False
    assert bool((G2[keep] == 5.0).all())
    out = plan.empty_flm()
    out.fill_(9.0)
    plan.sht_forward_columns(G, out, 5, 9)
    keep = torch.ones_like(out, dtype=torch.bool)
    keep[:, :, 5:9] = False
    assert bool((out[keep] == 9.0).all())
    for bad in [(-1, 3), (4, 2), (0, 2 * L)]:
        with pytest.raises(lib.S2WError):
            plan.sht_inverse_columns(a, G, *bad)
    with pytest.raises(lib.S2WError):
        plan.sht_inverse_rings(G, f, 0, L + 1)
    plan.check()
    plan.close()


def test_driver_one_rank_nccl(lib):
    """ShardedSHT over a one-rank NCCL group: the all-to-all with itself and the packing."""
    import os
    import socket

    import torch
    import torch.distributed as dist
    from paper_2402_01282_gb300.shard import ShardedSHT
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("nccl", rank=0, world_size=1, device_id=torch.device("cuda", torch.cuda.current_device()))
    try:
        L, B = 32, 2
        plan = lib.Plan(L, 2, 2.0, 0, spin=0, reality=True, batch=B, precision=4)
        sh = ShardedSHT(plan)
        rng = synth.rng_for(942, L)
        a = np.stack([synth.flm_random(L, rng, reality=True) for _ in range(B)])
        f = plan.empty_map()
        sh.inverse(to_dev(a[:, :, L - 1:]), f)
        ref = np.stack([harmonic.sht_inverse(a[b], L, 0).real for b in range(B)])
        assert rel(f.cpu().numpy(), ref) < TOL
        out = plan.empty_flm()
        sh.forward(f, out)
        assert rel(out.cpu().numpy(), a[:, :, L - 1:]) < TOL
        plan.check()
        plan.close()
    finally:
        dist.destroy_process_group()
