"""The m-sharded spin SHT's host logic on CPU ranks (gloo): the library's partition
(s2w_shard_layout) and the driver's block exchange (paper_2402_01282_gb300.shard).

The stages run in a stand-in built on the oracle (the GPU stage calls are covered by
test_gpu_shard.py): its column buffers start as NaN and every stage reads and writes only the
range it is given, so a block sent to the wrong rank, placed at the wrong rows or columns, or
missing leaves NaN or wrong values in the result.  Each rank's rings of the inverse and columns
of the forward transform are compared with the oracle's whole-map transforms."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import synth

CASES = [  # (L, spin, sampling, batch, world)
    (6, 0, 0, 2, 2),
    (5, 2, 1, 1, 2),
    (7, 1, 0, 2, 3),
    (4, 0, 1, 1, 3),
]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleStages:
    """The four SHT stage calls on CPU tensors, from the oracle (complex maps)."""

    def __init__(self, L, spin, sampling, batch):
        from paper_2402_01282_gb300 import rings
        self.L, self.spin, self.sampling, self.batch = L, spin, sampling, batch
        self.real = False
        self.R, self.Mc = rings(L, sampling), 2 * L - 1
        self.samp = "dh" if sampling == 1 else "mw"
        from oracle import sampling as smp
        ms = np.arange(-(L - 1), L)
        self.E = np.exp(1j * np.outer(ms, smp.phis(L)))   # [m, p]

    def empty_cols(self, device="cpu"):
        import torch
        return torch.full((self.batch, self.R, self.Mc), complex(float("nan"), float("nan")),
                          dtype=torch.complex128)

    def sht_inverse_columns(self, flm, cols, c0, c1):
        from oracle import harmonic
        for b in range(self.batch):
            f = harmonic.sht_inverse(flm[b].numpy(), self.L, self.spin, self.samp)
            G = f @ np.conj(self.E.T) / (2 * self.L - 1)   # [t, m]: f = G E
            cols[b, :, c0:c1] = _t(G[:, c0:c1])

    def sht_inverse_rings(self, cols, f, t0, t1):
        for b in range(self.batch):
            f[b, t0:t1] = _t(cols[b, t0:t1].numpy() @ self.E)

    def sht_forward_rings(self, f, cols, t0, t1):
        for b in range(self.batch):
            cols[b, t0:t1] = _t(f[b, t0:t1].numpy() @ np.conj(self.E.T) * (2 * np.pi / (2 * self.L - 1)))

    def sht_forward_columns(self, cols, flm, c0, c1):
        from oracle import harmonic
        for b in range(self.batch):
            G = np.zeros((self.R, self.Mc), dtype=np.complex128)
            G[:, c0:c1] = cols[b, :, c0:c1].numpy()   # only this rank's columns are read
            fpart = G @ self.E / (2 * np.pi)   # forward columns are 2 pi times the map's Fourier columns
            a = harmonic.sht_forward(fpart, self.L, self.spin, self.samp)
            flm[b, :, c0:c1] = _t(a[:, c0:c1])


def _t(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x))


def _worker(rank, world, port, case, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2402_01282_gb300.shard import ShardedSHT
    from oracle import harmonic
    L, spin, sampling, B = case
    st = OracleStages(L, spin, sampling, B)
    sh = ShardedSHT(st, None)
    rng = synth.rng_for(931, L)
    flm = np.stack([synth.flm_random(L, rng, spin=spin) for _ in range(B)])
    f = torch.full((B, st.R, 2 * L - 1), complex(float("nan"), float("nan")), dtype=torch.complex128)
    sh.inverse(_t(flm), f)
    t0, t1 = sh.rings
    ref = np.stack([harmonic.sht_inverse(flm[b], L, spin, st.samp) for b in range(B)])
    err_inv = float(np.abs(f[:, t0:t1].numpy() - ref[:, t0:t1]).max() / np.abs(ref).max()) if t1 > t0 else 0.0
    # forward: only this rank's rings of the input are valid
    fin = torch.full_like(f, complex(float("nan"), float("nan")))
    fin[:, t0:t1] = _t(ref[:, t0:t1])
    flm2 = torch.full((B, L, st.Mc), complex(float("nan"), float("nan")), dtype=torch.complex128)
    sh.forward(fin, flm2)
    c0, c1 = sh.columns
    err_fwd = float(np.abs(flm2[:, :, c0:c1].numpy() - flm[:, :, c0:c1]).max() / np.abs(flm).max()) if c1 > c0 else 0.0
    out[rank] = (sh.parts, err_inv, err_fwd)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("case", CASES)
def test_sharded_sht_exchange(case):
    *prob, world = case
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, tuple(prob), out), nprocs=world, join=True)
        res = dict(out)
    parts = res[0][0]
    assert all(res[r][0] == parts for r in range(world))   # every rank holds the same layout
    for r in range(world):
        assert res[r][1] < 1e-12 and res[r][2] < 1e-12, (r, res[r])


@pytest.mark.parametrize("L,spin,real,sampling", [(64, 0, True, 0), (33, 2, False, 0), (20, 1, False, 1),
                                                  (2, 0, True, 1)])
@pytest.mark.parametrize("nranks", [1, 2, 3, 7, 70])
def test_shard_layout_partitions(L, spin, real, sampling, nranks):
    """Column and ring ranges tile [0, Mc) and [0, R(L)) in rank order, and the column ranges
    split the contraction work (L - max(|m|, |spin|) degrees per column) evenly: each part is
    within one column's work of total/nranks."""
    from paper_2402_01282_gb300 import rings, shard_layout
    Mc, R = (L if real else 2 * L - 1), rings(L, sampling)
    parts = [shard_layout(L, spin, real, sampling, nranks, r) for r in range(nranks)]
    ms = np.arange(Mc) + (0 if real else -(L - 1))
    cost = L - np.maximum(np.abs(ms), abs(spin))
    total = cost.sum()
    c_prev, t_prev = 0, 0
    for c0, c1, t0, t1 in parts:
        assert c0 == c_prev and c1 >= c0 and t0 == t_prev and t1 >= t0
        c_prev, t_prev = c1, t1
        assert abs(cost[c0:c1].sum() - total / nranks) <= cost.max()
        assert (t1 - t0) in (R // nranks, R // nranks + 1)
    assert c_prev == Mc and t_prev == R


def test_shard_layout_rejects():
    from paper_2402_01282_gb300 import S2WError, shard_layout
    for args in [(1, 0, True, 0, 1, 0), (8, 0, True, 0, 2, 2), (8, 0, True, 0, 0, 0), (8, 8, False, 0, 1, 0),
                 (8, 1, True, 0, 1, 0), (8, 0, True, 5, 1, 0)]:
        with pytest.raises(S2WError):
            shard_layout(*args)
