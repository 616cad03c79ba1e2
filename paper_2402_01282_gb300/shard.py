"""m-sharded spin SHT over torch.distributed ranks.

The paper spreads its transforms over several GPUs (Sec. 4.3; timings on three GPUs in Sec. 4.4);
here the work is split over the order m.  Rank r of R owns a contiguous range of m columns of
near-equal contraction work and a contiguous range of colatitude rings (s2w_shard_layout).
The inverse transform contracts the rank's columns over l for every ring
(s2w_sht_inverse_columns), exchanges column blocks in one all-to-all (rank r sends rank q the
rows of q's rings in r's columns) and takes the azimuthal DFT of the rank's rings
(s2w_sht_inverse_rings).  The forward transform runs the
same steps in the opposite order: DFT of the rank's rings, all-to-all, contraction with the
colatitude quadrature of the rank's columns.

Every arithmetic step runs in the library's stage calls (include/s2w.h); this module packs the
blocks of the column buffer and calls the collective (NCCL between GPUs, gloo on CPU).  A
"plan" here is any object with the stage methods and layout attributes of ``Plan`` (L, spin,
real, sampling, batch, R, Mc, empty_cols and the four sht_*_columns / sht_*_rings calls).
"""
from __future__ import annotations

from . import shard_layout


class ShardedSHT:
    """One spin SHT of ``plan``'s batch split by m over the ranks of ``group``."""

    def __init__(self, plan, group=None):
        import torch.distributed as dist
        self.plan, self.group = plan, group
        self.nranks = dist.get_world_size(group)
        self.rank = dist.get_rank(group)
        # (c_begin, c_end, ring_begin, ring_end) of every rank, the same on all of them
        self.parts = [shard_layout(plan.L, plan.spin, plan.real, plan.sampling, self.nranks, q)
                      for q in range(self.nranks)]

    @property
    def columns(self):
        """This rank's column range [c_begin, c_end) (column c holds m = c + m_min)."""
        return self.parts[self.rank][:2]

    @property
    def rings(self):
        """This rank's ring range [ring_begin, ring_end)."""
        return self.parts[self.rank][2:]

    def _exchange(self, send_blocks, recv_shapes):
        """all-to-all of complex blocks: send_blocks[q] goes to rank q; returns the blocks
        received from every rank q, shaped recv_shapes[q]."""
        import math

        import torch
        import torch.distributed as dist
        dev = send_blocks[0].device
        send = torch.cat([b.reshape(-1) for b in send_blocks])
        n_out = [b.numel() for b in send_blocks]
        n_in = [math.prod(s) for s in recv_shapes]
        recv = torch.empty(sum(n_in), dtype=torch.complex128, device=dev)
        dist.all_to_all_single(torch.view_as_real(recv), torch.view_as_real(send), n_in, n_out, group=self.group)
        out, o = [], 0
        for s, n in zip(recv_shapes, n_in):
            out.append(recv[o:o + n].view(s))
            o += n
        return out

    def inverse(self, flm, f, cols=None):
        """flm (the whole batch of coefficients, on every rank) -> this rank's rings of f.
        cols: optional [batch, R(L), Mc] complex scratch (allocated when None)."""
        p = self.plan
        c0, c1, t0, t1 = self.parts[self.rank]
        G = cols if cols is not None else p.empty_cols(device=flm.device)
        p.sht_inverse_columns(flm, G, c0, c1)
        send = [G[:, q0:q1, c0:c1] for (_, _, q0, q1) in self.parts]
        shapes = [(p.batch, t1 - t0, e1 - e0) for (e0, e1, _, _) in self.parts]
        for (e0, e1, _, _), blk in zip(self.parts, self._exchange(send, shapes)):
            G[:, t0:t1, e0:e1] = blk
        p.sht_inverse_rings(G, f, t0, t1)
        return f

    def forward(self, f, flm, cols=None):
        """This rank's rings of f -> this rank's columns of flm (every l; other m untouched)."""
        p = self.plan
        c0, c1, t0, t1 = self.parts[self.rank]
        G = cols if cols is not None else p.empty_cols(device=f.device)
        p.sht_forward_rings(f, G, t0, t1)
        send = [G[:, t0:t1, e0:e1] for (e0, e1, _, _) in self.parts]
        shapes = [(p.batch, q1 - q0, c1 - c0) for (_, _, q0, q1) in self.parts]
        for (_, _, q0, q1), blk in zip(self.parts, self._exchange(send, shapes)):
            G[:, q0:q1, c0:c1] = blk
        p.sht_forward_columns(G, flm, c0, c1)
        return flm
