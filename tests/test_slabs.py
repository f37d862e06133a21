"""Axial slab decomposition, host side (Sec. "Communication": axial
partitions with two ghost layers, exchanged after every stage; the global
time step as the minimum over the partitions).

The partition and ghost-plane ranges are checked directly; the exchange and
the time-step reduction of ``slabs.DistSlab`` run over gloo with world sizes
2 and 3 (a middle slab has both cuts) on CPU tensors.  The slab stand-in
below steps a five-stage scheme whose residual reaches two planes along xi
(a fourth difference plus a first difference, the reach of the method's
dissipation), updates only its own interior planes and takes its step from
its own planes, as the library's slab contexts do; the decomposed run must
equal the undivided one bit for bit on every own plane."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2301_00817_gb300 import slabs  # noqa: E402

ALPHA = (1 / 4, 1 / 6, 3 / 8, 1 / 2, 1.0)


class FakeSlab:
    """CPU stand-in for a slab context: the phase calls and state_views."""

    def __init__(self, ni_local, glo, ghi, shape_jk=(3, 4)):
        import torch
        self.nl, self.glo, self.ghi = ni_local, glo, ghi
        self.SA = torch.zeros((5, ni_local) + shape_jk, dtype=torch.float64)
        self.SB = torch.zeros_like(self.SA)
        self.dt = None

    def les_state_load(self, Q):
        pass

    def les_state_store(self, Q):
        pass

    def _own(self):
        return self.glo, self.nl - self.ghi

    def les_step_begin(self, Q):
        a, b = self._own()
        return float(0.1 / (1.0 + Q[:, a:b].abs().max()))

    def les_step_set_dt(self, dt):
        self.dt = dt

    def _rhs(self, q):
        # reach two planes along xi, on the planes that have both neighbours
        r = q.clone().zero_()
        r[:, 2:-2] = (q[:, 4:] - 4 * q[:, 3:-1] + 6 * q[:, 2:-2] - 4 * q[:, 1:-3] + q[:, :-4]
                      + 0.5 * (q[:, 3:-1] - q[:, 1:-3]))
        return r

    def les_step_stage(self, l, Q):
        src = Q if l == 1 else (self.SA if l % 2 == 0 else self.SB)
        dst = Q if l == 5 else (self.SA if l % 2 == 1 else self.SB)
        r = self._rhs(src)
        # own interior planes only (physical faces and ghost planes untouched)
        a = max(self.glo, 2)
        b = min(self.nl - self.ghi, self.nl - 2)
        new = Q[:, a:b] - ALPHA[l - 1] * self.dt * r[:, a:b]
        if l < 5:
            dst.copy_(Q)
        dst[:, a:b] = new

    def les_step_end(self, Q):
        pass

    def state_views(self, l, Q):
        if l in (0, 5):
            return [Q]
        return [self.SA if l % 2 == 1 else self.SB]


def _initial(ni, shape_jk=(3, 4)):
    import torch
    g = torch.Generator().manual_seed(3)
    return torch.rand((5, ni) + shape_jk, generator=g, dtype=torch.float64)


def _undivided(ni, steps):
    Q = _initial(ni)
    s = FakeSlab(ni, 0, 0)
    dts = []
    for _ in range(steps):
        dt = s.les_step_begin(Q)
        s.les_step_set_dt(dt)
        for l in range(1, 6):
            s.les_step_stage(l, Q)
        dts.append(dt)
    return Q, dts


def test_partition_extent_and_ranges():
    for ni, n in ((48, 2), (49, 3), (288, 8), (10, 5)):
        parts = slabs.partition(ni, n)
        assert parts[0][0] == 0 and parts[-1][1] == ni
        assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
        assert all(i1 - i0 >= slabs.GHOST for i0, i1 in parts)
        for s, (i0, i1) in enumerate(parts):
            lo, hi, glo, ghi = slabs.extent(i0, i1, ni)
            assert (glo == 0) == (s == 0) and (ghi == 0) == (s == n - 1)
            nl = hi - lo
            snd, rcv = slabs.send_ranges(nl, glo, ghi), slabs.recv_ranges(nl, glo, ghi)
            if glo:
                # sent planes are the neighbour's ghost planes: global i0 .. i0+1
                assert snd[0] == (2, 4) and rcv[0] == (0, 2) and lo + snd[0][0] == i0
            if ghi:
                assert rcv[1] == (nl - 2, nl) and lo + rcv[1][0] == i1
                assert lo + snd[1][0] == i1 - 2
    with pytest.raises(ValueError):
        slabs.partition(5, 3)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, ni, steps, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    from paper_2301_00817_gb300 import slabs as sl
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        i0, i1 = sl.partition(ni, world)[rank]
        lo, hi, glo, ghi = sl.extent(i0, i1, ni)
        Q = _initial(ni)[:, lo:hi].clone()
        ctx = FakeSlab(hi - lo, glo, ghi)
        drv = sl.DistSlab(ctx, Q, ni, rank, world)
        dts = [drv.step() for _ in range(steps)]
        drv.ctx.les_state_store(Q)
        q.put((rank, i0, i1, glo, Q[:, glo:glo + (i1 - i0)].numpy(), dts))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_dist_slabs_match_the_undivided_run(world):
    import numpy as np
    import torch.multiprocessing as mp
    ni, steps = 23, 6
    ref, ref_dts = _undivided(ni, steps)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, ni, steps, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    covered = np.zeros(ni, bool)
    for rank, i0, i1, glo, own, dts in got:
        assert np.array_equal(own, ref[:, i0:i1].numpy()), rank
        assert dts == ref_dts  # every rank takes the global minimum
        covered[i0:i1] = True
    assert covered.all()
