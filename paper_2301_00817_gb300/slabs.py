"""Axial slab decomposition of the jet grid (Sec. "Communication": the
solver splits the domain into axial partitions that each carry two ghost
layers, exchanged after every Runge-Kutta stage, and takes the global time
step as the minimum over the partitions).

On one GB300 the whole grid fits a single context; slabs are for grids
spread over several GPUs (one context per GPU and rank) or over several
contexts of one process.  Each slab is a context over its own planes plus
two ghost planes at every cut (``slab_ghost``), stepped through the phase
calls of the C ABI (``les_step_begin`` ... ``les_step_end``):

    dt_i = les_step_begin(slab i)             own-plane CFL step of Q^n
    dt   = min_i dt_i                         (all-reduce MIN across ranks)
    les_step_set_dt(slab i, dt)
    for l in 1..5: les_step_stage(slab i, l); exchange the ghost planes
    les_step_end(slab i); exchange the ghost planes

A slab's own planes then hold, bit for bit, what the undivided grid holds
there: every own node's residual reads at most two planes away along xi,
which the ghost planes supply, and a ghost plane's own (wrong) values never
reach an own node.  ``LocalSlabs`` steps the slabs of one process and
exchanges through ``les_halo_copy`` (cudaMemcpy2DAsync between the
contexts' buffers); ``DistSlab`` steps this rank's slab and exchanges with
torch.distributed point-to-point calls (NCCL on GPUs, gloo on CPU tensors).
The partition, the ghost-plane index ranges and the exchange pattern are
plain host logic, shared by both.
"""
from __future__ import annotations

GHOST = 2  # ghost planes at a cut: the residual reaches two planes along xi


def partition(ni: int, nslabs: int):
    """Own planes [i0, i1) of each slab: near-equal consecutive ranges that
    cover 0 .. ni-1 (each slab owns at least GHOST planes)."""
    if nslabs < 1 or ni < GHOST * nslabs:
        raise ValueError(f"cannot split {ni} planes into {nslabs} slabs of >= {GHOST} planes")
    return [(s * ni // nslabs, (s + 1) * ni // nslabs) for s in range(nslabs)]


def extent(i0: int, i1: int, ni: int):
    """Local plane range [lo, hi) of the slab owning [i0, i1) and its ghost
    planes (glo, ghi): two at a cut, none at the entrance or the exit."""
    glo = GHOST if i0 > 0 else 0
    ghi = GHOST if i1 < ni else 0
    return i0 - glo, i1 + ghi, glo, ghi


def send_ranges(nl: int, glo: int, ghi: int):
    """Local planes a slab sends across its cuts: (low cut, high cut); None
    where the slab meets a physical face."""
    low = (glo, glo + GHOST) if glo else None
    high = (nl - ghi - GHOST, nl - ghi) if ghi else None
    return low, high


def recv_ranges(nl: int, glo: int, ghi: int):
    """Local ghost planes a slab receives: (low cut, high cut)."""
    low = (0, glo) if glo else None
    high = (nl - ghi, nl) if ghi else None
    return low, high


class LocalSlabs:
    """The slabs of one process (contexts on one GPU or on peer GPUs), each
    with its own state Q ([5, nl, nj, nk] FP64 on its device), stepped in
    lockstep; the exchange is les_halo_copy."""

    def __init__(self, ctxs, states):
        self.ctxs = list(ctxs)
        self.Q = list(states)
        for c, Q in zip(self.ctxs, self.Q):
            c.les_state_load(Q)

    def _exchange(self, l: int):
        for a in range(len(self.ctxs) - 1):
            lo, hi = self.ctxs[a], self.ctxs[a + 1]
            hi.les_halo_copy(self.Q[a + 1], lo, self.Q[a], l, 0)  # hi's low ghosts from lo
            lo.les_halo_copy(self.Q[a], hi, self.Q[a + 1], l, 1)  # lo's high ghosts from hi

    def step(self) -> float:
        dt = min(c.les_step_begin(Q) for c, Q in zip(self.ctxs, self.Q))
        for c in self.ctxs:
            c.les_step_set_dt(dt)
        for l in range(1, 6):
            for c, Q in zip(self.ctxs, self.Q):
                c.les_step_stage(l, Q)
            self._exchange(l)
        for c, Q in zip(self.ctxs, self.Q):
            c.les_step_end(Q)
        self._exchange(0)
        return dt

    def run(self, n: int):
        for _ in range(n):
            self.step()
        for c, Q in zip(self.ctxs, self.Q):
            c.les_state_store(Q)


class DistSlab:
    """This rank's slab of a decomposition over the ranks of a
    torch.distributed group (rank r owns partition()[r]).  ctx is any object
    with the phase calls and state_views (a Context, or a stand-in for
    tests); the ghost planes travel with send/recv of contiguous copies."""

    def __init__(self, ctx, Q, ni: int, rank: int, world: int, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.ctx, self.Q, self.group = ctx, Q, group
        self.rank, self.world = rank, world
        i0, i1 = partition(ni, world)[rank]
        self.lo, self.hi, self.glo, self.ghi = extent(i0, i1, ni)
        self.nl = self.hi - self.lo
        ctx.les_state_load(Q)

    def exchange(self, arrays):
        """Fill the ghost planes of every [5, nl, ...] array from the
        neighbouring ranks."""
        dist = self.dist
        send = send_ranges(self.nl, self.glo, self.ghi)
        recv = recv_ranges(self.nl, self.glo, self.ghi)
        peers = (self.rank - 1, self.rank + 1)
        for V in arrays:
            ops, incoming = [], []
            for side in (0, 1):
                if send[side] is not None:
                    a, b = send[side]
                    ops.append(dist.P2POp(dist.isend, V[:, a:b].contiguous(), peers[side],
                                          group=self.group))
                if recv[side] is not None:
                    a, b = recv[side]
                    buf = V[:, a:b].contiguous()
                    ops.append(dist.P2POp(dist.irecv, buf, peers[side], group=self.group))
                    incoming.append((a, b, buf))
            if ops:
                for r in dist.batch_isend_irecv(ops):
                    r.wait()
            for a, b, buf in incoming:
                V[:, a:b].copy_(buf)

    def step(self) -> float:
        import torch
        dist = self.dist
        dt_local = self.ctx.les_step_begin(self.Q)
        t = torch.tensor([dt_local], dtype=torch.float64, device=self.Q.device)
        dist.all_reduce(t, op=dist.ReduceOp.MIN, group=self.group)
        dt = float(t.item())
        self.ctx.les_step_set_dt(dt)
        for l in range(1, 6):
            self.ctx.les_step_stage(l, self.Q)
            self.exchange(self.ctx.state_views(l, self.Q))
        self.ctx.les_step_end(self.Q)
        self.exchange(self.ctx.state_views(0, self.Q))
        return dt

    def run(self, n: int):
        for _ in range(n):
            self.step()
        self.ctx.les_state_store(self.Q)
