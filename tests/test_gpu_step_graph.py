"""The FP32-mixed step replayed as a CUDA graph.  A context that replays its
captured step and one that runs every step as plain launches (the event
profiler keeps a context on plain launches) agree bit for bit over a
sequence that changes the parameters between runs (the graph must be
dropped and captured again), restarts the time and runs from a host buffer;
and the launch count grows by the same number of kernels per step either
way."""
import numpy as np
import pytest

from gpu_helpers import device_ctx

pytestmark = pytest.mark.gpu

SHAPE = (48, 24, 32)


@pytest.fixture(scope="module")
def lj():
    from paper_2301_00817_gb300 import _build
    _build.build()
    import paper_2301_00817_gb300 as lj
    lj.load_library()
    return lj


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def _sequence(lj, torch, ctx, Q0, plain):
    if plain:
        ctx.les_profile(True)
    Q = torch.from_numpy(Q0.copy()).cuda()
    out = []
    d1 = ctx.les_run_n_steps(4, Q)
    out.append((Q.cpu().numpy().copy(), d1.t, list(d1.totals)))
    # new parameters between runs: a smaller CFL number and the Vreman model
    ctx.les_set_params(lj.make_params(sgs_model=lj.SGS_VREMAN, cfl=0.3,
                                      precision=lj.PREC_MIXED))
    d2 = ctx.les_run_n_steps(3, Q)
    out.append((Q.cpu().numpy().copy(), d2.t, list(d2.totals)))
    # restart the clock, then steps from a pinned host buffer
    ctx.les_set_time(0.0)
    Qh = torch.from_numpy(Q.cpu().numpy().copy()).pin_memory()
    d3 = ctx.les_run_host(2, Qh, torch.zeros_like(Q))
    out.append((Qh.numpy().copy(), d3.t, list(d3.totals)))
    return out


def test_graph_replay_matches_plain_launches(lj, torch):
    xyz = lj.synth.jet_grid(*SHAPE)
    runs = []
    for plain in (False, True):
        ctx, xyz_d = device_ctx(lj, torch, SHAPE, xyz, sgs_model=lj.SGS_SMAGORINSKY,
                                precision=lj.PREC_MIXED)
        Qd = torch.empty((5,) + SHAPE, dtype=torch.float64, device="cuda")
        ctx.les_init_jet(xyz_d, 7, 1e-2, Qd)
        runs.append(_sequence(lj, torch, ctx, Qd.cpu().numpy(), plain))
    for (qa, ta, sa), (qb, tb, sb) in zip(*runs):
        assert np.array_equal(qa, qb)
        assert ta == tb and sa == sb


def test_graph_replay_counts_its_kernels(lj, torch):
    xyz = lj.synth.jet_grid(*SHAPE)
    ctx, xyz_d = device_ctx(lj, torch, SHAPE, xyz, sgs_model=lj.SGS_SMAGORINSKY,
                            precision=lj.PREC_MIXED)
    Q = torch.empty((5,) + SHAPE, dtype=torch.float64, device="cuda")
    ctx.les_init_jet(xyz_d, 7, 1e-2, Q)
    ctx.les_run_n_steps(2, Q)  # the first step plain, then the capture
    counts = []
    for n in (1, 5):
        c0 = ctx.les_launch_count()
        ctx.les_run_n_steps(n, Q)
        counts.append(ctx.les_launch_count() - c0)
    per_step = (counts[1] - counts[0]) / 4
    assert per_step == int(per_step) and per_step >= 8
    ctx.les_profile(True)  # plain launches
    c0 = ctx.les_launch_count()
    ctx.les_run_n_steps(5, Q)
    assert ctx.les_launch_count() - c0 == counts[1]
