"""Axial slabs on one GPU (Sec. "Communication": axial partitions with two
ghost layers): the jet configuration 48 x 24 x 32 split into two and three
slab contexts on the same device, stepped through the phase calls with the
ghost planes exchanged by les_halo_copy after every stage and after the
boundary conditions, and the global time step taken as the minimum of the
slabs' own.  Every own plane must equal the undivided run bit for bit (each
own node reads at most two planes away along xi, which the ghost planes
supply), in FP64 and in both mixed forms; the phase calls on an undivided
grid must equal les_rk_step bit for bit."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SHAPE = (48, 24, 32)


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2301_00817_gb300 import _build
    _build.build()
    import paper_2301_00817_gb300 as lj
    lj.load_library()
    return lj, torch


def _ctx(lj, torch, shape, xyz, **kw):
    ctx = lj.Context(lj.make_params(sgs_model=lj.SGS_SMAGORINSKY, **kw), shape, "cuda:0")
    ctx.les_set_grid(xyz)
    return ctx


@pytest.mark.parametrize("prec", ["fp64", "mixed", "compact"])
@pytest.mark.parametrize("nslabs", [2, 3])
def test_slabs_equal_the_undivided_run(env, prec, nslabs):
    lj, torch = env
    from paper_2301_00817_gb300 import slabs
    pc = {"fp64": lj.PREC_FP64, "mixed": lj.PREC_MIXED, "compact": lj.PREC_MIXED_COMPACT}[prec]
    ni = SHAPE[0]
    xyz = torch.from_numpy(lj.synth.jet_grid(*SHAPE)).cuda()
    whole = _ctx(lj, torch, SHAPE, xyz, precision=pc)
    Q0 = torch.empty((5,) + SHAPE, dtype=torch.float64, device="cuda")
    whole.les_init_jet(xyz, 0, 1e-2, Q0)
    steps = 12
    Qw = Q0.clone()
    diag = whole.les_run_n_steps(steps, Qw)
    ctxs, states, owns = [], [], []
    for (i0, i1) in slabs.partition(ni, nslabs):
        lo, hi, glo, ghi = slabs.extent(i0, i1, ni)
        shape = (hi - lo,) + SHAPE[1:]
        c = _ctx(lj, torch, shape, xyz[:, lo:hi].contiguous(), precision=pc, slab_ghost=(glo, ghi))
        ctxs.append(c)
        states.append(Q0[:, lo:hi].clone())
        owns.append((i0, i1, glo))
    run = slabs.LocalSlabs(ctxs, states)
    slab_dts = [run.step() for _ in range(steps)]
    for c, Q in zip(run.ctxs, run.Q):
        c.les_state_store(Q)
    torch.cuda.synchronize()
    assert slab_dts[-1] == diag.dt
    for (i0, i1, glo), Q in zip(owns, run.Q):
        assert torch.equal(Q[:, glo:glo + (i1 - i0)], Qw[:, i0:i1]), (prec, i0, i1)
    assert np.isfinite(Qw.cpu().numpy()).all()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_phase_calls_equal_rk_step(env, prec):
    lj, torch = env
    pc = lj.PREC_FP64 if prec == "fp64" else lj.PREC_MIXED
    xyz = torch.from_numpy(lj.synth.jet_grid(*SHAPE)).cuda()
    a = _ctx(lj, torch, SHAPE, xyz, precision=pc)
    b = _ctx(lj, torch, SHAPE, xyz, precision=pc)
    Q = torch.empty((5,) + SHAPE, dtype=torch.float64, device="cuda")
    a.les_init_jet(xyz, 1, 1e-2, Q)
    Qa, Qb = Q.clone(), Q.clone()
    a.les_run_n_steps(3, Qa)
    b.les_state_load(Qb)
    for _ in range(3):
        dt = b.les_step_begin(Qb)
        b.les_step_set_dt(dt)
        for l in range(1, 6):
            b.les_step_stage(l, Qb)
        b.les_step_end(Qb)
    b.les_state_store(Qb)
    torch.cuda.synchronize()
    assert torch.equal(Qa, Qb)


def test_slab_options_rejected(env):
    lj, torch = env
    with pytest.raises(lj.LesError):
        lj.Context(lj.make_params(slab_ghost=(1, 0)), (12, 8, 8), "cuda:0")
    with pytest.raises(lj.LesError):
        lj.Context(lj.make_params(slab_ghost=(2, 0), sgs_model=lj.SGS_DYNAMIC), (12, 8, 8), "cuda:0")
    with pytest.raises(lj.LesError):
        lj.Context(lj.make_params(slab_ghost=(2, 2)), (4, 8, 8), "cuda:0")
