"""GPU parity on a true centerline grid (Sec. "Centerline Boundary
Condition", Reading A27): ring j = 0 lies on the axis r = 0, where J^-1 = 0
exactly.  The CUDA path (FP64 and both mixed forms, through the C ABI) runs
with params.axis = 1 against the oracle's axis mode on the same grid and the
same initial bits.

Tolerances as in the annular parity tests: FP64 residual within 1e-13 of the
flux scale, one step within 1e-12 and 20 steps within 1e-10 (relative
L-inf); the mixed forms' residual within 2e-5 of the flux scale and 20 steps
within 1e-5 (relative L2) of FP64.
"""
import numpy as np
import pytest

from gpu_helpers import device_ctx, oracle_params, rel_l2, rel_linf

pytestmark = pytest.mark.gpu

AXIS_C1 = (48, 24, 32)
AXIS_RAGGED = (13, 9, 8)


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


def _axis_grid(lj, shape):
    xyz = lj.synth.jet_grid(*shape, r0=0.0)
    assert np.abs(xyz[1:, :, 0]).max() == 0.0  # ring 0 on the axis
    return xyz


def _flux_scale(M):
    # J^-1 |grad xi| is finite everywhere (0 on the axis)
    return (np.abs(M[9]) * np.sqrt(M[0] ** 2 + M[1] ** 2 + M[2] ** 2)).max()


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("shape", [AXIS_C1, AXIS_RAGGED])
def test_axis_metrics(orc, lj, torch, shape, form):
    """J^-1 = 0 exactly on the axis and the scaled metrics stored there; the
    other nodes as on any grid.  Each row is compared at the scale of its
    own magnitude (the axis rows are J^-1-scaled, the others are not)."""
    xyz = _axis_grid(lj, shape)
    ctx, _ = device_ctx(lj, torch, shape, xyz, axis=1, metric_form=form)
    Mg = ctx.les_metrics().cpu().numpy()
    Mo = orc.metrics(xyz, (0, 0, 1), None, form=form)
    assert (Mo[9][:, 0] == 0.0).all() and (Mg[9][:, 0] == 0.0).all()
    assert np.isfinite(Mg).all()
    for part in (np.s_[:, 0], np.s_[:, 1:]):
        for r in range(10):
            a, b = Mg[r][part], Mo[r][part]
            if r == 9:
                scale = np.abs(Mo[9][part]).max() + 1e-300
            else:
                scale = np.abs(Mo[3 * (r // 3):3 * (r // 3) + 3][(slice(None),) + part]).max()
            # the conservative form differences products: rounding follows the
            # coordinates' magnitudes times the derivatives, over J^-1
            if form == 1 and part == np.s_[:, 1:]:
                D = max(np.abs(np.gradient(xyz[c], axis=d)).max() for c in range(3) for d in range(3))
                scale = max(scale, np.abs(xyz).max() * D / np.abs(Mo[9][part]).min())
            assert np.abs(a - b).max() <= 1e-13 * scale, (r, part)


@pytest.mark.parametrize("sgs", [0, 1, 2])
def test_axis_mu_eff(orc, lj, torch, sgs):
    """An axis node's SGS viscosity is ring 1's azimuthal mean at its plane;
    its laminar part is its own."""
    shape = AXIS_C1
    xyz = _axis_grid(lj, shape)
    kw = dict(sgs_model=sgs, Re=2000.0, axis=1)
    ctx, _ = device_ctx(lj, torch, shape, xyz, **kw)
    P = oracle_params(orc, **kw)
    M = orc.metrics(xyz, (0, 0, 1))
    Q = orc.init_jet(P, xyz, seed=5, noise=2e-2)
    MK = torch.empty((2,) + shape, dtype=torch.float64, device="cuda")
    ctx.les_mu_eff(torch.from_numpy(Q).cuda(), MK)
    MKo = orc.mu_eff(P, Q, M)
    for r in range(2):
        assert np.abs(MK[r].cpu().numpy() - MKo[r]).max() <= 1e-13 * np.abs(MKo[r]).max()
    if sgs:
        # the axis values are constant around each plane
        ax = MK[0, :, 0].cpu().numpy()
        assert np.abs(ax - ax[:, :1]).max() <= 1e-13 * np.abs(ax).max()


@pytest.mark.parametrize("sgs", [0, 1, 2])
@pytest.mark.parametrize("shape", [AXIS_C1, AXIS_RAGGED])
def test_axis_rhs(orc, lj, torch, shape, sgs):
    xyz = _axis_grid(lj, shape)
    kw = dict(sgs_model=sgs, Re=2000.0, axis=1)
    P = oracle_params(orc, **kw)
    M = orc.metrics(xyz, (0, 0, 1))
    Q = orc.init_jet(P, xyz, seed=5, noise=2e-2)
    Ro = orc.rhs(P, Q, M)
    fscale = _flux_scale(M)
    for prec, tol in (("fp64", 1e-13), ("mixed", 2e-5), ("compact", 2e-5)):
        pc = {"fp64": lj.PREC_FP64, "mixed": lj.PREC_MIXED, "compact": lj.PREC_MIXED_COMPACT}[prec]
        ctx, _ = device_ctx(lj, torch, shape, xyz, precision=pc, **kw)
        R = torch.empty((5,) + shape, dtype=torch.float64, device="cuda")
        ctx.les_rhs(torch.from_numpy(Q).cuda(), R)
        Rg = R.cpu().numpy()
        assert np.isfinite(Rg).all(), prec
        for c in range(5):
            qs = np.abs(Q[c]).max() + (np.abs(Q[4]).max() if c in (1, 2, 3, 4) else 0.0)
            assert np.abs(Rg[c] - Ro[c]).max() <= tol * fscale * qs, (prec, c)
        assert np.abs(Rg[:, :, 0]).max() == 0.0  # the axis is a boundary


@pytest.mark.parametrize("sgs", [0, 1, 2])
def test_axis_steps(orc, lj, torch, sgs):
    """The small jet configuration on the centerline grid: 1 step <= 1e-12,
    20 steps <= 1e-10 against the oracle (FP64); the centerline rule leaves
    every axis node of a plane with the same state."""
    shape = AXIS_C1
    xyz = _axis_grid(lj, shape)
    kw = dict(sgs_model=sgs, axis=1)
    ctx, _ = device_ctx(lj, torch, shape, xyz, **kw)
    P = oracle_params(orc, **kw)
    M = orc.metrics(xyz, (0, 0, 1))
    Q0 = orc.init_jet(P, xyz, seed=0)
    Qd = torch.from_numpy(Q0).cuda()
    d1 = ctx.les_run_n_steps(1, Qd)
    Q1, dt1 = orc.rk_step(P, Q0, M, xyz, 0.0)
    assert abs(d1.dt - dt1) <= 1e-13 * dt1
    assert rel_linf(Qd.cpu().numpy(), Q1) <= 1e-12
    d20 = ctx.les_run_n_steps(19, Qd)
    Q20, t20 = orc.run(P, Q1, M, xyz, 19, t=dt1)
    assert abs(d20.t - t20) <= 1e-12 * t20
    Qg = Qd.cpu().numpy()
    assert rel_linf(Qg, Q20) <= 1e-10
    ax = Qg[:, 1:-1, 0]
    assert np.array_equal(ax, np.repeat(ax[:, :, :1], shape[2], axis=2))


def test_axis_mixed_against_fp64(orc, lj, torch):
    """Both mixed forms on the centerline grid: 20 steps within 1e-5 (rel
    L2) of the FP64 oracle."""
    shape = AXIS_C1
    xyz = _axis_grid(lj, shape)
    P = oracle_params(orc, sgs_model=1, axis=1)
    M = orc.metrics(xyz, (0, 0, 1))
    Q0 = orc.init_jet(P, xyz, seed=0)
    Qo, to = orc.run(P, Q0, M, xyz, 20)
    for pc in (lj.PREC_MIXED, lj.PREC_MIXED_COMPACT):
        ctx, _ = device_ctx(lj, torch, shape, xyz, sgs_model=1, axis=1, precision=pc)
        Qd = torch.from_numpy(Q0).cuda()
        d = ctx.les_run_n_steps(20, Qd)
        Qg = Qd.cpu().numpy()
        assert np.isfinite(Qg).all()
        assert rel_l2(Qg, Qo) <= 1e-5, pc
        assert abs(d.t - to) <= 1e-5 * to


def test_axis_free_stream(orc, lj, torch):
    """A uniform flow along the axis stays uniform on the centerline grid:
    the residual vanishes to round-off in FP64 (metrics of the separable
    grid, the J^-1-weighted interface means)."""
    shape = AXIS_C1
    xyz = _axis_grid(lj, shape)
    ctx, _ = device_ctx(lj, torch, shape, xyz, sgs_model=1, axis=1, bc=0)
    P = oracle_params(orc, sgs_model=1, axis=1, bc=0)
    M = orc.metrics(xyz, (0, 0, 1))
    Q = orc.prim_to_cons(P, lj.synth.uniform_prim(shape, u=0.7))
    R = torch.empty((5,) + shape, dtype=torch.float64, device="cuda")
    ctx.les_rhs(torch.from_numpy(Q).cuda(), R)
    assert np.abs(R.cpu().numpy()).max() <= 1e-13 * _flux_scale(M) * np.abs(Q).max()


def test_axis_options_rejected(lj, torch):
    """The dynamic model is not defined on a grid with an axis; the adjoint
    is provided for grids without one; an axis needs periodic {0, 0, 1}."""
    shape = AXIS_RAGGED
    with pytest.raises(lj.LesError) as e:
        lj.Context(lj.make_params(axis=1, sgs_model=lj.SGS_DYNAMIC), shape, "cuda:0")
    assert e.value.code in (lj.LES_ERR_UNSUPPORTED,)
    with pytest.raises(lj.LesError):
        lj.Context(lj.make_params(axis=1, bc=0, periodic=(1, 1, 1)), shape, "cuda:0")
    xyz = _axis_grid(lj, shape)
    ctx, xyz_d = device_ctx(lj, torch, shape, xyz, axis=1, dt_mode=lj.DT_FIXED, dt_fixed=1e-4)
    Q = torch.empty((5,) + shape, dtype=torch.float64, device="cuda")
    ctx.les_init_jet(xyz_d, 0, 1e-3, Q)
    with pytest.raises(lj.LesError) as e:
        ctx.les_adjoint_step(Q, 0.0, Q.clone(), torch.empty_like(Q), ctx.adjoint_workspace(1, 1))
    assert e.value.code == lj.LES_ERR_UNSUPPORTED
