"""The fused stage kernel's jet-grid instantiations on a grid that its 16 x 32
(eta, zeta) tiles cover exactly (24 x 32 x 32): xi and eta bounded, zeta
periodic, the shifted 16-byte staging and every thread owning a column are
then fixed at compile time.  Every variant of the stage kernel runs 20 steps
in both mixed forms against the FP64 oracle's 20 steps (relative L2 within
1e-5, the bar of the other mixed-form tests): the global step with each
static SGS model, local steps (Eq. localdt), the characteristic entrance
(Sec. "Entrance Boundary"), the dynamic model (Sec. "Dynamic Smagorinsky
Model") and the centerline grid (Sec. "Centerline Boundary Condition").
The other jet tests run on 48 x 24 x 32, whose eta extent the tiles do not
cover, and so exercise the instantiations that decide the cover at run
time."""
import numpy as np
import pytest

from gpu_helpers import device_ctx, oracle_params, rel_l2

pytestmark = pytest.mark.gpu

FULL = (24, 32, 32)
STEPS = 20


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


def _case(lj, name):
    """(options, ring-0 radius or None for the annular default, initial-state
    seed) of one variant."""
    jet = dict(periodic=(0, 0, 1), bc=lj.BC_JET)
    if name == "inviscid_sgs":
        return dict(jet, sgs_model=lj.SGS_NONE), None, 3
    if name == "smagorinsky":
        return dict(jet, sgs_model=lj.SGS_SMAGORINSKY), None, 4
    if name == "vreman":
        return dict(jet, sgs_model=lj.SGS_VREMAN), None, 5
    if name == "local_steps":
        return dict(jet, sgs_model=lj.SGS_SMAGORINSKY, dt_mode=lj.DT_LOCAL), None, 6
    if name == "characteristic_entrance":
        amp = tuple(lj.synth.forcing_amplitudes(2, scale=0.02))
        return dict(periodic=(0, 0, 1), bc=lj.BC_JET_CHAR, sgs_model=lj.SGS_SMAGORINSKY,
                    amp=amp), None, 7
    if name == "dynamic":
        return dict(jet, sgs_model=lj.SGS_DYNAMIC), None, 8
    if name == "axis":
        return dict(sgs_model=lj.SGS_SMAGORINSKY, axis=1), 0.0, 9
    raise ValueError(name)


@pytest.mark.parametrize("name", ["inviscid_sgs", "smagorinsky", "vreman", "local_steps",
                                  "characteristic_entrance", "dynamic", "axis"])
def test_full_tile_variants_against_the_oracle(orc, lj, torch, name):
    kw, r0, seed = _case(lj, name)
    xyz = lj.synth.jet_grid(*FULL) if r0 is None else lj.synth.jet_grid(*FULL, r0=r0)
    P = oracle_params(orc, **kw)
    M = orc.metrics(xyz, (0, 0, 1))
    Q0 = orc.init_jet(P, xyz, seed=seed, noise=1e-2)
    Qo, to = orc.run(P, Q0, M, xyz, STEPS)
    for pc in (lj.PREC_MIXED, lj.PREC_MIXED_COMPACT):
        ctx, _ = device_ctx(lj, torch, FULL, xyz, precision=pc, **kw)
        Qd = torch.from_numpy(Q0).cuda()
        d = ctx.les_run_n_steps(STEPS, Qd)
        Qg = Qd.cpu().numpy()
        assert d.status == 0 and np.isfinite(Qg).all(), (name, pc)
        err = rel_l2(Qg, Qo)
        assert err <= 1e-5, (name, pc, err)
        assert abs(d.t - to) <= 1e-5 * to, (name, pc)
