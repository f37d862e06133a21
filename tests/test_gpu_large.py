"""The largest jet workloads, FP32-mixed form.

* 2000 x 500 x 1024 (1.02e9 points) in the compact mixed form, the form that
  fits one GB300: one step checked at sampled interior nodes against the
  oracle, then a 20-step run that must stay finite with its status OK.  The
  oracle cannot run the whole grid, so each sampled node is checked against
  the oracle run on the 27^3 block around it with its faces frozen: one step
  reaches 12 nodes (five stages of the 2-node stencil, one node for the
  viscosity's derivatives, one for the block metrics' one-sided faces), less
  than the 13 from the centre to the block faces.
* 576 x 320 x 256 (47M points), Re_D = 1e6: FP64 and mixed side by side, one
  step at sampled nodes against the oracle (FP64 1e-12, mixed 2e-6), and the
  mixed form against FP64 after 200 steps.
* 1000 x 250 x 512 (the 1/8-size subgrid): the compact mixed form against
  plain FP64 after 20 steps, <= 1e-5 relative L2 on rho, rho u, rho E.
"""
import numpy as np
import pytest

from gpu_helpers import BLOCK_HALF, check_blocks, take_blocks

pytestmark = pytest.mark.gpu


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


def _free_bytes(torch):
    import gc
    gc.collect()
    torch.cuda.empty_cache()
    return torch.cuda.mem_get_info()[0]


def test_c5_compact_mixed_sampled_step_and_run(orc, lj, torch):
    shape = (2000, 500, 1024)
    ni, nj, nk = shape
    N = ni * nj * nk
    # state 40 + workspace 128 + coordinates 24 bytes per point, plus slack
    need = N * (40 + 129 + 24) + (4 << 30)
    free = _free_bytes(torch)
    if free < need:
        pytest.skip(f"needs {need / 1e9:.0f} GB of free device memory, {free / 1e9:.0f} GB free")
    ctx = lj.Context(lj.make_params(sgs_model=lj.SGS_SMAGORINSKY,
                                    precision=lj.PREC_MIXED_COMPACT), shape, "cuda:0")
    assert ctx.workspace.numel() <= 129 * N
    xyz = lj.synth.jet_grid_torch(ni, nj, nk, "cuda")
    ctx.les_set_grid(xyz)
    assert ctx.les_metrics() is None
    Q = torch.empty((5,) + shape, dtype=torch.float64, device="cuda")
    ctx.les_init_jet(xyz, 0, 1e-3, Q)
    del xyz
    torch.cuda.empty_cache()

    r = lj.synth.jet_radial(nj)
    centres = [(1000, int(np.argmin(np.abs(r - 0.5))), 300),
               (400, int(np.argmin(np.abs(r - 2.0))), 1000),
               (1700, nj - 1 - BLOCK_HALF - 5, 17)]
    blocks = take_blocks(torch, Q, centres, nk)
    d = ctx.les_run_n_steps(1, Q)
    assert d.status == 0 and d.dt > 0
    check_blocks(orc, lj.synth, shape, Q, centres, blocks, d.dt, 2e-6, sgs_model=1)
    d = ctx.les_run_n_steps(19, Q)
    assert d.status == 0
    assert bool(torch.isfinite(Q).all())
    assert np.all(np.isfinite(d.totals))


def test_subgrid_mixed_error_against_fp64(lj, torch):
    shape = (1000, 250, 512)
    N = shape[0] * shape[1] * shape[2]
    need = N * (24 + 2 * 40 + 300) + (4 << 30)
    free = _free_bytes(torch)
    if free < need:
        pytest.skip(f"needs {need / 1e9:.0f} GB of free device memory, {free / 1e9:.0f} GB free")
    xyz = lj.synth.jet_grid_torch(*shape, "cuda")
    out = {}
    for prec in (lj.PREC_FP64, lj.PREC_MIXED_COMPACT):
        ctx = lj.Context(lj.make_params(sgs_model=lj.SGS_SMAGORINSKY, precision=prec), shape,
                         "cuda:0")
        ctx.les_set_grid(xyz)
        Q = torch.empty((5,) + shape, dtype=torch.float64, device="cuda")
        ctx.les_init_jet(xyz, 0, 1e-3, Q)
        d = ctx.les_run_n_steps(20, Q)
        assert d.status == 0
        out[prec] = Q
        del ctx
        torch.cuda.empty_cache()
    a, b = out[lj.PREC_MIXED_COMPACT], out[lj.PREC_FP64]
    for c in (0, 1, 4):
        err = float(torch.linalg.vector_norm(a[c] - b[c]) / torch.linalg.vector_norm(b[c]))
        assert err <= 1e-5, (c, err)


def test_c3_fp64_and_mixed(orc, lj, torch):
    shape = (576, 320, 256)
    ni, nj, nk = shape
    xyz = lj.synth.jet_grid_torch(*shape, "cuda")
    r = lj.synth.jet_radial(nj)
    centres = [(300, int(np.argmin(np.abs(r - 0.5))), 40),
               (100, int(np.argmin(np.abs(r - 3.0))), 255),
               (ni - 1 - BLOCK_HALF, nj - 1 - BLOCK_HALF, 128)]
    out = {}
    for prec, tol in ((lj.PREC_FP64, 1e-12), (lj.PREC_MIXED, 2e-6)):
        ctx = lj.Context(lj.make_params(Re=1.0e6, sgs_model=lj.SGS_SMAGORINSKY, precision=prec),
                         shape, "cuda:0")
        ctx.les_set_grid(xyz)
        Q = torch.empty((5,) + shape, dtype=torch.float64, device="cuda")
        ctx.les_init_jet(xyz, 0, 1e-3, Q)
        blocks = take_blocks(torch, Q, centres, nk)
        d = ctx.les_run_n_steps(1, Q)
        check_blocks(orc, lj.synth, shape, Q, centres, blocks, d.dt, tol, Re=1.0e6, sgs_model=1)
        d = ctx.les_run_n_steps(199, Q)
        assert d.status == 0
        out[prec] = Q
        del ctx
    a, b = out[lj.PREC_MIXED], out[lj.PREC_FP64]
    for c in (0, 1, 4):
        err = float(torch.linalg.vector_norm(a[c] - b[c]) / torch.linalg.vector_norm(b[c]))
        assert err <= 1e-5, (c, err)
