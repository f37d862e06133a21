"""les_time_step_static: the time step for callers that cannot allocate
device memory (a hook running inside an application that has committed all
device memory to its own pool, or a tool handed only raw device pointers).

It must give the same time step as les_time_step, which uses the caller's
workspace, on consecutive calls; its scratch is one static device array in
the library, so a call must not see a previous call's contents.  Kept in a
file of its own that pytest collects last.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2301_00817_gb300 import _build
    _build.build()
    import paper_2301_00817_gb300 as lj
    lj.load_library()
    return lj, torch


def _jet_ctx(lj, torch, shape, **kw):
    ctx = lj.Context(lj.make_params(**kw), shape, "cuda:0")
    xyz = torch.from_numpy(lj.synth.jet_grid(*shape)).cuda()
    ctx.les_set_grid(xyz)
    return ctx, xyz


def test_static_time_step_matches_workspace_version(env):
    lj, torch = env
    big, xyz_big = _jet_ctx(lj, torch, (48, 24, 32))
    small, xyz_small = _jet_ctx(lj, torch, (13, 9, 7), cfl=0.9)
    cases = [(big, xyz_big, 1, 1e-3), (big, xyz_big, 2, 5e-2), (small, xyz_small, 3, 1e-2),
             (big, xyz_big, 4, 1e-3)]
    for ctx, xyz, seed, noise in cases:
        Q = torch.empty((5,) + ctx.shape, dtype=torch.float64, device="cuda")
        ctx.les_init_jet(xyz, seed, noise, Q)
        ref = ctx.les_time_step(Q)
        M = ctx.les_metrics().contiguous()
        got1 = ctx.les_time_step_static(Q, M)
        got2 = ctx.les_time_step_static(Q, M)
        assert abs(got1 - ref) <= 1e-14 * ref, (got1, ref)
        assert abs(got2 - ref) <= 1e-14 * ref, (got2, ref)


def test_static_time_step_needs_no_workspace(env):
    """A context that never received a workspace (les_create only) works."""
    lj, torch = env
    owner, xyz = _jet_ctx(lj, torch, (20, 12, 16))
    Q = torch.empty((5, 20, 12, 16), dtype=torch.float64, device="cuda")
    owner.les_init_jet(xyz, 9, 1e-3, Q)
    ref = owner.les_time_step(Q)
    h = C.c_void_p()
    p = lj.make_params()
    assert owner.lib.les_create(C.byref(p), 20, 12, 16, C.byref(h)) == lj.LES_OK
    out = C.c_double()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = owner.lib.les_time_step_static(h, C.c_void_p(Q.data_ptr()),
                                        C.c_void_p(owner.les_metrics().data_ptr()),
                                        C.byref(out), stream)
    assert rc == lj.LES_OK
    assert abs(out.value - ref) <= 1e-14 * ref
    owner.lib.les_destroy(h)


def test_static_time_step_rejects_oversize_and_bad_state(env):
    lj, torch = env
    h = C.c_void_p()
    p = lj.make_params()
    assert owner_create(lj, p, 16385, h) == lj.LES_OK
    lib = lj.load_library()
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = C.c_double()
    rc = lib.les_time_step_static(h, C.c_void_p(buf.data_ptr()), C.c_void_p(buf.data_ptr()),
                                  C.byref(out), None)
    assert rc == lj.LES_ERR_SHAPE
    assert b"LES_STATIC_MAX_NI" in lib.les_last_error(h)
    lib.les_destroy(h)
    ctx, xyz = _jet_ctx(lj, torch, (16, 10, 8))
    Q = torch.empty((5, 16, 10, 8), dtype=torch.float64, device="cuda")
    ctx.les_init_jet(xyz, 1, 1e-3, Q)
    Q[0, 5, 5, 5] = float("nan")
    with pytest.raises(lj.LesError) as e:
        ctx.les_time_step_static(Q, ctx.les_metrics().contiguous())
    assert e.value.code == lj.LES_ERR_NONFINITE


def owner_create(lj, p, ni, h):
    lib = lj.load_library()
    return lib.les_create(C.byref(p), ni, 5, 5, C.byref(h))
