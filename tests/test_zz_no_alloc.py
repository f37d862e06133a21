"""les_time_step_static: the time step for callers that cannot allocate
device memory (a hook running inside an application that has committed all
device memory to its own pool, or a tool handed only raw device pointers).

It must give the same time step as les_time_step, which uses the caller's
workspace, on consecutive calls; its scratch is one static device array in
the library, so a call must not see a previous call's contents.  Kept in a
file of its own that pytest collects last.
"""
import ctypes as C
import os
import subprocess
import sys

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


@pytest.mark.parametrize("mode", ["fixed", "local"])
def test_static_time_step_other_step_modes(env, mode):
    """dt_mode FIXED returns the configured step (the state is still checked);
    dt_mode LOCAL returns the clock's advance, the smallest per-node step,
    as les_time_step does (which also writes the per-node steps)."""
    lj, torch = env
    kw = dict(dt_mode=lj.DT_FIXED, dt_fixed=3.25e-4) if mode == "fixed" else dict(dt_mode=lj.DT_LOCAL)
    ctx, xyz = _jet_ctx(lj, torch, (30, 14, 16), **kw)
    Q = torch.empty((5,) + ctx.shape, dtype=torch.float64, device="cuda")
    for seed in (2, 3):
        ctx.les_init_jet(xyz, seed, 1e-2, Q)
        ref = ctx.les_time_step(Q)
        M = ctx.les_metrics().contiguous()
        for _ in range(2):
            got = ctx.les_time_step_static(Q, M)
            assert abs(got - ref) <= 1e-14 * ref, (mode, got, ref)
        if mode == "fixed":
            assert got == 3.25e-4


def test_static_time_step_on_a_mixed_contexts_metrics(env):
    """A mixed context keeps an FP64 metric copy: handed that copy, the
    static entry point gives the FP64 step of an FP64 context with the same
    grid and state; the mixed context's own step (FP32 radii) agrees to
    FP32 rounding."""
    lj, torch = env
    shape = (26, 12, 16)
    cm, xyz = _jet_ctx(lj, torch, shape, precision=lj.PREC_MIXED)
    c64, _ = _jet_ctx(lj, torch, shape)
    Q = torch.empty((5,) + shape, dtype=torch.float64, device="cuda")
    c64.les_init_jet(xyz, 4, 1e-2, Q)
    ref64 = c64.les_time_step(Q)
    Mm = cm.les_metrics()
    assert Mm is not None
    got = cm.les_time_step_static(Q, Mm.contiguous())
    assert abs(got - ref64) <= 1e-14 * ref64, (got, ref64)
    assert abs(got - cm.les_time_step(Q)) <= 1e-6 * ref64


_CONTEXT_CHANGE = r"""
import ctypes as C, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import oracle
import paper_2301_00817_gb300 as lj
shape = (20, 12, 16)
xyz = lj.synth.jet_grid(*shape)
P = oracle.params()
M = np.ascontiguousarray(oracle.metrics(xyz, (0, 0, 1)))
Q = np.ascontiguousarray(oracle.init_jet(P, xyz, seed=3, noise=1e-2))
ref = oracle.dt(P, Q, M)
cu = C.CDLL("libcuda.so.1")
def ok(r, what):
    if r != 0:
        raise SystemExit(f"driver call {what} returned {r}")
ok(cu.cuInit(0), "cuInit")
dev = C.c_int()
ok(cu.cuDeviceGet(C.byref(dev), 0), "cuDeviceGet")
lib = lj.load_library()
h = C.c_void_p()
p = lj.make_params()
assert lib.les_create(C.byref(p), *shape, C.byref(h)) == 0
def call_in(ctx):
    ok(cu.cuCtxPushCurrent_v2(ctx), "cuCtxPushCurrent")
    bufs = []
    for a in (Q, M):
        d = C.c_uint64()
        ok(cu.cuMemAlloc_v2(C.byref(d), C.c_size_t(a.nbytes)), "cuMemAlloc")
        ok(cu.cuMemcpyHtoD_v2(d, a.ctypes.data_as(C.c_void_p), C.c_size_t(a.nbytes)), "cuMemcpyHtoD")
        bufs.append(d)
    out = []
    for _ in range(2):
        dt = C.c_double()
        rc = lib.les_time_step_static(h, C.c_void_p(bufs[0].value), C.c_void_p(bufs[1].value),
                                      C.byref(dt), None)
        assert rc == 0, (rc, lib.les_last_error(h))
        out.append(dt.value)
    for d in bufs:
        ok(cu.cuMemFree_v2(d), "cuMemFree")
    popped = C.c_void_p()
    ok(cu.cuCtxPopCurrent_v2(C.byref(popped)), "cuCtxPopCurrent")
    return out
prim = C.c_void_p()
ok(cu.cuDevicePrimaryCtxRetain(C.byref(prim), dev), "cuDevicePrimaryCtxRetain")
other = C.c_void_p()
if hasattr(cu, "cuCtxCreate_v2"):
    ok(cu.cuCtxCreate_v2(C.byref(other), 0, dev), "cuCtxCreate")
else:
    ok(cu.cuCtxCreate_v4(C.byref(other), None, 0, dev), "cuCtxCreate")
ok(cu.cuCtxPopCurrent_v2(C.byref(C.c_void_p())), "cuCtxPopCurrent")
res = call_in(prim) + call_in(other) + call_in(prim)
ok(cu.cuCtxDestroy_v2(other), "cuCtxDestroy")
ok(cu.cuDevicePrimaryCtxRelease_v2(dev), "cuDevicePrimaryCtxRelease")
lib.les_destroy(h)
for v in res:
    assert abs(v - ref) <= 1e-13 * ref, (res, ref)
print("context change ok", res, ref)
"""


def test_static_time_step_across_a_context_change(env, tmp_path):
    """The scratch array lives in a module that every CUDA context loads at
    its own address.  A caller that switches contexts (here: the primary
    context, a second context created through the driver API, then the
    primary one again, in a fresh process) must get the right step in each,
    which holds only if the address is looked up for each context."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "ctx_change.py"
    script.write_text(_CONTEXT_CHANGE)
    r = subprocess.run([sys.executable, str(script), root], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    assert "context change ok" in r.stdout


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
