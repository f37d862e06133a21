"""GB300 (sm_103a) implementation of the LES hot path of arXiv 2301.00817.

Thin Python binding over the C ABI of ``liblesjet.so`` (``include/lesjet.h``).
The functions below only marshal arguments: every step of the residual and
the time step runs in the library's CUDA kernels.  PyTorch provides device
memory and streams.  There is no CPU fallback: importing the binding without
the built library, or calling it without a CUDA device, raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

from . import synth  # noqa: F401  (seeded synthetic inputs)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblesjet.so")

LES_OK = 0
LES_ERR_INVALID_ARG = -1
LES_ERR_SHAPE = -2
LES_ERR_ALIGN = -3
LES_ERR_CUDA = -4
LES_ERR_NONFINITE = -5
LES_ERR_UNSUPPORTED = -6
LES_ERR_STATE = -7

SGS_NONE, SGS_SMAGORINSKY, SGS_VREMAN, SGS_DYNAMIC = 0, 1, 2, 3
PREC_FP64, PREC_MIXED, PREC_MIXED_COMPACT = 0, 1, 2
BC_FROZEN, BC_JET, BC_JET_CHAR = 0, 1, 2
DT_CFL, DT_FIXED, DT_LOCAL = 0, 1, 2
METRIC_CROSS, METRIC_CONSERVATIVE = 0, 1


class LesError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"lesjet error {code}: {msg}")
        self.code = code


class LesParams(C.Structure):
    """Mirror of ``les_params`` in include/lesjet.h."""
    _fields_ = [
        ("gamma", C.c_double), ("Pr", C.c_double), ("Pr_sgs", C.c_double),
        ("Mj", C.c_double), ("Re", C.c_double), ("T_ref", C.c_double),
        ("k2", C.c_double), ("k4", C.c_double), ("Cs", C.c_double),
        ("cfl", C.c_double), ("dt_fixed", C.c_double), ("r_jet", C.c_double),
        ("theta_m", C.c_double), ("force_width", C.c_double),
        ("St", C.c_double * 4), ("amp", C.c_double * 16),
        ("sgs_model", C.c_int), ("periodic", C.c_int * 3), ("bc", C.c_int),
        ("dt_mode", C.c_int), ("freeze_visc", C.c_int), ("precision", C.c_int),
        ("metric_form", C.c_int),
        ("axis", C.c_int),
        ("slab_ghost", C.c_int * 2),
    ]


class LesDiag(C.Structure):
    _fields_ = [("t", C.c_double), ("dt", C.c_double), ("totals", C.c_double * 5),
                ("status", C.c_int), ("steps", C.c_int)]


class LesJetGrid(C.Structure):
    """Mirror of ``les_jet_grid`` in include/lesjet.h."""
    _fields_ = [("length", C.c_double), ("ratio", C.c_double), ("r0", C.c_double),
                ("r1", C.c_double), ("r_c", C.c_double), ("A", C.c_double),
                ("beta", C.c_double)]


def make_params(**kw) -> LesParams:
    """les_params with the jet workload's defaults, overridden by kw."""
    d = dict(gamma=1.4, Pr=0.72, Pr_sgs=0.9, Mj=1.4, Re=1.0e5, T_ref=288.15,
             k2=0.25, k4=0.016, Cs=0.148, cfl=0.5, dt_fixed=0.0, r_jet=0.5,
             theta_m=0.05, force_width=0.05, St=(0.25, 0.5, 0.75, 1.0),
             amp=(0.0,) * 16, sgs_model=SGS_NONE, periodic=(0, 0, 1), bc=BC_JET,
             dt_mode=DT_CFL, freeze_visc=1, precision=PREC_FP64, metric_form=METRIC_CROSS,
             axis=0, slab_ghost=(0, 0))
    d.update(kw)
    p = LesParams()
    for k, v in d.items():
        if k in ("St", "amp", "periodic", "slab_ghost"):
            arr = getattr(p, k)
            for i, x in enumerate(v):
                arr[i] = int(x) if k in ("periodic", "slab_ghost") else float(x)
        else:
            setattr(p, k, v)
    return p


_lib = None


def load_library(path: str = LIB_PATH):
    """Load liblesjet.so (built by ``_build.build()``); raises if missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    vp, i, d = C.c_void_p, C.c_int, C.c_double
    P = C.POINTER(LesParams)
    lib.les_create.argtypes = [P, i, i, i, C.POINTER(vp)]
    lib.les_destroy.argtypes = [vp]
    lib.les_last_error.argtypes = [vp]
    lib.les_last_error.restype = C.c_char_p
    lib.les_set_params.argtypes = [vp, P]
    lib.les_workspace_bytes.argtypes = [vp]
    lib.les_workspace_bytes.restype = C.c_size_t
    lib.les_set_grid.argtypes = [vp, vp, C.POINTER(d), vp, vp]
    lib.les_metrics.argtypes = [vp]
    lib.les_metrics.restype = vp
    lib.les_init_jet.argtypes = [vp, vp, C.c_uint64, d, vp, vp]
    lib.les_mu_eff.argtypes = [vp, vp, vp, vp]
    lib.les_rhs.argtypes = [vp, vp, vp, vp]
    lib.les_time_step.argtypes = [vp, vp, C.POINTER(d), vp]
    lib.les_apply_bc.argtypes = [vp, vp, d, vp]
    lib.les_set_time.argtypes = [vp, d, vp]
    lib.les_rk_step.argtypes = [vp, vp, vp]
    lib.les_run_n_steps.argtypes = [vp, i, vp, C.POINTER(LesDiag), vp]
    lib.les_run_host.argtypes = [vp, i, vp, vp, C.POINTER(LesDiag), vp]
    lib.les_totals.argtypes = [vp, vp, C.POINTER(d), vp]
    lib.les_launch_count.argtypes = [vp]
    lib.les_launch_count.restype = C.c_uint64
    lib.les_profile.argtypes = [vp, i]
    lib.les_profile.restype = C.c_int
    lib.les_profile_read.argtypes = [vp, C.POINTER(d), C.POINTER(C.c_uint64), vp]
    lib.les_profile_read.restype = C.c_int
    lib.les_profile_name.argtypes = [i]
    lib.les_profile_name.restype = C.c_char_p
    lib.les_measure_fma_peak.argtypes = [i, C.POINTER(d), vp]
    lib.les_dynamic_coefficients.argtypes = [vp, vp, C.POINTER(d), vp]
    lib.les_dynamic_coefficients.restype = C.c_int
    lib.les_grid_jet.argtypes = [i, i, i, C.POINTER(LesJetGrid), vp, vp]
    lib.les_grid_jet.restype = C.c_int
    lib.les_surface_functional.argtypes = [vp, vp, i, d, C.POINTER(d), vp]
    lib.les_time_step_static.argtypes = [vp, vp, vp, C.POINTER(d), vp]
    lib.les_time_step_static.restype = C.c_int
    lib.les_adjoint_workspace_bytes.argtypes = [vp, i, i]
    lib.les_adjoint_workspace_bytes.restype = C.c_size_t
    lib.les_rhs_jvp.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
    lib.les_rhs_vjp.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    lib.les_adjoint_step.argtypes = [vp, vp, d, vp, vp, C.POINTER(d), vp, vp]
    lib.les_adjoint_window.argtypes = [vp, vp, d, i, i, i, vp, C.POINTER(d), C.POINTER(d), vp]
    for name in ("les_rhs_jvp", "les_rhs_vjp", "les_adjoint_step", "les_adjoint_window"):
        getattr(lib, name).restype = C.c_int
    lib.les_step_begin.argtypes = [vp, vp, C.POINTER(d), vp]
    lib.les_step_set_dt.argtypes = [vp, d, vp]
    lib.les_step_stage.argtypes = [vp, i, vp, vp]
    lib.les_step_end.argtypes = [vp, vp, vp]
    lib.les_state_load.argtypes = [vp, vp, vp]
    lib.les_state_store.argtypes = [vp, vp, vp]
    lib.les_state_buffer.argtypes = [vp, i, C.POINTER(vp), C.POINTER(vp), C.POINTER(i)]
    lib.les_halo_copy.argtypes = [vp, vp, vp, vp, i, i, vp]
    for name in ("les_step_begin", "les_step_set_dt", "les_step_stage", "les_step_end",
                 "les_state_load", "les_state_store", "les_state_buffer", "les_halo_copy"):
        getattr(lib, name).restype = C.c_int
    for name in ("les_create", "les_destroy", "les_set_params", "les_set_grid", "les_init_jet",
                 "les_mu_eff", "les_rhs", "les_time_step", "les_apply_bc", "les_set_time",
                 "les_rk_step", "les_run_n_steps", "les_run_host", "les_totals"):
        getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("lesjet needs a CUDA device; there is no CPU fallback")
    return torch


def _ptr(t) -> int:
    assert t.is_cuda and t.is_contiguous(), "device tensors must be contiguous CUDA tensors"
    return t.data_ptr()


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def measure_fma_peak(precision: int, stream=None) -> float:
    """Measured FMA throughput (TFLOP/s) of the current device: FP64 for
    PREC_FP64, FP32 for the mixed precisions (les_measure_fma_peak)."""
    lib = load_library()
    out = C.c_double()
    rc = lib.les_measure_fma_peak(precision, C.byref(out), _stream(stream))
    if rc != LES_OK:
        raise LesError(rc, "les_measure_fma_peak failed")
    return out.value


def grid_jet(shape, xyz=None, length: float = 20.0, ratio: float = 0.0, r0: float = 0.02,
             r1: float = 10.0, r_c: float = 0.5, A: float = 0.9, beta: float = 8.0,
             stream=None):
    """The synthetic annular jet grid written on the device (les_grid_jet):
    coordinates [3, ni, nj, nk] FP64, into ``xyz`` when given.  ratio <= 0
    selects the axial stretching rule (1.01 up to 288 planes, 1.01^(288/ni)
    beyond)."""
    torch = _torch()
    lib = load_library()
    ni, nj, nk = (int(v) for v in shape)
    if xyz is None:
        xyz = torch.empty((3, ni, nj, nk), dtype=torch.float64, device="cuda")
    assert xyz.dtype == torch.float64 and xyz.numel() == 3 * ni * nj * nk
    g = LesJetGrid(length, ratio, r0, r1, r_c, A, beta)
    rc = lib.les_grid_jet(ni, nj, nk, C.byref(g), _ptr(xyz), _stream(stream))
    if rc != LES_OK:
        raise LesError(rc, "les_grid_jet failed")
    return xyz


class Context:
    """Owns a les_ctx and the device workspace tensor bound to it."""

    def __init__(self, params: LesParams, shape, device="cuda:0"):
        self.lib = load_library()
        torch = _torch()
        self.params = params
        self.shape = tuple(int(x) for x in shape)
        self.device = torch.device(device)
        h = C.c_void_p()
        rc = self.lib.les_create(C.byref(params), *self.shape, C.byref(h))
        if rc != LES_OK:
            raise LesError(rc, "les_create rejected the parameters or the shape")
        self.h = h
        nbytes = int(self.lib.les_workspace_bytes(h))
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.N = self.shape[0] * self.shape[1] * self.shape[2]

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            self.lib.les_destroy(h)
            self.h = None

    def _check(self, rc: int):
        if rc != LES_OK:
            raise LesError(rc, self.lib.les_last_error(self.h).decode())

    # --- C-ABI mirrors -----------------------------------------------------
    def les_set_params(self, params: LesParams):
        self._check(self.lib.les_set_params(self.h, C.byref(params)))
        self.params = params

    def les_set_grid(self, xyz, shift=None, stream=None):
        sh = (C.c_double * 9)(*([0.0] * 9 if shift is None else [float(x) for x in shift]))
        self._check(self.lib.les_set_grid(self.h, _ptr(xyz), sh, _ptr(self.workspace),
                                          _stream(stream)))

    def les_metrics(self):
        """FP64 metrics [10, ni, nj, nk] (a view of the workspace), or None for
        a compact mixed context, which keeps FP32 metrics only."""
        torch = _torch()
        ptr = self.lib.les_metrics(self.h)
        if not ptr:
            return None
        off = ptr - self.workspace.data_ptr()
        return self.workspace[off:off + 80 * self.N].view(torch.float64).view(10, *self.shape)

    def les_init_jet(self, xyz, seed: int, noise: float, Q, stream=None):
        self._check(self.lib.les_init_jet(self.h, _ptr(xyz), seed, noise, _ptr(Q), _stream(stream)))

    def les_mu_eff(self, Q, MK, stream=None):
        self._check(self.lib.les_mu_eff(self.h, _ptr(Q), _ptr(MK), _stream(stream)))

    def les_dynamic_coefficients(self, Q, stream=None) -> dict:
        """The dynamic SGS procedure on Q (les_dynamic_coefficients): the six
        averaged terms and C_ds, C_I, Pr_sgs."""
        out = (C.c_double * 9)()
        self._check(self.lib.les_dynamic_coefficients(self.h, _ptr(Q), out, _stream(stream)))
        keys = ("numC", "denC", "numI", "denI", "numP", "denP", "Cd", "CI", "Prt")
        return dict(zip(keys, list(out)))

    def les_rhs(self, Q, R, stream=None):
        self._check(self.lib.les_rhs(self.h, _ptr(Q), _ptr(R), _stream(stream)))

    def les_time_step(self, Q, stream=None) -> float:
        out = C.c_double()
        self._check(self.lib.les_time_step(self.h, _ptr(Q), C.byref(out), _stream(stream)))
        return out.value

    def les_surface_functional(self, Q, j_surface: int, w: float, stream=None) -> float:
        """w * sum over the eta surface j_surface of (p - 1/gamma)^2 dA."""
        out = C.c_double()
        self._check(self.lib.les_surface_functional(self.h, _ptr(Q), j_surface, w, C.byref(out),
                                                    _stream(stream)))
        return out.value

    def les_time_step_static(self, Q, M, stream=None) -> float:
        """Time step without workspace or allocation (static library scratch)."""
        out = C.c_double()
        self._check(self.lib.les_time_step_static(self.h, _ptr(Q), _ptr(M), C.byref(out),
                                                  _stream(stream)))
        return out.value

    # --- discrete adjoint (FP64) -------------------------------------------
    def adjoint_workspace(self, nsteps: int = 1, ckpt_every: int = 1):
        torch = _torch()
        nbytes = int(self.lib.les_adjoint_workspace_bytes(self.h, nsteps, ckpt_every))
        return torch.empty(nbytes, dtype=torch.uint8, device=self.device)

    def les_rhs_jvp(self, Q, dQ, dMK, R, dR, aw, stream=None):
        opt = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None
        self._check(self.lib.les_rhs_jvp(self.h, _ptr(Q), _ptr(dQ), opt(dMK), opt(R), _ptr(dR),
                                         _ptr(aw), _stream(stream)))

    def les_rhs_vjp(self, Q, lamR, lamQ, lamMK, aw, stream=None):
        self._check(self.lib.les_rhs_vjp(self.h, _ptr(Q), _ptr(lamR), _ptr(lamQ), _ptr(lamMK),
                                         _ptr(aw), _stream(stream)))

    def les_adjoint_step(self, Qn, t_n: float, lam_next, lam_out, aw, stream=None):
        g = (C.c_double * 16)()
        self._check(self.lib.les_adjoint_step(self.h, _ptr(Qn), t_n, _ptr(lam_next), _ptr(lam_out),
                                              g, _ptr(aw), _stream(stream)))
        return list(g)

    def les_adjoint_window(self, Q_start, t0: float, nsteps: int, ckpt_every: int,
                           j_surface: int, aw, stream=None):
        J = C.c_double()
        g = (C.c_double * 16)()
        self._check(self.lib.les_adjoint_window(self.h, _ptr(Q_start), t0, nsteps, ckpt_every,
                                                j_surface, _ptr(aw), C.byref(J), g,
                                                _stream(stream)))
        return J.value, list(g)

    def les_apply_bc(self, Q, t: float, stream=None):
        self._check(self.lib.les_apply_bc(self.h, _ptr(Q), t, _stream(stream)))

    def les_set_time(self, t: float, stream=None):
        self._check(self.lib.les_set_time(self.h, t, _stream(stream)))

    def les_rk_step(self, Q, stream=None):
        self._check(self.lib.les_rk_step(self.h, _ptr(Q), _stream(stream)))

    def les_run_n_steps(self, n: int, Q, stream=None) -> LesDiag:
        diag = LesDiag()
        self._check(self.lib.les_run_n_steps(self.h, n, _ptr(Q), C.byref(diag), _stream(stream)))
        return diag

    # --- one step in phases (axial slabs; see slabs.py) -------------------
    def les_step_begin(self, Q, stream=None) -> float:
        """Viscosity and the CFL step of this slab's own planes; synchronises."""
        out = C.c_double()
        self._check(self.lib.les_step_begin(self.h, _ptr(Q), C.byref(out), _stream(stream)))
        return out.value

    def les_step_set_dt(self, dt: float, stream=None):
        self._check(self.lib.les_step_set_dt(self.h, dt, _stream(stream)))

    def les_step_stage(self, l: int, Q, stream=None):
        self._check(self.lib.les_step_stage(self.h, l, _ptr(Q), _stream(stream)))

    def les_step_end(self, Q, stream=None):
        self._check(self.lib.les_step_end(self.h, _ptr(Q), _stream(stream)))

    def les_state_load(self, Q, stream=None):
        self._check(self.lib.les_state_load(self.h, _ptr(Q), _stream(stream)))

    def les_state_store(self, Q, stream=None):
        self._check(self.lib.les_state_store(self.h, _ptr(Q), _stream(stream)))

    def state_views(self, l: int, Q):
        """The arrays holding the state after stage l (les_state_buffer), as
        [5, ni, nj, nk] views: the caller's Q, a stage buffer of the
        workspace, or the float pair (hi, lo) of the mixed forms."""
        torch = _torch()
        a, b, e = C.c_void_p(), C.c_void_p(), C.c_int()
        self._check(self.lib.les_state_buffer(self.h, l, C.byref(a), C.byref(b), C.byref(e)))
        if not a.value:
            return [Q]
        dt = torch.float32 if e.value == 4 else torch.float64
        out = []
        for ptr in (a.value, b.value):
            if not ptr:
                continue
            off = ptr - self.workspace.data_ptr()
            nbytes = 5 * self.N * e.value
            out.append(self.workspace[off:off + nbytes].view(dt).view(5, *self.shape))
        return out

    def les_halo_copy(self, Q, src, Q_src, l: int, side: int, stream=None):
        """Ghost planes of this slab from the neighbouring slab src (same
        process): side 0, src lies below along xi; side 1, above."""
        self._check(self.lib.les_halo_copy(self.h, _ptr(Q), src.h, _ptr(Q_src), l, side,
                                           _stream(stream)))

    def les_run_host(self, n: int, Q_host, Q_dev, stream=None) -> LesDiag:
        assert not Q_host.is_cuda and Q_host.is_contiguous()
        diag = LesDiag()
        self._check(self.lib.les_run_host(self.h, n, C.c_void_p(Q_host.data_ptr()), _ptr(Q_dev),
                                          C.byref(diag), _stream(stream)))
        return diag

    def les_totals(self, Q, stream=None):
        out = (C.c_double * 5)()
        self._check(self.lib.les_totals(self.h, _ptr(Q), out, _stream(stream)))
        return list(out)

    def les_launch_count(self) -> int:
        return int(self.lib.les_launch_count(self.h))

    def les_profile(self, enable: bool):
        self._check(self.lib.les_profile(self.h, 1 if enable else 0))

    def les_profile_read(self, stream=None) -> dict:
        ms = (C.c_double * 16)()
        n = (C.c_uint64 * 16)()
        self._check(self.lib.les_profile_read(self.h, ms, n, _stream(stream)))
        out = {}
        for k in range(16):
            name = self.lib.les_profile_name(k).decode()
            if name:
                out[name] = (float(ms[k]), int(n[k]))
        return out


@dataclass
class Solver:
    """Convenience wrapper: a context, its grid and a device state."""
    params: LesParams
    shape: tuple
    xyz: object = None
    shift: object = None
    ctx: Context = field(init=False)

    def __post_init__(self):
        torch = _torch()
        self.ctx = Context(self.params, self.shape)
        if self.xyz is None:
            self.xyz = synth.jet_grid(*self.shape)
        xyz = torch.as_tensor(self.xyz, dtype=torch.float64).to(self.ctx.device).contiguous()
        self.ctx.les_set_grid(xyz, self.shift)
        self._xyz_dev = xyz

    def new_state(self):
        torch = _torch()
        return torch.empty((5,) + tuple(self.shape), dtype=torch.float64, device=self.ctx.device)

    def init_jet(self, seed: int = 0, noise: float = 1.0e-3):
        Q = self.new_state()
        self.ctx.les_init_jet(self._xyz_dev, seed, noise, Q)
        return Q

    def rhs(self, Q):
        R = self.new_state()
        self.ctx.les_rhs(Q, R)
        return R

    def step(self, Q):
        """One time step in place (Delta t, five RK stages, boundary conditions)."""
        self.ctx.les_rk_step(Q)
        return Q

    def run(self, Q, n: int) -> LesDiag:
        return self.ctx.les_run_n_steps(n, Q)


def window_functional(ctx: "Context", amplitudes, Q_start, t0: float, nsteps: int,
                      ckpt_every: int, j_surface: int, aw=None):
    """Differentiable far-field functional of the 16 inflow forcing amplitudes.

    Returns J (0-d float64 tensor) whose backward gives dJ/da from the
    hand-written discrete adjoint (les_adjoint_window)."""
    torch = _torch()

    class _Window(torch.autograd.Function):
        @staticmethod
        def forward(fctx, amps):
            p = LesParams.from_buffer_copy(ctx.params)
            for k in range(16):
                p.amp[k] = float(amps[k])
            ctx.les_set_params(p)
            ws = aw if aw is not None else ctx.adjoint_workspace(nsteps, ckpt_every)
            J, g = ctx.les_adjoint_window(Q_start, t0, nsteps, ckpt_every, j_surface, ws)
            fctx.save_for_backward(torch.tensor(g, dtype=torch.float64))
            return torch.tensor(J, dtype=torch.float64)

        @staticmethod
        def backward(fctx, gJ):
            (g,) = fctx.saved_tensors
            return gJ * g

    return _Window.apply(torch.as_tensor(amplitudes, dtype=torch.float64))
