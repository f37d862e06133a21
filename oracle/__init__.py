"""Plain FP64 CPU oracle of the LES residual / RK5 step of arXiv 2301.00817.

TEST INFRASTRUCTURE.  Only the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library (``paper_2301_00817_gb300``) and the library never
imports it.

The arithmetic lives in ``les_oracle.c`` (plain loops, FP64, no fused
multiply-add); this module only compiles it with gcc and marshals numpy
arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "les_oracle.c")
_HDR = os.path.join(_HERE, "les_oracle.h")
_LIB = os.path.join(_HERE, "liblesoracle.so")
_lock = threading.Lock()
_lib = None

GCC_FLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
             "-shared", "-std=c99"]


def build(force: bool = False) -> str:
    """Compile the oracle shared library in place (gcc, no FMA contraction)."""
    stale = (not os.path.exists(_LIB) or
             os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", *GCC_FLAGS, "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class OrcParams(C.Structure):
    _fields_ = [
        ("gamma", C.c_double), ("Pr", C.c_double), ("Pr_sgs", C.c_double),
        ("Mj", C.c_double), ("Re", C.c_double), ("T_ref", C.c_double),
        ("k2", C.c_double), ("k4", C.c_double), ("Cs", C.c_double),
        ("cfl", C.c_double), ("dt_fixed", C.c_double), ("r_jet", C.c_double),
        ("theta_m", C.c_double), ("force_width", C.c_double),
        ("St", C.c_double * 4), ("amp", C.c_double * 16),
        ("sgs_model", C.c_int), ("periodic", C.c_int * 3), ("bc", C.c_int),
        ("dt_mode", C.c_int), ("freeze_visc", C.c_int), ("axis", C.c_int),
    ]


def params(**kw) -> OrcParams:
    """Oracle parameters; defaults are the jet configuration's values."""
    d = dict(gamma=1.4, Pr=0.72, Pr_sgs=0.9, Mj=1.4, Re=1.0e5, T_ref=288.15,
             k2=0.25, k4=0.016, Cs=0.148, cfl=0.5, dt_fixed=0.0, r_jet=0.5,
             theta_m=0.05, force_width=0.05, St=(0.25, 0.5, 0.75, 1.0),
             amp=(0.0,) * 16, sgs_model=0, periodic=(0, 0, 1), bc=1, dt_mode=0,
             freeze_visc=1, axis=0)
    d.update(kw)
    p = OrcParams()
    for k, v in d.items():
        if k in ("St", "amp", "periodic"):
            arr = getattr(p, k)
            for i, x in enumerate(v):
                arr[i] = x
        else:
            setattr(p, k, v)
    return p


_dp = C.POINTER(C.c_double)


def _lib_handle():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            P = C.POINTER(OrcParams)
            i = C.c_int
            lib.orc_metrics.argtypes = [i, i, i, C.POINTER(C.c_int), _dp, _dp, _dp]
            lib.orc_metrics_conservative.argtypes = [i, i, i, C.POINTER(C.c_int), _dp, _dp, _dp]
            lib.orc_prim_to_cons.argtypes = [P, C.c_size_t, _dp, _dp]
            lib.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32),
                                               C.POINTER(C.c_uint32)]
            lib.orc_normals3.argtypes = [C.c_uint64, C.c_uint64, _dp]
            lib.orc_init_jet.argtypes = [P, i, i, i, _dp, C.c_uint64, C.c_double, _dp]
            lib.orc_mu_eff.argtypes = [P, i, i, i, _dp, _dp, _dp]
            lib.orc_rhs.argtypes = [P, i, i, i, _dp, _dp, _dp, _dp]
            lib.orc_interface_flux.argtypes = [P, i, i, i, _dp, _dp, _dp, i, i, i, i, _dp]
            lib.orc_dt.argtypes = [P, i, i, i, _dp, _dp]
            lib.orc_dt.restype = C.c_double
            lib.orc_bc_jet.argtypes = [P, i, i, i, _dp, _dp, _dp, C.c_double]
            lib.orc_rk_step.argtypes = [P, i, i, i, _dp, _dp, _dp, C.c_double]
            lib.orc_rk_step.restype = C.c_double
            lib.orc_totals.argtypes = [i, i, i, _dp, _dp, _dp]
            lib.orc_surface_functional.argtypes = [P, i, i, i, _dp, _dp, i, C.c_double]
            lib.orc_surface_functional.restype = C.c_double
            lib.orc_num_threads.restype = C.c_int
            lib.orc_set_num_threads.argtypes = [i]
            RHSFN = C.CFUNCTYPE(None, C.c_void_p, _dp, _dp)
            lib.orc_rk5.argtypes = [i, C.c_size_t, _dp, C.POINTER(C.c_ubyte), _dp,
                                    C.c_double, _dp, RHSFN, C.c_void_p]
            lib.orc_dt_local.argtypes = [P, i, i, i, _dp, _dp, _dp]
            lib.orc_dynamic_coefficients.argtypes = [P, i, i, i, _dp, _dp, _dp]
            lib.orc_test_filter.argtypes = [i, i, i, C.POINTER(C.c_int), _dp, _dp]
            lib._RHSFN = RHSFN
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], (a.dtype, a.flags)
    return a.ctypes.data_as(_dp)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(_lib_handle().orc_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the oracle's OpenMP loops (its results do not depend on it)."""
    _lib_handle().orc_set_num_threads(int(n))


def metrics(xyz, periodic=(0, 0, 1), shift=None, form: int = 0) -> np.ndarray:
    """xyz [3, ni, nj, nk] -> M [10, ni, nj, nk] (metrics then J^-1).
    form 0: the cross-product formulas; 1: the conservative form."""
    xyz = _f64(xyz)
    _, ni, nj, nk = xyz.shape
    sh = _f64(np.zeros(9) if shift is None else np.asarray(shift).reshape(9))
    per = (C.c_int * 3)(*periodic)
    M = np.empty((10, ni, nj, nk))
    fn = _lib_handle().orc_metrics_conservative if form == 1 else _lib_handle().orc_metrics
    fn(ni, nj, nk, per, _ptr(sh), _ptr(xyz), _ptr(M))
    return M


def prim_to_cons(P: OrcParams, prim) -> np.ndarray:
    prim = _f64(prim)
    Q = np.empty_like(prim)
    _lib_handle().orc_prim_to_cons(C.byref(P), prim[0].size, _ptr(prim), _ptr(Q))
    return Q


def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    _lib_handle().orc_philox4x32_10(c, k, o)
    return tuple(int(x) for x in o)


def normals3(seed: int, n: int) -> np.ndarray:
    z = np.empty(3)
    _lib_handle().orc_normals3(seed, n, _ptr(z))
    return z


def init_jet(P: OrcParams, xyz, seed: int, noise: float = 1.0e-3) -> np.ndarray:
    xyz = _f64(xyz)
    _, ni, nj, nk = xyz.shape
    Q = np.empty((5, ni, nj, nk))
    _lib_handle().orc_init_jet(C.byref(P), ni, nj, nk, _ptr(xyz), seed, noise, _ptr(Q))
    return Q


def mu_eff(P: OrcParams, Q, M) -> np.ndarray:
    """[mu_eff, kappa_eff] (and sigma_ll for the dynamic model)."""
    Q, M = _f64(Q), _f64(M)
    _, ni, nj, nk = Q.shape
    MK = np.empty((3 if P.sgs_model == 3 else 2, ni, nj, nk))
    _lib_handle().orc_mu_eff(C.byref(P), ni, nj, nk, _ptr(Q), _ptr(M), _ptr(MK))
    return MK


def rhs(P: OrcParams, Q, M, MK=None) -> np.ndarray:
    """RHS with viscosity from the same state unless MK is given."""
    Q, M = _f64(Q), _f64(M)
    if MK is None:
        MK = mu_eff(P, Q, M)
    MK = _f64(MK)
    _, ni, nj, nk = Q.shape
    R = np.empty_like(Q)
    _lib_handle().orc_rhs(C.byref(P), ni, nj, nk, _ptr(Q), _ptr(M), _ptr(MK), _ptr(R))
    return R


def interface_flux(P: OrcParams, Q, M, MK, d: int, i: int, j: int, k: int) -> np.ndarray:
    Q, M, MK = _f64(Q), _f64(M), _f64(MK)
    _, ni, nj, nk = Q.shape
    F = np.empty(5)
    _lib_handle().orc_interface_flux(C.byref(P), ni, nj, nk, _ptr(Q), _ptr(M), _ptr(MK),
                                     d, i, j, k, _ptr(F))
    return F


def dt(P: OrcParams, Q, M) -> float:
    Q, M = _f64(Q), _f64(M)
    _, ni, nj, nk = Q.shape
    return float(_lib_handle().orc_dt(C.byref(P), ni, nj, nk, _ptr(Q), _ptr(M)))


def test_filter(f, periodic=(1, 1, 1)) -> np.ndarray:
    """The dynamic model's test filter applied to the node field f."""
    f = _f64(f)
    ni, nj, nk = f.shape
    out = np.empty_like(f)
    _lib_handle().orc_test_filter(ni, nj, nk, (C.c_int * 3)(*periodic), _ptr(f), _ptr(out))
    return out


def dynamic_coefficients(P: OrcParams, Q, M) -> dict:
    """The dynamic Smagorinsky procedure on Q: the averaged numerators and
    denominators and the coefficients C_ds, C_I, Pr_sgs."""
    Q, M = _f64(Q), _f64(M)
    _, ni, nj, nk = Q.shape
    out = np.empty(9)
    _lib_handle().orc_dynamic_coefficients(C.byref(P), ni, nj, nk, _ptr(Q), _ptr(M), _ptr(out))
    keys = ("numC", "denC", "numI", "denI", "numP", "denP", "Cd", "CI", "Prt")
    return dict(zip(keys, out.tolist()))


def dt_local(P: OrcParams, Q, M) -> np.ndarray:
    """Per-node local time steps [ni, nj, nk]."""
    Q, M = _f64(Q), _f64(M)
    _, ni, nj, nk = Q.shape
    out = np.empty((ni, nj, nk))
    _lib_handle().orc_dt_local(C.byref(P), ni, nj, nk, _ptr(Q), _ptr(M), _ptr(out))
    return out


def bc_jet(P: OrcParams, Q, M, xyz, t: float) -> np.ndarray:
    Q = _f64(Q).copy()
    M, xyz = _f64(M), _f64(xyz)
    _, ni, nj, nk = Q.shape
    _lib_handle().orc_bc_jet(C.byref(P), ni, nj, nk, _ptr(Q), _ptr(M), _ptr(xyz), t)
    return Q


def rk5(Q, rhs_fn, dt: float, update=None, Jinv=None, dtn=None) -> np.ndarray:
    """Generic 5-stage driver; rhs_fn(Q_array) -> R_array of Q's shape."""
    Q = _f64(Q).copy()
    shape = Q.shape
    ncomp = shape[0]
    N = Q[0].size

    lib = _lib_handle()

    def cb(_user, qp, rp):
        qa = np.ctypeslib.as_array(qp, shape=(ncomp * N,)).reshape(shape)
        ra = np.ctypeslib.as_array(rp, shape=(ncomp * N,)).reshape(shape)
        ra[...] = rhs_fn(qa.copy())

    fn = lib._RHSFN(cb)
    upd = None
    if update is not None:
        upd_arr = np.ascontiguousarray(update, dtype=np.uint8).reshape(-1)
        upd = upd_arr.ctypes.data_as(C.POINTER(C.c_ubyte))
    jp = None
    if Jinv is not None:
        Jinv = _f64(Jinv)
        jp = _ptr(Jinv)
    dp = None
    if dtn is not None:
        dtn = _f64(dtn)
        assert dtn.size == N
        dp = _ptr(dtn)
    lib.orc_rk5(ncomp, N, _ptr(Q), upd, jp, dt, dp, fn, None)
    return Q


def rk_step(P: OrcParams, Q, M, xyz, t: float):
    """One full step; returns (Q_next, dt)."""
    Q = _f64(Q).copy()
    M, xyz = _f64(M), _f64(xyz)
    _, ni, nj, nk = Q.shape
    d = _lib_handle().orc_rk_step(C.byref(P), ni, nj, nk, _ptr(Q), _ptr(M), _ptr(xyz), t)
    return Q, float(d)


def run(P: OrcParams, Q, M, xyz, nsteps: int, t: float = 0.0):
    """nsteps full steps; returns (Q, t)."""
    for _ in range(nsteps):
        Q, d = rk_step(P, Q, M, xyz, t)
        t += d
    return Q, t


def surface_functional(P: OrcParams, Q, M, j_surface: int, w: float = 1.0) -> float:
    """w sum_{i,k} (p - 1/gamma)^2 J^-1 |grad eta| on the ring j = j_surface."""
    Q, M = _f64(Q), _f64(M)
    _, ni, nj, nk = Q.shape
    if not 0 <= j_surface < nj:
        raise ValueError("j_surface out of range")
    return float(_lib_handle().orc_surface_functional(C.byref(P), ni, nj, nk, _ptr(Q), _ptr(M),
                                                      j_surface, w))


def window_functional(P: OrcParams, Q, M, xyz, nsteps: int, t0: float, j_surface: int) -> float:
    """The adjoint window's functional along an oracle run: the sum over the
    steps n = 1..nsteps of dt times the surface functional of Q^n (the state
    after step n and its boundary conditions)."""
    J, t = 0.0, t0
    for _ in range(nsteps):
        Q, d = rk_step(P, Q, M, xyz, t)
        t += d
        J += surface_functional(P, Q, M, j_surface, d)
    return J


def totals(Q, M) -> np.ndarray:
    Q, M = _f64(Q), _f64(M)
    _, ni, nj, nk = Q.shape
    out = np.empty(5)
    _lib_handle().orc_totals(ni, nj, nk, _ptr(Q), _ptr(M), _ptr(out))
    return out
