"""The C-ABI library builds, loads and exports every symbol include/lesjet.h
declares; host-only entry points validate their arguments.  No compute call
is made (these run without a GPU)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lesjet.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2301_00817_gb300 import _build
    _build.build()
    import paper_2301_00817_gb300 as lj
    return lj.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(les_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("les_create", "les_set_grid", "les_init_jet", "les_rhs", "les_rk_step",
                     "les_run_n_steps", "les_time_step", "les_apply_bc", "les_mu_eff",
                     "les_grid_jet"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_create_validates_and_sizes_workspace(lib):
    import paper_2301_00817_gb300 as lj
    h = C.c_void_p()
    p = lj.make_params()
    assert lib.les_create(C.byref(p), 48, 24, 32, C.byref(h)) == lj.LES_OK
    ws = lib.les_workspace_bytes(h)
    N = 48 * 24 * 32
    assert ws >= N * 8 * (10 + 2 + 10)  # metrics, viscosity, two stage states
    assert lib.les_destroy(h) == lj.LES_OK
    assert lib.les_create(C.byref(p), 4, 24, 32, C.byref(h)) == lj.LES_ERR_SHAPE
    bad = lj.make_params(sgs_model=7)
    assert lib.les_create(C.byref(bad), 8, 8, 8, C.byref(h)) == lj.LES_ERR_INVALID_ARG
    bad = lj.make_params(periodic=(1, 1, 1), bc=lj.BC_JET)
    assert lib.les_create(C.byref(bad), 8, 8, 8, C.byref(h)) == lj.LES_ERR_INVALID_ARG
    bad = lj.make_params(dt_mode=lj.DT_FIXED, dt_fixed=0.0)
    assert lib.les_create(C.byref(bad), 8, 8, 8, C.byref(h)) == lj.LES_ERR_INVALID_ARG
    mixed = lj.make_params(precision=lj.PREC_MIXED)
    assert lib.les_create(C.byref(mixed), 48, 24, 32, C.byref(h)) == lj.LES_OK
    ws_mixed = lib.les_workspace_bytes(h)
    assert ws_mixed > 0
    lib.les_destroy(h)
    # the compact mixed form drops exactly the FP64 metrics (up to alignment)
    compact = lj.make_params(precision=lj.PREC_MIXED_COMPACT)
    assert lib.les_create(C.byref(compact), 48, 24, 32, C.byref(h)) == lj.LES_OK
    ws_compact = lib.les_workspace_bytes(h)
    assert abs((ws_mixed - ws_compact) - 80 * N) <= 256
    lib.les_destroy(h)
    # 2000 x 500 x 1024 points fit the mixed forms' 32-bit field indexing; the
    # compact workspace is 128 bytes per point (float metrics 40, mu/kappa 8,
    # two stage states 40, the state as a float pair 40)
    assert lib.les_create(C.byref(compact), 2000, 500, 1024, C.byref(h)) == lj.LES_OK
    assert lib.les_workspace_bytes(h) <= 129 * 2000 * 500 * 1024
    lib.les_destroy(h)
    assert lib.les_create(C.byref(compact), 3000, 1000, 1024, C.byref(h)) == lj.LES_ERR_SHAPE
    bad = lj.make_params(precision=3)
    assert lib.les_create(C.byref(bad), 8, 8, 8, C.byref(h)) == lj.LES_ERR_INVALID_ARG


def test_calls_before_grid_are_rejected_without_touching_the_device(lib):
    import paper_2301_00817_gb300 as lj
    h = C.c_void_p()
    p = lj.make_params()
    assert lib.les_create(C.byref(p), 8, 8, 8, C.byref(h)) == lj.LES_OK
    assert lib.les_rk_step(h, C.c_void_p(16), None) == lj.LES_ERR_STATE
    assert b"les_set_grid" in lib.les_last_error(h)
    assert lib.les_set_grid(h, C.c_void_p(3), None, C.c_void_p(16), None) == lj.LES_ERR_ALIGN
    lib.les_destroy(h)


def test_grid_jet_validates_before_touching_the_device(lib):
    import paper_2301_00817_gb300 as lj
    good = lj.LesJetGrid(20.0, 0.0, 0.02, 10.0, 0.5, 0.9, 8.0)
    ptr = C.c_void_p(16)
    assert lib.les_grid_jet(1, 8, 8, C.byref(good), ptr, None) == lj.LES_ERR_SHAPE
    assert lib.les_grid_jet(8, 8, 8, None, ptr, None) == lj.LES_ERR_INVALID_ARG
    assert lib.les_grid_jet(8, 8, 8, C.byref(good), None, None) == lj.LES_ERR_INVALID_ARG
    assert lib.les_grid_jet(8, 8, 8, C.byref(good), C.c_void_p(24), None) == lj.LES_ERR_ALIGN
    for field, value in (("length", 0.0), ("r_c", 0.01), ("r_c", 10.0), ("A", 1.0),
                         ("beta", 0.0), ("r0", -1.0)):
        bad = lj.LesJetGrid(20.0, 0.0, 0.02, 10.0, 0.5, 0.9, 8.0)
        setattr(bad, field, value)
        assert lib.les_grid_jet(8, 8, 8, C.byref(bad), ptr, None) == lj.LES_ERR_INVALID_ARG, field


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes mirrors have the C structs' sizes and field offsets (the
    header compiled as plain C by gcc)."""
    import paper_2301_00817_gb300 as lj
    fields = {"les_params": (lj.LesParams, ["Re", "St", "amp", "sgs_model", "periodic", "bc",
                                            "precision", "metric_form", "axis",
                                            "slab_ghost"]),
              "les_diag": (lj.LesDiag, ["dt", "totals", "status", "steps"]),
              "les_jet_grid": (lj.LesJetGrid, ["ratio", "r_c", "beta"])}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void) {"]
    for st, (_, names) in fields.items():
        lines.append(f'  printf("{st} size %zu\\n", sizeof({st}));')
        for f in names:
            lines.append(f'  printf("{st} {f} %zu\\n", offsetof({st}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-std=c11", "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    for line in out.splitlines():
        st, what, value = line.split()
        cls = fields[st][0]
        got = C.sizeof(cls) if what == "size" else getattr(cls, what).offset
        assert got == int(value), (st, what, got, value)


def test_plain_c_client(lib, tmp_path):
    """tests/c_client.c, which includes only lesjet.h and links only
    liblesjet.so, compiles as C11 without warnings and its host-only checks
    (creation, validation, workspace sizes, call order, grid arguments)
    hold."""
    import subprocess
    import paper_2301_00817_gb300 as lj
    libdir = os.path.dirname(lj.LIB_PATH)
    exe = tmp_path / "c_client"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-I",
                    os.path.join(ROOT, "include"), "-o", str(exe),
                    os.path.join(ROOT, "tests", "c_client.c"), "-L", libdir, "-llesjet",
                    "-Wl,-rpath," + libdir], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr


def test_local_time_steps_are_chosen_at_creation(lib):
    """Per-node steps need workspace: a context created with a global step
    cannot switch to LES_DT_LOCAL, and creating with it grows the workspace
    by one value per point."""
    import paper_2301_00817_gb300 as lj
    h = C.c_void_p()
    p = lj.make_params()
    assert lib.les_create(C.byref(p), 16, 12, 8, C.byref(h)) == lj.LES_OK
    base = lib.les_workspace_bytes(h)
    q = lj.make_params(dt_mode=lj.DT_LOCAL)
    assert lib.les_set_params(h, C.byref(q)) == lj.LES_ERR_INVALID_ARG
    assert b"creation" in lib.les_last_error(h)
    lib.les_destroy(h)
    for prec, size in ((lj.PREC_FP64, 8), (lj.PREC_MIXED, 4)):
        h0, h1 = C.c_void_p(), C.c_void_p()
        a, b = lj.make_params(precision=prec), lj.make_params(precision=prec, dt_mode=lj.DT_LOCAL)
        assert lib.les_create(C.byref(a), 16, 12, 8, C.byref(h0)) == lj.LES_OK
        assert lib.les_create(C.byref(b), 16, 12, 8, C.byref(h1)) == lj.LES_OK
        grow = lib.les_workspace_bytes(h1) - lib.les_workspace_bytes(h0)
        assert size * 16 * 12 * 8 <= grow <= size * 16 * 12 * 8 + 256
        assert lib.les_set_params(h1, C.byref(a)) == lj.LES_OK  # and back is fine
        lib.les_destroy(h0)
        lib.les_destroy(h1)
    assert base > 0


def test_dynamic_model_is_chosen_at_creation(lib):
    """The dynamic SGS model needs its scratch in the workspace, chosen at
    creation: about 408 more bytes per point in FP64; in the mixed forms 236
    (50 FP32 procedure fields, 8 FP32 node fields, the third viscosity
    field)."""
    import paper_2301_00817_gb300 as lj
    for prec in (lj.PREC_MIXED, lj.PREC_MIXED_COMPACT):
        h0, h1 = C.c_void_p(), C.c_void_p()
        a = lj.make_params(sgs_model=lj.SGS_SMAGORINSKY, precision=prec)
        b = lj.make_params(sgs_model=lj.SGS_DYNAMIC, precision=prec)
        assert lib.les_create(C.byref(a), 16, 12, 8, C.byref(h0)) == lj.LES_OK
        assert lib.les_create(C.byref(b), 16, 12, 8, C.byref(h1)) == lj.LES_OK
        N = 16 * 12 * 8
        grow = lib.les_workspace_bytes(h1) - lib.les_workspace_bytes(h0)
        assert 236 * N <= grow <= 236 * N + 1024, grow / N
        lib.les_destroy(h0)
        lib.les_destroy(h1)
    h0, h1 = C.c_void_p(), C.c_void_p()
    a, b = lj.make_params(sgs_model=lj.SGS_SMAGORINSKY), lj.make_params(sgs_model=lj.SGS_DYNAMIC)
    assert lib.les_create(C.byref(a), 16, 12, 8, C.byref(h0)) == lj.LES_OK
    assert lib.les_create(C.byref(b), 16, 12, 8, C.byref(h1)) == lj.LES_OK
    N = 16 * 12 * 8
    grow = lib.les_workspace_bytes(h1) - lib.les_workspace_bytes(h0)
    assert 408 * N <= grow <= 408 * N + 512
    assert lib.les_set_params(h0, C.byref(b)) == lj.LES_ERR_INVALID_ARG
    assert b"creation" in lib.les_last_error(h0)
    assert lib.les_set_params(h1, C.byref(a)) == lj.LES_OK
    out = (C.c_double * 9)()
    assert lib.les_dynamic_coefficients(h1, C.c_void_p(16), out, None) == lj.LES_ERR_STATE
    lib.les_destroy(h0)
    lib.les_destroy(h1)
