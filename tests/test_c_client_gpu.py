"""The plain-C client on the device (tests/c_client_gpu.c): the header and
the library alone, with buffers the client allocates itself, run the jet
configuration 48 x 24 x 32 for 20 steps in FP64 and FP32-mixed; the FP64
state after 20 steps matches the oracle run from the same initial state
(<= 1e-10 relative L-inf), and so does the FP64 residual of the final state
(within 1e-13 of the flux scale)."""
import os
import subprocess

import numpy as np
import pytest

from gpu_helpers import rel_linf

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _cuda_home():
    for cand in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "include", "cuda_runtime.h")):
            return cand
    pytest.skip("CUDA toolkit headers not found")


def test_c_client_runs_the_method(orc, tmp_path):
    from paper_2301_00817_gb300 import _build
    _build.build()
    import paper_2301_00817_gb300 as lj
    cuda = _cuda_home()
    libdir = os.path.dirname(lj.LIB_PATH)
    exe = tmp_path / "c_client_gpu"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-I",
                    os.path.join(ROOT, "include"), "-I", os.path.join(cuda, "include"),
                    "-o", str(exe), os.path.join(ROOT, "tests", "c_client_gpu.c"),
                    "-L", libdir, "-llesjet", "-L", os.path.join(cuda, "lib64"), "-lcudart",
                    "-lm", "-Wl,-rpath," + libdir, "-Wl,-rpath," + os.path.join(cuda, "lib64")],
                   check=True)
    out = tmp_path / "states.bin"
    r = subprocess.run([str(exe), str(out)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
    t_c = float(r.stdout.split()[1])
    shape = (48, 24, 32)
    data = np.fromfile(out, dtype=np.float64).reshape(4, 5, *shape)
    Q0, Q64, Qm, R64 = data
    xyz = lj.synth.jet_grid(*shape)
    P = orc.params(sgs_model=1)
    M = orc.metrics(xyz, (0, 0, 1))
    Qo, to = orc.run(P, Q0, M, xyz, 20)
    assert rel_linf(Q64, Qo) <= 1e-10
    assert abs(t_c - to) <= 1e-12 * to
    Ro = orc.rhs(P, Q64, M)
    fscale = (np.abs(M[9]) * np.sqrt(M[0] ** 2 + M[1] ** 2 + M[2] ** 2)).max()
    for c in range(5):
        qs = np.abs(Q64[c]).max() + (np.abs(Q64[4]).max() if c else 0.0)
        assert np.abs(R64[c] - Ro[c]).max() <= 1e-13 * fscale * qs, c
    assert rel_linf(Qm, Qo) <= 1e-6
