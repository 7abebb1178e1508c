"""The C ABI used from plain C: tests/c/isam_c_client.c, compiled with gcc
against include/isam.h and linked with libisam and the CUDA runtime, applies
A and A^H; its outputs equal the Python binding's bit for bit and the
oracle's within the FP32 bar (1e-5)."""
import os
import subprocess

import numpy as np
import pytest

from oracle import isam_oracle as O
from paper_1905_06058_gb300 import inputs as I

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def torch():
    import torch as T
    if not T.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    return T


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_c_client_matches_binding_and_oracle(torch, tmp_path):
    from paper_1905_06058_gb300 import isam as B
    cuda = "/usr/local/cuda"
    exe = tmp_path / "client"
    libdir = os.path.dirname(B.LIB_PATH)
    subprocess.run(["gcc", "-O2", "-I" + os.path.join(ROOT, "include"), "-I" + cuda + "/include",
                    os.path.join(ROOT, "tests", "c", "isam_c_client.c"), "-o", str(exe),
                    "-L" + libdir, "-lisam", "-L" + cuda + "/lib64", "-lcudart",
                    "-Wl,-rpath," + libdir + ":" + cuda + "/lib64"], check=True)
    wl = I.small_bscan(nx=32, nk=64, nz=128, seed=60)
    g = wl.geom
    eta = I.random_image((1, g.nx, g.nz), 61).astype(np.complex64)
    (tmp_path / "eta.bin").write_bytes(eta.tobytes())
    disp = list(g.disp) + [0.0] * (4 - len(g.disp))
    args = [str(exe), str(g.nx), str(g.nk), str(g.nz)] + [repr(float(v)) for v in (
        g.k_min, g.k_max, g.dx, g.na, g.z0, *disp)] + [
        str(tmp_path / "eta.bin"), str(tmp_path / "s.bin"), str(tmp_path / "a.bin")]
    r = subprocess.run(args, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    s_c = np.frombuffer((tmp_path / "s.bin").read_bytes(), np.float32).reshape(1, g.nx, g.nk)
    a_c = np.frombuffer((tmp_path / "a.bin").read_bytes(), np.complex64).reshape(1, g.nx, g.nz)
    plan = B.Plan(g)
    s_py = plan.forward(torch.from_numpy(eta).cuda()).cpu().numpy()
    a_py = plan.adjoint(torch.from_numpy(s_py).cuda()).cpu().numpy()
    plan.close()
    assert np.array_equal(s_c, s_py) and np.array_equal(a_c, a_py)
    op = O.IsamOracle(g, "nufft")
    assert rel(s_c, op.forward(eta.astype(np.complex128))) < 1e-5
    assert rel(a_c, op.adjoint(s_c.astype(np.float64))) < 1e-5
