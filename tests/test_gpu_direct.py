"""The direct reconstruction of Eq. 9 and the 1-D per-A-scan model of Eq. 10
(ISAM_FLAG_AXIAL_MODEL) on the GPU against the FP64 oracle.

Bars: Eq. 9 within 1e-5 (FP32) / 1e-10 (FP64) relative L2 of the oracle's
direct sum (the oracle evaluates e^{-j 2 k z} at arguments up to
2 k_max z_max ~ 1e5 rad, so its own FP64 phase rounding reaches ~1e-11); the axial-model A and A^H within 1e-5 / 1e-10 of the oracle's
per-A-scan NUFFT model; its adjoint within the NUFFT error (2e-5) of Eq. 9;
its FISTA solve within 1e-3 / 1e-6 of the oracle's."""
import numpy as np
import pytest

from oracle import isam_oracle as O
from paper_1905_06058_gb300 import inputs as I

pytestmark = pytest.mark.gpu


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


def dev(torch, a, dt):
    return torch.from_numpy(np.ascontiguousarray(a.astype(dt))).cuda()


SIZES = [dict(nx=8, nk=64, nz=64), dict(nx=4, nk=32, nz=128),
         dict(nx=4, ny=2, nk=256, nz=256), dict(nx=2, nk=2048, nz=2048), dict(nx=1, nk=16, nz=16)]


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("fp64", 1e-10)])
@pytest.mark.parametrize("kw", SIZES, ids=lambda k: "x".join(str(v) for v in k.values()))
def test_dispersion_compensated_ifft(torch, prec, tol, kw):
    from paper_1905_06058_gb300.isam import Plan
    g = I.small_bscan(seed=2, **kw).geom
    y = I.random_spectra((g.ny, g.nx, g.nk), 3)
    plan = Plan(g, precision=prec)
    rt = np.float64 if prec == "fp64" else np.float32
    got = plan.dispersion_compensated_ifft(dev(torch, y, rt)).cpu().numpy()
    plan.close()
    ref = O.dispersion_compensated_ifft(g, y)
    assert rel(got, ref) < tol


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("fp64", 1e-10)])
@pytest.mark.parametrize("kw", SIZES[:4], ids=lambda k: "x".join(str(v) for v in k.values()))
def test_axial_model_matches_oracle(torch, prec, tol, kw):
    from paper_1905_06058_gb300.isam import Plan
    g = I.small_bscan(seed=4, **kw).geom
    op = O.AxialModelOracle(g, "nufft")
    eta = I.random_image(op.image_shape, 5)
    y = I.random_spectra(op.spec_shape, 6)
    ct, rt = (np.complex128, np.float64) if prec == "fp64" else (np.complex64, np.float32)
    plan = Plan(g, precision=prec, axial_model=True)
    s = plan.forward(dev(torch, eta, ct)).cpu().numpy()
    a = plan.adjoint(dev(torch, y, rt)).cpu().numpy()
    d = plan.dispersion_compensated_ifft(dev(torch, y, rt)).cpu().numpy()
    plan.close()
    assert rel(s, op.forward(eta)) < tol
    assert rel(a, op.adjoint(y)) < tol
    assert rel(a, d) < 2e-5           # A^H of the 1-D model is Eq. 9 up to the NUFFT error


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-3), ("fp64", 1e-6)])
def test_axial_model_solve_matches_oracle(torch, prec, tol):
    from paper_1905_06058_gb300.isam import Plan
    wl = I.small_bscan(nx=16, nk=64, nz=128, seed=8, n_points=10)
    g = wl.geom
    op = O.AxialModelOracle(g, "nufft")
    s = I.add_noise(op.forward(wl.eta), 30.0, np.random.default_rng(8))
    L = O.power_iteration(op.forward, op.adjoint, I.start_vector(op.image_shape, 8), 300, 1e-13)
    lam = O.lambda_from_data(op.adjoint, s, 0.05)
    ref = O.fista(op.forward, op.adjoint, s, lam, L, max_iter=40, shape=op.image_shape)
    rt = np.float64 if prec == "fp64" else np.float32
    plan = Plan(g, precision=prec, axial_model=True)
    out, info = plan.solve(dev(torch, s, rt), lambda_abs=lam, L=L, max_iter=40)
    plan.close()
    assert rel(out.cpu().numpy(), ref.eta) < tol
