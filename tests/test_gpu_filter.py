"""The filter B(q, k) of Eq. 3 (isam_set_filter) on the GPU against the oracle.

Bars: A and A^H within 1e-5 (FP32) / 1e-10 (FP64) of the filtered oracle, with
the Stolt table and with positions evaluated on the fly; a filtered FISTA
solve within 1e-3; <dA/dtheta x, y> with a filter within 1e-5 of the bound;
removing the filter gives the unfiltered plan's results bit for bit."""
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


def random_filter(g, seed):
    rng = np.random.default_rng(seed)
    shape = ((g.ny // 2 + 1) if g.ny > 1 else 1, g.nx // 2 + 1, g.nk)
    return rng.uniform(0.3, 1.2, shape) * np.exp(1j * rng.uniform(-0.5, 0.5, shape))


CASES = [dict(nx=32, nk=64, nz=64), dict(nx=8, ny=4, nk=32, nz=64), dict(nx=48, nk=64, nz=128),
         dict(nx=4, nk=2048, nz=2048)]


@pytest.mark.parametrize("table", [True, False], ids=["stolt_table", "stolt_evaluated"])
@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("fp64", 1e-10)])
@pytest.mark.parametrize("kw", CASES, ids=lambda k: "x".join(str(v) for v in k.values()))
def test_filtered_operators_match_oracle(torch, kw, prec, tol, table):
    from paper_1905_06058_gb300.isam import Plan
    g = I.small_bscan(seed=30, **kw).geom
    filt = random_filter(g, 31)
    op = O.IsamOracle(g, "nufft", filt=filt)
    eta = I.random_image(op.image_shape, 32)
    y = I.random_spectra(op.spec_shape, 33)
    ct, rt = (np.complex128, np.float64) if prec == "fp64" else (np.complex64, np.float32)
    plan = Plan(g, precision=prec, stolt_table=table)
    plan.set_filter(filt)
    s = plan.forward(dev(torch, eta, ct)).cpu().numpy()
    a = plan.adjoint(dev(torch, y, rt)).cpu().numpy()
    x = dev(torch, eta, ct)
    gr = plan.param_grad(x, dev(torch, y, rt))
    plan.close()
    assert rel(s, op.forward(eta)) < tol
    assert rel(a, op.adjoint(y)) < tol
    ref = O.param_grad(op, eta, y)
    D = O.phase_log_derivatives(g, op.grid)
    S = op.phase * op.axial_forward(O.lateral_fft(eta))
    Fy = O.lateral_fft(y.astype(np.complex128))
    bound = np.array([np.sum(np.abs(D[i]) * np.abs(Fy) * np.abs(S)) for i in range(5)])
    assert np.all(np.abs(gr - ref) <= tol * bound)


def test_filtered_solve_and_removal(torch):
    from paper_1905_06058_gb300.isam import Plan
    wl = I.small_bscan(nx=32, nk=64, nz=128, seed=34, n_points=10)
    g = wl.geom
    filt = random_filter(g, 35)
    op = O.IsamOracle(g, "nufft", filt=filt)
    s = I.add_noise(op.forward(wl.eta), 30.0, np.random.default_rng(34))
    L = O.power_iteration(op.forward, op.adjoint, I.start_vector(op.image_shape, 34), 300, 1e-13)
    lam = O.lambda_from_data(op.adjoint, s, 0.05)
    ref = O.fista(op.forward, op.adjoint, s, lam, L, max_iter=40, shape=op.image_shape)
    plan = Plan(g)
    eta = dev(torch, wl.eta, np.complex64)
    s0 = plan.forward(eta)
    plan.set_filter(filt)
    out, _ = plan.solve(dev(torch, s, np.float32), lambda_abs=lam, L=L, max_iter=40)
    assert rel(out.cpu().numpy(), ref.eta) < 1e-3
    plan.set_filter(None)
    assert torch.equal(plan.forward(eta), s0)
    plan.close()
