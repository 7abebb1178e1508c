"""The Haar-depth and TV priors against the oracle's FISTA with the same
prox: within 1e-3 (FP32) / 1e-6 (FP64) after the stated iterations; refused
with weights, with a stop rule (and, for TV, a resumed state); a batch entry
with the prior equals its plan's solve."""
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


def problem(seed, **kw):
    wl = I.small_bscan(seed=seed, n_points=10, **kw)
    op = O.IsamOracle(wl.geom, "nufft")
    s = I.add_noise(op.forward(wl.eta), 30.0, np.random.default_rng(seed))
    L = O.power_iteration(op.forward, op.adjoint, I.start_vector(op.image_shape, seed), 300, 1e-13)
    return wl, op, s, L


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-3), ("fp64", 1e-6)])
@pytest.mark.parametrize("kw", [dict(nx=32, nk=64, nz=128), dict(nx=8, ny=4, nk=32, nz=64),
                                dict(nx=4, nk=2048, nz=2048)],
                         ids=["bscan", "volume", "nz2048"])
def test_haar_prior_solve_matches_oracle(torch, prec, tol, kw):
    from paper_1905_06058_gb300.isam import Plan
    wl, op, s, L = problem(40, **kw)
    lam = O.lambda_from_data(op.adjoint, s, 0.05)
    ref = O.fista(op.forward, op.adjoint, s, lam, L, max_iter=30, shape=op.image_shape,
                  prox=O.haar_prox)
    dt = np.float64 if prec == "fp64" else np.float32
    plan = Plan(wl.geom, precision=prec)
    sd = torch.from_numpy(s.astype(dt)).cuda()
    out, info = plan.solve(sd, lambda_abs=lam, L=L, max_iter=30, prior="haar_depth")
    plan.close()
    assert rel(out.cpu().numpy(), ref.eta) < tol
    # the prior changes the result (against the l1 solve)
    l1 = O.fista(op.forward, op.adjoint, s, lam, L, max_iter=30, shape=op.image_shape)
    assert rel(l1.eta, ref.eta) > 10 * tol


def test_haar_prior_refusals_and_batch(torch):
    from paper_1905_06058_gb300.isam import Batch, IsamError, Plan
    wl, op, s, L = problem(41, nx=16, nk=64, nz=64)
    plan = Plan(wl.geom)
    sd = torch.from_numpy(s.astype(np.float32)).cuda()
    w = torch.ones(64, dtype=torch.float32, device="cuda")
    for kw in (dict(w=w), dict(tol=1e-3)):
        with pytest.raises(IsamError) as e:
            plan.solve(sd, L=L, max_iter=5, prior="haar_depth", **kw)
        assert e.value.status == 6
    ref, _ = plan.solve(sd, lambda_rel=0.03, L=L, max_iter=25, prior="haar_depth")
    out = torch.empty_like(ref)
    b = Batch([(plan, sd, out, dict(lambda_rel=0.03, L=L, max_iter=25, prior="haar_depth"))])
    info = b.run()
    assert info[0]["status"] == 0
    assert rel(out.cpu().numpy(), ref.cpu().numpy()) < 1e-5
    b.close()
    plan.close()


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-3), ("fp64", 1e-6)])
@pytest.mark.parametrize("kw", [dict(nx=32, nk=64, nz=128), dict(nx=8, ny=4, nk=32, nz=64)],
                         ids=["bscan", "volume"])
def test_tv_prior_solve_matches_oracle(torch, prec, tol, kw):
    """Isotropic TV over (x, z): the oracle runs the same fast dual gradient
    projection (10 steps per prox, warm started) inside its FISTA."""
    from paper_1905_06058_gb300.isam import Plan
    wl, op, s, L = problem(42, **kw)
    lam = O.lambda_from_data(op.adjoint, s, 0.02)
    ref = O.fista(op.forward, op.adjoint, s, lam, L, max_iter=20, shape=op.image_shape,
                  prox=O.TVProx(10))
    dt = np.float64 if prec == "fp64" else np.float32
    plan = Plan(wl.geom, precision=prec)
    sd = torch.from_numpy(s.astype(dt)).cuda()
    out, info = plan.solve(sd, lambda_abs=lam, L=L, max_iter=20, prior="tv", prior_iters=10)
    plan.close()
    assert rel(out.cpu().numpy(), ref.eta) < tol
    l1 = O.fista(op.forward, op.adjoint, s, lam, L, max_iter=20, shape=op.image_shape)
    assert rel(l1.eta, ref.eta) > 10 * tol


def test_tv_prior_refusals_and_batch(torch):
    from paper_1905_06058_gb300.isam import Batch, IsamError, Plan
    wl, op, s, L = problem(43, nx=16, nk=64, nz=64)
    plan = Plan(wl.geom)
    sd = torch.from_numpy(s.astype(np.float32)).cuda()
    w = torch.ones(64, dtype=torch.float32, device="cuda")
    for kw in (dict(w=w), dict(tol=1e-3)):
        with pytest.raises(IsamError) as e:
            plan.solve(sd, L=L, max_iter=5, prior="tv", **kw)
        assert e.value.status == 6
    st = {"z1": torch.zeros(plan.image_shape, dtype=torch.complex64, device="cuda"),
          "z2": torch.zeros(plan.image_shape, dtype=torch.complex64, device="cuda"), "k": 3}
    with pytest.raises(IsamError) as e:
        plan.solve(sd, L=L, max_iter=5, prior="tv", state=st)
    assert e.value.status == 6
    ref, _ = plan.solve(sd, lambda_rel=0.02, L=L, max_iter=15, prior="tv", prior_iters=8)
    out = torch.empty_like(ref)
    b = Batch([(plan, sd, out, dict(lambda_rel=0.02, L=L, max_iter=15, prior="tv",
                                    prior_iters=8))])
    assert b.run()[0]["status"] == 0
    assert rel(out.cpu().numpy(), ref.cpu().numpy()) < 1e-5
    b.close()
    plan.close()
