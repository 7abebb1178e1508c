"""GPU calibration derivatives (theta = a1..a4, z0) against the FP64 oracle.

Bars: <dA/dtheta x, y> within 1e-5 (FP32) / 1e-10 (FP64) of the bound
sum |D||F y||S_x|; the unrolled iterate equal to isam_solve bit for bit; the
unrolled gradient within 1e-3 (FP32) / 1e-7 (FP64) of the oracle's reverse
recursion; the autograd data-fidelity gradient within 1e-3 of central finite
differences (h = 1e-4 in phase-radian / range-fraction units) and of the
oracle gradient."""
import dataclasses

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


def dev(torch, a, dt):
    return torch.from_numpy(np.ascontiguousarray(a.astype(dt))).cuda()


def types(prec):
    return (np.complex128, np.float64) if prec == "fp64" else (np.complex64, np.float32)


def grad_bound(op, x, y):
    """sum_{q,k} |D_theta| |F y| |S_x|: the scale of <dA/dtheta x, y>."""
    D = O.phase_log_derivatives(op.g, op.grid)
    S = op.phase * op.axial_forward(O.lateral_fft(x))
    Fy = O.lateral_fft(y.astype(np.complex128))
    return np.array([np.sum(np.abs(D[i]) * np.abs(Fy) * np.abs(S)) for i in range(5)])


GEOMS = [
    ("bscan_32x64", dict(nx=32, nk=64, nz=64)),
    ("bscan_16x128_nz256", dict(nx=16, nk=128, nz=256)),
    ("ascan_q0", dict(nx=1, nk=64, nz=64)),
    ("volume_4x8x32", dict(nx=8, ny=4, nk=32, nz=32)),
    ("evanescent_edge", dict(nx=32, nk=64, nz=64, dx_scale=0.08)),
    ("bscan_4x2048", dict(nx=4, nk=2048, nz=2048)),
]


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("fp64", 1e-10)])
@pytest.mark.parametrize("name,kw", GEOMS)
def test_param_grad_matches_oracle(torch, prec, tol, name, kw):
    from paper_1905_06058_gb300.isam import Plan
    wl = I.small_bscan(seed=21, **kw)
    op = O.IsamOracle(wl.geom, "nufft")
    rng = np.random.default_rng(3)
    x = rng.standard_normal(op.image_shape) + 1j * rng.standard_normal(op.image_shape)
    y = rng.standard_normal(op.spec_shape)
    ref = O.param_grad(op, x, y)
    ct, rt = types(prec)
    plan = Plan(wl.geom, precision=prec)
    got = plan.param_grad(dev(torch, x, ct), dev(torch, y, rt))
    plan.close()
    bound = grad_bound(op, x, y)
    assert np.all(np.abs(got - ref) <= tol * bound), (got, ref, bound)
    if kw.get("nx") == 1:
        assert got[4] == 0.0


@pytest.mark.parametrize("table", [True, False])
def test_set_model_matches_fresh_plan(torch, table):
    from paper_1905_06058_gb300.isam import Plan
    wl = I.small_bscan(nx=32, nk=128, nz=128, seed=4)
    g2 = dataclasses.replace(wl.geom, disp=(1e-7, 3e-10, -2e-15, 0.0), z0=wl.geom.z0 * 0.5)
    eta = dev(torch, I.random_image((1, 32, 128), 5), np.complex64)
    p1 = Plan(wl.geom, stolt_table=table)
    p1.forward(eta)
    p1.set_model(g2.disp, g2.z0)
    p2 = Plan(g2, stolt_table=table)
    assert torch.equal(p1.forward(eta), p2.forward(eta))
    y = p2.forward(eta)
    assert torch.equal(p1.adjoint(y), p2.adjoint(y))
    p1.close()
    p2.close()


def unrolled_problem(nx=16, nk=64, nz=64, seed=31, n_points=8):
    wl = I.small_bscan(nx=nx, nk=nk, nz=nz, seed=seed, n_points=n_points)
    op = O.IsamOracle(wl.geom, "nufft")
    s = I.add_noise(op.forward(wl.eta), 30.0, np.random.default_rng(seed))
    L = O.power_iteration(op.forward, op.adjoint, I.start_vector(op.image_shape, seed), 300, 1e-13)
    lam = O.lambda_from_data(op.adjoint, s, 0.05)
    return wl, op, s, L, lam


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_unrolled_equals_solve_and_checkpoints(torch, prec):
    from paper_1905_06058_gb300.isam import Plan
    wl, op, s, L, lam = unrolled_problem()
    ct, rt = types(prec)
    plan = Plan(wl.geom, precision=prec)
    sd = dev(torch, s, rt)
    K, every = 12, 5
    z, ck = plan.fista_unrolled(sd, lam, L, K, every)
    ref, _ = plan.solve(sd, lambda_abs=lam, L=L, max_iter=K)
    assert torch.equal(z, ref)
    assert ck.shape[0] == 6
    st = {"z1": torch.zeros_like(z), "z2": torch.zeros_like(z), "k": 0}
    plan.solve(sd, lambda_abs=lam, L=L, max_iter=every, state=st)
    assert torch.equal(ck[2], st["z1"]) and torch.equal(ck[3], st["z2"])
    assert not torch.any(ck[0]) and not torch.any(ck[1])
    plan.close()


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-3), ("fp64", 1e-7)])
@pytest.mark.parametrize("K,every", [(10, 4), (7, 1), (6, 6)])
def test_unrolled_vjp_matches_oracle(torch, prec, tol, K, every):
    from paper_1905_06058_gb300.isam import Plan
    wl, op, s, L, lam = unrolled_problem()
    w = I.depth_weights(op.grid.nz)
    rng = np.random.default_rng(7)
    zbar = rng.standard_normal(op.image_shape) + 1j * rng.standard_normal(op.image_shape)
    ref = O.fista_unrolled_vjp(op, s, lam, L, K, zbar, w=w[None, None, :])
    ct, rt = types(prec)
    plan = Plan(wl.geom, precision=prec)
    sd, wd = dev(torch, s, rt), dev(torch, w, rt)
    z, ck = plan.fista_unrolled(sd, lam, L, K, every, w=wd)
    assert np.linalg.norm(z.cpu().numpy() - ref.z) <= tol * np.linalg.norm(ref.z)
    g, sb = plan.fista_unrolled_vjp(sd, lam, L, K, every, ck, dev(torch, zbar, ct),
                                    want_s_bar=True, w=wd)
    plan.close()
    assert np.linalg.norm(g - ref.theta_bar) <= tol * np.linalg.norm(ref.theta_bar) or \
        np.all(np.abs(g - ref.theta_bar) <= tol * np.abs(ref.theta_bar))
    for i in range(5):
        assert abs(g[i] - ref.theta_bar[i]) <= tol * abs(ref.theta_bar[i]) + 1e-12 * np.abs(
            ref.theta_bar[i]), O.PARAM_NAMES[i]
    sbv = sb.cpu().numpy()
    assert np.linalg.norm(sbv - ref.s_bar) <= tol * np.linalg.norm(ref.s_bar)


def test_autograd_gradient_matches_fd_and_oracle(torch):
    """Data fidelity 1/2||A z^K(theta) - s||^2 through K = 8 unrolled iterations (FP64)."""
    from paper_1905_06058_gb300 import calib
    from paper_1905_06058_gb300.isam import Plan
    wl, op, s, L, lam = unrolled_problem(seed=41)
    g = wl.geom
    plan = Plan(g, precision="fp64")
    sd = dev(torch, s, np.float64)
    K, every = 8, 3
    theta0 = np.array(list(g.disp) + [g.z0], dtype=np.float64)
    th = torch.tensor(theta0, requires_grad=True)
    loss = calib.data_fidelity(sd, th, plan, lam, L, K, every)
    loss.backward()
    grad = th.grad.numpy().copy()
    # central differences, each step a phase change of at most 1e-4 rad
    # (a_i: at the band edge; z0: at the largest 2k + beta of the grid)
    D = O.phase_log_derivatives(g, op.grid)
    for i in (1, 2, 4):
        h = 1e-4 / np.abs(D[i]).max()
        vals = []
        for sgn in (1, -1):
            t = theta0.copy()
            t[i] += sgn * h
            with torch.no_grad():
                vals.append(float(calib.data_fidelity(sd, torch.tensor(t), plan, lam, L, K, every)))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert grad[i] == pytest.approx(fd, rel=1e-3), O.PARAM_NAMES[i]
    # oracle: d/dtheta = <dA z^K, r> + d<A^H r, z^K>/dtheta with r = A z^K - s
    zK = O.fista_unrolled_vjp(op, s, lam, L, K, np.zeros(op.image_shape)).z
    r = op.forward(zK) - s
    ref = O.param_grad(op, zK, r) + O.fista_unrolled_vjp(op, s, lam, L, K, op.adjoint(r)).theta_bar
    for i in range(5):
        assert grad[i] == pytest.approx(ref[i], rel=1e-6, abs=1e-9 * np.abs(ref).max()), O.PARAM_NAMES[i]
    plan.close()


def test_model_and_adjoint_autograd(torch):
    """Gradients of <A eta, y> and <A^H y, x> by autograd equal the direct calls."""
    from paper_1905_06058_gb300 import calib
    from paper_1905_06058_gb300.isam import Plan
    wl = I.small_bscan(nx=16, nk=64, nz=64, seed=8)
    g = wl.geom
    plan = Plan(g, precision="fp64")
    th = torch.tensor(list(g.disp) + [g.z0], dtype=torch.float64, requires_grad=True)
    rng = np.random.default_rng(8)
    eta = dev(torch, rng.standard_normal((1, 16, 64)) + 1j * rng.standard_normal((1, 16, 64)),
              np.complex128).requires_grad_(True)
    y = dev(torch, rng.standard_normal((1, 16, 64)), np.float64).requires_grad_(True)
    (calib.model(eta, th, plan) * y).sum().backward()
    assert torch.allclose(eta.grad, plan.adjoint(y.detach()), rtol=0, atol=0)
    assert np.array_equal(th.grad.numpy(), plan.param_grad(eta.detach(), y.detach()))
    th.grad = None
    eta.grad = None
    y.grad = None
    x = eta.detach()
    torch.real(torch.vdot(x.flatten(), calib.model_adjoint(y, th, plan).flatten())).backward()
    assert torch.allclose(y.grad, plan.forward(x), rtol=0, atol=0)
    assert np.allclose(th.grad.numpy(), plan.param_grad(x, y.detach()), rtol=1e-12)
    plan.close()


def test_calibration_recovers_hidden_theta(torch):
    """Two B-scans made with hidden (a2, a3, z0); Adam from a perturbed start."""
    from paper_1905_06058_gb300 import calib
    from paper_1905_06058_gb300.isam import Plan
    rng = np.random.default_rng(12)
    wl = I.small_bscan(nx=64, nk=256, nz=256, seed=12, n_points=30)
    g = wl.geom
    truth = np.array(list(g.disp) + [g.z0], dtype=np.float64)
    op = O.IsamOracle(g, "nufft")
    spectra, lams = [], []
    for b in range(2):
        eta = I.point_scatterers(np.random.default_rng(100 + b), op.image_shape, 30)
        s = I.add_noise(op.forward(eta), 40.0, rng)
        spectra.append(dev(torch, s, np.float32))
        lams.append(O.lambda_from_data(op.adjoint, s, 0.02))
    plan = Plan(g)
    L = plan.lipschitz()
    scale = calib.theta_scales(g)
    start = truth.copy()
    start[1] += 0.6 * scale[1]
    start[2] -= 0.4 * scale[2]
    start[4] += 0.01 * scale[4]
    res = calib.calibrate(plan, spectra, start, lams, L, K=20, every=5, steps=60)
    plan.close()
    err0 = np.abs((start - truth) / scale)[[1, 2, 4]]
    err1 = np.abs((res.theta - truth) / scale)[[1, 2, 4]]
    assert res.losses[-1] < 0.5 * res.losses[0]
    # the annealed step settles: the last loss is within 5 % of the best seen
    assert res.losses[-1] <= 1.05 * res.best_loss, (res.losses[-1], res.best_loss)
    assert np.all(err1 < 0.2 * err0), (err0, err1)


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("fp64", 1e-6)])
def test_data_fidelity_matches_oracle(torch, prec, tol):
    """isam_data_fidelity: 1/2 ||A eta - s||^2 and the residual A eta - s against
    the oracle (Eq. 12 data term, per-application bars), and the autograd
    Function built on it returns exactly A^H r and <dA/dtheta z, r>."""
    from paper_1905_06058_gb300 import calib
    from paper_1905_06058_gb300.isam import Plan
    wl = I.small_bscan(nx=32, nk=128, nz=128, seed=61, n_points=10)
    op = O.IsamOracle(wl.geom, "nufft")
    s = I.add_noise(op.forward(wl.eta), 20.0, np.random.default_rng(61))
    eta = wl.eta + 0.3 * I.random_image(op.image_shape, 62)
    r_ref = op.forward(eta) - s
    ct, rt = types(prec)
    plan = Plan(wl.geom, precision=prec)
    ed, sd = dev(torch, eta, ct), dev(torch, s, rt)
    value, r = plan.data_fidelity(ed, sd)
    assert np.linalg.norm(r.cpu().numpy() - r_ref) <= tol * np.linalg.norm(r_ref)
    assert value == pytest.approx(0.5 * np.sum(r_ref * r_ref), rel=2 * tol)
    z = ed.clone().requires_grad_(True)
    th = torch.tensor(list(wl.geom.disp) + [wl.geom.z0], dtype=torch.float64,
                      requires_grad=True)
    loss = calib.DataFidelity.apply(z, th, plan, sd)
    assert float(loss.detach()) == value
    loss.backward()
    assert torch.equal(z.grad, plan.adjoint(r))
    assert np.array_equal(th.grad.numpy(), plan.param_grad(ed, r))
    plan.close()
