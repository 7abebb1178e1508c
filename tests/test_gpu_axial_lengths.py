"""The fused gradient kernel at the compile-time axial lengths, K = 2048 and
4096 (nz = 1024, 2048), which FP32 plans run in radix-16 form, against the
oracle.

With lambda = 0 the iteration of Alg. 1 is linear (z^k = eta^k - g^k / L, the
soft threshold of Eq. 14 passes everything), so after four iterations the image
is a short composition of A and A^H applications and must agree with the
oracle's within the per-application bar, 1e-5 relative L2.  Covered: every
neighbour count J, the u_hat output (no residual check) and the gradient
output (check on every iteration), a geometry with evanescent columns whose
Stolt maps span up to 4.35 K (several scatter chunks), and the unrolled
solve's vector-Jacobian product (the instance that also writes the model
spectra) at K = 4096."""
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


def linear_steps(torch, wl, J, check, iters=4, L=4.0):
    from paper_1905_06058_gb300.isam import Plan
    ref = O.IsamOracle(wl.geom, "nufft", J=J)
    s = I.add_noise(ref.forward(wl.eta), 30.0, np.random.default_rng(40))
    res = O.fista(ref.forward, ref.adjoint, s, 0.0, L, max_iter=iters, shape=ref.image_shape)
    plan = Plan(wl.geom, J=J)
    kw = dict(lambda_rel=0.0, L=L, max_iter=iters)
    if check:
        kw.update(tol=1e-300, check_every=1)
    out, info = plan.solve(torch.from_numpy(s.astype(np.float32)).cuda(), **kw)
    plan.close()
    assert info["iterations"] == iters
    return rel(out.cpu().numpy(), res.eta)


@pytest.mark.parametrize("check", [False, True], ids=["u_hat", "gradient"])
@pytest.mark.parametrize("nz,J", [(1024, 4), (1024, 6), (1024, 8), (2048, 4), (2048, 6),
                                  (2048, 8)])
def test_linear_steps_compile_time_lengths(torch, nz, J, check):
    wl = I.small_bscan(nx=16, nk=nz, nz=nz, n_points=10, seed=40)
    assert linear_steps(torch, wl, J, check) < 1e-5


@pytest.mark.parametrize("check", [False, True], ids=["u_hat", "gradient"])
def test_linear_steps_evanescent_k4096(torch, check):
    wl = I.small_bscan(nx=16, nk=2048, nz=2048, dx_scale=0.1, n_points=6, seed=42)
    assert linear_steps(torch, wl, 6, check) < 1e-5


def test_unrolled_vjp_k4096(torch):
    """Reverse recursion through 6 unrolled iterations (checkpoints every 3) at
    nz = 2048 against the oracle's, FP32 bar 1e-3 (as at the small sizes)."""
    from paper_1905_06058_gb300.isam import Plan
    wl = I.small_bscan(nx=8, nk=2048, nz=2048, seed=41, n_points=8)
    op = O.IsamOracle(wl.geom, "nufft")
    s = I.add_noise(op.forward(wl.eta), 30.0, np.random.default_rng(41))
    L = 1.05 * O.power_iteration(op.forward, op.adjoint, I.start_vector(op.image_shape, 41), 40,
                                 1e-8)
    lam = O.lambda_from_data(op.adjoint, s, 0.05)
    rng = np.random.default_rng(9)
    zbar = rng.standard_normal(op.image_shape) + 1j * rng.standard_normal(op.image_shape)
    K, every = 6, 3
    ref = O.fista_unrolled_vjp(op, s, lam, L, K, zbar)
    plan = Plan(wl.geom)
    sd = torch.from_numpy(s.astype(np.float32)).cuda()
    z, ck = plan.fista_unrolled(sd, lam, L, K, every)
    assert rel(z.cpu().numpy(), ref.z) < 1e-3
    g, sb = plan.fista_unrolled_vjp(sd, lam, L, K, every, ck,
                                    torch.from_numpy(zbar.astype(np.complex64)).cuda(),
                                    want_s_bar=True)
    plan.close()
    for i in range(5):
        assert abs(g[i] - ref.theta_bar[i]) <= 1e-3 * abs(ref.theta_bar[i]) + 1e-12, \
            O.PARAM_NAMES[i]
    assert rel(sb.cpu().numpy(), ref.s_bar) < 1e-3
