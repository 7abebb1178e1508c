"""The stop rule of Alg. 1 (relative residual, Eq. 15) on geometries whose
lateral update blocks hold fewer than 32 threads, or a partial last warp.

The update kernel sums the three norms of Eq. 15 per block.  A block has
(L/8) * TP threads for a lateral length L >= 8 and TP threads below it: 8 for
an A-scan (nx = 1) and for nx = 8, 24 for nx = 24 = 3 * 8, 48 (one full warp and
one of 16 lanes) for nx = 48, and 8 again in the y pass of an 8 x 8 volume.
Each case runs the oracle's FISTA with tol = 1e-3 and the GPU solve with the
same tolerance checked on every iteration: the iteration count at which the
rule fires and r_r there must agree (FP64: the same count, r_r within 1e-6;
FP32: the count within one, r_r within 1e-3 when the counts agree), and the
images must agree at the solver bars (1e-6 FP64, 1e-3 FP32)."""
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


CASES = {
    "ascan_nx1": dict(nx=1, nk=64, nz=128, n_points=4),
    "nx8": dict(nx=8, nk=64, nz=128, n_points=6),
    "nx24": dict(nx=24, nk=64, nz=64, n_points=6),
    "nx48": dict(nx=48, nk=64, nz=64, n_points=8),
    "volume_8x8": dict(nx=8, ny=8, nk=32, nz=64, n_points=6),
}


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_stop_rule_small_lateral_blocks(torch, case, prec):
    from paper_1905_06058_gb300.isam import Plan
    kw = CASES[case]
    wl = I.small_bscan(seed=31, **kw)
    ref = O.IsamOracle(wl.geom, "nufft")
    s = I.add_noise(ref.forward(wl.eta), 30.0, np.random.default_rng(31))
    L = O.power_iteration(ref.forward, ref.adjoint, I.start_vector(ref.image_shape, 31), 300,
                          1e-13)
    lam = O.lambda_from_data(ref.adjoint, s, 0.05)
    res = O.fista(ref.forward, ref.adjoint, s, lam, L, max_iter=3000, tol=1e-3,
                  shape=ref.image_shape)
    assert 3 < res.iterations < 3000          # the rule fires, after a few iterations
    dt = np.float64 if prec == "fp64" else np.float32
    plan = Plan(wl.geom, precision=prec)
    sd = torch.from_numpy(np.ascontiguousarray(s.astype(dt))).cuda()
    out, info = plan.solve(sd, lambda_abs=lam, L=L, max_iter=3000, tol=1e-3, check_every=1,
                           eps=1e-12)
    plan.close()
    if prec == "fp64":
        assert info["iterations"] == res.iterations
        assert info["rr"] == pytest.approx(res.rr, rel=1e-6)
        assert rel(out.cpu().numpy(), res.eta) < 1e-6
    else:
        assert abs(info["iterations"] - res.iterations) <= 1
        if info["iterations"] == res.iterations:
            assert info["rr"] == pytest.approx(res.rr, rel=1e-3)
            assert rel(out.cpu().numpy(), res.eta) < 1e-3
        assert info["rr"] < 1e-3


@pytest.mark.parametrize("ny", [1, 4], ids=["bscan", "volume"])
def test_device_stop_returns_the_stopping_iterate(torch, ny):
    """The stop rule runs on the device and the host queues a further check
    interval before it reads a check's outcome; kernels queued past the stop
    return at once.  So a solve that stops at check k returns exactly (bit for
    bit) the iterate, count and r_r of a solve with the same checks that ends
    at iteration k."""
    from paper_1905_06058_gb300.isam import Plan
    wl = I.small_bscan(nx=16, ny=ny, nk=64, nz=64, n_points=6, seed=23)
    ref = O.IsamOracle(wl.geom, "nufft")
    s = ref.forward(wl.eta)
    plan = Plan(wl.geom, precision="fp32", stolt_table=False)
    sd = torch.from_numpy(s.astype(np.float32)).cuda()
    kw = dict(lambda_rel=0.05, L=4.0, check_every=10)
    # r_r at iteration 20, then a tolerance the rule meets at check 10 or 20
    _, probe = plan.solve(sd, max_iter=20, tol=1e-300, **kw)
    z, info = plan.solve(sd, max_iter=200, tol=probe["rr"] * 1.0001, **kw)
    k = info["iterations"]
    assert k in (10, 20)
    z_ref, info_ref = plan.solve(sd, max_iter=k, tol=1e-300, **kw)
    assert info_ref["iterations"] == k
    assert info["rr"] == info_ref["rr"]
    assert torch.equal(z, z_ref)
    plan.close()
