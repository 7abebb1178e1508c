"""isam_autotune: picks a feasible lateral tile and Stolt-table mode and
leaves every result unchanged (to FP32 rounding, 1e-6) — solves before and
after tuning agree, including the stop rule's iteration count."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("kw", [dict(nx=64, nk=128, nz=128), dict(nx=384, nk=64, nz=64),
                                dict(nx=8, ny=16, nk=64, nz=64), dict(nx=16, nk=2048, nz=2048)],
                         ids=["bscan", "bscan_radix3", "volume", "nz2048"])
def test_autotune_keeps_results(torch, kw):
    from paper_1905_06058_gb300.isam import Plan
    wl = I.small_bscan(seed=14, **kw)
    plan = Plan(wl.geom)
    eta = torch.from_numpy(I.random_image(plan.image_shape, 3).astype(np.complex64)).cuda()
    s = plan.forward(eta)
    L = plan.lipschitz(iters=50, rtol=1e-6) * 1.01
    out0, info0 = plan.solve(s, lambda_rel=0.05, L=L, max_iter=40, tol=1e-4, check_every=5)
    choice = plan.autotune()
    L8 = (kw["ny"] if kw.get("ny", 1) > 1 else kw["nx"]) // 8
    assert choice["lateral_tile"] in (1, 2, 4, 8) and choice["lateral_tile"] * max(L8, 1) <= 512
    out1, info1 = plan.solve(s, lambda_rel=0.05, L=L, max_iter=40, tol=1e-4, check_every=5)
    assert info1["iterations"] == info0["iterations"]
    a, b = out0.cpu().numpy(), out1.cpu().numpy()
    assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(a)
    plan.close()
