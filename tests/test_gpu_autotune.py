"""isam_autotune_ex: picks a feasible lateral tile, Stolt-table mode and FFT
radices and leaves every result unchanged up to FP32 rounding (1e-5; the
radix changes the order of rounding) — solves before and after tuning agree,
including the stop rule's iteration count; the radix-8 and radix-16 forms
agree; isam_set_tuning refuses what does not fit."""
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
    assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(a)
    plan.close()


@pytest.mark.parametrize("kw", [dict(nx=16, nk=2048, nz=2048), dict(nx=1024, nk=64, nz=64),
                                dict(nx=256, nk=64, nz=64)],
                         ids=["axial_K4096", "lateral_L1024", "lateral_L256"])
def test_radix8_and_radix16_forms_agree(torch, kw):
    """Where both FFT forms exist (FP32 axial K = 2048 / 4096; lateral tiles of
    L = 1024 x 4 pairs and L = 256 x 8 pairs) they compute the same operators
    and solves up to rounding: A and A^H within 1e-6, a 30-iteration solve
    within 1e-5 relative L2."""
    from paper_1905_06058_gb300.isam import Plan
    wl = I.small_bscan(seed=15, n_points=8, **kw)
    plan = Plan(wl.geom)
    eta = torch.from_numpy(I.random_image(plan.image_shape, 4).astype(np.complex64)).cuda()
    y = torch.from_numpy(I.random_spectra(plan.spec_shape, 5).astype(np.float32)).cuda()
    res = {}
    for r in (8, 16):
        plan.set_tuning(axial_radix=r, lateral_radix=r)
        t = plan.tuning()
        assert t["axial_radix"] == r and t["lateral_radix"] == r
        s = plan.forward(eta)
        a = plan.adjoint(y)
        z, info = plan.solve(y, lambda_rel=0.05, L=4.0, max_iter=30)
        res[r] = (s.cpu().numpy(), a.cpu().numpy(), z.cpu().numpy())
    plan.close()
    for i, bar in enumerate((1e-6, 1e-6, 1e-5)):
        u, v = res[8][i], res[16][i]
        assert np.linalg.norm(u - v) <= bar * np.linalg.norm(v), i


def test_set_tuning_validates(torch):
    from paper_1905_06058_gb300.isam import IsamError, Plan
    g = I.small_bscan(nx=64, nk=64, nz=64, seed=16).geom
    plan = Plan(g, stolt_table=False)
    for kw, status in ((dict(axial_radix=4), 1), (dict(lateral_tile=16), 1),
                       (dict(lateral_tile=3), 1), (dict(stolt_table=True), 6)):
        with pytest.raises(IsamError) as e:
            plan.set_tuning(**kw)
        assert e.value.status == status, kw
    plan.set_tuning(lateral_tile=2, stolt_table=False, axial_radix=8, lateral_radix=16)
    assert plan.tuning() == {"lateral_tile": 2, "stolt_table": False, "axial_radix": 8,
                             "lateral_radix": 16}
    plan.close()
