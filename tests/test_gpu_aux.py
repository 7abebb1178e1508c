"""Auxiliary subsystems on the GPU: the plan allocator hook (a host framework's
pool, and injected allocation failures), the Eq. 12 objective in the solve
info, and the autotune cache file."""
import os

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


def test_allocator_hook_and_injected_failures(torch):
    from paper_1905_06058_gb300 import isam as B
    wl = I.small_bscan(nx=32, nk=64, nz=64, seed=50)
    g = wl.geom
    eta = torch.from_numpy(wl.eta.astype(np.complex64)).cuda()
    ref = B.Plan(g)
    s_ref = ref.forward(eta)
    L = ref.lipschitz(iters=50, rtol=1e-6) * 1.01
    z_ref, _ = ref.solve(s_ref, L=L, max_iter=10)
    ref.close()
    live = {}

    def alloc(n):
        p = torch.cuda.caching_allocator_alloc(n)
        live[p] = n
        return p

    def free(p):
        live.pop(p)
        torch.cuda.caching_allocator_delete(p)

    try:
        B.use_torch_allocator()                 # the packaged helper works
        B.Plan(g).close()
        B.set_allocator(alloc, free)
        plan = B.Plan(g)
        assert len(live) > 0
        assert torch.equal(plan.forward(eta), s_ref)
        z, _ = plan.solve(s_ref, L=L, max_iter=10)
        assert torch.equal(z, z_ref)
        plan.close()
        assert not live
        for n_ok in (0, 3, 7):                  # the (n_ok + 1)-th allocation fails
            count = [0]

            def failing(n, n_ok=n_ok, count=count):
                if count[0] >= n_ok:
                    return 0
                count[0] += 1
                return alloc(n)
            B.set_allocator(failing, free)
            with pytest.raises(B.IsamError) as e:
                B.Plan(g)
            assert e.value.status == 2
            assert not live                     # the partly built plan was released
        B.set_allocator(alloc, free)
        plan = B.Plan(g)
        B.set_allocator(lambda n: 0, free)      # the solve's workspace cannot be had
        with pytest.raises(B.IsamError) as e:
            plan.solve(s_ref, L=L, max_iter=3)
        assert e.value.status == 2
        B.set_allocator(alloc, free)
        z, _ = plan.solve(s_ref, L=L, max_iter=10)
        assert torch.equal(z, z_ref)
        plan.close()
        assert not live
    finally:
        B.set_allocator()


@pytest.mark.parametrize("weighted", [False, True])
def test_objective_matches_oracle(torch, weighted):
    from paper_1905_06058_gb300.isam import Plan
    wl = I.small_bscan(nx=32, nk=64, nz=128, seed=51, n_points=10)
    op = O.IsamOracle(wl.geom, "nufft")
    s = I.add_noise(op.forward(wl.eta), 30.0, np.random.default_rng(51))
    w = I.depth_weights(op.grid.nz) if weighted else np.ones(op.grid.nz)
    plan = Plan(wl.geom)
    sd = torch.from_numpy(s.astype(np.float32)).cuda()
    wd = torch.from_numpy(w.astype(np.float32)).cuda() if weighted else None
    z, info = plan.solve(sd, lambda_rel=0.03, max_iter=30, w=wd, objective=True)
    _, info0 = plan.solve(sd, lambda_rel=0.03, max_iter=30, w=wd)
    plan.close()
    assert info0["objective"] == -1.0
    ref = O.objective(op.forward, z.cpu().numpy().astype(np.complex128), s, info["lam"],
                      w[None, None, :])
    assert info["objective"] == pytest.approx(ref, rel=1e-5)


def test_autotune_cache_file(torch, tmp_path):
    from paper_1905_06058_gb300.isam import Plan
    path = tmp_path / "tune.txt"
    os.environ["ISAM_AUTOTUNE_CACHE"] = str(path)
    try:
        g = I.small_bscan(nx=64, nk=128, nz=128, seed=52).geom
        p1 = Plan(g)
        c1 = p1.autotune()
        lines = path.read_text().splitlines()
        assert len(lines) == 1 and f"tile={c1['lateral_tile']}" in lines[0]
        p2 = Plan(g)
        assert p2.autotune() == c1
        assert len(path.read_text().splitlines()) == 1       # served from the cache
        key = lines[0].split(" -> ")[0]
        with open(path, "a") as f:                          # a later entry wins
            f.write(f"{key} -> tile=1 stolt=2\n")
        p3 = Plan(g)
        # (a line without radices, as earlier builds wrote them, means 16/16)
        assert p3.autotune() == {"lateral_tile": 1, "stolt_table": False, "axial_radix": 16,
                                 "lateral_radix": 16}
        for p in (p1, p2, p3):
            p.close()
    finally:
        del os.environ["ISAM_AUTOTUNE_CACHE"]


@pytest.mark.parametrize("prec,cdt", [("fp32", np.complex64), ("fp64", np.complex128)])
def test_max_abs_propagates_nan(torch, prec, cdt):
    """lambda = c ||A^H s||_inf must not come silently from corrupted data: a NaN
    anywhere in the image makes the max NaN; an infinite element gives inf."""
    from paper_1905_06058_gb300.isam import Plan
    wl = I.small_bscan(nx=64, nk=256, nz=256, seed=53)
    plan = Plan(wl.geom, precision=prec)
    x = I.random_image(plan.image_shape, 53).astype(cdt)
    ref = float(np.abs(x).max())
    assert plan.max_abs(torch.from_numpy(x).cuda()) == pytest.approx(ref, rel=1e-6)
    for pos in ((0, 0, 0), (0, 17, 100), (0, 63, 255)):      # first, inner, last element
        y = x.copy()
        y[pos] = complex(np.nan, 0.0)
        assert np.isnan(plan.max_abs(torch.from_numpy(y).cuda()))
    y = x.copy()
    y[0, 5, 7] = complex(0.0, np.inf)
    assert plan.max_abs(torch.from_numpy(y).cuda()) == np.inf
    plan.close()
