"""Batched solves recorded as one CUDA graph (isam_batch_*).

Each entry of an uneven batch (own geometry, dispersion, NA, lambda, iteration
count) equals the same plan's isam_solve within 1e-5 (FP32 rounding of
lambda / L is formed in another order) and one entry matches the oracle's
FISTA within 1e-3; a replay after overwriting s_d follows the new data (the
relative lambda is evaluated on the device); bad batches are refused and a
non-finite entry is reported without touching the others; the stop rule runs
inside the graph."""
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


SHAPES = [dict(nx=32, nk=64, nz=64, na=0.08), dict(nx=48, nk=128, nz=128, na=0.2),
          dict(nx=24, nk=64, nz=128, na=0.12), dict(nx=64, nk=128, nz=128, na=0.15)]


def entries(torch, seed0=50):
    from paper_1905_06058_gb300.isam import Plan
    out = []
    for i, kw in enumerate(SHAPES):
        wl = I.small_bscan(seed=seed0 + i, n_points=6 + 2 * i, **kw)
        op = O.IsamOracle(wl.geom, "nufft")
        s = I.add_noise(op.forward(wl.eta), 30.0, np.random.default_rng(seed0 + i))
        plan = Plan(wl.geom)
        L = plan.lipschitz()
        sd = torch.from_numpy(s.astype(np.float32)).cuda()
        res = torch.empty(plan.image_shape, dtype=torch.complex64, device="cuda")
        kw2 = dict(lambda_rel=0.02 + 0.01 * i, max_iter=20 + 10 * i, L=L)
        out.append((plan, sd, res, kw2, wl, op, s))
    return out


def test_batch_matches_individual_solves_and_oracle(torch):
    from paper_1905_06058_gb300.isam import Batch
    ents = entries(torch)
    b = Batch([(p, sd, res, kw) for p, sd, res, kw, *_ in ents])
    assert b.kernel_count() > 2 * sum(e[3]["max_iter"] for e in ents)
    infos = b.run()
    for (p, sd, res, kw, wl, op, s), info in zip(ents, infos):
        assert info["status"] == 0 and info["iterations"] == kw["max_iter"]
        ref, rinfo = p.solve(sd, **kw)
        assert info["lam"] == pytest.approx(rinfo["lam"], rel=1e-12)
        assert rel(res.cpu().numpy(), ref.cpu().numpy()) < 1e-5
    p, sd, res, kw, wl, op, s = ents[0]
    lam = O.lambda_from_data(op.adjoint, s, kw["lambda_rel"])
    ref = O.fista(op.forward, op.adjoint, s, lam, kw["L"], max_iter=kw["max_iter"],
                  shape=op.image_shape)
    assert rel(res.cpu().numpy(), ref.eta) < 1e-3
    b.close()
    for e in ents:
        e[0].close()


@pytest.mark.parametrize("addback", [False, True])
def test_batch_stop_rule(torch, addback):
    """Alg. 1's stop rule inside the graph (evaluated on the device): every
    entry stops at the same check as its own isam_solve with the same
    tolerance, with the same r_r and image (1e-5), and the graph's output is
    that check's iterate (and its residual add-back), not the last queued one;
    a replay starts over (the stop flag is reset by the graph)."""
    from paper_1905_06058_gb300.isam import Batch
    ents = entries(torch, seed0=90)
    for i, e in enumerate(ents):
        e[3].update(max_iter=200, tol=[3e-2, 1e-2, 2e-2, 1e-9][i], check_every=5,
                    addback=addback)
    b = Batch([(p, sd, res, kw) for p, sd, res, kw, *_ in ents])
    for rep in range(2):
        infos = b.run()
        for (p, sd, res, kw, *_), info in zip(ents, infos):
            ref, rinfo = p.solve(sd, **kw)
            assert info["status"] == 0
            assert info["iterations"] == rinfo["iterations"]
            assert info["rr"] == pytest.approx(rinfo["rr"], rel=1e-4)
            assert rel(res.cpu().numpy(), ref.cpu().numpy()) < 1e-5
    assert infos[3]["iterations"] == 200 and min(i["iterations"] for i in infos[:3]) < 200
    b.close()
    for e in ents:
        e[0].close()


def test_batch_replay_follows_new_data(torch):
    from paper_1905_06058_gb300.isam import Batch
    ents = entries(torch, seed0=60)
    b = Batch([(p, sd, res, kw) for p, sd, res, kw, *_ in ents])
    b.run()
    for p, sd, res, kw, wl, op, s in ents:
        sd.mul_(-0.5).add_(torch.randn_like(sd) * 0.01)
    infos = b.run()
    for (p, sd, res, kw, *_), info in zip(ents, infos):
        ref, rinfo = p.solve(sd, **kw)
        assert info["lam"] == pytest.approx(rinfo["lam"], rel=1e-12)
        assert rel(res.cpu().numpy(), ref.cpu().numpy()) < 1e-5
    b.close()


def test_batch_refusals_and_nonfinite_entry(torch):
    from paper_1905_06058_gb300.isam import Batch, IsamError
    ents = entries(torch, seed0=70)[:3]
    p, sd, res, kw = ents[0][:4]
    with pytest.raises(IsamError):
        Batch([(p, sd, res, kw), (p, sd, res, kw)])          # one plan twice
    import ctypes
    from paper_1905_06058_gb300 import isam as B
    o = p._opts(0.01, 0.0, 10, -1.0, 1, None, False, 1.0, 0.0)
    h = ctypes.c_void_p()
    arr = (ctypes.c_void_p * 1)(p._h)
    st = B.lib().isam_batch_create(arr, 1, (ctypes.c_void_p * 1)(sd.data_ptr()), ctypes.byref(o),
                                   (ctypes.c_void_p * 1)(res.data_ptr()), None, ctypes.byref(h))
    assert st == 1 and not h.value                           # tol < 0 refused
    ents[1][1][0, 3, 5] = float("nan")
    b = Batch([(p, sd, res, kw) for p, sd, res, kw, *_ in ents])
    infos = b.run()
    assert [i["status"] for i in infos] == [0, 4, 0]
    b.close()


def test_batch_pins_its_plans(torch):
    """While a batch's graph records a plan, calls that would change the
    recorded tables or shapes are refused; after destroy they work again."""
    from paper_1905_06058_gb300.isam import Batch, IsamError
    ents = entries(torch, seed0=80)[:2]
    p, sd, res, kw = ents[0][:4]
    b = Batch([(e[0], e[1], e[2], e[3]) for e in ents])
    g = ents[0][4].geom
    for call in (lambda: p.set_model(g.disp, g.z0), lambda: p.set_filter(None), p.autotune,
                 lambda: p.set_tuning(axial_radix=8)):
        with pytest.raises(IsamError) as e:
            call()
        assert e.value.status == 1
    b.run()
    b.close()
    p.set_model(g.disp, g.z0)
    p.autotune()
    for e in ents:
        e[0].close()


def test_batch_mixes_volumes_and_bscans(torch):
    """A volume entry (2-D lateral transform) beside B-scans in one graph:
    each equals its plan's isam_solve, the volume also the oracle's FISTA."""
    from paper_1905_06058_gb300.isam import Batch, Plan
    ents = entries(torch, seed0=90)[:2]
    wl = I.small_bscan(nx=16, ny=24, nk=64, nz=64, na=0.12, seed=95, n_points=8)
    op = O.IsamOracle(wl.geom, "nufft")
    s = I.add_noise(op.forward(wl.eta), 30.0, np.random.default_rng(95))
    plan = Plan(wl.geom)
    kw = dict(lambda_rel=0.03, max_iter=15, L=plan.lipschitz())
    sd = torch.from_numpy(s.astype(np.float32)).cuda()
    res = torch.empty(plan.image_shape, dtype=torch.complex64, device="cuda")
    items = [(plan, sd, res, kw)] + [(p, d, r, k) for p, d, r, k, *_ in ents]
    b = Batch(items)
    infos = b.run()
    for (p, d, r, k), info in zip(items, infos):
        assert info["status"] == 0 and info["iterations"] == k["max_iter"]
        ref, _ = p.solve(d, **k)
        assert rel(r.cpu().numpy(), ref.cpu().numpy()) < 1e-5
    lam = O.lambda_from_data(op.adjoint, s, kw["lambda_rel"])
    ref = O.fista(op.forward, op.adjoint, s, lam, kw["L"], max_iter=kw["max_iter"],
                  shape=op.image_shape)
    assert rel(res.cpu().numpy(), ref.eta) < 1e-3
    b.close()
    for p, *_ in items:
        p.close()


def test_batch_entry_latencies(torch):
    """isam_batch_entry_ms: per-entry completion times of the last replay, from
    timing events recorded inside the graph.  Refused before the first run;
    afterwards every entry's time is positive and no later than the replay's
    host wall time, and the last entry to finish ends the graph."""
    import time
    from paper_1905_06058_gb300.isam import Batch, IsamError
    ents = entries(torch, seed0=70)
    b = Batch([(p, sd, res, kw) for p, sd, res, kw, *_ in ents])
    with pytest.raises(IsamError) as e:
        b.entry_ms()
    assert e.value.status == 1
    b.run()
    t0 = time.perf_counter()
    b.run()
    wall_ms = (time.perf_counter() - t0) * 1e3
    ms = b.entry_ms()
    assert len(ms) == len(ents)
    assert all(0.0 < m <= wall_ms for m in ms), (ms, wall_ms)
    b.close()
    for p, *_ in ents:
        p.close()
