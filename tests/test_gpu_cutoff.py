"""The ion-ion cutoff (Sec. 5 switching function) on the GPU against the oracle:
forces on injected states in an elongated domain, 30 coupled steps with every integer
event identical, the cutoff beyond the domain reproducing the all-pairs run, bitwise
determinism and exact checkpoints."""
import math

import numpy as np
import pytest

import oracle
import paper_2205_06557_gb300 as od
from paper_2205_06557_gb300 import workloads as W

pytestmark = pytest.mark.gpu
EPS0 = 8.8541878128e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2205_06557_gb300 import build

    build.build()
    od.lib()


def _tube(H=2e-3, **kw):
    """the ~2,000-ion plasma in a tube of radius 0.2 mm and length H (10,050 ions at 2 mm)"""
    p = W.tiny()
    p.update(H=H, n_ions=0, charge_model="given")
    p.update(kw)
    return p


RC, RS = 3e-4, 1.5e-4  # cutoff and start of the switching zone, m (lambda_De = 1.66 mm)


def _scales(x, lam, kii, rc):
    """per ion: sum_j |a_ij| over pairs inside the cutoff (plain Yukawa magnitude, an upper
    bound of the switched one up to the switch's slope term)"""
    n = len(x)
    out = np.zeros(n)
    for i0 in range(0, n, 512):
        d = x[i0: i0 + 512, None, :] - x[None, :, :]
        r = np.sqrt((d * d).sum(-1))
        with np.errstate(divide="ignore", invalid="ignore"):
            f = kii * (1 + r / lam) * np.exp(-r / lam) / (r * r) * (1 + 6 * r / rc)
        f[~np.isfinite(f) | (r >= rc)] = 0.0
        out[i0: i0 + 512] = f.sum(1)
    return out


@pytest.mark.parametrize("n", [1, 700, 4099, 10050])
def test_cutoff_forces_on_injected_states(n):
    p = _tube(n_ions=max(n, 1), r_cut=RC, r_switch=RS)
    p["alpha"] = oracle.Oracle(dict(p, n_ions=1)).alpha()
    o = oracle.Oracle(p)
    x, v, ids = W.random_ions(n, p["R"], p["H"], seed=700 + n, dust=p["dust"])
    o.set_ions(x, v, ids)
    acc_ref, fo_ref = o.forces()
    run = od.Run(p)
    od.od_set_cutoff(run.h, RC, RS)
    run.set_ions(x, v, ids, next_id=n)
    _, _, a_gpu, _ = run.get_ions()
    d = o.derived()
    kii = d["q"] ** 2 / (4 * math.pi * EPS0 * d["m"])
    scale = _scales(x, d["lam"], kii, RC) + np.linalg.norm(acc_ref, axis=1)
    dev = np.linalg.norm(a_gpu - acc_ref, axis=1)
    assert np.linalg.norm(a_gpu - acc_ref) <= 1e-5 * np.linalg.norm(acc_ref)
    err = dev / scale
    assert err.max() < 1e-5, (err.max(), int(err.argmax()))
    _, fo_gpu = run.dust_now()
    assert np.allclose(fo_gpu, fo_ref, rtol=1e-5, atol=1e-5 * np.abs(fo_ref).max())
    run.close()


def test_cutoff_steps_match_the_oracle_event_for_event():
    p = _tube(H=1.2e-3, charge_model="consistent", r_cut=RC, r_switch=RS)
    p["alpha"] = oracle.Oracle(dict(p, n_ions=1)).alpha()
    o = oracle.Oracle(p)
    run = od.Run(p)
    od.od_set_cutoff(run.h, RC, RS)
    steps = 30
    o.step(steps)
    for _ in range(steps):
        run.step(1)
    _, ev_o = o.records(1, steps)
    _, ev_g = run.series(1, steps)
    bad = np.nonzero((ev_o != ev_g).any(1))[0]
    assert len(bad) == 0, bad
    xo, _, _, io = o.get_ions()
    xg, _, _, ig = run.get_ions()
    assert np.array_equal(io, ig) and np.abs(xo - xg).max() < 1e-10
    run.close()


def test_cutoff_beyond_the_domain_reproduces_all_pairs():
    p = _tube(H=1.2e-3)
    a, b = od.Run(p), od.Run(p)
    diam = math.hypot(2 * p["R"], p["H"])
    od.od_set_cutoff(b.h, 3 * diam, 2 * diam)
    a.step(20)
    b.step(20)
    assert np.array_equal(a.series(1, 20)[1], b.series(1, 20)[1])
    xa, _, _, ia = a.get_ions()
    xb, _, _, ib = b.get_ions()
    assert np.array_equal(ia, ib) and np.abs(xa - xb).max() < 1e-12


def test_cutoff_is_deterministic_and_checkpoints_exactly(tmp_path):
    p = _tube()
    a, b = od.Run(p), od.Run(p)
    for r in (a, b):
        od.od_set_cutoff(r.h, RC, RS)
        r.step(8)
    path = str(tmp_path / "cut.ckpt")
    a.save(path)
    a.step(7)
    b.step(7)
    c = od.Run.load(path)
    c.step(7)
    xa, va, aa, _ = a.get_ions()
    for r in (b, c):
        x, v, acc, _ = r.get_ions()
        assert np.array_equal(x, xa) and np.array_equal(v, va) and np.array_equal(acc, aa)
    assert np.array_equal(a.series(1, 15)[0], c.series(1, 15)[0])
    with pytest.raises(od.OdError):
        od.od_tune(c.h, 1)
    od.od_set_cutoff(c.h, 0.0)
    c.step(2)


def test_uneven_density_matches_the_oracle(tmp_path):
    """All 16,384 ions of a 12 mm tube gathered within |z| < r_cut / 2: each of the 32 tiles
    then neighbours all 32 (a uniform density gives about 3).  The tile pairs' sums go to
    one fixed-point accumulator per ion, so no per-neighbour storage can run short; the
    forces match the oracle; the cutoff set on the gathered state gives the same bits; a
    checkpoint of it loads and continues exactly."""
    n = 16384
    p = _tube(H=1.2e-2, n_ions=n, r_cut=RC, r_switch=RS)
    p["alpha"] = oracle.Oracle(dict(p, n_ions=1)).alpha()
    x, v, ids = W.random_ions(n, p["R"], RC, seed=4242, dust=p["dust"])
    run = od.Run(p)
    od.od_set_cutoff(run.h, RC, RS)
    run.set_ions(x, v, ids, next_id=n)
    o = oracle.Oracle(p)
    o.set_ions(x, v, ids)
    acc_ref, fo_ref = o.forces()
    _, _, a_gpu, _ = run.get_ions()
    d = o.derived()
    kii = d["q"] ** 2 / (4 * math.pi * EPS0 * d["m"])
    dev = np.linalg.norm(a_gpu - acc_ref, axis=1)
    assert np.linalg.norm(a_gpu - acc_ref) <= 1e-5 * np.linalg.norm(acc_ref)
    err = dev / (_scales(x, d["lam"], kii, RC) + np.linalg.norm(acc_ref, axis=1))
    assert err.max() < 1e-5, (err.max(), int(err.argmax()))
    _, fo_gpu = run.dust_now()
    assert np.allclose(fo_gpu, fo_ref, rtol=1e-5, atol=1e-5 * np.abs(fo_ref).max())
    late = od.Run(p)
    late.set_ions(x, v, ids, next_id=n)
    od.od_set_cutoff(late.h, RC, RS)
    assert np.array_equal(late.get_ions()[2], a_gpu)
    late.close()
    path = str(tmp_path / "gathered.ckpt")
    run.save(path)
    back = od.Run.load(path)
    run.step(3)
    back.step(3)
    for got, want in zip(back.get_ions(), run.get_ions()):
        assert np.array_equal(got, want)
    run.close()
    back.close()


def test_bad_cutoffs_are_rejected():
    run = od.Run(W.tiny())
    for rc, rs in [(1e-4, 2e-4), (1e-4, -1e-5), (float("nan"), 0.0)]:
        with pytest.raises(od.OdError) as ei:
            od.od_set_cutoff(run.h, rc, rs)
        assert ei.value.code == -1
    run.close()
