"""Batched persistent launch against the FP64 oracle (one persistent launch per step for
runs of uneven size, Sec. 4 sweeps).

* Four runs of 2,011, ~6,800 (four grains), ~10,000 and ~20,300 ions stepped together
  for 25 steps with the ordered-pair plan and with the symmetric tile-pair plan (two
  tile sizes): every run's per-step integer events (absorbed per grain, outflow,
  injected per face, collided) equal the oracle's run of the same parameters, ion ids
  are the oracle's and positions agree within 1e-10 m.
* A ~100,000-ion run batched with a small one: after one batched step, sampled target
  ions' accelerations are within 1e-5 of their pair-term sums of the oracle's, and the
  sampled force array agrees normwise within 1e-5, with both plans.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2205_06557_gb300 as od
from paper_2205_06557_gb300 import workloads as W

pytestmark = pytest.mark.gpu

QE = 1.602176634e-19
EPS0 = 8.8541878128e-12
STEPS = 25


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2205_06557_gb300 import build

    build.build()
    od.lib()


def _scaled(p, f, **kw):
    """the ~2,000-ion plasma in a domain f times larger per axis (f^3 times the ions)"""
    q = dict(p)
    q.update(R=p["R"] * f, H=p["H"] * f, n_ions=0, avg_start=1)
    q.update(kw)
    q["alpha"] = oracle.Oracle(dict(q, n_ions=1)).alpha()
    return q


def _members():
    four = [dict(x=0.0, y=0.0, z=-1.2e-4, a=1.5e-5, q0=-8e4 * QE), dict(x=6e-5, y=0.0, z=-2e-5, a=1.0e-5, q0=-5e4 * QE),
            dict(x=-4e-5, y=5e-5, z=8e-5, a=8e-6, q0=-4e4 * QE), dict(x=0.0, y=-7e-5, z=1.6e-4, a=1.2e-5, q0=-6e4 * QE)]
    return [_scaled(W.tiny(seed=1), 1.0),
            _scaled(W.tiny(seed=2), 1.5, mach=0.6, dust=four),
            _scaled(W.tiny(seed=3), 1.71, mach=1.4, nu=5e6),
            _scaled(W.tiny(seed=4), 2.16)]


_ORACLE = {}


def _oracle_runs():
    """the members' oracle runs over STEPS steps (computed once for every plan)"""
    if "runs" not in _ORACLE:
        ps = _members()
        outs = []
        for p in ps:
            o = oracle.Oracle(p)
            o.step(STEPS)
            _, ev = o.records(1, STEPS)
            x, _, _, ids = o.get_ions()
            outs.append((ev, x, ids))
            o.close()
        _ORACLE.update(ps=ps, runs=outs)
    return _ORACLE["ps"], _ORACLE["runs"]


@pytest.mark.parametrize("tpt,chunk", [(2, 4096), (4, 0), (8, 0)])
def test_batch_members_match_the_oracle_event_for_event(tpt, chunk):
    ps, refs = _oracle_runs()
    batch = od.Batch(ps)
    od.od_batch_set_config(batch.b, tpt, chunk)
    Ns = [r.N for r in batch.runs]
    assert max(Ns) >= 20000 and len(set(Ns)) == len(Ns)
    batch.step(STEPS)
    for r, p, (ev_o, x_o, id_o) in zip(batch.runs, ps, refs):
        _, ev_g = r.series(1, STEPS)
        bad = np.nonzero((ev_g != ev_o).any(1))[0]
        assert len(bad) == 0, (r.N, int(bad[0]) + 1, ev_o[bad[0]].tolist(), ev_g[bad[0]].tolist())
        assert ev_o[:, 8].sum() > 50  # outflow and re-injection happened
        x_g, _, _, id_g = r.get_ions()
        assert np.array_equal(id_g, id_o)
        assert np.abs(x_g - x_o).max() < 1e-10
    assert ps[1]["dust"] and len(ps[1]["dust"]) == 4
    assert refs[1][0][:, :4].sum() > 0  # the four-grain run absorbed ions
    batch.close()


@pytest.mark.parametrize("tpt,chunk", [(4, 4096), (8, 0)])
def test_batch_forces_of_a_100k_ion_member(tpt, chunk):
    big = _scaled(W.tiny(seed=5), 3.68, dust=[dict(x=0.0, y=0.0, z=-2e-4, a=2e-5, q0=-1e5 * QE),
                                              dict(x=0.0, y=0.0, z=2e-4, a=1.5e-5, q0=-7e4 * QE)])
    small = _scaled(W.tiny(seed=6), 1.0)
    batch = od.Batch([big, small])
    od.od_batch_set_config(batch.b, tpt, chunk)
    batch.step(1)
    r = batch.runs[0]
    assert r.N > 95000
    x, v, a, ids = r.get_ions()
    # the step's forces used the initial charges
    o = oracle.Oracle(dict(big, n_ions=1))
    o.load_ions(x, v, ids)
    d = o.derived()
    kii = d["q"] ** 2 / (4 * math.pi * EPS0 * d["m"])
    N = len(x)
    got, want = [], []
    for i0 in (0, N // 2, N - 32):
        ref, _ = o.forces(i0, i0 + 32)
        for k in range(32):
            i = i0 + k
            rr = np.linalg.norm(x - x[i], axis=1)
            rr[i] = 1.0
            f = kii * (1 + rr / d["lam"]) * np.exp(-rr / d["lam"]) / (rr * rr)
            f[i] = 0.0
            ts = f.sum()
            err = np.linalg.norm(a[i] - ref[k]) / (ts + np.linalg.norm(ref[k]))
            assert err < 1e-5, (i, err)
        got.append(a[i0: i0 + 32])
        want.append(ref)
    got, want = np.concatenate(got), np.concatenate(want)
    assert np.linalg.norm(got - want) <= 1e-5 * np.linalg.norm(want)
    o.close()
    batch.close()
