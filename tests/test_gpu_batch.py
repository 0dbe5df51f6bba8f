"""Batched persistent launch: runs stepped together in one launch per step must
reproduce the same runs stepped alone (integer events bit-exact, the same ion ids,
positions equal up to the pair-sum order of the different tiling)."""
import numpy as np
import pytest

import paper_2205_06557_gb300 as od
from paper_2205_06557_gb300 import workloads as W

pytestmark = pytest.mark.gpu

QE = 1.602176634e-19


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2205_06557_gb300 import build

    build.build()
    od.lib()


def _params():
    ps = [W.tiny(seed=s) for s in range(3)]
    big = W.tiny(seed=7)
    big["R"] *= 1.6
    big["H"] *= 1.6
    big["mach"] = 0.6
    big["dust"] = [dict(x=0.0, y=0.0, z=-8e-5, a=1.5e-5, q0=-6e4 * QE), dict(x=5e-5, y=0.0, z=9e-5, a=1e-5, q0=-4e4 * QE)]
    ps.append(big)
    for p in ps:
        p["avg_start"] = 1
    return ps


def _compare(batch_run, single, steps):
    _, ev_b = batch_run.series(1, steps)
    _, ev_s = single.series(1, steps)
    bad = np.nonzero((ev_b != ev_s).any(1))[0]
    assert len(bad) == 0, (bad[:3], ev_b[bad[:1]].tolist(), ev_s[bad[:1]].tolist())
    xb, vb, _, ib = batch_run.get_ions()
    xs, vs, _, is_ = single.get_ions()
    assert np.array_equal(ib, is_)
    assert np.abs(xb - xs).max() < 1e-10
    qb, Fb = batch_run.dust_state()
    qs, Fs = single.dust_state()
    assert np.allclose(qb, qs, rtol=1e-9)


def test_batch_reproduces_single_runs():
    ps = _params()
    batch = od.Batch(ps)
    singles = [od.Run(p) for p in ps]
    assert [r.N for r in batch.runs] == [s.N for s in singles]
    assert len(set(r.N for r in batch.runs)) >= 2  # uneven sizes
    batch.step(25)
    for s in singles:
        s.step(25)
    for r, s in zip(batch.runs, singles):
        _compare(r, s, 25)
        assert r.counters()[13] == 25
    batch.close()


def test_batch_tuning_keeps_results():
    ps = _params()[:2]
    batch = od.Batch(ps)
    ms, ipt, jc = batch.tune(reps=1)
    assert ms.shape == (3, 4) and ms.min() > 0 and ipt in od.BATCH_TPT and jc in od.BATCH_CHUNKS
    assert ms[od.BATCH_TPT.index(ipt), od.BATCH_CHUNKS.index(jc)] == ms.min()
    singles = [od.Run(p) for p in ps]
    batch.step(15)
    for s in singles:
        s.step(15)
    for r, s in zip(batch.runs, singles):
        _compare(r, s, 15)
    batch.close()


@pytest.mark.parametrize("tpt", od.BATCH_TPT)
def test_batch_symmetric_plan_reproduces_single_runs(tpt):
    """the batch's symmetric tile pairs (each unordered pair once) give the same events
    and trajectories as the runs stepped alone"""
    ps = _params()
    batch = od.Batch(ps)
    od.od_batch_set_config(batch.b, tpt, 0)
    singles = [od.Run(p) for p in ps]
    batch.step(20)
    for s in singles:
        s.step(20)
    for r, s in zip(batch.runs, singles):
        _compare(r, s, 20)
    batch.close()


def test_batch_member_cannot_be_stepped_alone():
    batch = od.Batch(_params()[:1])
    with pytest.raises(od.OdError) as ei:
        od.od_step(batch.runs[0].h, 1)
    assert ei.value.code == -1
    batch.close()
