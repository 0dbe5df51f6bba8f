"""The OML charge model (Sec. 2 "oml": each grain held at its isolated-sphere floating
charge in the run's flow), solved on the device at run creation.

* the device's floating charge against the oracle's (oracle/oml.py, adaptive quadrature
  and Brent's method) for four plasmas and grains, within 1e-6;
* 25 coupled steps of a two-grain run with the OML model against the oracle given the
  oracle's OML charges as fixed charges: every integer event per step, the ids and the
  positions (1e-10 m), and the recorded charges and grain forces;
* batch members with the OML model get the same charges as single runs.
"""
import numpy as np
import pytest

import oracle
import paper_2205_06557_gb300 as od
from oracle import oml
from paper_2205_06557_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2205_06557_gb300 import build

    build.build()
    od.lib()


def _oml_ref(p, a):
    return oml.oml_charge(a, p["n_inf"], p["m_i"], p["T_i"], p["T_e"], p["mach"])


@pytest.mark.parametrize("mach,nu,a", [(1.0, 1e6, 2e-5), (0.3, 0.0, 8e-6), (2.0, 5e6, 1.5e-5), (1e-9, 0.0, 1e-5)])
def test_device_oml_charge_matches_oracle(mach, nu, a):
    p = dict(W.tiny(), mach=mach, nu=nu, n_ions=64, charge_model="oml")
    p["dust"] = [dict(x=0.0, y=0.0, z=0.0, a=a, q0=0.0)]
    run = od.Run(p)
    q, _ = run.dust_now()
    ref = _oml_ref(p, a)
    assert abs(q[0] / ref - 1) < 1e-6, (q[0], ref)
    run.close()


def _two_grains(model):
    p = W.tiny(seed=11)
    p.update(R=p["R"] * 1.3, H=p["H"] * 1.3, n_ions=0, charge_model=model, avg_start=1)
    p["dust"] = [dict(x=0.0, y=0.0, z=-8e-5, a=2e-5, q0=0.0), dict(x=3e-5, y=0.0, z=9e-5, a=1.2e-5, q0=0.0)]
    return p


def test_oml_run_matches_oracle_event_for_event():
    p = _two_grains("oml")
    q_ref = [_oml_ref(p, g["a"]) for g in p["dust"]]
    po = dict(p, charge_model="given")
    po["dust"] = [dict(g, q0=q) for g, q in zip(p["dust"], q_ref)]
    p["alpha"] = po["alpha"] = oracle.Oracle(dict(po, n_ions=1)).alpha()
    o = oracle.Oracle(po)
    run = od.Run(p)
    steps = 25
    o.step(steps)
    for _ in range(steps):
        run.step(1)
    rec_o, ev_o = o.records(1, steps)
    rec_g, ev_g = run.series(1, steps)
    bad = np.nonzero((ev_o != ev_g).any(1))[0]
    assert len(bad) == 0, (int(bad[0]) + 1, ev_o[bad[0]].tolist(), ev_g[bad[0]].tolist())
    assert ev_o[:, 8].sum() > 50
    xo, _, _, io = o.get_ions()
    xg, _, _, ig = run.get_ions()
    assert np.array_equal(io, ig) and np.abs(xo - xg).max() < 1e-10
    # constant charges, equal to the oracle's OML charges
    assert np.allclose(rec_g[:, :, 0], np.array(q_ref)[None, :], rtol=1e-6, atol=0)
    assert np.all(rec_g[:, :, 0] == rec_g[0, :, 0])
    fo_scale = np.abs(rec_o[:, :, 1:4]).max()
    assert np.abs(rec_g[:, :, 1:4] - rec_o[:, :, 1:4]).max() < 1e-4 * fo_scale
    run.close()


def test_batch_members_get_the_oml_charges():
    ps = [_two_grains("oml"), dict(_two_grains("oml"), mach=1.7, seed=3)]
    batch = od.Batch(ps)
    for r, p in zip(batch.runs, ps):
        q, _ = r.dust_now()
        ref = [_oml_ref(p, g["a"]) for g in p["dust"]]
        assert np.allclose(q, ref, rtol=1e-6, atol=0)
    batch.step(3)
    for r in batch.runs:
        rec, _ = r.series(1, 3)
        assert np.all(rec[:, :, 0] == rec[0, :, 0])
    batch.close()
