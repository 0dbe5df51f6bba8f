"""Pins for the oracle's collisions (Sec. 2), absorption and charging (Eq. 3, Sec. 2
charging models), the OML charge, and the printed values of Tables 2 and 3.

* collisional drift: the discrete Andersen scheme's steady mean drift is exactly
  (1 - p) a dt / p; for small nu dt it is the mobility drift e E / (m_i nu);
* collision counts follow Binomial(N steps, T_coll / 2^32);
* collisions relax the velocity variance to k T_n / m_i;
* a radial shot is absorbed at the step its end point enters the grain, with the
  momentum m v / dt of Eq. 3; overlapping grains: the lowest index wins;
* with absorption off the charge follows Q' = -e Gamma_e(Q) whose closed-form
  solution Q(t) = -(C k T_e / e) ln(1 + t / tau) the forward-Euler recurrence
  approaches at first order in dt;
* OML ion current: the textbook stationary-Maxwellian and cold-beam limits;
* Table 2's preset charge agrees with the OML charge; Table 3's (E, nu) pairs follow
  the drift law u = e E / (m_i nu) with u = c_s (Mach 1).
"""
import json
import math
import os

import numpy as np

import oracle
from oracle import oml
from paper_2205_06557_gb300 import workloads as W

QE = 1.602176634e-19
KB = 1.380649e-23
EPS0 = 8.8541878128e-12
GOLD = os.path.join(os.path.dirname(__file__), "golden")
FREE = oracle.F_NO_IONION | oracle.F_NO_EOUT | oracle.F_NO_BOUNDARY


def test_collisional_drift():
    p = dict(W.tiny(), n_ions=20000, dust=[], mach=0.0, E_ext=1000.0, nu=1e7, charge_model="given",
             oracle_flags=FREE)
    o = oracle.Oracle(p)
    d = o.derived()
    o.step(400)  # two relaxation times
    means = []
    for _ in range(30):
        o.step(100)
        means.append(o.get_ions()[1][:, 2].mean())
    means = np.array(means)
    se = means.std(ddof=1) / math.sqrt(len(means)) * 2.0  # blocks of 100 steps are ~correlated over 2
    a = QE * 1000.0 / p["m_i"]
    pc = d["pcoll"]
    assert abs(pc + math.expm1(-1e7 * p["dt"])) < 1e-18
    discrete = (1 - pc) * a * p["dt"] / pc
    assert abs(means.mean() - discrete) < 3 * se + 1e-3 * discrete
    mobility = a / 1e7
    assert abs(means.mean() / mobility - 1) < 0.01
    assert abs(d["u"] - mobility) < 1e-9 * mobility  # initial drift from the same law


def test_collision_counts_and_thermalisation():
    p = dict(W.tiny(), n_ions=5000, dust=[], mach=0.0, nu=1e7, T_n=600.0, charge_model="given",
             oracle_flags=FREE)
    o = oracle.Oracle(p)
    d = o.derived()
    assert d["Tcoll"] == math.floor(d["pcoll"] * 2 ** 32)
    n = 3000
    o.step(n)
    _, ev = o.records()
    tot = ev[:, 12].sum()
    pt = d["Tcoll"] / 2 ** 32
    mu = 5000 * n * pt
    assert abs(tot - mu) < 4 * math.sqrt(mu * (1 - pt))
    v = o.get_ions()[1]
    var = v.var(0)
    target = KB * 600.0 / p["m_i"]
    assert np.all(np.abs(var / target - 1) < 0.05)


def _shot(dust, x0, v0, **kw):
    p = dict(W.tiny(), n_ions=1, mach=0.0, nu=0.0, charge_model="given", dust=dust,
             oracle_flags=oracle.F_NO_IONION | oracle.F_NO_EOUT | oracle.F_NO_BOUNDARY)
    p.update(kw)
    o = oracle.Oracle(p)
    o.set_ions(np.array([x0]), np.array([v0]), np.array([0], dtype=np.uint64))
    return o, p


def test_radial_shot_absorption_and_momentum():
    dust = [dict(x=0.0, y=0.0, z=0.0, a=2e-5, q0=0.0)]
    o, p = _shot(dust, [1.0001e-4, 0.0, 0.0], [-1000.0, 0.0, 0.0])
    o.step(170)
    rec, ev = o.records()
    hit = np.nonzero(ev[:, 0])[0]
    # end point enters the grain after ceil((1.0001e-4 - 2e-5) / 5e-7) = 161 steps
    assert list(hit) == [160] and ev[160, 0] == 1
    fc = rec[160, 0, 7:10]
    assert np.allclose(fc, [p["m_i"] * -1000.0 / p["dt"], 0.0, 0.0], rtol=1e-12)
    assert np.all(rec[:160, 0, 7:10] == 0.0)
    # the replacement came in through the boundary with the next id
    assert ev[160, 9:12].sum() == 1 and o.get_ions()[3][0] == 1


def test_overlapping_grains_lowest_index_wins():
    dust = [dict(x=0.0, y=0.0, z=0.0, a=1e-5, q0=0.0), dict(x=0.0, y=0.0, z=0.0, a=2e-5, q0=0.0)]
    o, _ = _shot(dust, [0.0, 0.0, 0.5e-5], [0.0, 0.0, -1.0])
    o.step(1)
    _, ev = o.records()
    assert ev[0, 0] == 1 and ev[0, 1] == 0


def _charge_run(dt, t_end, a=2e-5):
    dust = [dict(x=0.0, y=0.0, z=0.0, a=a, q0=0.0)]
    p = dict(W.tiny(), n_ions=1, mach=0.0, nu=0.0, dt=dt, charge_model="consistent", dust=dust,
             oracle_flags=FREE | oracle.F_NO_ABSORB)
    o = oracle.Oracle(p)
    o.set_ions(np.array([[1.5e-4, 0, 0]]), np.zeros((1, 3)), np.array([0], dtype=np.uint64))
    n = int(round(t_end / dt))
    o.step(n)
    return o.dust_q()[0], p


def test_charging_follows_closed_form():
    t_end = 2.5e-6
    q1, p = _charge_run(5e-10, t_end)
    q2, _ = _charge_run(2.5e-10, t_end)
    a, Te = 2e-5, p["T_e"]
    C = 4 * math.pi * EPS0 * a
    ve = math.sqrt(8 * KB * Te / (math.pi * 9.1093837015e-31))
    I0 = QE * p["n_inf"] * math.pi * a * a * ve  # electron current at zero potential
    tau = C * KB * Te / (QE * I0)
    exact = -(C * KB * Te / QE) * math.log(1 + t_end / tau)
    e1, e2 = abs(q1 / exact - 1), abs(q2 / exact - 1)
    assert e1 < 2e-3
    assert 1.6 < e1 / e2 < 2.4  # first order in dt


def test_oml_limits():
    a, n, m, Ti = 2e-5, 4e13, W.AR_MASS, 300.0
    phi = -3.0
    # stationary Maxwellian: I = e n pi a^2 sqrt(8 k T_i / (pi m)) (1 - e phi / k T_i)
    ref0 = QE * n * math.pi * a * a * math.sqrt(8 * KB * Ti / (math.pi * m)) * (1 - QE * phi / (KB * Ti))
    assert abs(oml.ion_current(a, phi, n, m, Ti, 0.0) / ref0 - 1) < 1e-8
    # cold beam: I = e n pi a^2 u (1 - 2 e phi / (m u^2))
    u = 40 * math.sqrt(KB * Ti / m)
    refb = QE * n * math.pi * a * a * u * (1 - 2 * QE * phi / (m * u * u))
    assert abs(oml.ion_current(a, phi, n, m, Ti, u) / refb - 1) < 2e-3


def test_table2_preset_charge_matches_oml():
    g = json.load(open(os.path.join(GOLD, "table2_preset_charge.json")))
    pl = g["plasma"]
    Q = oml.oml_charge(g["grain"]["radius_m"], pl["n_inf_m3"], pl["m_i_kg"], pl["T_i_K"], pl["T_e_K"], pl["mach"])
    assert abs(-Q / QE / g["preset_charge_e"] - 1) < 0.02


def test_table3_field_for_mach_one():
    g = json.load(open(os.path.join(GOLD, "table3_field_driven.json")))
    pl = g["plasma"]
    for pair in g["pairs"]:
        p = dict(W.tiny(), n_ions=1, dust=[], m_i=pl["m_i_kg"], T_e=pl["T_e_K"], T_i=pl["T_i_K"],
                 n_inf=pl["n_inf_m3"], mach=1.0, nu=pair["nu_Hz"], oracle_flags=oracle.F_NO_EOUT)
        E = oracle.Oracle(p).derived()["E"]
        assert abs(E / pair["E_ext_V_per_m"] - 1) < 1e-3, (E, pair)
