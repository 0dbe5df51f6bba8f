"""Pins for the oracle's grain records and their averages (Eqs. 1, 2, 4; the time
averages of Sec. 2's results).

* Eq. 2: two grains, no ions: the recorded grain-grain force is Coulomb's law;
* Eq. 4: the recorded driving-field force is Q E with E = m_i nu c_s M / e (Table 3's
  relation for field-driven flow at Mach M);
* Eq. 1 for one ion: the screened Coulomb force q Q (1 + r/lambda) e^(-r/lambda) / (4 pi
  eps0 r^2), directed from the ion to the grain's far side;
* Eq. 1 against the ion-side forces: as lambda_De -> infinity the grain-side Yukawa sum
  and the ions' bare Coulomb accelerations (computed by different code) balance
  (Newton's third law);
* window means and batch-means standard errors: equal to the mean of the per-step
  records over the window and to the spread of 20 equal batch means, computed here.
"""
import math

import numpy as np

import oracle
from paper_2205_06557_gb300 import workloads as W

QE = 1.602176634e-19
EPS0 = 8.8541878128e-12
K = 1.0 / (4 * math.pi * EPS0)


def _grains(q0, q1):
    return [dict(x=0.0, y=0.0, z=-5e-5, a=1e-5, q0=q0), dict(x=3e-5, y=-2e-5, z=6e-5, a=8e-6, q0=q1)]


def test_grain_grain_force_is_coulomb():
    p = W.tiny()
    p.update(dust=_grains(-2e4 * QE, 7e3 * QE), charge_model="given", n_ions=0,
             oracle_flags=oracle.F_NO_EOUT | oracle.F_NO_BOUNDARY)
    o = oracle.Oracle(p)
    o.step(1)
    rec, _ = o.records(1, 1)
    g0, g1 = p["dust"]
    d = np.array([g0["x"] - g1["x"], g0["y"] - g1["y"], g0["z"] - g1["z"]])
    f = K * g0["q0"] * g1["q0"] * d / np.linalg.norm(d) ** 3
    assert np.allclose(rec[0, 0, 4:7], f, rtol=1e-13)
    assert np.allclose(rec[0, 1, 4:7], -f, rtol=1e-13)


def test_driving_field_force_is_q_times_e():
    p = W.tiny()
    p.update(charge_model="given")
    o = oracle.Oracle(p)
    o.step(2)
    rec, _ = o.records(1, 2)
    kB, m = 1.380649e-23, 39.948 * 1.66053906660e-27
    E = m * p["nu"] * p["mach"] * math.sqrt(kB * p["T_e"] / m) / QE
    Q = p["dust"][0]["q0"]
    assert np.allclose(rec[:, 0, 12], Q * E, rtol=1e-12)
    assert np.all(rec[:, 0, 10:12] == 0.0)


def test_orbit_force_of_one_ion_is_screened_coulomb():
    p = W.tiny()
    p.update(n_ions=1, charge_model="given", dust=[dict(x=0.0, y=0.0, z=0.0, a=1e-5, q0=-3e4 * QE)],
             oracle_flags=oracle.F_NO_EOUT)
    o = oracle.Oracle(p)
    xi = np.array([[3e-5, -4e-5, 5e-5]])
    o.set_ions(xi, np.zeros((1, 3)), np.array([0], dtype=np.uint64))
    _, fo = o.forces()
    d = o.derived()
    r = np.linalg.norm(xi[0])
    lam = d["lam"]
    f = K * d["q"] * p["dust"][0]["q0"] * (1 + r / lam) * math.exp(-r / lam) / r ** 2 * (-xi[0] / r)
    assert np.allclose(fo[0], f, rtol=1e-12)


def test_grain_and_ion_forces_balance_as_screening_vanishes():
    p = W.tiny()
    # n_inf tiny -> lambda_De of ~50 km: Yukawa -> Coulomb, and the asymmetric model becomes
    # symmetric: the force on the grain is minus the sum of the grain's forces on the ions
    p.update(n_ions=7, n_inf=4e13 * 1e-18, charge_model="given", weight=1.0,
             dust=[dict(x=0.0, y=0.0, z=1e-5, a=1e-5, q0=-3e4 * QE)],
             oracle_flags=oracle.F_NO_EOUT | oracle.F_NO_IONION)
    p["mach"] = 0.0
    p["nu"] = 0.0
    o = oracle.Oracle(p)
    x, v, ids = W.random_ions(7, p["R"], p["H"], seed=4, dust=p["dust"])
    o.set_ions(x, v, ids)
    acc, fo = o.forces()
    d = o.derived()
    assert d["lam"] > 1e4
    on_ions = (acc * d["m"]).sum(0)
    assert np.allclose(fo[0], -on_ions, rtol=1e-9, atol=1e-9 * np.abs(on_ions).max())


def test_window_means_and_batch_errors_follow_their_definition():
    p = W.tiny()
    p["avg_start"] = 41
    o = oracle.Oracle(p)
    o.step(120)  # window of 80 records: 20 batches of 4
    rec, _ = o.records(1, 120)
    mean, se = o.dust_terms()
    win = rec[40:120, : o.D, :]
    assert np.allclose(mean, win.mean(0), rtol=1e-12, atol=0)
    bm = win.reshape(20, 4, o.D, -1).mean(1)
    se_ref = bm.std(0, ddof=1) / math.sqrt(20)
    assert np.allclose(se, se_ref, rtol=1e-9, atol=1e-300)
