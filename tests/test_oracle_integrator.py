"""Pins for the oracle's velocity-Verlet push (Sec. 2).

* constant field: Verlet is exact for a constant force, x(t) = x0 + v0 t + a t^2 / 2;
* time reversal: flipping every velocity retraces the trajectory;
* energy conservation with boundaries, collisions and absorption switched off,
  including the ion-grain Coulomb energy and the cavity potential q P(r, z): the
  error is bounded and scales as dt^2.
"""
import math

import numpy as np

import oracle
from paper_2205_06557_gb300 import workloads as W

QE = 1.602176634e-19
EPS0 = 8.8541878128e-12
PA = [0, 1, 0, 1, 2, 0, 2, 1, 3, 0, 2, 3, 1, 4, 0]
PB = [0, 0, 1, 1, 0, 2, 1, 2, 0, 3, 2, 1, 3, 0, 4]

NOB = oracle.F_NO_BOUNDARY | oracle.F_NO_ABSORB


def test_constant_field_parabola():
    # E_ext with a negligible collision frequency (threshold floor(5e-10 * 2^32) = 2)
    p = dict(W.tiny(), n_ions=3, dust=[], mach=0.0, E_ext=1000.0, nu=1.0, charge_model="given",
             oracle_flags=oracle.F_NO_IONION | oracle.F_NO_EOUT | NOB)
    o = oracle.Oracle(p)
    x0, _, _, ids = o.get_ions()
    v0 = np.array([[300.0, -200.0, 100.0], [0.0, 50.0, -400.0], [-10.0, 0.0, 0.0]])
    o.set_ions(x0, v0, ids)
    n = 100
    o.step(n)
    x, v, _, ids2 = o.get_ions()
    _, ev = o.records()
    assert ev[:, 12].sum() == 0 and np.all(ids2 == ids)
    t = n * p["dt"]
    a = np.array([0.0, 0.0, QE * 1000.0 / p["m_i"]])
    assert np.allclose(x, x0 + v0 * t + 0.5 * a * t * t, rtol=0, atol=1e-17)
    assert np.allclose(v, v0 + a * t, rtol=0, atol=1e-10)


def _closed_system(n_ions, dt, q_dust=-2000.0):
    p = dict(W.tiny(), n_ions=n_ions, mach=0.0, nu=0.0, dt=dt, charge_model="given", oracle_flags=NOB)
    p["dust"] = [dict(x=0.0, y=0.0, z=0.0, a=2e-5, q0=q_dust * QE)]
    return p


def test_time_reversal():
    p = _closed_system(60, 5e-10)
    o = oracle.Oracle(p)
    x0, v0, _, ids = o.get_ions()
    o.step(40)
    x, v, _, _ = o.get_ions()
    o.set_ions(x, -v, ids)
    o.step(40)
    xb, vb, _, _ = o.get_ions()
    assert np.abs(xb - x0).max() < 1e-12 * p["R"] * 1e3
    assert np.abs(vb + v0).max() < 1e-6


def _energy(o, p):
    x, v, _, _ = o.get_ions()
    d = o.derived()
    q, m, lam = d["q"], d["m"], d["lam"]
    al = o.alpha()
    K = 0.5 * m * (v * v).sum()
    diff = x[:, None, :] - x[None, :, :]
    r = np.sqrt((diff * diff).sum(-1))
    iu = np.triu_indices(len(x), 1)
    U = (q * q * np.exp(-r[iu] / lam) / (4 * math.pi * EPS0 * r[iu])).sum()
    for g in p["dust"]:
        rd = np.sqrt(((x - [g["x"], g["y"], g["z"]]) ** 2).sum(1))
        U += (q * g["q0"] / (4 * math.pi * EPS0 * rd)).sum()
    r2 = x[:, 0] ** 2 + x[:, 1] ** 2
    z2 = x[:, 2] ** 2
    U += q * sum(al[t] * r2 ** PA[t] * z2 ** PB[t] for t in range(15)).sum()
    return K + U


def _max_energy_error(dt, t_end):
    p = _closed_system(40, dt)
    o = oracle.Oracle(p)
    E0 = _energy(o, p)
    errs = []
    n = int(round(t_end / dt))
    for _ in range(10):
        o.step(n // 10)
        errs.append(abs(_energy(o, p) - E0))
    K0 = 0.5 * o.derived()["m"] * (o.get_ions()[1] ** 2).sum()
    return max(errs) / K0


def test_energy_conservation_dt2():
    e1 = _max_energy_error(2e-9, 4e-7)
    e2 = _max_energy_error(1e-9, 4e-7)
    assert e1 < 5e-4
    ratio = e1 / e2
    assert 2.5 < ratio < 6.0, ratio
