"""Pins for the oracle's force routine (Sec. 2 ion model, Eq. 1, App. A field).

* every acceleration equals -grad U / m, with U written as a potential energy
  (Yukawa pair energy, Coulomb ion-grain energy, q P(r, z) of the fitted cavity
  potential, -q E z of the driving field) and differentiated numerically;
* Newton's third law for the ion-ion part;
* Coulomb's law in the limit lambda_De -> infinity (ion-ion and ion-grain), where the
  asymmetric ion-grain model becomes symmetric;
* the Debye length against the NRL formulary's 7430 sqrt(T_e[eV]/n[m^-3]) m.
"""
import math

import numpy as np

import oracle
from paper_2205_06557_gb300 import workloads as W

QE = 1.602176634e-19
EPS0 = 8.8541878128e-12
PA = [0, 1, 0, 1, 2, 0, 2, 1, 3, 0, 2, 3, 1, 4, 0]
PB = [0, 0, 1, 1, 0, 2, 1, 2, 0, 3, 2, 1, 3, 0, 4]


def _params(n, dust_q=(-1000.0, 500.0), **kw):
    p = W.tiny()
    p["n_ions"] = n
    places = [(0.0, 0.0, -6e-5), (4e-5, 0.0, 7e-5)]
    p["dust"] = [dict(x=c[0], y=c[1], z=c[2], a=1e-5, q0=qe * QE) for c, qe in zip(places, dust_q)]
    p["charge_model"] = "given"
    p.update(kw)
    return p


def _ion_energy(i, x, q, lam, dust, alpha, E, eout=True):
    """potential energy terms that involve ion i"""
    d = x - x[i]
    r = np.sqrt((d * d).sum(1))
    r[i] = np.inf
    U = (q * q * np.exp(-r / lam) / (4 * math.pi * EPS0 * r)).sum()
    for g in dust:
        rd = math.sqrt((x[i, 0] - g["x"]) ** 2 + (x[i, 1] - g["y"]) ** 2 + (x[i, 2] - g["z"]) ** 2)
        U += q * g["q0"] / (4 * math.pi * EPS0 * rd)
    if eout:
        r2 = x[i, 0] ** 2 + x[i, 1] ** 2
        z2 = x[i, 2] ** 2
        U += q * sum(alpha[t] * r2 ** PA[t] * z2 ** PB[t] for t in range(15))
    U -= q * E * x[i, 2]
    return U


def test_forces_are_minus_gradient_of_energy():
    p = _params(14)
    o = oracle.Oracle(p)
    x, v, ids = W.random_ions(14, p["R"], p["H"], seed=3, dust=p["dust"])
    o.set_ions(x, v, ids)
    acc, _ = o.forces()
    d = o.derived()
    alpha = o.alpha()
    h = 2e-9
    for i in range(14):
        for c in range(3):
            xp = x.copy()
            xm = x.copy()
            xp[i, c] += h
            xm[i, c] -= h
            Up = _ion_energy(i, xp, d["q"], d["lam"], p["dust"], alpha, d["E"])
            Um = _ion_energy(i, xm, d["q"], d["lam"], p["dust"], alpha, d["E"])
            f_fd = -(Up - Um) / (2 * h)
            f = acc[i, c] * d["m"]
            scale = np.abs(acc[i]).max() * d["m"]
            assert abs(f_fd - f) <= 2e-6 * scale, (i, c, f_fd, f)


def test_newton_third_law_ion_ion():
    p = _params(300, dust_q=(), mach=0.0, nu=0.0, oracle_flags=oracle.F_NO_EOUT)
    o = oracle.Oracle(p)
    x, v, ids = W.random_ions(300, p["R"], p["H"], seed=5)
    o.set_ions(x, v, ids)
    acc, _ = o.forces()
    tot = acc.sum(0)
    assert np.all(np.abs(tot) <= 1e-12 * np.abs(acc).sum(0))


def test_coulomb_limit_two_ions_and_grain():
    # n_inf tiny => lambda_De ~ 1e4 m; the Yukawa factor (1 + r/lam) exp(-r/lam) -> 1
    p = _params(2, dust_q=(-3000.0,), mach=0.0, nu=0.0, n_inf=1.0, oracle_flags=oracle.F_NO_EOUT)
    p["dust"][0].update(x=0.0, y=0.0, z=0.0)
    o = oracle.Oracle(p)
    assert o.derived()["lam"] > 1e3
    x = np.array([[5e-5, 0.0, 0.0], [5e-5, 0.0, 3e-5]])
    o.set_ions(x, np.zeros((2, 3)), np.arange(2, dtype=np.uint64))
    acc, fo = o.forces()
    m = p["m_i"]
    Q = p["dust"][0]["q0"]
    k = 1.0 / (4 * math.pi * EPS0)
    # ion 0: pushed by ion 1 along -z, attracted by the grain along -x
    d01 = 3e-5
    exp0 = np.array([k * QE * Q / (5e-5) ** 2, 0.0, -k * QE * QE / d01 ** 2]) / m
    assert np.allclose(acc[0], exp0, rtol=1e-8, atol=0)
    # grain: attracted by both ions; in this limit equal and opposite to the ion-side forces
    f_ions_from_grain = np.zeros(3)
    for xi in x:
        r = np.linalg.norm(xi)
        f_ions_from_grain += k * QE * Q * xi / r ** 3
    assert np.allclose(fo[0], -f_ions_from_grain, rtol=1e-8, atol=0)


def test_asymmetric_ion_grain_model():
    """finite lambda: the grain feels the screened force, the ion the bare one"""
    p = _params(1, dust_q=(-5000.0,), mach=0.0, nu=0.0, oracle_flags=oracle.F_NO_EOUT)
    p["dust"][0].update(x=0.0, y=0.0, z=0.0)
    o = oracle.Oracle(p)
    lam = o.derived()["lam"]
    r = 1.5e-4
    o.set_ions(np.array([[0.0, r, 0.0]]), np.zeros((1, 3)), np.zeros(1, dtype=np.uint64))
    acc, fo = o.forces()
    f_ion = acc[0] * p["m_i"]
    ratio = -fo[0][1] / f_ion[1]
    assert abs(ratio - (1 + r / lam) * math.exp(-r / lam)) < 1e-12
    assert ratio < 1.0


def test_debye_length_nrl():
    o = oracle.Oracle(dict(W.tiny(), n_ions=1, dust=[]))
    lam = o.derived()["lam"]
    nrl = 7430.0 * math.sqrt(2.0 / 4e13)
    assert abs(lam / nrl - 1) < 2e-3
