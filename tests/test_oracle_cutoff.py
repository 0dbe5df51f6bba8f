"""Pins for the oracle's ion-ion cutoff (Sec. 5: a switching function that vanishes
beyond a fixed distance; the form is a reading: the Yukawa pair energy times
S(x) = 1 - 10 x^3 + 15 x^4 - 6 x^5 between r_switch and r_cut).

* forces equal minus the numerical gradient of the switched pair energy, summed over
  pairs (the energy is all that is written here: a wrong sign, factor or derivative of
  the switch in the oracle's force fails);
* two ions: the plain Yukawa force inside r_switch, exactly zero at and beyond r_cut,
  and the force continuous with a vanishing slope at both ends of the switching zone
  (S(0) = 1, S(1) = 0, S'(0) = S'(1) = 0);
* a cutoff beyond the domain's diameter gives the forces without a cutoff bit for bit;
* Newton's third law holds with the cutoff.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2205_06557_gb300 import workloads as W

EPS0 = 8.8541878128e-12


def _params(n, **kw):
    p = W.tiny()
    p.update(n_ions=n, dust=[], charge_model="given", mach=0.0, nu=0.0, oracle_flags=oracle.F_NO_EOUT)
    p.update(kw)
    return p


def _switch(r, rs, rc):
    x = np.clip((r - rs) / (rc - rs), 0.0, 1.0)
    return np.where(r >= rc, 0.0, 1.0 - 10 * x ** 3 + 15 * x ** 4 - 6 * x ** 5)


def _energy_of(i, x, q, lam, rs, rc):
    d = x - x[i]
    r = np.sqrt((d * d).sum(1))
    r[i] = np.inf
    with np.errstate(invalid="ignore"):
        u = q * q * np.exp(-r / lam) / (4 * math.pi * EPS0 * r) * _switch(r, rs, rc)
    u[i] = 0.0
    return u.sum()


def test_cutoff_forces_are_minus_gradient_of_switched_energy():
    # ions spread over ~1.5 mm of z so that pairs fall on both sides of and inside the
    # switching zone; lambda_De = 1.66 mm
    n = 16
    rc, rs = 5e-4, 2e-4
    p = _params(n, R=4e-4, H=1.5e-3, r_cut=rc, r_switch=rs)
    o = oracle.Oracle(p)
    x, v, ids = W.random_ions(n, p["R"], p["H"], seed=5)
    o.set_ions(x, v, ids)
    acc, _ = o.forces()
    d = o.derived()
    r = np.sqrt(((x[:, None, :] - x[None, :, :]) ** 2).sum(-1))
    inside = ((r > rs) & (r < rc)).sum() // 2
    beyond = (r >= rc).sum() // 2
    assert inside >= 5 and beyond >= 5
    h = 2e-10
    for i in range(n):
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, c] += h
            xm[i, c] -= h
            f_fd = -(_energy_of(i, xp, d["q"], d["lam"], rs, rc) - _energy_of(i, xm, d["q"], d["lam"], rs, rc)) / (2 * h)
            f = acc[i, c] * d["m"]
            scale = np.abs(acc[i]).max() * d["m"]
            assert abs(f_fd - f) <= 1e-6 * scale, (i, c, f_fd, f)


def _pair_force(o, r):
    x = np.array([[0.0, 0.0, -0.5 * r], [0.0, 0.0, 0.5 * r]])
    o.set_ions(x, np.zeros((2, 3)), np.array([0, 1], dtype=np.uint64))
    acc, _ = o.forces()
    return acc[1, 2] * o.derived()["m"]  # force on the upper ion along +z


def test_two_ions_regions_and_smoothness():
    rc, rs = 5e-4, 3e-4
    p = _params(2, R=2e-4, H=1.2e-3, r_cut=rc, r_switch=rs)
    o = oracle.Oracle(p)
    plain = oracle.Oracle(_params(2, R=2e-4, H=1.2e-3))
    d = o.derived()
    k = d["q"] ** 2 / (4 * math.pi * EPS0)
    lam = d["lam"]
    for r in (5e-5, 1.5e-4, 2.9e-4):
        yuk = k * (1 + r / lam) * math.exp(-r / lam) / (r * r)
        assert _pair_force(o, r) == pytest.approx(yuk, rel=1e-12)
        assert _pair_force(o, r) == _pair_force(plain, r)
    for r in (rc, 5.5e-4, 1.0e-3):
        assert _pair_force(o, r) == 0.0
    # continuity at both ends and a vanishing slope there (cubic approach)
    eps = 1e-9
    assert _pair_force(o, rs + eps) == pytest.approx(_pair_force(o, rs - eps), rel=1e-6)
    f1, f2 = _pair_force(o, rc - 1e-6), _pair_force(o, rc - 2e-6)
    assert 0 < f1 < f2 and f2 / f1 == pytest.approx(4.0, rel=0.05)  # F ~ (r_c - r)^2 near r_c
    # inside the zone the force stays repulsive; the energy switch adds -U S' > 0, so
    # early in the zone it exceeds the plain force and late in it falls below
    zone = [_pair_force(o, r) for r in np.linspace(rs, rc, 9)[1:-1]]
    assert min(zone) > 0.0
    assert zone[0] > _pair_force(plain, np.linspace(rs, rc, 9)[1]) and zone[-1] < _pair_force(plain, np.linspace(rs, rc, 9)[-2])


def test_cutoff_beyond_the_domain_changes_nothing():
    n = 40
    p = _params(n)
    x, v, ids = W.random_ions(n, p["R"], p["H"], seed=9)
    a0 = oracle.Oracle(p)
    a0.set_ions(x, v, ids)
    diam = math.hypot(2 * p["R"], p["H"])
    a1 = oracle.Oracle(dict(p, r_cut=3 * diam, r_switch=2 * diam))
    a1.set_ions(x, v, ids)
    assert np.array_equal(a0.forces()[0], a1.forces()[0])


def test_newton_third_law_with_cutoff():
    n = 60
    p = _params(n, R=4e-4, H=1.5e-3, r_cut=4e-4, r_switch=1e-4)
    o = oracle.Oracle(p)
    x, v, ids = W.random_ions(n, p["R"], p["H"], seed=11)
    o.set_ions(x, v, ids)
    acc, _ = o.forces()
    tot = acc.sum(0)
    assert np.abs(tot).max() <= 1e-12 * np.abs(acc).sum(0).max()


def test_bad_cutoff_is_rejected():
    with pytest.raises(Exception):
        oracle.Oracle(_params(4, r_cut=1e-4, r_switch=2e-4))
