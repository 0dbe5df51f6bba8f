"""Pins for the oracle's confinement field E_out (App. A).

The cavity potential needs I(r, z) = int_cyl exp(-|r-r'|/lam)/|r-r'| d^3r'.  Its
quadrature is pinned by
* the screened Poisson equation, (laplacian - 1/lam^2) I = -4 pi inside the cylinder,
  checked by finite differences at off-axis points (any error in the ray-boundary
  geometry breaks it);
* the on-axis value, where the transverse integral is elementary and leaves a 1-D
  integral done here by scipy;
* the Coulomb limit on the axis (closed form for a uniformly charged cylinder);
* the infinite-medium limit 4 pi lam^2.
The 15-term fit (Eq. Polinomial) and its gradient (Eq. extField) are pinned by the
fit residual, by the numerical gradient of the quadrature potential, and by the
field pointing inward (confining for ions).
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_2205_06557_gb300 import workloads as W

QE = 1.602176634e-19
EPS0 = 8.8541878128e-12
PA = [0, 1, 0, 1, 2, 0, 2, 1, 3, 0, 2, 3, 1, 4, 0]
PB = [0, 0, 1, 1, 0, 2, 1, 2, 0, 3, 2, 1, 3, 0, 4]


def _geom(kind):
    p = W.tiny()
    p["n_ions"] = 1
    p["dust"] = []
    if kind == "wide":  # R = 3 lam, H = 6 lam as in Table 2's domain (in Debye lengths)
        lam = 1.6622799639830418e-3
        p["R"], p["H"] = 3 * lam, 6 * lam
    return p


def _lam(p):
    return math.sqrt(EPS0 * 1.380649e-23 * p["T_e"] / (p["n_inf"] * QE * QE))


@pytest.mark.parametrize("kind", ["tiny", "wide"])
def test_screened_poisson_identity(kind):
    p = _geom(kind)
    lam = _lam(p)
    R, hz = p["R"], 0.5 * p["H"]
    I = lambda r, z: oracle.cyl_integral(p, r, z)
    h = 2e-3 * R
    for (r, z) in [(0.5 * R, 0.3 * hz), (0.8 * R, -0.6 * hz), (0.25 * R, 0.85 * hz)]:
        c = I(r, z)
        irr = (I(r + h, z) - 2 * c + I(r - h, z)) / h ** 2
        ir = (I(r + h, z) - I(r - h, z)) / (2 * h)
        izz = (I(r, z + h) - 2 * c + I(r, z - h)) / h ** 2
        lap = irr + ir / r + izz
        assert abs((lap - c / lam ** 2) / (-4 * math.pi) - 1) < 2e-4, (r, z, lap - c / lam ** 2)


@pytest.mark.parametrize("kind", ["tiny", "wide"])
def test_on_axis_one_dimensional(kind):
    p = _geom(kind)
    lam = _lam(p)
    R, hz = p["R"], 0.5 * p["H"]
    for z0 in (0.0, 0.4 * hz, hz):
        f = lambda t: 2 * math.pi * lam * (math.exp(-abs(t) / lam) - math.exp(-math.sqrt(R * R + t * t) / lam))
        ref, _ = integrate.quad(f, -hz - z0, hz - z0, points=[0.0] if -hz - z0 < 0 < hz - z0 else None,
                                epsabs=0, epsrel=1e-13, limit=200)
        assert abs(oracle.cyl_integral(p, 0.0, z0) / ref - 1) < 1e-10


def test_coulomb_limit_on_axis():
    p = dict(_geom("tiny"), n_inf=1.0)  # lam ~ 1e4 m
    R, hz = p["R"], 0.5 * p["H"]

    def F(L):  # int_0^L (sqrt(R^2 + t^2) - t) dt
        return 0.5 * (L * math.sqrt(R * R + L * L) + R * R * math.asinh(L / R)) - 0.5 * L * L

    lam = _lam(p)
    for z0 in (0.0, 0.5 * hz, hz):
        # exp(-s/lam)/s = 1/s - 1/lam + O(s/lam^2): the second term integrates to -V/lam
        ref = 2 * math.pi * (F(hz - z0) + F(hz + z0)) - math.pi * R * R * p["H"] / lam
        assert abs(oracle.cyl_integral(p, 0.0, z0) / ref - 1) < 1e-10


def test_infinite_medium_limit():
    p = _geom("tiny")
    lam = _lam(p)
    p["R"], p["H"] = 25 * lam, 50 * lam
    assert abs(oracle.cyl_integral(p, 0.0, 0.0) / (4 * math.pi * lam * lam) - 1) < 1e-9


def _poly(al, r, z):
    return sum(al[t] * (r * r) ** PA[t] * (z * z) ** PB[t] for t in range(15))


@pytest.mark.parametrize("kind", ["tiny", "wide"])
def test_fit_residual_gradient_and_direction(kind):
    p = _geom(kind)
    o = oracle.Oracle(p)
    al = o.alpha()
    R, hz = p["R"], 0.5 * p["H"]
    pref = QE * p["n_inf"] / (4 * math.pi * EPS0)
    phi = lambda r, z: -pref * oracle.cyl_integral(p, r, z)
    # residual on a coarse sub-grid of the fit grid
    vals, fits = [], []
    for k in range(0, 41, 5):
        for q in range(0, 41, 5):
            r, z = k / 40 * R, q / 40 * hz
            vals.append(phi(r, z))
            fits.append(_poly(al, r, z))
    vals, fits = np.array(vals), np.array(fits)
    rng = vals.max() - vals.min()
    res = vals - fits - np.mean(vals - fits)
    # the 15-term fit is an approximation of the method: worst at the rim, small elsewhere
    assert np.abs(res).max() < 1e-2 * rng
    assert np.sqrt(np.mean(res ** 2)) < 2e-3 * rng
    # fitted field vs numerical gradient of the quadrature potential, off the grid
    h = 1e-4 * R
    Es = []
    for (r, z) in [(0.33 * R, 0.21 * hz), (0.71 * R, 0.55 * hz), (0.93 * R, -0.37 * hz), (0.12 * R, 0.9 * hz)]:
        Er_num = -(phi(r + h, z) - phi(r - h, z)) / (2 * h)
        Ez_num = -(phi(r, z + h) - phi(r, z - h)) / (2 * h)
        E = o.eout(r, 0.0, z)
        Es.append((E[0], E[2], Er_num, Ez_num))
        # confining: field points back toward the centre
        assert E[0] < 0 and E[2] * z < 0 and E[1] == 0.0
    Es = np.array(Es)
    scale = np.abs(Es[:, 2:]).max()
    assert np.abs(Es[:, 0] - Es[:, 2]).max() < 1e-2 * scale
    assert np.abs(Es[:, 1] - Es[:, 3]).max() < 1e-2 * scale
    # symmetry: no field at the centre
    assert np.all(o.eout(0.0, 0.0, 0.0) == 0.0)
