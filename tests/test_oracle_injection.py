"""Pins for the oracle's re-injection rule (App. B) and open boundary (Sec. 2).

* face frequencies follow p_face = J_face / sum J (chi-square);
* sampled velocities follow the flux-weighted distributions; the reference CDFs are
  built here by numerical integration of v phi(v) (scipy), not from the oracle's
  closed forms; the side's radial speed is Rayleigh, its axial speed the flow
  Maxwellian and its tangential speed the thermal Maxwellian;
* positions are uniform on each face;
* flux conservation: with no grain and no forces the long-run density stays uniform
  and equal to the initial one.
"""
import math

import numpy as np
from scipy import integrate, stats

import oracle
from paper_2205_06557_gb300 import workloads as W


def _sampler(mach=0.3, **kw):
    p = dict(W.tiny(), n_ions=1, dust=[], mach=mach, nu=0.0, charge_model="given")
    p.update(kw)
    return oracle.Oracle(p), p


def _draw(o, n, step=7):
    P = np.zeros((n, 3))
    V = np.zeros((n, 3))
    F = np.zeros(n, int)
    for i in range(n):
        P[i], V[i], F[i] = o.inject_sample(10 ** 6 + i, step)
    return P, V, F


def _flux_cdf(u, sig, lo, hi):
    """CDF of the density |v| N(v; u, sig^2) on [lo, hi] by numerical integration"""
    pdf = lambda v: abs(v) * math.exp(-0.5 * ((v - u) / sig) ** 2)
    tot, _ = integrate.quad(pdf, lo, hi, epsabs=0, epsrel=1e-12, limit=200)

    def cdf(x):
        x = np.atleast_1d(x)
        return np.array([integrate.quad(pdf, lo, min(max(xi, lo), hi), epsabs=0, epsrel=1e-10, limit=200)[0]
                         for xi in x]) / tot

    return cdf


def test_face_frequencies():
    o, p = _sampler(mach=0.3)
    d = o.derived()
    _, _, F = _draw(o, 20000)
    cnt = np.bincount(F, minlength=3)
    exp = 20000 * np.array([d["pb"], d["pt"], d["ps"]])
    chi2 = ((cnt - exp) ** 2 / exp).sum()
    assert chi2 < 13.8  # chi-square, 2 dof, p = 0.001
    # the probabilities follow the App. B flux integrals, done here numerically
    u, sig = d["u"], d["sig"]
    phi = lambda v: math.exp(-0.5 * ((v - u) / sig) ** 2) / (sig * math.sqrt(2 * math.pi))
    jb = math.pi * p["R"] ** 2 * integrate.quad(lambda v: v * phi(v), 0, np.inf)[0]
    jt = -math.pi * p["R"] ** 2 * integrate.quad(lambda v: v * phi(v), -np.inf, 0)[0]
    js = 2 * math.pi * p["R"] * p["H"] * integrate.quad(
        lambda v: v * math.exp(-0.5 * (v / sig) ** 2) / (sig * math.sqrt(2 * math.pi)), 0, np.inf)[0]
    J = jb + jt + js
    assert np.allclose([d["pb"], d["pt"], d["ps"]], [jb / J, jt / J, js / J], rtol=1e-9)
    assert d["Tb"] == math.floor(d["pb"] * 2 ** 32)


def test_velocity_distributions():
    o, p = _sampler(mach=0.3)
    d = o.derived()
    u, sig = d["u"], d["sig"]
    P, V, F = _draw(o, 12000)
    bot, top, side = V[F == 0], V[F == 1], V[F == 2]
    assert stats.kstest(bot[:, 2], _flux_cdf(u, sig, 0.0, u + 12 * sig)).pvalue > 1e-3
    assert stats.kstest(top[:, 2], _flux_cdf(u, sig, min(u, 0) - 12 * sig, 0.0)).pvalue > 1e-3
    for c in (0, 1):
        assert stats.kstest(bot[:, c] / sig, "norm").pvalue > 1e-3
    # side: radial (inward) Rayleigh, tangential N(0, sig^2), axial N(u, sig^2)
    ps = P[F == 2]
    rhat = ps[:, :2] / np.linalg.norm(ps[:, :2], axis=1, keepdims=True)
    that = np.stack([-rhat[:, 1], rhat[:, 0]], 1)
    vr = -(side[:, :2] * rhat).sum(1)
    vt = (side[:, :2] * that).sum(1)
    assert np.all(vr > 0)
    assert stats.kstest(vr / sig, "rayleigh").pvalue > 1e-3
    assert stats.kstest(vt / sig, "norm").pvalue > 1e-3
    assert stats.kstest((side[:, 2] - u) / sig, "norm").pvalue > 1e-3


def test_paper_literal_side_has_no_tangential_speed():
    o, p = _sampler(mach=0.3, oracle_flags=oracle.F_PAPER_SIDE)
    P, V, F = _draw(o, 3000)
    ps, vs = P[F == 2], V[F == 2]
    cross = ps[:, 0] * vs[:, 1] - ps[:, 1] * vs[:, 0]
    assert np.abs(cross).max() < 1e-12 * p["R"] * np.abs(vs).max()


def test_positions_uniform_on_faces():
    o, p = _sampler(mach=0.3)
    P, V, F = _draw(o, 12000)
    R, H = p["R"], p["H"]
    bt = P[F < 2]
    assert np.allclose(np.abs(bt[:, 2]), 0.5 * H, rtol=0, atol=0)
    rho2 = (bt[:, 0] ** 2 + bt[:, 1] ** 2) / R ** 2
    assert stats.kstest(rho2, "uniform").pvalue > 1e-3
    sd = P[F == 2]
    assert np.allclose(np.hypot(sd[:, 0], sd[:, 1]), R, rtol=1e-14)
    assert stats.kstest(sd[:, 2] / H + 0.5, "uniform").pvalue > 1e-3
    ang = (np.arctan2(sd[:, 1], sd[:, 0]) / (2 * np.pi)) % 1.0
    assert stats.kstest(ang, "uniform").pvalue > 1e-3


def test_flux_conservation_keeps_density_uniform():
    # free streaming (no forces, no grain, no collisions): the open boundary with
    # flux-weighted injection must reproduce the homogeneous stationary plasma
    p = dict(W.tiny(), n_ions=3000, dust=[], mach=0.5, nu=0.0, charge_model="given",
             oracle_flags=oracle.F_NO_IONION | oracle.F_NO_EOUT)
    o = oracle.Oracle(p)
    R, H = p["R"], p["H"]
    inner, upper, vz = [], [], []
    for _ in range(40):
        o.step(25)
        x, v, _, _ = o.get_ions()
        inner.append(np.mean(x[:, 0] ** 2 + x[:, 1] ** 2 < 0.25 * R * R))
        upper.append(np.mean(x[:, 2] > 0))
        vz.append(v[:, 2].mean())
    _, ev = o.records()
    assert o.n_ions == 3000
    assert ev[:, 8].sum() == ev[:, 9:12].sum()  # 1:1 replacement
    # inner quarter of the cross-section and upper half of the height
    assert abs(np.mean(inner) - 0.25) < 0.02
    assert abs(np.mean(upper) - 0.5) < 0.02
    assert abs(np.mean(vz) / o.derived()["u"] - 1) < 0.05
