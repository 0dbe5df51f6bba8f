"""Pins for the oracle's flux-driven injection (the number of superions entering per step
follows the App. B fluxes instead of replacing each removed ion, so N varies).

* the per-step count is Poisson with mean n_inf (J_bottom + J_top + J_side) dt / w: a
  chi-square test against the exact Poisson probabilities at the ~2,000-ion plasma's
  mean (~6.5), and mean and variance where the mean is split into chunks (~150);
* the same count for the same step and seed, a different one for another seed;
* flux conservation (App. B: injecting the flux-weighted distribution through the faces
  keeps a free-streaming gas at the density n_inf): with no ion-ion or grain forces, no
  field and no collisions, the long-run mean ion count is n_inf V / w, with and without
  drift;
* without the flag N stays fixed (1:1 replacement).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2205_06557_gb300 import workloads as W

stats = pytest.importorskip("scipy.stats")

QUIET = oracle.F_NO_IONION | oracle.F_NO_EOUT | oracle.F_FLUX_INJECT


def _lam(p):
    """n_inf (J_b + J_t + J_s) dt / w from the App. B flux formulas (written out here)"""
    kB, amu = 1.380649e-23, 1.66053906660e-27
    m = p["m_i"] if "m_i" in p else 39.948 * amu
    sig = math.sqrt(kB * p["T_i"] / m)
    cs = math.sqrt(kB * p["T_e"] / m)
    u = p["mach"] * cs
    z = u / sig
    R, H = p["R"], p["H"]
    Jb = math.pi * R * R * (u * stats.norm.cdf(z) + sig * stats.norm.pdf(z))
    Jt = math.pi * R * R * (-u * stats.norm.cdf(-z) + sig * stats.norm.pdf(z))
    Js = 2 * math.pi * R * H * sig / math.sqrt(2 * math.pi)
    return p["n_inf"] / p.get("weight", 1.0) * (Jb + Jt + Js) * p["dt"]


def test_injection_count_is_poisson_with_the_flux_mean():
    p = W.tiny()
    p.update(n_ions=10, oracle_flags=QUIET)
    o = oracle.Oracle(p)
    lam = _lam(p)
    assert 6.0 < lam < 7.0
    k = np.array([o.injections(s) for s in range(1, 20001)])
    assert abs(k.mean() - lam) < 4 * math.sqrt(lam / len(k))
    obs = np.bincount(k, minlength=25)[:25]
    exp = stats.poisson.pmf(np.arange(25), lam) * len(k)
    keep = exp > 5
    chi2 = (((obs[keep] - exp[keep]) ** 2) / exp[keep]).sum()
    assert stats.chi2.sf(chi2, keep.sum() - 1) > 1e-3


def test_chunked_mean_stays_poisson():
    p = W.tiny()
    p.update(n_ions=10, n_inf=4e13 * 23.0, oracle_flags=QUIET)  # mean ~150: chunks of 64, 64, 22
    o = oracle.Oracle(p)
    lam = _lam(p)
    assert 128 < lam < 192
    k = np.array([o.injections(s) for s in range(1, 8001)], dtype=np.float64)
    assert abs(k.mean() - lam) < 4 * math.sqrt(lam / len(k))
    assert abs(k.var() / lam - 1) < 0.1


def test_count_is_a_function_of_seed_and_step():
    p = W.tiny()
    p.update(n_ions=10, oracle_flags=QUIET)
    a, b, c = oracle.Oracle(p), oracle.Oracle(p), oracle.Oracle(dict(p, seed=5))
    ka = [a.injections(s) for s in range(1, 200)]
    assert ka == [b.injections(s) for s in range(1, 200)]
    assert ka != [c.injections(s) for s in range(1, 200)]


@pytest.mark.parametrize("mach", [0.0, 1.0])
def test_flux_injection_keeps_the_free_gas_at_n_inf(mach):
    p = W.tiny()
    # a small box (~250 ions at n_inf) with free-streaming ions: no forces, no collisions
    p.update(R=1e-4, H=2e-4, dust=[], mach=mach, nu=0.0, n_ions=0, dt=2e-9, oracle_flags=QUIET)
    o = oracle.Oracle(p)
    n_eq = p["n_inf"] * math.pi * p["R"] ** 2 * p["H"]
    o.step(300)  # forget the initial state (transit ~ 0.2 mm / 250 m/s = 400 steps of 2 ns)
    counts = []
    for _ in range(200):
        o.step(25)
        counts.append(o.n_ions)
    c = np.array(counts, dtype=np.float64)
    # the mean within 3% (statistical error ~1%, plus the O(u dt / H) ~ 2% bias of placing
    # injected ions on the faces at the end of a step); the spread is Poisson-like
    assert abs(c.mean() - n_eq) < 0.03 * n_eq, (c.mean(), n_eq)
    assert 0.7 < c.std() / math.sqrt(n_eq) < 1.3


def test_without_the_flag_n_is_fixed():
    p = W.tiny()
    p.update(R=1e-4, H=2e-4, dust=[], nu=0.0, n_ions=0, dt=2e-9, oracle_flags=oracle.F_NO_IONION | oracle.F_NO_EOUT)
    o = oracle.Oracle(p)
    n0 = o.n_ions
    o.step(200)
    assert o.n_ions == n0
