"""Seeded synthetic inputs shared by the CUDA library's tests/bench and the oracle.

This module holds parameter sets and random input generators only: none of the
method's arithmetic (forces, pushes, sampling rules, charging) lives here.  Every
value is SI.  The parameter sets follow the shapes of the paper's workloads
(Sec. 4 test cases: one or a few grains on the axis of a cylinder filled with a
flowing Ar+ plasma) at the sizes used for measurement.

Parameter dict keys (both sides read the same dict):
  m_i, Z, T_i, T_n, T_e, n_inf, mach | E_ext, nu, R, H, dt, weight, n_ions,
  dust: [{x, y, z, a, q0}], charge_model ('given' | 'consistent'), seed, avg_start.
"""
import math

import numpy as np

AMU = 1.66053906660e-27
E_CHARGE = 1.602176634e-19
EV_IN_K = 11604.51812  # 1 eV / k_B

AR_MASS = 39.948 * AMU

# OML floating charge of a 20 um grain in the plasma below (Mach 1), computed once
# with the oracle's OML routine (oracle/oml.py) and stated here as an input value:
# any initial charge is a valid input; this one starts the grain near equilibrium.
Q0_A20_M1 = -108087.329 * E_CHARGE


def plasma_ar(mach=1.0, nu=1e6):
    """Ar+ plasma: T_i = T_n = 300 K, T_e = 2 eV, n = 4e13 m^-3, flow along +z."""
    return dict(m_i=AR_MASS, Z=1.0, T_i=300.0, T_n=300.0, T_e=2.0 * EV_IN_K, n_inf=4e13,
                mach=mach, E_ext=0.0, nu=nu, weight=1.0)


def tiny(steps=200, seed=0, charge_model="consistent"):
    """~2,000 ions, one 20 um grain on the axis of R = 0.2 mm, H = 0.4 mm, dt = 0.5 ns."""
    p = plasma_ar()
    p.update(R=2e-4, H=4e-4, dt=5e-10, n_ions=0, seed=seed, charge_model=charge_model,
             dust=[dict(x=0.0, y=0.0, z=0.0, a=2e-5, q0=Q0_A20_M1)], avg_start=steps // 2 + 1)
    p["steps"] = steps
    return p


def at_scale(steps=20000, seed=0):
    """Same physics with the domain scaled at fixed density and aspect to ~200,000 ions."""
    p = plasma_ar()
    p.update(R=9.267e-4, H=1.853e-3, dt=5e-10, n_ions=0, seed=seed, charge_model="consistent",
             dust=[dict(x=0.0, y=0.0, z=0.0, a=2e-5, q0=Q0_A20_M1)], avg_start=steps // 2 + 1)
    p["steps"] = steps
    return p


def dust_chain(n_dust=4, mach=1.0, nu=1e6, seed=0, steps=2000):
    """~1,000,000 ions in R = 1 mm, H = 8 mm; 2-8 grains (radii 5-20 um) along the
    axis, spaced 1-3 ion Debye lengths (0.189 mm at 300 K, 4e13 m^-3)."""
    rng = np.random.default_rng(1000 + seed)
    lam_di = 1.8903e-4
    radii = rng.uniform(5e-6, 2e-5, n_dust)
    gaps = rng.uniform(1.0, 3.0, max(n_dust - 1, 0)) * lam_di
    zs = np.concatenate([[0.0], np.cumsum(gaps)])
    zs -= zs.mean()
    p = plasma_ar(mach, nu)
    p.update(R=1e-3, H=8e-3, dt=5e-10, n_ions=0, seed=seed, charge_model="consistent",
             dust=[dict(x=0.0, y=0.0, z=float(z), a=float(a), q0=Q0_A20_M1 * float(a) / 2e-5)
                   for z, a in zip(zs, radii)], avg_start=steps // 2 + 1)
    p["steps"] = steps
    return p


def sweep_run(seed, steps=2000):
    """One run of the 64-run sweep: N log-uniform in [1e4, 2e5] at fixed density with
    H = 2R, Mach U(0.3, 2), 1-4 grains (radii U(5, 20) um) at random positions within
    the inner half of the domain."""
    rng = np.random.default_rng(seed)
    n_target = math.exp(rng.uniform(math.log(1e4), math.log(2e5)))
    # volume pi R^2 (2R) = n_target / n_inf
    R = (n_target / (4e13 * 2.0 * math.pi)) ** (1.0 / 3.0)
    H = 2.0 * R
    mach = float(rng.uniform(0.3, 2.0))
    nd = int(rng.integers(1, 5))
    dust = []
    while len(dust) < nd:
        a = float(rng.uniform(5e-6, 2e-5))
        r = 0.5 * R * math.sqrt(rng.uniform())
        ph = rng.uniform(0, 2 * math.pi)
        z = rng.uniform(-0.25 * H, 0.25 * H)
        g = dict(x=r * math.cos(ph), y=r * math.sin(ph), z=float(z), a=a, q0=Q0_A20_M1 * a / 2e-5)
        if all((g["x"] - o["x"]) ** 2 + (g["y"] - o["y"]) ** 2 + (g["z"] - o["z"]) ** 2 > (2 * (a + o["a"])) ** 2
               for o in dust):
            dust.append(g)
    p = plasma_ar(mach, 1e6)
    p.update(R=R, H=H, dt=5e-10, n_ions=0, seed=seed, charge_model="consistent", dust=dust,
             avg_start=steps // 2 + 1)
    p["steps"] = steps
    return p


def sweep(n_runs=64, steps=2000):
    return [sweep_run(s, steps) for s in range(n_runs)]


def random_ions(n, R, H, seed, speed=250.0, dust=()):
    """Uniform positions in the cylinder (outside any grain) and Maxwellian-like
    velocities of scale `speed`; ids 0..n-1.  For force and kernel tests."""
    rng = np.random.default_rng(seed)
    x = np.zeros((n, 3))
    k = 0
    while k < n:
        m = 2 * (n - k) + 16
        rho = R * np.sqrt(rng.uniform(size=m))
        ph = rng.uniform(0, 2 * np.pi, m)
        c = np.stack([rho * np.cos(ph), rho * np.sin(ph), H * (rng.uniform(size=m) - 0.5)], 1)
        ok = np.ones(m, bool)
        for g in dust:
            d = c - np.array([g["x"], g["y"], g["z"]])
            ok &= (d * d).sum(1) > (1.5 * g["a"]) ** 2
        c = c[ok][: n - k]
        x[k: k + len(c)] = c
        k += len(c)
    v = rng.normal(0.0, speed, (n, 3))
    ids = np.arange(n, dtype=np.uint64)
    return x, v, ids
