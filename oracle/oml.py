"""Orbital-motion-limited (OML) charge of an isolated grain (Sec. 2 charging models).

TEST INFRASTRUCTURE ONLY (part of the oracle).  Used to pick physically sensible
initial grain charges for test and benchmark inputs and to pin the charging
formulas against the paper's Table 2 preset charge.

* Electron current (Boltzmann electrons, repelled by a negative grain):
      I_e = e n_e pi a^2 sqrt(8 k T_e / (pi m_e)) exp(e phi / k T_e).
* Ion current for ions drifting at u with thermal speed sig = sqrt(k T_i / m_i),
  OML cross-section pi a^2 (1 - 2 Z e phi / (m_i v^2)) for phi < 0:
      I_i = Z e n int d^3v f(v) v sigma(v),
  reduced to one speed integral with the angular factor of the shifted Maxwellian.
* The floating potential solves I_i = I_e; Q = 4 pi eps0 a phi.
"""
import math

from scipy import integrate, optimize

QE = 1.602176634e-19
KB = 1.380649e-23
EPS0 = 8.8541878128e-12
ME = 9.1093837015e-31


def ion_current(a, phi, n, m_i, T_i, u, Z=1.0):
    """OML ion current (A) onto a sphere of radius a at potential phi <= 0."""
    sig = math.sqrt(KB * T_i / m_i)

    def integrand(v):
        if v <= 0.0:
            return 0.0
        cross = math.pi * a * a * (1.0 - 2.0 * Z * QE * phi / (m_i * v * v))
        if u == 0.0:
            ang = 4.0 * math.pi * math.exp(-v * v / (2 * sig * sig))
        else:
            x = v * u / (sig * sig)
            # 2 pi int_{-1}^{1} exp(-(v^2 - 2 v u mu + u^2)/(2 sig^2)) dmu
            ang = 2.0 * math.pi * (math.exp(-(v - u) ** 2 / (2 * sig * sig))
                                   - math.exp(-(v + u) ** 2 / (2 * sig * sig))) / x
        return v * v * v * cross * ang

    vmax = u + 14.0 * sig
    pts = [u] if u > 0 else None
    val, _ = integrate.quad(integrand, 0.0, vmax, points=pts, limit=500, epsabs=0.0, epsrel=1e-12)
    return Z * QE * n * val * (2 * math.pi * sig * sig) ** -1.5


def electron_current(a, phi, n_e, T_e):
    return QE * n_e * math.pi * a * a * math.sqrt(8 * KB * T_e / (math.pi * ME)) * math.exp(QE * phi / (KB * T_e))


def floating_potential(a, n, m_i, T_i, T_e, u, Z=1.0):
    f = lambda phi: ion_current(a, phi, n, m_i, T_i, u, Z) - electron_current(a, phi, Z * n, T_e)
    return optimize.brentq(f, -200.0 * KB * T_e / QE, -1e-12 * KB * T_e / QE, xtol=1e-15, rtol=1e-14)


def oml_charge(a, n, m_i, T_i, T_e, mach, Z=1.0):
    """OML grain charge (C) in a flow of Mach number `mach` (c_s = sqrt(Z k T_e / m_i))."""
    u = mach * math.sqrt(Z * KB * T_e / m_i)
    phi = floating_potential(a, n, m_i, T_i, T_e, u, Z)
    return 4 * math.pi * EPS0 * a * phi
