"""Flux-driven injection (a Poisson number of ions per step from the App. B fluxes, N
varies) on the GPU against the oracle: every event and the ion count per step for 50
coupled steps, flux conservation of a free-streaming gas, the capacity overflow report,
exact checkpoints, and the combinations that are refused."""
import math

import numpy as np
import pytest

import oracle
import paper_2205_06557_gb300 as od
from paper_2205_06557_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2205_06557_gb300 import build

    build.build()
    od.lib()


@pytest.mark.parametrize("variant", [None, 12, 17])  # default plan, sym2<128,2>, sym2<64,8>
def test_flux_injection_matches_the_oracle_step_by_step(variant):
    """the count varies identically; with the packed symmetric kernels the last tiles of
    the capacity hold only dummies, so their tile pairs are skipped or give zero slots"""
    p = W.tiny()
    p["alpha"] = oracle.Oracle(dict(p, n_ions=1)).alpha()
    o = oracle.Oracle(dict(p, oracle_flags=oracle.F_FLUX_INJECT))
    run = od.Run(dict(p, flags=od.F_FLUX_INJECT))
    if variant is not None:
        od.od_set_force_config(run.h, variant, 8, 0)
    n_o, n_g = [], []
    for _ in range(50):
        o.step(1)
        run.step(1)
        n_o.append(o.n_ions)
        n_g.append(int(run.counters()[14]))
    assert n_o == n_g and len(set(n_g)) > 1  # the count varies, identically
    _, ev_o = o.records(1, 50)
    _, ev_g = run.series(1, 50)
    bad = np.nonzero((ev_o != ev_g).any(1))[0]
    assert len(bad) == 0, bad
    xo, _, _, io = o.get_ions()
    xg, _, _, ig = run.get_ions()
    assert np.array_equal(io, ig) and np.abs(xo - xg).max() < 1e-10
    run.close()


def test_flux_injection_keeps_the_free_gas_at_n_inf():
    p = W.tiny()
    # ~20,000 free-streaming ions (no forces, no collisions, no grains)
    p.update(R=4e-4, H=1e-3, dust=[], nu=0.0, n_ions=0,
             flags=od.F_FLUX_INJECT | od.F_NO_IONION | od.F_NO_EOUT)
    run = od.Run(p)
    n_eq = p["n_inf"] * math.pi * p["R"] ** 2 * p["H"]
    run.step(1500)  # a few transit times (drift 2,200 m/s over 1 mm: 900 steps)
    counts = []
    for _ in range(100):
        run.step(20)
        counts.append(run.counters()[14])
    c = np.array(counts, dtype=np.float64)
    assert abs(c.mean() - n_eq) < 0.02 * n_eq, (c.mean(), n_eq)
    run.close()


def test_capacity_overflow_is_reported():
    p = W.tiny()
    p.update(n_ions=100, flags=od.F_FLUX_INJECT)  # equilibrium ~2,000 ions, capacity 356
    run = od.Run(p)
    assert int(run.info()["capacity"]) == 356
    with pytest.raises(od.OdError) as ei:
        for _ in range(600):
            run.step(1)
    assert ei.value.code == -5 and "capacity" in str(ei.value)
    run.close()


def test_flux_run_checkpoints_exactly(tmp_path):
    p = dict(W.tiny(), flags=od.F_FLUX_INJECT)
    a = od.Run(p)
    a.step(20)
    path = str(tmp_path / "flux.ckpt")
    a.save(path)
    a.step(20)
    b = od.Run.load(path)
    b.step(20)
    xa, va, _, ia = a.get_ions()
    xb, vb, _, ib = b.get_ions()
    assert np.array_equal(ia, ib) and np.array_equal(xa, xb) and np.array_equal(va, vb)
    assert np.array_equal(a.series(1, 40)[1], b.series(1, 40)[1])


def test_flux_rule_is_refused_where_the_count_must_stay_fixed():
    run = od.Run(dict(W.tiny(), flags=od.F_FLUX_INJECT))
    with pytest.raises(od.OdError):
        od.od_set_cutoff(run.h, 3e-4, 1e-4)
    run.close()
    with pytest.raises(od.OdError):
        od.Batch([dict(W.tiny(), flags=od.F_FLUX_INJECT)])
