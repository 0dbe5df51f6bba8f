"""GPU-vs-oracle parity of the CUDA library, called through its C ABI.

* forces on identical injected states (ragged sizes that span several tiles, 0-8
  grains): per-ion error relative to sum_j |a_ij| + |a_i| within 1e-5, grain force
  (Eq. 1) relative to its own term sum within 1e-5;
* 50 coupled steps of the ~2,000-ion workload: every integer event (absorbed per
  grain, outflow, injected per face, collided) bit-exact per step, ion ids identical,
  positions within 1e-10 m, per-step grain records within tolerance;
* 25 coupled steps of ~19,700 ions with the ordered, symmetric and packed symmetric
  pair kernels: every integer event and every position as the oracle's;
* 200 steps: window means of charge and force within 2 combined standard errors;
* the ~200,000-ion workload in the benchmark's launch configuration: sampled target
  ions and the grain force against the oracle;
* failure paths: a non-finite ion state reports OD_ENAN, too many ions OD_EOVERFLOW.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2205_06557_gb300 as od
from paper_2205_06557_gb300 import workloads as W

pytestmark = pytest.mark.gpu

QE = 1.602176634e-19
EPS0 = 8.8541878128e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2205_06557_gb300 import build

    build.build()
    od.lib()


def _alpha(p):
    return oracle.Oracle(dict(p, n_ions=1)).alpha()


def _pair_scale(x, lam, kii):
    """sum_j |a_ij| for every i (the scale of the cancellation-aware per-ion error)"""
    n = len(x)
    out = np.zeros(n)
    for i0 in range(0, n, 512):
        d = x[i0: i0 + 512, None, :] - x[None, :, :]
        r = np.sqrt((d * d).sum(-1))
        with np.errstate(divide="ignore", invalid="ignore"):
            f = kii * (1 + r / lam) * np.exp(-r / lam) / (r * r)
        f[~np.isfinite(f)] = 0.0
        out[i0: i0 + 512] = f.sum(1)
    return out


def _grain_scale(x, dust, q, lam, Qs):
    out = []
    for g, Q in zip(dust, Qs):
        d = x - np.array([g["x"], g["y"], g["z"]])
        r = np.sqrt((d * d).sum(1))
        out.append(abs(q * Q) / (4 * math.pi * EPS0) * ((1 + r / lam) * np.exp(-r / lam) / (r * r)).sum())
    return np.array(out)


GRAINS = [(0.0, 0.0, -6e-5, 1.0e-5, -1500.0), (4e-5, 0.0, 7e-5, 1.2e-5, 800.0), (-5e-5, 3e-5, 0.0, 0.8e-5, -300.0),
          (0.0, -6e-5, 1.2e-4, 0.6e-5, -900.0), (6e-5, 6e-5, -1.2e-4, 0.5e-5, -200.0),
          (-8e-5, -4e-5, 1.4e-4, 0.7e-5, -1200.0), (2e-5, 1e-4, -1.5e-4, 0.9e-5, 400.0),
          (-1e-4, 1e-5, -0.5e-4, 0.6e-5, -700.0)]


def _force_case(n, n_dust, flags=0, variant=None):
    p = W.tiny()
    p.update(n_ions=max(n, 1), charge_model="given")
    p["dust"] = [dict(x=g[0], y=g[1], z=g[2], a=g[3], q0=g[4] * QE) for g in GRAINS[:n_dust]]
    p["alpha"] = _alpha(p)
    p["flags"] = flags
    o = oracle.Oracle(dict(p, oracle_flags=flags))
    x, v, ids = W.random_ions(n, p["R"], p["H"], seed=100 + n, dust=p["dust"])
    o.set_ions(x, v, ids)
    acc_ref, fo_ref = o.forces()
    run = od.Run(p)
    if variant is not None:
        od.od_set_force_config(run.h, variant, 8, 0)
    run.set_ions(x, v, ids, next_id=n)
    _, _, a_gpu, id_gpu = run.get_ions()
    _, fo_gpu = run.dust_now()
    d = o.derived()
    return p, d, x, acc_ref, fo_ref, a_gpu, fo_gpu, id_gpu, ids


def _check_forces(p, d, x, acc_ref, fo_ref, a_gpu, fo_gpu):
    kii = d["q"] ** 2 / (4 * math.pi * EPS0 * d["m"])
    scale = _pair_scale(x, d["lam"], kii) + np.linalg.norm(acc_ref, axis=1)
    dev = np.linalg.norm(a_gpu - acc_ref, axis=1)
    # the force array to 1e-5 (normwise) and every ion to 1e-5 of its term sum (the
    # close-pair correction removes the FP32 rounding of close pairs' positions)
    assert np.linalg.norm(a_gpu - acc_ref) <= 1e-5 * np.linalg.norm(acc_ref)
    err = dev / scale
    assert err.max() < 1e-5, (err.max(), int(err.argmax()))
    if len(p["dust"]):
        gs = _grain_scale(x, p["dust"], d["q"], d["lam"], [g["q0"] for g in p["dust"]])
        gs = gs + np.linalg.norm(fo_ref, axis=1)
        gerr = np.linalg.norm(fo_gpu - fo_ref, axis=1) / gs
        assert gerr.max() < 1e-5, gerr


@pytest.mark.parametrize("n,n_dust", [(1, 1), (2, 2), (33, 2), (255, 1), (256, 0), (257, 3), (2011, 1), (5000, 8)])
def test_forces_on_injected_states(n, n_dust):
    p, d, x, acc_ref, fo_ref, a_gpu, fo_gpu, id_gpu, ids = _force_case(n, n_dust)
    assert np.array_equal(id_gpu, ids)
    _check_forces(p, d, x, acc_ref, fo_ref, a_gpu, fo_gpu)


@pytest.mark.parametrize("variant", range(len(od.FORCE_VARIANTS)))
@pytest.mark.parametrize("n", [1, 300, 2500, 4099])
def test_every_pair_kernel_variant(variant, n):
    """every variant, ordered-pair and symmetric, on one tile, several tiles and ragged
    tails (the symmetric tiles hold 256-1024 ions); a second evaluation of the same state
    gives the same bits (fixed summation order)"""
    p, d, x, acc_ref, fo_ref, a_gpu, fo_gpu, id_gpu, ids = _force_case(n, 2, variant=variant)
    _check_forces(p, d, x, acc_ref, fo_ref, a_gpu, fo_gpu)
    _, _, _, _, _, a2, fo2, _, _ = _force_case(n, 2, variant=variant)
    assert np.array_equal(a2, a_gpu) and np.array_equal(fo2, fo_gpu)


def test_forces_without_ion_ion_term():
    p, d, x, acc_ref, fo_ref, a_gpu, fo_gpu, _, _ = _force_case(700, 2, flags=od.F_NO_IONION)
    err = np.linalg.norm(a_gpu - acc_ref, axis=1) / np.linalg.norm(acc_ref, axis=1)
    assert err.max() < 1e-6


# App. A polynomial P(r, z) = sum_t alpha_t r^(2 A_t) z^(2 B_t) in the paper's term order
_POW_R = (0, 1, 0, 1, 2, 0, 2, 1, 3, 0, 2, 3, 1, 4, 0)
_POW_Z = (0, 0, 1, 1, 0, 2, 1, 2, 0, 3, 2, 1, 3, 0, 4)


def _field_of(alpha, x, y, z):
    """E = -grad P of the fitted polynomial at (x, y, z)"""
    r2, z2 = x * x + y * y, z * z
    g = sum(a * 2 * A * r2 ** (A - 1) * z2 ** B for a, A, B in zip(alpha, _POW_R, _POW_Z) if A > 0)
    k = sum(a * 2 * B * r2 ** A * z2 ** (B - 1) for a, A, B in zip(alpha, _POW_R, _POW_Z) if B > 0)
    return np.array([-x * g, -y * g, -z * k])


@pytest.mark.parametrize("shape", ["tiny", "chain"])
def test_library_eout_fit_matches_oracle(shape):
    """the library's App. A quadrature (slices of the cylinder, in-plane radial integral in
    closed form) and least-squares fit against the oracle's (spherical rays about each
    node, QR): the field of the two fits within 1e-6 of the field's scale"""
    p = W.tiny() if shape == "tiny" else W.dust_chain(n_dust=2)
    run = od.Run(dict(p, n_ions=1))
    o = oracle.Oracle(dict(p, n_ions=1))
    al_gpu = run.info()["alpha"]
    E_ref, E_gpu = [], []
    for r, z in [(0.0, 0.0), (0.2, 0.1), (0.5, -0.6), (0.9, 0.95), (0.99, -0.3), (1.0, 1.0)]:
        pt = (r * p["R"], 0.0, z * 0.5 * p["H"])
        E_ref.append(o.eout(*pt))
        E_gpu.append(_field_of(al_gpu, *pt))
    E_ref, E_gpu = np.array(E_ref), np.array(E_gpu)
    assert np.abs(E_gpu - E_ref).max() < 1e-6 * np.abs(E_ref).max()
    # the polynomial restated here is the oracle's field for the oracle's own coefficients
    assert np.allclose([_field_of(o.alpha(), r * p["R"], 0.0, z * 0.5 * p["H"]) for r, z in [(0.5, 0.5), (0.9, -0.2)]],
                       [o.eout(r * p["R"], 0.0, z * 0.5 * p["H"]) for r, z in [(0.5, 0.5), (0.9, -0.2)]],
                       rtol=1e-12, atol=0)


def _coupled(p, steps):
    o = oracle.Oracle(p)
    run = od.Run(p)
    xo, vo, ao, ido = o.get_ions()
    xg, vg, ag, idg = run.get_ions()
    assert np.array_equal(ido, idg)
    assert np.abs(xo - xg).max() < 1e-18 + 1e-14 * p["R"]
    assert np.abs(vo - vg).max() < 1e-9
    return o, run


def test_tiny_50_steps_events_bit_exact():
    p = W.tiny()
    p["alpha"] = _alpha(p)
    o, run = _coupled(p, 50)
    o.step(50)
    for _ in range(50):
        run.step(1)
    rec_o, ev_o = o.records(1, 50)
    rec_g, ev_g = run.series(1, 50)
    bad = np.nonzero((ev_o != ev_g).any(1))[0]
    assert len(bad) == 0, "first mismatched step %d: oracle %s gpu %s" % (
        bad[0] + 1, ev_o[bad[0]].tolist(), ev_g[bad[0]].tolist())
    assert ev_o[:, 8].sum() > 100 and ev_o[:, 12].sum() > 10  # the run exercised outflow and collisions
    xo, vo, _, ido = o.get_ions()
    xg, vg, _, idg = run.get_ions()
    assert np.array_equal(ido, idg)
    assert np.abs(xo - xg).max() < 1e-10
    assert np.abs(vo - vg).max() < 1e-3
    # grain records: charge and the force terms
    assert np.allclose(rec_g[:, :, 0], rec_o[:, :, 0], rtol=1e-9, atol=0)
    fo_scale = np.abs(rec_o[:, :, 1:4]).max()
    assert np.abs(rec_g[:, :, 1:4] - rec_o[:, :, 1:4]).max() < 1e-4 * fo_scale
    # collected momentum (Eq. 3) and driving-field force (Eq. 4), per step as vectors
    for j0 in (7, 10):
        dv = np.linalg.norm(rec_g[:, :, j0:j0 + 3] - rec_o[:, :, j0:j0 + 3], axis=-1)
        assert np.all(dv <= 1e-5 * np.linalg.norm(rec_o[:, :, j0:j0 + 3], axis=-1) + 1e-30)
    c = run.counters()
    assert c[13] == 50 and c[14] == o.n_ions


_BIG = {}


def _big_oracle_run(steps):
    """~19,700 ions (the ~2,000-ion plasma in a domain 2.14x larger per axis): one oracle
    run shared by the kernel variants below"""
    if "o" not in _BIG:
        p = W.tiny()
        p.update(R=p["R"] * 2.14, H=p["H"] * 2.14, n_ions=0)
        p["alpha"] = _alpha(p)
        o = oracle.Oracle(p)
        o.step(steps)
        _BIG.update(p=p, o=o)
    return _BIG["p"], _BIG["o"]


@pytest.mark.parametrize("variant", [None, 9, 15])  # default (ordered), sym<128,4>, sym2<256,4>
def test_coupled_steps_at_20k_ions_every_kernel(variant):
    steps = 25
    p, o = _big_oracle_run(steps)
    run = od.Run(p)
    if variant is not None:
        od.od_set_force_config(run.h, variant, 8, 0)
    for _ in range(steps):
        run.step(1)
    _, ev_o = o.records(1, steps)
    _, ev_g = run.series(1, steps)
    bad = np.nonzero((ev_o != ev_g).any(1))[0]
    assert len(bad) == 0, "first mismatched step %d" % (bad[0] + 1)
    assert ev_o[:, 8].sum() > 100
    xo, _, _, ido = o.get_ions()
    xg, _, _, idg = run.get_ions()
    assert np.array_equal(ido, idg) and np.abs(xo - xg).max() < 1e-10
    run.close()


def test_tiny_200_steps_long_run_means():
    p = W.tiny(steps=200)
    p["alpha"] = _alpha(p)
    o = oracle.Oracle(p)
    run = od.Run(p)
    o.step(200)
    run.step(200)
    mo, so = o.dust_terms()
    mg, sg = run.dust_terms()
    for j in (0, 1, 2, 3, 7, 8, 9):
        se = math.sqrt(so[0, j] ** 2 + sg[0, j] ** 2)
        assert abs(mo[0, j] - mg[0, j]) <= 2 * se + 1e-9 * abs(mo[0, j]), (j, mo[0, j], mg[0, j], se)
    q, F = run.dust_state()
    assert np.isclose(q[0], mg[0, 0]) and np.allclose(F[0], mg[0, 1:4] + mg[0, 4:7] + mg[0, 7:10] + mg[0, 10:13])


@pytest.mark.parametrize("config", ["tuned", "symmetric"])
def test_at_scale_sampled_forces(config):
    """the ~200,000-ion workload with the autotuner's choice (the benchmark's launch
    configuration, same cache) and with the largest-tile symmetric kernel"""
    p = W.at_scale()
    p["alpha"] = _alpha(p)  # both sides use the oracle's cavity-field fit
    run = od.Run(p)
    if config == "tuned":
        import torch

        od.tune_cached(run.h, "%s|N=%d" % (torch.cuda.get_device_name(0), run.N))
    else:
        od.od_set_force_config(run.h, od.FORCE_VARIANTS.index((256, 4, 1)), 8, 0)
    run.step(3)
    x, v, a, ids = run.get_ions()
    rec, _ = run.series(2, 1)
    Q_used = rec[0, :, 0]  # charges the ions felt in step 3
    po = dict(p, n_ions=1)
    po["dust"] = [dict(g, q0=float(Q)) for g, Q in zip(p["dust"], Q_used)]
    o = oracle.Oracle(po)
    o.load_ions(x, v, ids)
    N = len(x)
    d = o.derived()
    kii = d["q"] ** 2 / (4 * math.pi * EPS0 * d["m"])
    a_s, ref_s = [], []
    for i0 in (0, N // 2, N - 24):
        acc_ref, fo_ref = o.forces(i0, i0 + 24)
        scale = np.linalg.norm(acc_ref, axis=1)
        for k, i in enumerate(range(i0, i0 + 24)):
            dd = x[i] - x
            r = np.sqrt((dd * dd).sum(1))
            r[i] = 1.0
            f = kii * (1 + r / d["lam"]) * np.exp(-r / d["lam"]) / (r * r)
            f[i] = 0.0
            scale[k] += f.sum()
        err = np.linalg.norm(a[i0: i0 + 24] - acc_ref, axis=1) / scale
        assert err.max() < 1e-5, err.max()
        a_s.append(a[i0: i0 + 24])
        ref_s.append(acc_ref)
    # the sampled force array normwise
    a_s, ref_s = np.concatenate(a_s), np.concatenate(ref_s)
    assert np.linalg.norm(a_s - ref_s) <= 1e-5 * np.linalg.norm(ref_s)
    _, fo_gpu = run.dust_now()
    gs = _grain_scale(x, po["dust"], d["q"], d["lam"], Q_used) + np.linalg.norm(fo_ref, axis=1)
    assert (np.linalg.norm(fo_gpu - fo_ref, axis=1) / gs).max() < 1e-5


def test_nan_state_reports_enan():
    p = W.tiny()
    run = od.Run(p)
    x, v, a, ids = run.get_ions()
    x[5, 0] = np.nan
    run.set_ions(x, v, ids, next_id=run.N)
    with pytest.raises(od.OdError) as ei:
        run.step(1)
    assert ei.value.code == -4
    run.close()


def test_too_many_ions_reports_overflow():
    p = W.tiny()
    run = od.Run(p)
    x, v, ids = W.random_ions(run.N + 1, p["R"], p["H"], seed=1)
    with pytest.raises(od.OdError) as ei:
        run.set_ions(x, v, ids, next_id=run.N + 1)
    assert ei.value.code == -5
    run.close()


def test_restart_round_trip_is_exact():
    p = W.tiny()
    a_run = od.Run(p)
    a_run.step(10)
    x, v, acc, ids = a_run.get_ions()
    nid = int(a_run.counters()[15])
    a_run.step(10)
    b_run = od.Run(p)
    b_run.step(10)
    b_run.set_ions(x, v, ids, next_id=nid, a=acc)
    b_run.step(10)
    xa, va, _, ia = a_run.get_ions()
    xb, vb, _, ib = b_run.get_ions()
    assert np.array_equal(ia, ib) and np.array_equal(xa, xb) and np.array_equal(va, vb)


def test_bounded_wait_reports_timeout_and_gpu_stays_usable():
    """the scan's look-back wait on a prefix nobody publishes gives up with OD_ETIMEOUT"""
    bad = od.Run(W.tiny())
    assert od.od_selftest_wait_timeout(bad.h, 2000) == -6
    assert "wait" in od.od_last_error(bad.h)
    bad.close()
    good = od.Run(W.tiny(steps=10))
    good.step(10)
    assert good.counters()[13] == 10


def test_tuned_configuration_keeps_results():
    p = W.tiny()
    ref = od.Run(p)
    tuned = od.Run(p)
    ms, v, g, b = od.od_tune(tuned.h, reps=1)
    # the choice comes from a final round among the three fastest settings of the sweep
    assert ms[v, [4, 8, 16, 32].index(g), [0, 4, 2].index(b)] <= np.sort(ms[ms > 0])[:3].max()
    assert od.od_get_force_config(tuned.h)[:3] == (v, g, b)
    ref.step(20)
    tuned.step(20)
    _, ev_r = ref.series(1, 20)
    _, ev_t = tuned.series(1, 20)
    assert np.array_equal(ev_r, ev_t)
    xr, _, _, ir = ref.get_ions()
    xt, _, _, it = tuned.get_ions()
    assert np.array_equal(ir, it) and np.abs(xr - xt).max() < 1e-12


@pytest.mark.parametrize("variant", [16, 17])  # sym2<128,8>, sym2<64,8>
def test_unit_queue_results_do_not_depend_on_the_grid(variant):
    """The packed kernel takes its tile pairs from a queue, so the CTA that evaluates a unit
    varies from launch to launch; each unit writes fixed slots, so every grid size gives the
    same bits, and the queue is reset after each launch (repeated evaluations agree)."""
    p = W.at_scale(steps=100)
    p.update(n_ions=40000)
    run = od.Run(p)
    x, v, _, ids = run.get_ions()
    accs = []
    for bps in (0, 1, 2, 0):
        od.od_set_force_config(run.h, variant, 8, bps)
        for _ in range(2):
            run.set_ions(x, v, ids, next_id=len(ids))
            accs.append(run.get_ions()[2])
    for a in accs[1:]:
        assert np.array_equal(a, accs[0])
    run.step(3)
    assert run.counters()[13] == 3
    run.close()
