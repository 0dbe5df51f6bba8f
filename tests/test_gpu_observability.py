"""Observability and restart through the C ABI: checkpoints continue bit for bit, the
density map equals a host binning of the same positions, ion dumps hold the exact state."""
import math

import numpy as np
import pytest

import paper_2205_06557_gb300 as od
from paper_2205_06557_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2205_06557_gb300 import build

    build.build()
    od.lib()


def _medium():
    """~40,000 ions: above the size where the untuned run uses the symmetric kernel"""
    p = W.tiny()
    p["R"] *= 2.72
    p["H"] *= 2.72
    p["n_ions"] = 0
    return p


@pytest.mark.parametrize("make", [W.tiny, _medium])
def test_checkpoint_continues_bit_for_bit(make, tmp_path):
    p = make()
    p["avg_start"] = 5
    a = od.Run(p)
    a.step(12)
    path = str(tmp_path / "run.ckpt")
    a.save(path)
    a.step(13)
    b = od.Run.load(path)
    assert b.D == a.D and b.N == a.N
    assert od.od_get_force_config(b.h)[:3] == od.od_get_force_config(a.h)[:3]
    b.step(13)
    ra, ea = a.series(1, 25)
    rb, eb = b.series(1, 25)
    assert np.array_equal(ea, eb) and np.array_equal(ra, rb)
    xa, va, aa, ia = a.get_ions()
    xb, vb, ab, ib = b.get_ions()
    assert np.array_equal(ia, ib) and np.array_equal(xa, xb) and np.array_equal(va, vb) and np.array_equal(aa, ab)
    for fa, fb in zip(a.dust_state() + a.dust_terms(), b.dust_state() + b.dust_terms()):
        assert np.array_equal(fa, fb)
    assert np.array_equal(a.counters(), b.counters())
    a.close()
    b.close()


def _bin(x, R, H, nr, nz):
    """host binning with the library's stated FP64 formula (numpy does not contract)"""
    r = np.sqrt(x[:, 0] * x[:, 0] + x[:, 1] * x[:, 1])
    ir = np.clip(np.floor(r * (nr / R)).astype(np.int64), 0, nr - 1)
    iz = np.clip(np.floor((x[:, 2] + 0.5 * H) * (nz / H)).astype(np.int64), 0, nz - 1)
    out = np.zeros((nz, nr), dtype=np.uint64)
    np.add.at(out, (iz, ir), 1)
    return out


@pytest.mark.parametrize("nr,nz", [(16, 32), (128, 128)])  # shared-memory and global-atomic paths
def test_density_map_equals_host_binning(nr, nz):
    p = W.tiny()
    run = od.Run(p)
    run.step(3)
    od.od_density_enable(run.h, nr, nz)
    ref = np.zeros((nz, nr), dtype=np.uint64)
    for _ in range(15):
        run.step(1)
        ref += _bin(run.get_ions()[0], p["R"], p["H"], nr, nz)
    counts, dens, n = od.od_density_read(run.h, nr, nz)
    assert n == 15 and np.array_equal(counts, ref)
    assert int(counts.sum()) == 15 * run.N
    # density x annulus volume, summed, gives back the ion count per step
    r = np.linspace(0, p["R"], nr + 1)
    vol = math.pi * (r[1:] ** 2 - r[:-1] ** 2)[None, :] * (p["H"] / nz)
    assert np.isclose((dens * vol).sum(), run.N, rtol=1e-12)
    # mean density is the ion count over the cylinder volume
    assert np.isclose((dens * vol).sum() / (math.pi * p["R"] ** 2 * p["H"]), run.N / (math.pi * p["R"] ** 2 * p["H"]))
    od.od_density_enable(run.h, 0, 0)
    run.step(2)
    with pytest.raises(od.OdError):
        od.od_density_read(run.h, nr, nz)
    run.close()


def test_bad_density_map_sizes_are_rejected():
    run = od.Run(W.tiny())
    for nr, nz in [(-1, 4), (5000, 4), (4096, 4096), (0, 3)]:
        with pytest.raises(od.OdError) as ei:
            od.od_density_enable(run.h, nr, nz)
        assert ei.value.code == -1
    run.close()


def test_ion_dumps_hold_the_exact_state(tmp_path):
    run = od.Run(W.tiny())
    run.step(4)
    x, v, _, ids = run.get_ions()
    xyz = str(tmp_path / "ions.xyz")
    csv = str(tmp_path / "ions.csv")
    run.write_ions(xyz, od.DUMP_XYZ)
    run.write_ions(csv, od.DUMP_CSV)
    lines = open(xyz).read().splitlines()
    assert int(lines[0]) == run.N and "step=4" in lines[1]
    body = np.array([ln.split()[1:] for ln in lines[2:]], dtype=np.float64)
    assert np.array_equal(body[:, :3], x) and np.array_equal(body[:, 3:6], v)
    assert np.array_equal(np.array([ln.split()[7] for ln in lines[2:]], dtype=np.uint64), ids)
    c = np.loadtxt(csv, delimiter=",", skiprows=1, dtype=np.float64)
    assert np.array_equal(c[:, 1:4], x) and np.array_equal(c[:, 4:7], v)
    assert np.array_equal(np.loadtxt(csv, delimiter=",", skiprows=1, usecols=0, dtype=np.uint64), ids)
    run.close()


def test_kernel_times_span_more_steps_than_the_event_ring():
    """per-kernel profiling records events for every step and reads them 64 steps at a
    time: a call of 70 steps and one of 5 count 75 launches of each stage, and the
    profiled (directly launched) steps give the same bits as graph-replayed ones (75 steps
    in one call: four 16-step graphs and eleven one-step graphs), state and records"""
    p = W.tiny(steps=200)
    prof, ref = od.Run(p), od.Run(p)
    od.od_set_profiling(prof.h, 1)
    prof.step(70)
    prof.step(5)
    ms, n = od.od_kernel_times(prof.h)
    assert n.tolist() == [75] * 4 and (ms > 0).all()
    od.od_set_profiling(prof.h, 0)
    ref.step(75)
    for a, b in zip(prof.get_ions(), ref.get_ions()):
        assert np.array_equal(a, b)
    for a, b in zip(prof.series(1, 75), ref.series(1, 75)):
        assert np.array_equal(a, b)
    prof.close()
    ref.close()


def test_step_graph_lengths_give_the_same_bits():
    """od_step replays 16-step graphs while 16 or more steps remain and one-step graphs for
    the rest: 40 steps as one call, as 16 + 1 + 23, and one at a time end in the same state
    and records"""
    p = W.tiny(steps=200)
    runs = [od.Run(p) for _ in range(3)]
    runs[0].step(40)
    for k in (16, 1, 23):
        runs[1].step(k)
    for _ in range(40):
        runs[2].step(1)
    ref_state, ref_series = runs[0].get_ions(), runs[0].series(1, 40)
    for r in runs[1:]:
        for a, b in zip(r.get_ions(), ref_state):
            assert np.array_equal(a, b)
        for a, b in zip(r.series(1, 40), ref_series):
            assert np.array_equal(a, b)
    for r in runs:
        r.close()
