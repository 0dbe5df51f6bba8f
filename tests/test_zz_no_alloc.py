"""The pair-force entry point that allocates no device memory (od_pair_accel_static).

It exists for callers that cannot allocate on the device: work recorded into a
CUDA graph, loops that must not risk an allocation's implicit device
synchronisation, and hosts whose framework owns every device allocation.  Its
scratch is a fixed array inside the library, shared by all calls.

The test calls it through the C ABI twice in a row, the second time on fewer ions
so that the first call's scratch is still in the shared array.  Each result is
checked against the accelerations that the run-based entry points (od_set_ions,
then od_get_ions) produce for the same ions with no grains, no cavity field and no
driving field, to the tolerance of the other force tests.  This file is collected
last so that a failure here comes after every other test has run.
"""
import math

import numpy as np
import pytest

import paper_2205_06557_gb300 as od
from paper_2205_06557_gb300 import workloads as W

pytestmark = pytest.mark.gpu

EPS0 = 8.8541878128e-12


def _reference(n, seed):
    p = dict(W.tiny(), n_ions=n, dust=[], mach=0.0, nu=0.0, charge_model="given", flags=od.F_NO_EOUT)
    run = od.Run(p)
    x, v, ids = W.random_ions(n, p["R"], p["H"], seed=seed)
    run.set_ions(x, v, ids, next_id=n)
    _, _, a_ref, _ = run.get_ions()
    info = run.info()
    run.close()
    k = info["q"] ** 2 / (4 * math.pi * EPS0 * info["m"])
    return x, a_ref, info["lam"], k


def _term_sums(x, lam, k):
    out = np.zeros(len(x))
    for i0 in range(0, len(x), 512):
        d = x[i0: i0 + 512, None, :] - x[None, :, :]
        r = np.sqrt((d * d).sum(-1))
        with np.errstate(divide="ignore", invalid="ignore"):
            f = k * (1 + r / lam) * np.exp(-r / lam) / (r * r)
        f[~np.isfinite(f)] = 0.0
        out[i0: i0 + 512] = f.sum(1)
    return out


def test_static_pair_accel_matches_run_forces_twice():
    torch = pytest.importorskip("torch")
    from paper_2205_06557_gb300 import build

    build.build()
    for n, seed in ((3000, 7), (1100, 8)):
        x, a_ref, lam, k = _reference(n, seed)
        xd = torch.tensor(x, dtype=torch.float64, device="cuda")
        ad = torch.full((n, 3), float("nan"), dtype=torch.float32, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        od.od_pair_accel_static(xd.data_ptr(), n, lam, k, ad.data_ptr(), stream)
        torch.cuda.synchronize()
        a = ad.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(a))
        assert np.linalg.norm(a - a_ref) <= 1e-5 * np.linalg.norm(a_ref)
        err = np.linalg.norm(a - a_ref, axis=1) / _term_sums(x, lam, k)
        assert err.max() < 1e-5, (n, err.max())


def test_static_pair_accel_rejects_too_many_ions():
    from paper_2205_06557_gb300 import build

    build.build()
    with pytest.raises(od.OdError) as ei:
        od.od_pair_accel_static(0, od.STATIC_MAX_IONS + 1, 1e-3, 1.0, 0)
    assert ei.value.code == -1
    assert "n must be" in od.od_last_error()
