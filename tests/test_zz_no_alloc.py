"""The pair-force entry point that allocates no device memory (od_pair_accel_static).

It exists for callers that cannot allocate on the device: host applications whose
framework owns every device allocation, and loops in which an allocation's implicit
device synchronisation is not acceptable.  Its scratch is a fixed array inside the
library, shared by all calls.

The test calls it through the C ABI twice in a row, the second time on fewer ions so
that the first call's scratch is still in the shared array.  Each result is checked,
ion by ion to 1e-5 of its pair-term sum, against

* the accelerations that the run-based entry points (od_set_ions, then od_get_ions)
  produce for the same ions with no grains, no cavity field and no driving field, and
* the FP64 oracle's pair accelerations of the same positions;

and the device's free memory is the same before and after the second call.  This file
is collected last so that a failure here comes after every other test has run.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2205_06557_gb300 as od
from paper_2205_06557_gb300 import workloads as W

pytestmark = pytest.mark.gpu

EPS0 = 8.8541878128e-12


def _params(n):
    return dict(W.tiny(), n_ions=n, dust=[], mach=0.0, nu=0.0, charge_model="given")


def _run_reference(x, ids):
    """pair accelerations from the run-based entry points, and (lambda_De, k)"""
    n = len(x)
    run = od.Run(dict(_params(n), flags=od.F_NO_EOUT))
    run.set_ions(x, np.zeros_like(x), ids, next_id=n)
    _, _, a_ref, _ = run.get_ions()
    info = run.info()
    run.close()
    return a_ref, info["lam"], info["q"] ** 2 / (4 * math.pi * EPS0 * info["m"])


def _oracle_reference(x, ids):
    """the FP64 oracle's accelerations of the same ions (pair forces only)"""
    o = oracle.Oracle(dict(_params(len(x)), oracle_flags=oracle.F_NO_EOUT))
    o.set_ions(x, np.zeros_like(x), ids)
    acc, _ = o.forces()
    o.close()
    return acc


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


def test_static_pair_accel_matches_run_forces_and_oracle_twice():
    torch = pytest.importorskip("torch")
    from paper_2205_06557_gb300 import build

    build.build()
    for call, (n, seed) in enumerate(((3000, 7), (1100, 8))):
        p = _params(n)
        x, _, ids = W.random_ions(n, p["R"], p["H"], seed=seed)
        a_run, lam, k = _run_reference(x, ids)
        a_orc = _oracle_reference(x, ids)
        xd = torch.tensor(x, dtype=torch.float64, device="cuda")
        ad = torch.full((n, 3), float("nan"), dtype=torch.float32, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        od.od_pair_accel_static(xd.data_ptr(), n, lam, k, ad.data_ptr(), stream)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        if call == 1:  # a warm call (the first may load the library's device code)
            assert free1 == free0, (free0, free1)
        a = ad.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(a))
        ts = _term_sums(x, lam, k)
        for ref in (a_run, a_orc):
            assert np.linalg.norm(a - ref) <= 1e-5 * np.linalg.norm(ref)
            err = np.linalg.norm(a - ref, axis=1) / (ts + np.linalg.norm(ref, axis=1))
            assert err.max() < 1e-5, (n, err.max())


def test_static_pair_accel_rejects_too_many_ions():
    from paper_2205_06557_gb300 import build

    build.build()
    with pytest.raises(od.OdError) as ei:
        od.od_pair_accel_static(0, od.STATIC_MAX_IONS + 1, 1e-3, 1.0, 0)
    assert ei.value.code == -1
    assert "n must be" in od.od_last_error()
