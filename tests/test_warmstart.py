"""Warm-start pipeline: host-side pieces on CPU (features, targets, convergence
criterion), and a small end-to-end run on the GPU showing what the trained network
gains over starting the consistent charge iteration from zero and from the OML charge
(the usual starting point)."""
import math

import numpy as np
import pytest

from paper_2205_06557_gb300 import build


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def test_features_and_targets_are_consistent():
    from paper_2205_06557_gb300 import warmstart as ws

    p = ws.study_run(3, 1000)
    x, m = ws.features(p)
    D = len(p["dust"])
    assert 1 <= D <= 4 and m.sum() == D and np.all(m[D:] == 0)
    assert np.all(np.abs(x[:D, 3:6]) <= 1.0) and np.all(np.abs(x[:D, 6]) <= 1.0)
    # q0 is the OML charge, so its potential offset target is zero
    q = np.array([g["q0"] for g in p["dust"]])
    t = ws.targets(p, q, np.zeros((D, 3)))
    assert np.allclose(t[:D, 0], 0.0, atol=1e-6)
    # the network's charge map inverts the target map
    assert all(g["q0"] < 0 for g in p["dust"])


def test_chain_runs_are_valid_inputs():
    """held-out dust-chain runs: 2-8 grains on the axis, inside the domain, not overlapping,
    features in the ranges the network was trained on"""
    from paper_2205_06557_gb300 import warmstart as ws

    for seed in range(6):
        p = ws.chain_run(seed, 1000)
        D = len(p["dust"])
        assert 2 <= D <= 8
        zs = np.array([g["z"] for g in p["dust"]])
        a = np.array([g["a"] for g in p["dust"]])
        assert np.all(np.diff(zs) > a[1:] + a[:-1])
        assert np.all(np.abs(zs) + a < 0.5 * p["H"])
        x, m = ws.features(p)
        assert m.sum() == D and np.all(np.abs(x[:D, 3:6]) <= 1.0)
        assert all(g["q0"] < 0 for g in p["dust"])


def test_steps_to_converge():
    from paper_2205_06557_gb300.warmstart import steps_to_converge

    t = np.arange(1000)
    q = -1e5 * (1 - np.exp(-t / 100.0))
    # |q - q_ref| <= 1% |q_ref| from exp(-t/100) <= 0.01, i.e. t >= 461
    assert steps_to_converge(q, -1e5, 0.01) == math.ceil(100 * math.log(100))
    assert steps_to_converge(np.full(10, -1e5), -1e5, 0.01) == 0


def test_force_convergence_criterion():
    from paper_2205_06557_gb300.warmstart import batch_se, steps_to_force

    rng = np.random.default_rng(1)
    # white noise: batch-means SE equals sigma / sqrt(n)
    x = rng.normal(0.0, 2.0, 200_000)
    assert abs(batch_se(x) / (2.0 / np.sqrt(len(x))) - 1) < 0.4
    # a relaxing mean plus noise: the first window that agrees starts after the transient
    t = np.arange(40_000)
    f = 5.0 + 3.0 * np.exp(-t / 2000.0) + rng.normal(0.0, 1.0, len(t))
    n = steps_to_force(f, 5.0, 0.0, 10_000)
    assert 10_000 < n < 30_000
    # a series that never reaches the reference
    assert steps_to_force(f + 1.0, 5.0, 0.0, 10_000) == len(f) + 1


@pytest.mark.gpu
def test_warm_start_pipeline_beats_zero_and_oml_starts():
    from paper_2205_06557_gb300 import warmstart as ws

    # a dense plasma (charging time ~2,400 steps) in a small domain (~6,000 ions) keeps
    # the label and evaluation runs short enough to converge in a test
    dom = dict(n_inf=1e15, R=1e-4, H=2e-4)
    plist, X, M, T = ws.generate(96, 10000, seed0=0, batch_runs=96, **dom)
    assert X.shape == (96, 8, 7) and np.isfinite(T).all()
    net, norm, losses, vlosses = ws.train(X, M, T, iters=800, batch=32)
    assert losses[-30:].mean() < losses[:30].mean()
    evalp = [ws.study_run(10_000 + s, 8000, **dom) for s in range(8)]
    steps, err0 = ws.evaluate(net, norm, evalp, 8000, tol=0.02)
    print("WARMSTART median initial charge error zero %.3f oml %.3f net %.3f; median steps to 2%% zero %d oml %d "
          "net %d" % (np.median(err0["zero"]), np.median(err0["oml"]), np.median(err0["net"]),
                      np.median(steps["zero"]), np.median(steps["oml"]), np.median(steps["net"])))
    # starting from zero charge is far from converged; the network starts closer than the
    # OML charge and reaches the converged charge in fewer steps (median over the grains)
    assert np.median(err0["net"]) < 0.2 * np.median(err0["zero"])
    assert steps["net"].mean() < steps["zero"].mean()
    assert np.median(err0["net"]) < np.median(err0["oml"])
    assert np.median(steps["net"]) < np.median(steps["oml"])
    net.close()
