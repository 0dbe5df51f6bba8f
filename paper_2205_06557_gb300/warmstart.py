"""Learned warm start of the self-consistent grain charge.

The network (od_sur_*, a set-pooled MLP) maps a run's (Mach number, collision
frequency, T_e/T_i) and each grain's position and radius to the grain's converged
charge and force.  Its only use is to pick the initial charges q0 of a run with the
"consistent" charging model (Sec. 2); the method then converges by itself and its own
long-run result judges the prediction.

* generate():  labels from batched runs of the method (one launch per step for all
  runs): each run starts from the grains' OML charges and its window means of charge
  and total force become the targets;
* train():     the library's forward/backward/Adam kernels on standardised targets;
* evaluate():  held-out runs started from q0 = 0, from the OML charge and from the
  network's prediction, stepped together; for each grain the number of steps until the
  charge stays within a tolerance of the converged value is reported.

Targets are dimensionless: the grain potential e Q / (4 pi eps0 a k T_e) minus its OML
value, and the total force over n_inf k T_e pi a^2.
"""
import math

import numpy as np

from . import Batch, Surrogate, od_oml_charge
from . import workloads as W

QE = 1.602176634e-19
KB = 1.380649e-23
EPS0 = 8.8541878128e-12
TE_TI_REF = 2.0 * W.EV_IN_K / 300.0


def study_run(seed, steps, n_inf=4e13, R=2e-4, H=4e-4):
    """A small-domain run of the sweep's physics: Mach U(0.3, 2), collision frequency
    from {1e5, 1e6, 5e6} /s, 1-4 grains of radius U(10, 20) um inside the inner half of
    the cylinder (by default R = 0.2 mm, H = 0.4 mm at 4e13 m^-3: ~2,000 ions),
    consistent charging from the OML charges.  The charging time scales as 1 / n_inf."""
    rng = np.random.default_rng(50_000 + seed)
    p = W.plasma_ar(mach=float(rng.uniform(0.3, 2.0)), nu=float(rng.choice([1e5, 1e6, 5e6])))
    p["n_inf"] = n_inf
    nd = int(rng.integers(1, 5))
    dust = []
    tries = 0
    while len(dust) < nd and tries < 1000:
        tries += 1
        a = float(rng.uniform(1e-5, 2e-5))
        r = 0.5 * R * math.sqrt(rng.uniform())
        ph = rng.uniform(0, 2 * math.pi)
        g = dict(x=r * math.cos(ph), y=r * math.sin(ph), z=float(rng.uniform(-0.25 * H, 0.25 * H)), a=a, q0=0.0)
        if math.hypot(g["x"], g["y"]) + a < R and abs(g["z"]) + a < 0.5 * H and all(
                (g["x"] - o["x"]) ** 2 + (g["y"] - o["y"]) ** 2 + (g["z"] - o["z"]) ** 2 > (1.5 * (a + o["a"])) ** 2
                for o in dust):
            dust.append(g)
    p.update(R=R, H=H, dt=5e-10, n_ions=0, seed=seed, charge_model="consistent", dust=dust,
             avg_start=steps // 2 + 1)
    for g in p["dust"]:
        g["q0"] = od_oml_charge(p, g["a"])
    return p


def chain_run(seed, steps, n_inf=1e15, R=1.5e-4, H=1.2e-3):
    """A dust-chain run (the shape of the paper's chain tests): 2-8 grains of radius
    U(10, 20) um on the axis of an elongated cylinder, centred, spaced U(1, 3) ion Debye
    lengths apart along the flow; Mach U(0.3, 2), collision frequency from {1e5, 1e6, 5e6}
    /s, consistent charging from the OML charges (by default ~85,000 ions at 1e15 m^-3)."""
    rng = np.random.default_rng(70_000 + seed)
    p = W.plasma_ar(mach=float(rng.uniform(0.3, 2.0)), nu=float(rng.choice([1e5, 1e6, 5e6])))
    p["n_inf"] = n_inf
    lam_di = math.sqrt(EPS0 * KB * p["T_i"] / (n_inf * QE * QE))
    nd = int(rng.integers(2, 9))
    radii = rng.uniform(1e-5, 2e-5, nd)
    gaps = np.maximum(rng.uniform(1.0, 3.0, nd - 1) * lam_di, 1.2 * (radii[1:] + radii[:-1]))
    zs = np.concatenate([[0.0], np.cumsum(gaps)])
    zs -= zs.mean()
    dust = [dict(x=0.0, y=0.0, z=float(z), a=float(a), q0=0.0) for z, a in zip(zs, radii)]
    p.update(R=R, H=H, dt=5e-10, n_ions=0, seed=seed, charge_model="consistent", dust=dust,
             avg_start=steps // 2 + 1)
    for g in p["dust"]:
        g["q0"] = od_oml_charge(p, g["a"])
    return p


def _psi_scale(p, a):
    return 4 * math.pi * EPS0 * a * KB * p["T_e"] / QE  # charge per unit dimensionless potential


def features(p):
    x = np.zeros((8, 7), dtype=np.float32)
    m = np.zeros(8, dtype=np.float32)
    glob = [p["mach"], math.log10(max(p["nu"], 1.0) / 1e6), math.log10(p["T_e"] / p["T_i"] / TE_TI_REF)]
    for k, g in enumerate(p["dust"]):
        x[k] = glob + [g["x"] / p["R"], g["y"] / p["R"], g["z"] / (0.5 * p["H"]), (g["a"] - 1.5e-5) / 5e-6]
        m[k] = 1.0
    return x, m


def targets(p, q, F):
    t = np.zeros((8, 4), dtype=np.float32)
    for k, g in enumerate(p["dust"]):
        a = g["a"]
        psi = q[k] / _psi_scale(p, a)
        psi_oml = od_oml_charge(p, a) / _psi_scale(p, a)
        f0 = p["n_inf"] * KB * p["T_e"] * math.pi * a * a
        t[k] = [psi - psi_oml, F[k][2] / f0, F[k][0] / f0, F[k][1] / f0]
    return t


def generate(n_runs, steps, seed0=0, batch_runs=256, stream=None, **domain):
    """(params, x[n, 8, 7], mask[n, 8], targets[n, 8, 4]) from runs of the method; the
    window means cover the second half of each run"""
    plist, X, M, T = [], [], [], []
    for c0 in range(0, n_runs, batch_runs):
        ps = [study_run(seed0 + s, steps, **domain) for s in range(c0, min(n_runs, c0 + batch_runs))]
        b = Batch(ps, stream=stream)
        b.tune(reps=1)  # the batch's pair plan (ordered chunks or symmetric tile pairs)
        b.step(steps)
        for p, run in zip(ps, b.runs):
            mean, _ = run.dust_terms()
            q = mean[:, 0]
            F = mean[:, 1:4] + mean[:, 4:7] + mean[:, 7:10] + mean[:, 10:13]
            x, m = features(p)
            X.append(x)
            M.append(m)
            T.append(targets(p, q, F))
        b.close()
        plist.extend(ps)
    return plist, np.array(X), np.array(M), np.array(T)


def train(X, M, T, iters=3000, batch=128, lr=1e-3, seed=0, stream=None, val_fraction=0.15):
    """Adam with a decaying rate on standardised targets; a held-out fraction of the runs
    picks the iteration with the lowest validation loss (the parameters returned).
    Returns (network, (mean, std) of the targets, training losses, validation losses)."""
    present = M > 0
    mu = T[present].mean(0)
    sd = T[present].std(0) + 1e-6
    Tn = ((T - mu) / sd) * present[..., None]
    rng = np.random.default_rng(seed)
    perm = rng.permutation(len(X))
    n_val = int(round(val_fraction * len(X))) if len(X) >= 10 else 0
    val, tr = perm[:n_val], perm[n_val:]
    net = Surrogate(max_batch=max(batch, n_val), seed=seed, stream=stream)
    losses, vlosses = [], []
    best, best_params = np.inf, None
    for it in range(iters):
        idx = rng.choice(tr, size=min(batch, len(tr)), replace=False)
        lr_it = lr * (0.1 ** (it / max(iters, 1)))
        losses.append(net.train_step(X[idx], M[idx], Tn[idx], lr_it))
        if n_val and (it % 25 == 24 or it == iters - 1):
            vl, _ = net.gradients(X[val], M[val], Tn[val])
            vlosses.append(vl)
            if vl < best:
                best, best_params = vl, net.get_params()
    if best_params is not None:
        net.set_params(best_params)
    return net, (mu, sd), np.array(losses), np.array(vlosses)


def predict_q0(net, norm, plist):
    mu, sd = norm
    out = []
    for c0 in range(0, len(plist), 128):
        ps = plist[c0: c0 + 128]
        xs = np.array([features(p)[0] for p in ps])
        ms = np.array([features(p)[1] for p in ps])
        y = net.forward(xs, ms) * sd + mu
        for p, yy in zip(ps, y):
            out.append(np.array([(od_oml_charge(p, g["a"]) / _psi_scale(p, g["a"]) + yy[k, 0]) * _psi_scale(p, g["a"])
                                 for k, g in enumerate(p["dust"])]))
    return out


def steps_to_converge(q, q_ref, tol):
    """first step after which |q - q_ref| <= tol |q_ref| at every later step"""
    bad = np.nonzero(np.abs(q - q_ref) > tol * abs(q_ref))[0]
    return 0 if len(bad) == 0 else int(bad[-1]) + 1


def batch_se(x, nb=20):
    """standard error of the mean of a correlated series by batch means (nb batches)"""
    m = len(x) // nb
    if m < 1:
        return float("nan")
    b = np.asarray(x[: m * nb], dtype=np.float64).reshape(nb, m).mean(1)
    return float(b.std(ddof=1) / np.sqrt(nb))


def steps_to_force(f, f_ref, se_ref, window, stride=250):
    """steps that must be simulated before a window mean of the per-step force agrees
    with the converged force: the smallest t + window such that the mean of f over
    [t, t + window) is within 2 combined standard errors (batch means of that window and
    se_ref) of f_ref; len(f) + 1 if no window qualifies"""
    c = np.concatenate([[0.0], np.cumsum(np.asarray(f, dtype=np.float64))])
    for t in range(0, len(f) - window + 1, stride):
        m = (c[t + window] - c[t]) / window
        se = np.hypot(batch_se(f[t: t + window]), se_ref)
        if abs(m - f_ref) <= 2.0 * se:
            return t + window
    return len(f) + 1


def evaluate(net, norm, plist, steps, tol=0.01, stream=None, details=False):
    """Held-out runs from q0 = 0, OML and network predictions, stepped in one batch.
    Returns per-strategy arrays of steps to converge (one per grain) and the initial
    charge errors relative to the converged charge; with details=True also the steps to
    a converged axial force (window of steps/4, 2 standard errors) and the batch's
    device time per step."""
    q_net = predict_q0(net, norm, plist)
    runs = []
    for p, qn in zip(plist, q_net):
        for strat in ("zero", "oml", "net"):
            r = {k: v for k, v in p.items() if k != "dust"}
            r["dust"] = [dict(g) for g in p["dust"]]
            for k, g in enumerate(r["dust"]):
                g["q0"] = 0.0 if strat == "zero" else (od_oml_charge(p, g["a"]) if strat == "oml" else float(qn[k]))
            r["avg_start"] = steps - steps // 4 + 1
            runs.append(r)
    b = Batch(runs, stream=stream)
    b.tune(reps=1)  # the batch's pair plan (ordered chunks or symmetric tile pairs)
    import time

    t0 = time.perf_counter()
    b.step(steps)  # synchronises on the error word at the end
    t_step = (time.perf_counter() - t0) / steps
    res = {s: [] for s in ("zero", "oml", "net")}
    resf = {s: [] for s in ("zero", "oml", "net")}
    err0 = {s: [] for s in ("zero", "oml", "net")}
    window = steps // 4
    for i, p in enumerate(plist):
        recs = [b.runs[3 * i + j].series(1, steps)[0] for j in range(3)]
        series = [r[:, :, 0] for r in recs]
        # total axial force per step: orbit + grain-grain + collection + driving field
        fz = [r[:, :, 3] + r[:, :, 6] + r[:, :, 9] + r[:, :, 12] for r in recs]
        tail = steps - window
        # converged charge and force: last quarter of the runs started near it (OML and
        # network)
        q_ref = np.mean([s[tail:].mean(0) for s in series[1:]], axis=0)
        for j, strat in enumerate(("zero", "oml", "net")):
            q0 = np.array([g["q0"] for g in runs[3 * i + j]["dust"]])
            for k in range(len(p["dust"])):
                res[strat].append(steps_to_converge(series[j][:, k], q_ref[k], tol))
                err0[strat].append(abs(q0[k] - q_ref[k]) / abs(q_ref[k]))
                if details:
                    f_ref = 0.5 * (fz[1][tail:, k].mean() + fz[2][tail:, k].mean())
                    se_ref = 0.5 * np.hypot(batch_se(fz[1][tail:, k]), batch_se(fz[2][tail:, k]))
                    resf[strat].append(steps_to_force(fz[j][:, k], f_ref, se_ref, window))
    b.close()
    out = ({s: np.array(v) for s, v in res.items()}, {s: np.array(v) for s, v in err0.items()})
    if details:
        out = out + ({s: np.array(v) for s, v in resf.items()}, t_step)
    return out
