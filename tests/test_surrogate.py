"""The warm-start network: its FP64 CPU reference is pinned by central finite
differences; the GPU's hand-written forward/backward (BF16 products, FP32
accumulation, on either matrix-product engine) is checked against that reference with
the same BF16 roundings; and a learning test shows the GPU training loop fits a smooth
synthetic target."""
import numpy as np
import pytest

from oracle import surrogate as ref

N_PARAMS = sum(o * i + o for o, i in ref.SHAPES)


def _inputs(B, seed):
    rng = np.random.default_rng(seed)
    x = rng.normal(0.0, 1.0, (B, 8, 7))
    mask = (rng.uniform(size=(B, 8)) < 0.5).astype(np.float64)
    mask[:, 0] = 1.0
    t = rng.normal(0.0, 1.0, (B, 8, 4))
    return x, mask, t


def _params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    p = []
    for o, i in ref.SHAPES:
        W = rng.normal(0.0, scale / np.sqrt(i), (o, i))
        if (o, i) == ref.SHAPES[0]:
            W[:, 7:] = 0.0
        if (o, i) == ref.SHAPES[-1]:
            W[4:, :] = 0.0
        p.append(W.ravel())
        p.append(rng.normal(0.0, 0.1, o) * (np.arange(o) < (4 if o == 16 else o)))
    return np.concatenate(p)


def test_reference_gradients_match_finite_differences():
    x, mask, t = _inputs(3, 1)
    p = _params(2)
    loss, g, _ = ref.loss_and_grad(p, x, mask, t, bf=False)
    rng = np.random.default_rng(3)
    # live parameters of every layer (padding columns/rows carry no gradient)
    offs, off = [], 0
    for o, i in ref.SHAPES:
        offs.append((off, o, i))
        off += o * i + o
    idx = []
    for off, o, i in offs:
        for _ in range(6):
            r, c = rng.integers(0, 4 if o == 16 else o), rng.integers(0, 7 if i == 16 else i)
            idx.append(off + r * i + c)
        idx.append(off + o * i + rng.integers(0, 4 if o == 16 else o))
    for k in idx:
        h = 1e-6 * max(1.0, abs(p[k]))
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (ref.loss_and_grad(pp, x, mask, t, bf=False)[0] - ref.loss_and_grad(pm, x, mask, t, bf=False)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1e-3, abs(g[k])) + 1e-9, (k, fd, g[k])


def test_reference_pooling_is_permutation_invariant():
    x, mask, t = _inputs(2, 4)
    p = _params(5)
    l0, g0, y0 = ref.loss_and_grad(p, x, mask, t, bf=False)
    perm = np.array([3, 1, 7, 0, 5, 2, 6, 4])
    l1, g1, y1 = ref.loss_and_grad(p, x[:, perm], mask[:, perm], t[:, perm], bf=False)
    assert abs(l0 - l1) < 1e-12 * abs(l0) and np.allclose(y0[:, perm], y1, rtol=1e-12, atol=1e-12)
    assert np.allclose(g0, g1, rtol=1e-9, atol=1e-12)


@pytest.mark.gpu
@pytest.mark.parametrize("engine", ["tcgen05", "mma_sync"])
def test_gpu_gradients_match_reference(engine):
    import paper_2205_06557_gb300 as od

    s = od.Surrogate(max_batch=16, seed=7)
    s.set_gemm(od.GEMM_TCGEN05 if engine == "tcgen05" else od.GEMM_MMA_SYNC)
    p = s.get_params().astype(np.float64)
    assert p.size == N_PARAMS
    x, mask, t = _inputs(6, 11)
    loss_g, g_g = s.gradients(x, mask, t)
    loss_r, g_r, y_r = ref.loss_and_grad(p, x, mask, t, bf=True)
    assert abs(loss_g - loss_r) <= 1e-4 * abs(loss_r)
    y_g = s.forward(x, mask)
    assert np.abs(y_g - y_r).max() <= 1e-3 * np.abs(y_r).max()
    off = 0
    for o, i in ref.SHAPES:
        for n in (o * i, o):
            a, b = g_g[off: off + n].astype(np.float64), g_r[off: off + n]
            off += n
            if np.linalg.norm(b) == 0:
                assert np.linalg.norm(a) == 0
                continue
            assert np.linalg.norm(a - b) <= 5e-3 * np.linalg.norm(b), (o, i, n)
            assert a @ b / (np.linalg.norm(a) * np.linalg.norm(b)) > 0.9999
    s.close()


@pytest.mark.gpu
def test_gpu_training_fits_a_smooth_target():
    import paper_2205_06557_gb300 as od

    rng = np.random.default_rng(0)
    B = 64
    x = rng.uniform(-1, 1, (512, 8, 7))
    mask = (rng.uniform(size=(512, 8)) < 0.4).astype(np.float64)
    mask[:, 0] = 1.0
    # per-grain target mixing the grain's own features, the globals and the set mean
    setmean = (mask[:, :, None] * x).sum(1) / mask.sum(1)[:, None]
    t = np.stack([np.sin(x[..., 0] + x[..., 3]), x[..., 4] * x[..., 1], np.cos(x[..., 5]) - 0.5,
                  setmean[:, None, 6].repeat(8, 1) + 0.3 * x[..., 2]], -1)
    s = od.Surrogate(max_batch=B, seed=1)
    first = None
    for it in range(600):
        sl = slice((it * B) % 512, (it * B) % 512 + B)
        loss = s.train_step(x[sl], mask[sl], t[sl], lr=2e-3)
        if first is None:
            first = loss
    _, _, y = ref.loss_and_grad(s.get_params(), x[:64], mask[:64], t[:64], bf=True)
    err = ((y - t[:64]) ** 2 * mask[:64, :, None]).sum() / (mask[:64].sum() * 4)
    assert loss < first / 20 and err < first / 20, (first, loss, err)
    s.close()
