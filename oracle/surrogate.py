"""FP64 CPU reference of the warm-start network (TEST INFRASTRUCTURE ONLY, part of the
oracle): forward pass, mean-squared-error loss and analytic gradients of the
set-pooled MLP that the CUDA library trains.

    h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2)        per grain (x: 7 features, padded to 16)
    c  = mean of h2 over the sample's present grains
    h3 = relu(W3 [h2, c] + b3), h4 = relu(W4 h3 + b4)  per grain
    y  = W5 h4 + b5                                    4 outputs (padded to 16)
    loss = sum over present grains and the 4 outputs of (y - t)^2 / (count * 4)

With bf16=True every operand of a matrix product (weights and the activation entering
it, and the backpropagated errors entering the weight-gradient and input-gradient
products) is rounded to bfloat16 as the GPU does; the arithmetic itself is FP64.
The parameter vector is layer by layer W (out x in, row-major) then b (out).
"""
import numpy as np

SHAPES = ((256, 16), (256, 256), (256, 512), (256, 256), (16, 256))
G = 8


def bf16(a):
    """round to the nearest bfloat16 (ties to even), returned as float64"""
    x = np.asarray(a, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(p):
    out, off = [], 0
    for o, i in SHAPES:
        W = np.asarray(p[off: off + o * i], dtype=np.float64).reshape(o, i)
        off += o * i
        b = np.asarray(p[off: off + o], dtype=np.float64)
        off += o
        out.append((W, b))
    return out


def pack(grads):
    return np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])


def loss_and_grad(p, x, mask, t, bf=True):
    r = bf16 if bf else (lambda a: np.asarray(a, dtype=np.float64))
    B = x.shape[0]
    M = B * G
    X = np.zeros((M, 16))
    X[:, :7] = np.asarray(x, dtype=np.float64).reshape(M, 7)
    m = np.asarray(mask, dtype=np.float64).reshape(M)
    T = np.asarray(t, dtype=np.float64).reshape(M, 4)
    (W1, b1), (W2, b2), (W3, b3), (W4, b4), (W5, b5) = unpack(p)
    X0 = r(X)
    z1 = X0 @ r(W1).T + b1
    a1 = np.maximum(z1, 0.0)
    z2 = r(a1) @ r(W2).T + b2
    a2 = np.maximum(z2, 0.0)
    mb = m.reshape(B, G)
    n = mb.sum(1)
    c = np.where(n[:, None] > 0, (mb[:, :, None] * a2.reshape(B, G, 256)).sum(1) / np.maximum(n, 1)[:, None], 0.0)
    X3 = np.concatenate([r(a2), r(np.repeat(c, G, axis=0))], axis=1)
    z3 = X3 @ r(W3).T + b3
    a3 = np.maximum(z3, 0.0)
    z4 = r(a3) @ r(W4).T + b4
    a4 = np.maximum(z4, 0.0)
    y = r(a4) @ r(W5).T + b5
    count = (m > 0).sum() * 4
    e = (y[:, :4] - T) * (m[:, None] > 0)
    loss = (e * e).sum() / count
    dy = np.zeros((M, 16))
    dy[:, :4] = 2.0 * e / count
    # the GPU keeps its backpropagated errors in FP32 before rounding them for the products
    f32 = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64) if bf else a
    dy = f32(dy)
    g5 = (r(dy).T @ r(a4), dy.sum(0))
    d4 = f32(r(dy) @ r(W5)) * (a4 > 0)
    g4 = (r(d4).T @ r(a3), d4.sum(0))
    d3 = f32(r(d4) @ r(W4)) * (a3 > 0)
    g3 = (r(d3).T @ X3, d3.sum(0))
    dX3 = f32(r(d3) @ r(W3))
    dc = (mb[:, :, None] * dX3[:, 256:].reshape(B, G, 256)).sum(1) / np.maximum(n, 1)[:, None]
    d2 = dX3[:, :256] + m[:, None] * np.repeat(dc, G, axis=0)
    d2 = f32(d2) * (a2 > 0)
    g2 = (r(d2).T @ r(a1), d2.sum(0))
    d1 = f32(r(d2) @ r(W2)) * (a1 > 0)
    g1 = (r(d1).T @ X0, d1.sum(0))
    return loss, pack([g1, g2, g3, g4, g5]), y[:, :4].reshape(B, G, 4)
