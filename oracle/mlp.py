"""FP64 CPU reference of the surrogate network -- TEST INFRASTRUCTURE ONLY.

Plain numpy forward and backward pass of the MLP the CUDA library trains:
inputs (alpha, beta, a/M, q, theta0) normalised to about [-1, 1], plus the polar form
(rho, cos psi, sin psi) of the scaled pixel direction and (cos, sin) of theta0, zero
padded to 16 columns,
layers 16 -> 256 -> 256 -> 256 -> 256 -> 16 with SiLU between them, output
(escape logit, end-direction vector, 12 unused), loss
    mean( BCE(logit, y) + w * y * |d_pred - d|^2 ),
where y = 1 for escaped rays and d = (sin th cos ph, sin th sin ph, cos th) of the end
position.  With `bf=True` the values are rounded where the GPU stores them in 16 bits,
round to nearest even: each forward product is split-precision bfloat16 -- the layer
input, rounded to float32 as the GPU holds it, and the weight are each carried as a pair
hi = bf16(v), lo = bf16(v - hi), and the product is x_hi w_hi + x_lo w_hi + x_hi w_lo --
and the backward products take bfloat16 operands (the transposed layer inputs of the
weight gradient, the weights of the input gradient and the gradients themselves), so
that GPU and CPU results can be compared closely; with `bf=False` it is the exact FP64
network, whose gradient a finite-difference test pins.
"""
from __future__ import annotations

import math

import numpy as np

IN = (16, 256, 256, 256, 256)
OUT = (256, 256, 256, 256, 16)


def n_params() -> int:
    return sum(o * i + o for i, o in zip(IN, OUT))


def split(params: np.ndarray):
    """Weights [out, in] and biases of each layer from the flat parameter vector."""
    ws, bs, off = [], [], 0
    for i, o in zip(IN, OUT):
        ws.append(params[off:off + o * i].reshape(o, i))
        off += o * i
        bs.append(params[off:off + o])
        off += o
    return ws, bs


def bf16(x) -> np.ndarray:
    """Round to bfloat16 (nearest even) through float32; returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def features(alpha, beta, spin, q, theta0, r0=15.0, fov_deg=75.0, spin_max=0.99, q_max=2.0,
             th_min=5 * math.pi / 180, th_max=math.pi / 2):
    V = math.tan(0.5 * fov_deg / 180 * math.pi) / r0
    H = math.atan(math.tan(V))
    X = np.zeros((len(alpha), 16))
    a = np.asarray(alpha, dtype=np.float64) / H
    b = np.asarray(beta, dtype=np.float64) / V
    th = np.asarray(theta0, dtype=np.float64)
    X[:, 0] = a
    X[:, 1] = b
    X[:, 2] = np.asarray(spin) * (2 / spin_max) - 1
    X[:, 3] = np.asarray(q) / q_max
    X[:, 4] = th * (2 / (th_max - th_min)) - (th_max + th_min) / (th_max - th_min)
    rho = np.hypot(a, b)
    X[:, 5] = rho
    X[:, 6] = a / np.maximum(rho, 1e-3)   # cos psi
    X[:, 7] = b / np.maximum(rho, 1e-3)   # sin psi
    X[:, 8] = np.cos(th)
    X[:, 9] = np.sin(th)
    return X


def labels(status, th, ph):
    y = (np.asarray(status) == 0).astype(np.float64)
    d = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], axis=1)
    return y, d * y[:, None]


def silu(z):
    return z / (1 + np.exp(-z))


def dsilu(z):
    s = 1 / (1 + np.exp(-z))
    return s * (1 + z * (1 - s))


def split_bf16(x):
    """The bf16 pair (hi, lo) of x as the GPU forms it: x rounded to float32, hi = bf16(x),
    lo = bf16(x - hi) (the difference is exact in float32); hi + lo carries x to about
    2^-17 relative."""
    x32 = np.asarray(x, dtype=np.float32).astype(np.float64)
    hi = bf16(x32)
    return hi, bf16(x32 - hi)


def split_product(A, W):
    """A W^T by the split-precision rule x_hi w_hi + x_lo w_hi + x_hi w_lo."""
    a_hi, a_lo = split_bf16(A)
    w_hi, w_lo = split_bf16(W)
    return a_hi @ w_hi.T + a_lo @ w_hi.T + a_hi @ w_lo.T


def forward(params, X0, bf=True):
    """Returns the unrounded layer inputs A[0..4] and the pre-activations Z[0..4]; with
    bf=True each product is the split-precision bf16 product of the GPU."""
    ws, bs = split(params)
    As, Zs = [np.asarray(X0, dtype=np.float64)], []
    for l in range(5):
        if bf:
            Z = split_product(As[-1], ws[l]) + bs[l]
        else:
            Z = As[-1] @ ws[l].T + bs[l]
        Zs.append(Z)
        if l < 4:
            As.append(silu(Z))
    return As, Zs


def loss_and_grad(params, X0, y, d, w_dir, bf=True):
    r = bf16 if bf else (lambda a: np.asarray(a, dtype=np.float64))
    ws, _ = split(params)
    As, Zs = forward(params, X0, bf)
    n = X0.shape[0]
    z = Zs[4]
    zl = z[:, 0]
    bce = np.maximum(zl, 0) - zl * y + np.log1p(np.exp(-np.abs(zl)))
    diff = z[:, 1:4] - d
    loss = np.mean(bce + w_dir * y * np.sum(diff * diff, axis=1))
    dZ = np.zeros_like(z)
    dZ[:, 0] = (1 / (1 + np.exp(-zl)) - y) / n
    dZ[:, 1:4] = 2 * w_dir * y[:, None] * diff / n
    grads = []
    for l in range(4, -1, -1):
        dW = r(dZ).T @ r(As[l])
        db = dZ.sum(axis=0)
        grads.append((l, dW, db))
        if l > 0:
            dX = r(dZ) @ r(ws[l])
            dZ = dX * dsilu(Zs[l - 1])
    g = np.zeros_like(params, dtype=np.float64)
    gw, gb = split(g)
    for l, dW, db in grads:
        gw[l][...] = dW
        gb[l][...] = db
    return loss, g, z


def init_params(seed=0):
    """Seeded LeCun-normal weights, zero biases (for CPU-only tests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    p = np.zeros(n_params())
    ws, _ = split(p)
    for l, w in enumerate(ws):
        fan = 10 if l == 0 else IN[l]
        w[...] = rng.normal(0, 1 / math.sqrt(fan), w.shape)
    return p
