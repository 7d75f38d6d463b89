"""Plain FP64 reference of the surrogate network: a multilayer perceptron
with ReLU hidden layers and a linear output, its mean-squared-error loss,
the gradients by the chain rule, and the Adam update.

TEST INFRASTRUCTURE ONLY: imported by the tests, never by the product path.
It shares no code with the CUDA library.

Definitions (the network has no counterpart in the paper):
  Z_l = A_{l-1} W_l^T + b_l,  A_l = max(Z_l, 0) for hidden layers,
  Y = Z_L * s + c (linear output with an optional per-output map (c, s)),
  A_0 = X (rows = samples);
  loss = mean over samples and outputs of (Y - T)^2;
  Adam (Kingma & Ba 2015, Algorithm 1): m <- b1 m + (1-b1) g,
  v <- b2 v + (1-b2) g^2, w <- w - lr mhat / (sqrt(vhat) + eps) with
  mhat = m / (1 - b1^t), vhat = v / (1 - b2^t).

emulate_bf16=True rounds to bfloat16 (round to nearest, ties to even, from
the binary32 value) exactly where the CUDA kernels store bfloat16 operands:
the weights, the network input, every hidden activation A_l, and the
back-propagated pre-activation gradients dZ_l that feed the weight and
input-gradient products.  Sums stay FP64 here (FP32 on the GPU).
"""
from __future__ import annotations

import numpy as np


def bf16_round(a):
    """Nearest bfloat16 of each value's binary32 rounding (ties to even),
    returned as FP64."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def _q(a, on):
    return bf16_round(a) if on else np.asarray(a, dtype=np.float64)


def forward(params, X, emulate_bf16=False, out_map=None):
    """Returns (Y, cache) with cache = (A_0 .. A_{L-1}, Z_1 .. Z_L);
    out_map = (shift, scale) per output, or None for the identity."""
    A = _q(X, emulate_bf16)
    As, Zs = [A], []
    L = len(params)
    for l, (W, b) in enumerate(params):
        Z = A @ _q(W, emulate_bf16).T + b
        Zs.append(Z)
        if l < L - 1:
            A = _q(np.maximum(Z, 0.0), emulate_bf16)
            As.append(A)
    Y = Zs[-1] if out_map is None else Zs[-1] * out_map[1] + out_map[0]
    return Y, (As, Zs)


def loss(Y, T):
    return float(np.mean((Y - T) ** 2))


def grads(params, X, T, emulate_bf16=False, out_map=None):
    """(loss, [(dW_l, db_l)]) of the mean-squared error by back-propagation."""
    Y, (As, Zs) = forward(params, X, emulate_bf16, out_map)
    B, m = Y.shape
    dZ = 2.0 * (Y - T) / (B * m)
    if out_map is not None:
        dZ = dZ * out_map[1]
    out = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        W = _q(params[l][0], emulate_bf16)
        dZq = _q(dZ, emulate_bf16)
        out[l] = (dZq.T @ As[l], dZ.sum(axis=0))
        if l > 0:
            dA = dZq @ W
            dZ = dA * (Zs[l - 1] > 0.0)
    return loss(Y, T), out


def adam(params, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step at step number t >= 1 on lists of arrays; returns the
    new (params, m, v)."""
    P, M, V = [], [], []
    for w, gg, mm, vv in zip(params, g, m, v):
        mm = b1 * mm + (1.0 - b1) * gg
        vv = b2 * vv + (1.0 - b2) * gg * gg
        mh = mm / (1.0 - b1 ** t)
        vh = vv / (1.0 - b2 ** t)
        P.append(w - lr * mh / (np.sqrt(vh) + eps))
        M.append(mm)
        V.append(vv)
    return P, M, V


def flatten(params):
    """Parameter vector in the order W_0 (row-major), b_0, W_1, b_1, ..."""
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in params])


def unflatten(vec, dims):
    out, o = [], 0
    for a, b in zip(dims[:-1], dims[1:]):
        W = vec[o:o + a * b].reshape(b, a)
        o += a * b
        out.append((W, vec[o:o + b]))
        o += b
    return out
