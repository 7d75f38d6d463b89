"""Pins of the FP64 surrogate-network oracle (oracle/mlp_oracle.py) to facts
outside itself: finite differences, closed forms, a library rounding
routine, a library loss, and invariants of Adam."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import mlp_oracle as M


def small_net(seed=3, dims=(7, 6, 5, 4)):
    return W.mlp_init(list(dims), seed)


def test_bf16_rounding_matches_torch():
    import torch
    rng = np.random.Generator(np.random.PCG64(1))
    x = np.concatenate([rng.normal(size=20000) * 10.0 ** rng.uniform(-30, 30, size=20000),
                        [0.0, -0.0, 1.0, -1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, 65504.0, 1e-40]])
    want = torch.tensor(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    got = M.bf16_round(x)
    assert np.array_equal(got, want)


def test_loss_is_the_library_mean_squared_error():
    from sklearn.metrics import mean_squared_error
    rng = np.random.Generator(np.random.PCG64(2))
    Y, T = rng.normal(size=(9, 5)), rng.normal(size=(9, 5))
    assert M.loss(Y, T) == pytest.approx(mean_squared_error(T, Y), rel=1e-15)


@pytest.mark.parametrize("seed,mapped", [(0, False), (1, False), (2, True)])
def test_gradients_match_central_differences(seed, mapped):
    """Every weight and bias gradient of a 3-layer ReLU network against
    central differences of the FP64 loss (h = 1e-6), with random biases so
    that no pre-activation sits on the ReLU kink (checked)."""
    rng = np.random.Generator(np.random.PCG64(10 + seed))
    params = [(Wl, rng.normal(size=bl.size) * 0.5) for Wl, bl in small_net(seed)]
    X = rng.normal(size=(11, 7))
    T = rng.normal(size=(11, 4))
    om = (rng.normal(size=4), rng.uniform(0.1, 3.0, size=4)) if mapped else None
    _, (_, Zs) = M.forward(params, X)
    assert min(np.abs(z).min() for z in Zs[:-1]) > 1e-4
    _, g = M.grads(params, X, T, out_map=om)
    dims = [7, 6, 5, 4]
    vec = M.flatten(params)
    gvec = M.flatten(g)
    h = 1e-6
    worst = 0.0
    for idx in range(vec.size):
        vp, vm = vec.copy(), vec.copy()
        vp[idx] += h
        vm[idx] -= h
        fp = M.loss(M.forward(M.unflatten(vp, dims), X, out_map=om)[0], T)
        fm = M.loss(M.forward(M.unflatten(vm, dims), X, out_map=om)[0], T)
        fd = (fp - fm) / (2 * h)
        worst = max(worst, abs(fd - gvec[idx]) / (abs(gvec[idx]) + 1e-6))
    assert worst < 1e-5, worst


def test_single_linear_layer_gradient_closed_form():
    """No hidden layer: loss = |X W^T + b - T|^2 / (B m), so
    dL/dW = 2 (X W^T + b - T)^T X / (B m) and dL/db = column sums of the
    same residual; the minimiser is the least-squares solution."""
    rng = np.random.Generator(np.random.PCG64(4))
    X = rng.normal(size=(30, 5))
    T = rng.normal(size=(30, 3))
    Wt = rng.normal(size=(3, 5))
    bt = rng.normal(size=3)
    _, g = M.grads([(Wt, bt)], X, T)
    R = X @ Wt.T + bt - T
    assert np.allclose(g[0][0], 2.0 * R.T @ X / (30 * 3), rtol=1e-13, atol=1e-15)
    assert np.allclose(g[0][1], 2.0 * R.sum(axis=0) / (30 * 3), rtol=1e-13, atol=1e-15)
    # at the least-squares solution (numpy lstsq) the gradient vanishes
    Xa = np.hstack([X, np.ones((30, 1))])
    sol = np.linalg.lstsq(Xa, T, rcond=None)[0]
    _, g2 = M.grads([(sol[:5].T, sol[5])], X, T)
    assert np.abs(g2[0][0]).max() < 1e-13 and np.abs(g2[0][1]).max() < 1e-13


def test_identity_output_map_changes_nothing():
    params = small_net(4)
    rng = np.random.Generator(np.random.PCG64(12))
    X, T = rng.normal(size=(6, 7)), rng.normal(size=(6, 4))
    idm = (np.zeros(4), np.ones(4))
    assert np.array_equal(M.forward(params, X)[0], M.forward(params, X, out_map=idm)[0])
    a, b = M.grads(params, X, T), M.grads(params, X, T, out_map=idm)
    assert a[0] == b[0] and all(np.array_equal(x[0], y[0]) for x, y in zip(a[1], b[1]))


def test_relu_special_cases():
    """All hidden pre-activations positive: the network is the product of
    its linear maps.  All negative: the output is the last bias and no
    gradient reaches the hidden weights."""
    rng = np.random.Generator(np.random.PCG64(5))
    X = np.abs(rng.normal(size=(8, 4))) + 0.1
    W1 = np.abs(rng.normal(size=(6, 4)))
    W2 = rng.normal(size=(3, 6))
    b1, b2 = np.abs(rng.normal(size=6)), rng.normal(size=3)
    Y, _ = M.forward([(W1, b1), (W2, b2)], X)
    assert np.allclose(Y, (X @ W1.T + b1) @ W2.T + b2, rtol=1e-14)
    Y2, _ = M.forward([(-W1, -b1), (W2, b2)], X)
    assert np.array_equal(Y2, np.broadcast_to(b2, Y2.shape))
    _, g = M.grads([(-W1, -b1), (W2, b2)], X, rng.normal(size=(8, 3)))
    assert not g[0][0].any() and not g[0][1].any()


def test_adam_with_constant_gradient_moves_by_lr_per_step():
    """With bias correction, a constant gradient g gives mhat = g and
    vhat = g^2 at every step, so each step moves a weight by
    lr g / (|g| + eps): after t steps w = w0 - t lr g / (|g| + eps)."""
    rng = np.random.Generator(np.random.PCG64(6))
    w0 = rng.normal(size=50)
    g = rng.normal(size=50) * 10.0 ** rng.uniform(-3, 2, size=50)
    w, m, v = [w0.copy()], [np.zeros(50)], [np.zeros(50)]
    lr, eps = 1e-3, 1e-8
    for t in range(1, 8):
        w, m, v = M.adam(w, [g], m, v, t, lr=lr, eps=eps)
        want = w0 - t * lr * g / (np.abs(g) + eps)
        assert np.allclose(w[0], want, rtol=1e-12, atol=1e-15), t


def test_adam_is_invariant_to_gradient_scale():
    """Adam's step depends on the gradient only through g / sqrt(v): scaling
    every gradient by c > 0 leaves the trajectory unchanged when eps = 0."""
    rng = np.random.Generator(np.random.PCG64(7))
    w0 = rng.normal(size=20)
    gs = [rng.normal(size=20) for _ in range(6)]
    runs = []
    for c in (1.0, 1e3):
        w, m, v = [w0.copy()], [np.zeros(20)], [np.zeros(20)]
        for t, g in enumerate(gs, 1):
            w, m, v = M.adam(w, [c * g], m, v, t, eps=0.0)
        runs.append(w[0])
    assert np.allclose(runs[0], runs[1], rtol=1e-12)


def test_bf16_emulation_stays_within_bfloat16_error():
    """The emulated forward differs from the exact one by the rounding it
    inserts: a few units of 2^-8 relative at most on a 259-256x4-256 net."""
    dims = W.mlp_dims()
    params = W.mlp_init(dims, 1602)
    rng = np.random.Generator(np.random.PCG64(8))
    X = rng.uniform(-1, 1, size=(32, dims[0]))
    Y, _ = M.forward(params, X)
    Yb, _ = M.forward(params, X, emulate_bf16=True)
    rel = np.linalg.norm(Yb - Y) / np.linalg.norm(Y)
    assert 0.0 < rel < 8 * 2.0 ** -8, rel


def test_flatten_roundtrip_and_layout():
    dims = [5, 4, 3]
    params = W.mlp_init(dims, 9)
    vec = M.flatten(params)
    assert vec.size == 5 * 4 + 4 + 4 * 3 + 3
    assert np.array_equal(vec[:20], params[0][0].ravel())
    back = M.unflatten(vec, dims)
    for (a, b), (c, d) in zip(params, back):
        assert np.array_equal(a, c) and np.array_equal(b, d)


def test_mlp_init_is_he_uniform():
    dims = W.mlp_dims()
    params = W.mlp_init(dims, 1)
    for (Wl, bl), fan in zip(params, dims[:-1]):
        lim = math.sqrt(6.0 / fan)
        assert np.abs(Wl).max() <= lim and np.abs(Wl).max() > 0.95 * lim
        assert abs(Wl.var() - lim * lim / 3.0) < 0.05 * lim * lim / 3.0
        assert not bl.any()
