"""Surrogate network kernels (include/fargo_mlp.h) against the FP64 oracle.

The oracle runs with bfloat16 rounding at the points where the kernels
store bfloat16 operands, so the two differ by FP32-versus-FP64 accumulation
and by the rare activation whose bfloat16 rounding flips between them.
Tolerances (relative L2): forward 2e-3, loss 1e-4, each layer's weight and
bias gradient 1e-2 (one flipped rounding of a hidden activation moves a
gradient row by about 2^-8), Adam 1e-6 (FP32 arithmetic on identical
gradients).
"""
import numpy as np
import pytest

import workloads as W
from oracle import mlp_oracle as M
from tests.gpu_util import record

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(np.asarray(a, dtype=np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def net_and_params(dims, seed, max_batch=512):
    import paper_1602_02359_b300.mlp as fm
    rng = np.random.Generator(np.random.PCG64(seed + 100))
    params = [(Wl, 0.1 * rng.normal(size=bl.size)) for Wl, bl in W.mlp_init(dims, seed)]
    vec = M.flatten(params).astype(np.float32)
    params32 = M.unflatten(vec.astype(np.float64), dims)
    net = fm.Mlp(dims, max_batch)
    net.set_params(vec)
    return net, vec, params32


def dev(a):
    import torch
    return torch.tensor(np.asarray(a, dtype=np.float32), device="cuda").contiguous()


CASES = [(W.mlp_dims(), 77), (W.mlp_dims(), 256), ([7, 5, 3], 3), ([33, 70, 65, 9], 130)]


@pytest.mark.parametrize("dims,batch", CASES)
def test_forward_matches_oracle(dims, batch):
    import torch
    net, vec, p = net_and_params(dims, 1)
    rng = np.random.Generator(np.random.PCG64(2))
    X = rng.uniform(-1, 1, size=(batch, dims[0])).astype(np.float32)
    y = torch.empty(batch, dims[-1], device="cuda")
    net.forward(dev(X), y)
    Yo, _ = M.forward(p, X.astype(np.float64), emulate_bf16=True)
    net.status()
    e = rel_l2(y.cpu().numpy(), Yo)
    record(f"mlp_forward_{'x'.join(map(str, dims))}_b{batch}", rel_l2=e)
    assert e < 2e-3
    net.close()


@pytest.mark.parametrize("dims,batch", CASES)
def test_inference_kernel_agrees_with_the_training_forward(dims, batch):
    """Inference runs the whole network in one kernel; back-propagation runs
    the layer-by-layer products.  The loss back-propagation reports must be
    the mean squared error of the inference output against the same targets
    (both FP32 over the same bfloat16 operands)."""
    import torch
    net, vec, p = net_and_params(dims, 4)
    rng = np.random.Generator(np.random.PCG64(5))
    X = dev(rng.uniform(-1, 1, size=(batch, dims[0])))
    T = dev(rng.normal(size=(batch, dims[-1])))
    y = torch.empty(batch, dims[-1], device="cuda")
    net.forward(X, y)
    loss = torch.zeros(1, device="cuda")
    net.backward(X, T, loss)
    net.status()
    mse = float(((y.double() - T.double()) ** 2).mean())
    got = float(loss.item())
    record(f"mlp_inference_vs_training_forward_{'x'.join(map(str, dims))}_b{batch}", rel=abs(got - mse) / mse)
    assert abs(got - mse) <= 1e-5 * mse, (got, mse)
    net.close()


@pytest.mark.parametrize("dims,batch", CASES)
def test_gradients_match_oracle(dims, batch):
    import torch
    net, vec, p = net_and_params(dims, 3)
    rng = np.random.Generator(np.random.PCG64(4))
    X = rng.uniform(-1, 1, size=(batch, dims[0])).astype(np.float32)
    T = rng.normal(size=(batch, dims[-1])).astype(np.float32)
    loss = torch.zeros(1, device="cuda")
    net.backward(dev(X), dev(T), loss)
    g = net.get_grads()
    lo, go = M.grads(p, X.astype(np.float64), T.astype(np.float64), emulate_bf16=True)
    assert abs(loss.item() - lo) <= 1e-4 * lo
    gl = M.unflatten(g.astype(np.float64), dims)
    record(f"mlp_grads_{'x'.join(map(str, dims))}_b{batch}",
           worst_dW=max(rel_l2(a[0], b[0]) for a, b in zip(gl, go)),
           worst_db=max(rel_l2(a[1], b[1]) for a, b in zip(gl, go)))
    for l, ((dW, db), (oW, ob)) in enumerate(zip(gl, go)):
        assert rel_l2(dW, oW) < 1e-2, (l, rel_l2(dW, oW))
        assert rel_l2(db, ob) < 1e-2, (l, rel_l2(db, ob))
    net.close()


def test_adam_step_matches_oracle():
    import torch
    dims = [33, 70, 65, 9]
    net, vec, p = net_and_params(dims, 5)
    net.set_optimizer(lr=3e-3, b1=0.8, b2=0.99, eps=1e-7)
    rng = np.random.Generator(np.random.PCG64(6))
    X = dev(rng.uniform(-1, 1, size=(40, 33)))
    T = dev(rng.normal(size=(40, 9)))
    w = [vec.astype(np.float64)]
    m, v = [np.zeros(vec.size)], [np.zeros(vec.size)]
    for t in range(1, 4):
        net.backward(X, T)
        g = net.get_grads().astype(np.float64)
        net.adam()
        w, m, v = M.adam(w, [g], m, v, t, lr=3e-3, b1=0.8, b2=0.99, eps=1e-7)
        got = net.get_params()
        assert rel_l2(got, w[0]) < 1e-6, t
        w = [got.astype(np.float64)]     # continue from the device's FP32 weights
    net.close()


def test_train_step_graph_equals_backward_plus_adam_and_learns():
    """train_step (one captured graph) and backward + adam (direct launches)
    run the same kernels: bit-identical weights.  Training a smooth
    regression lowers the loss at least tenfold."""
    import torch
    dims = [16, 64, 64, 8]
    x, y = W.regression_set(1024, 16, 8, seed=7)
    X, T = dev(x[:256]), dev(y[:256])
    a, vec, _ = net_and_params(dims, 8)
    b, _, _ = net_and_params(dims, 8)
    loss = torch.zeros(1, device="cuda")
    first = None
    for it in range(300):
        a.train_step(X, T, loss)
        if it == 0:
            torch.cuda.synchronize()
            first = loss.item()
        b.backward(X, T)
        b.adam()
    torch.cuda.synchronize()
    assert np.array_equal(a.get_params(), b.get_params())
    a.backward(X, T, loss)
    torch.cuda.synchronize()
    assert loss.item() < 0.1 * first, (first, loss.item())
    a.close()
    b.close()


def test_output_map_forward_and_gradients():
    import torch
    dims = [33, 70, 65, 9]
    net, vec, p = net_and_params(dims, 12)
    rng = np.random.Generator(np.random.PCG64(13))
    sh = rng.normal(size=9).astype(np.float32)
    sc = rng.uniform(0.01, 2, size=9).astype(np.float32)
    net.set_output_map(sh, sc)
    om = (sh.astype(np.float64), sc.astype(np.float64))
    X = rng.uniform(-1, 1, size=(50, 33)).astype(np.float32)
    T = rng.normal(size=(50, 9)).astype(np.float32)
    y = torch.empty(50, 9, device="cuda")
    net.forward(dev(X), y)
    Yo, _ = M.forward(p, X.astype(np.float64), emulate_bf16=True, out_map=om)
    assert rel_l2(y.cpu().numpy(), Yo) < 2e-3
    loss = torch.zeros(1, device="cuda")
    net.backward(dev(X), dev(T), loss)
    lo, go = M.grads(p, X.astype(np.float64), T.astype(np.float64), emulate_bf16=True, out_map=om)
    assert abs(loss.item() - lo) <= 1e-4 * lo
    gl = M.unflatten(net.get_grads().astype(np.float64), dims)
    for (dW, db), (oW, ob) in zip(gl, go):
        assert rel_l2(dW, oW) < 1e-2 and rel_l2(db, ob) < 1e-2
    net.close()


def test_input_map_is_applied_before_the_first_layer():
    import torch
    dims = [12, 32, 5]
    net, vec, p = net_and_params(dims, 9)
    rng = np.random.Generator(np.random.PCG64(10))
    X = rng.normal(size=(20, 12)).astype(np.float32) * 5 + 3
    shift = rng.normal(size=12).astype(np.float32)
    scale = rng.uniform(0.1, 2, size=12).astype(np.float32)
    net.set_input_map(shift, scale)
    y = torch.empty(20, 5, device="cuda")
    net.forward(dev(X), y)
    Xs = (X - shift) * scale
    Yo, _ = M.forward(p, Xs.astype(np.float64), emulate_bf16=True)
    assert rel_l2(y.cpu().numpy(), Yo) < 2e-3
    net.close()


def test_ensemble_statistics():
    import torch
    import paper_1602_02359_b300.mlp as fm
    rng = np.random.Generator(np.random.PCG64(11))
    ys = rng.normal(size=(4, 37, 256)).astype(np.float32) * 0.05 + 1.0
    mean = torch.empty(37, 256, device="cuda")
    spread = torch.empty(37, device="cuda")
    fm.ensemble(dev(ys), mean, spread)
    torch.cuda.synchronize()
    mu = ys.astype(np.float64).mean(axis=0)
    sd = ys.astype(np.float64).std(axis=0, ddof=1)
    want = np.linalg.norm(sd, axis=1) / np.linalg.norm(mu, axis=1)
    assert rel_l2(mean.cpu().numpy(), mu) < 1e-6
    assert rel_l2(spread.cpu().numpy(), want) < 1e-5


def test_bad_arguments():
    import torch
    import paper_1602_02359_b300 as fb
    import paper_1602_02359_b300.mlp as fm
    with pytest.raises(fb.FargoError) as e:
        fm.Mlp([4, 0, 3], 8)
    assert e.value.code == -1
    net = fm.Mlp([4, 8, 3], 8)
    with pytest.raises(fb.FargoError) as e:
        net.forward(torch.zeros(9, 4, device="cuda"), torch.zeros(9, 3, device="cuda"))
    assert e.value.code == -6
    with pytest.raises(fb.FargoError) as e:
        net.set_params(np.zeros(5))
    assert e.value.code == -6
    net.close()
