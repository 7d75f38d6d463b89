"""The learned surrogate of the batched disk sweep, end to end at a reduced
scale (disks of 24..32 radial cells, 5 orbits): training data from the
batched FP32 solver, a 4-member ensemble trained by the network kernels,
judged by the FP64 solver.

What the network gains over the method without it (the solver alone):
answers at a stated error in a small fraction of the solver's time.  The
test also checks that the network learned the sweep (its error is well
below that of the best constant answer, the training-mean profile) and that
the fallback hands every query above the threshold to the solver."""
import time

import numpy as np
import pytest

import workloads as W
from tests.gpu_util import record

pytestmark = pytest.mark.gpu

ORBITS = 5.0


@pytest.fixture(scope="module")
def trained():
    import torch
    import paper_1602_02359_b300 as fb
    import paper_1602_02359_b300.surrogate as S
    params = W.surrogate_params(n=448, seed=1602, nr=(24, 32))
    bins = W.surrogate_bins()
    X = np.stack([S.features(p, bins) for p in params])
    ntr, ncal = 320, 64
    Y, solver_s, _ = S.solve(params[:ntr], ORBITS, precision=fb.F32)
    Ycal, _, _ = S.solve(params[ntr:ntr + ncal], ORBITS, precision=fb.F32)
    ev = params[ntr + ncal:]
    t0 = time.perf_counter()
    Yev32, solver_ev_s, _ = S.solve(ev, ORBITS, precision=fb.F32)
    solver_ev_wall = time.perf_counter() - t0
    Yev64, _, _ = S.solve(ev, ORBITS, precision=fb.F64)
    ens = S.Ensemble(k=4, seed=1602, max_batch=512)
    hist = ens.fit(X[:ntr], Y, epochs=400, lr=2e-3)
    ens.calibrate(X[ntr:ntr + ncal], Ycal)
    yield dict(S=S, ens=ens, params=params, X=X, Y=Y, ev=ev, Xev=X[ntr + ncal:], Yev32=Yev32, Yev64=Yev64,
               solver_ev_s=solver_ev_s, solver_ev_wall=solver_ev_wall, hist=hist)
    ens.close()


def test_training_lowers_the_loss(trained):
    hist = trained["hist"]
    assert hist[-1][1] < 0.05 * hist[0][1], hist


def test_surrogate_beats_the_best_constant_answer(trained):
    S = trained["S"]
    mean, _ = trained["ens"].predict(trained["Xev"])
    err = S.rel_err(mean.cpu().numpy(), trained["Yev64"])
    naive = S.rel_err(np.broadcast_to(trained["Y"].mean(axis=0), trained["Yev64"].shape), trained["Yev64"])
    record("surrogate_small", median=np.median(err), p90=np.quantile(err, 0.9), naive_median=np.median(naive))
    assert np.median(err) < 0.5 * np.median(naive), (np.median(err), np.median(naive))
    assert np.median(err) < 0.05


def test_surrogate_answers_far_faster_than_the_solver(trained):
    import torch
    ens, Xev = trained["ens"], trained["Xev"]
    ens.predict(Xev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(10):
        ens.predict(Xev)
    torch.cuda.synchronize()
    t_sur = (time.perf_counter() - t0) / 10
    record("surrogate_small_speed", surrogate_s=t_sur, solver_s=trained["solver_ev_s"])
    assert t_sur * 20 < trained["solver_ev_s"], (t_sur, trained["solver_ev_s"])


def test_fallback_returns_the_solver_answer(trained):
    """Threshold 0: every query goes to the FP32 batched solver, bit for bit
    its answer.  Threshold infinite: none does.  The calibrated threshold:
    every accepted answer's reported error is within it, and most accepted
    answers' actual error is too."""
    S, ens, ev = trained["S"], trained["ens"], trained["ev"]
    prof, rep, fall = S.query(ens, ev, ORBITS, threshold=0.0)
    assert fall.all() and np.array_equal(prof, trained["Yev32"])
    prof, rep, fall = S.query(ens, ev, ORBITS, threshold=np.inf)
    assert not fall.any()
    prof, rep, fall = S.query(ens, ev, ORBITS, threshold=0.05)
    assert (rep[~fall] <= 0.05).all()
    err = S.rel_err(prof, trained["Yev64"])
    record("surrogate_small_fallback", fallback_fraction=fall.mean(),
           accepted_max=err[~fall].max() if (~fall).any() else 0.0)
    if (~fall).any():
        assert (err[~fall] <= 0.05).mean() >= 0.8
    assert np.allclose(prof[fall], trained["Yev32"][fall], rtol=0, atol=0)
