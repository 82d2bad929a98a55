"""Learned warm start, end to end at a small scale: discharges run by the
library give cycle-averaged profiles, the library's MLP kernels learn them,
and runs of held-out (U, p) loaded from the predicted profiles start closer
to their own late-time profiles than the cold (uniform) start does."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_warm_start_beats_cold_start(torch_cuda):
    from paper_0705_0497_gb300 import api, inputs, warmstart as W, xsec
    procs = xsec.oxygen_set()
    sweep = inputs.batch_sweep(14, seed=321, count_range=(1.0e4, 1.0e4))
    T = (3.0, 0.026, 0.026)
    runs = [(cfg, W.cold_state(cfg, counts, T, seed=i)) for i, (cfg, counts, _) in enumerate(sweep)]
    gs = W.make_discharges(api, runs, procs)
    ref, _ = W.run_cycles(api, gs, cycles=150, window=50)
    for g in gs:
        g.close()
    train, held = list(range(12)), [12, 13]
    X = np.stack([W.features(sweep[i][0]) for i in train])
    Y = np.stack([W.to_target(ref[i]) for i in train])
    mlp = api.MLP([4, 256, 256, 256, 768], seed=1)
    losses = W.train(api, mlp, X, Y, steps=1500)
    assert losses[-1] < 0.1 * losses[0], losses[::10]
    pred = W.predict(mlp, [sweep[i][0] for i in held])
    cases = []
    for k, i in enumerate(held):
        cfg, counts, _ = sweep[i]
        cases.append((cfg, W.warm_state(cfg, pred[k], T, seed=100 + k)))
        cases.append((cfg, W.cold_state(cfg, counts, T, seed=200 + k)))
    gs = W.make_discharges(api, cases, procs)
    _, hist = W.run_cycles(api, gs, cycles=10, window=10)
    err_warm = [np.mean(W.profile_error(hist[0][2 * k], ref[i])) for k, i in enumerate(held)]
    err_cold = [np.mean(W.profile_error(hist[0][2 * k + 1], ref[i])) for k, i in enumerate(held)]
    print("first 10 cycles, rms profile error vs the 150-cycle reference: warm", err_warm, "cold", err_cold)
    assert np.mean(err_warm) < np.mean(err_cold)
    mlp.close()
