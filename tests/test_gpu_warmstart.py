"""Learned warm start, end to end at a small scale: discharges run by the
library give cycle-averaged density and mean-energy profiles, the library's
MLP kernels learn them, and held-out (U, p, L, C) loaded from the predicted
profiles reach their converged profiles in far fewer RF cycles than the
cold (uniform) start of the same discharge."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# a warm start must reach the tolerance at least this many times sooner (in
# RF cycles, mean over the held-out discharges) than the cold start
MIN_CYCLE_RATIO = 3.0


def cycles_to(errors, tol, window):
    return next(((w + 1) * window for w, e in enumerate(errors) if e < tol), None)


def test_warm_start_reaches_tolerance_sooner(torch_cuda):
    from paper_0705_0497_gb300 import api, inputs, warmstart as W, xsec
    procs = xsec.oxygen_set()
    N, n_train, held = 20000, 16, [16, 17, 18]
    sweep = inputs.batch_sweep(n_train + len(held), seed=321, count_range=(N, N))
    rng = np.random.Generator(np.random.PCG64(5))
    for cfg, _, _ in sweep:
        cfg["C_meta"] = float(rng.uniform(0.1, 1.0 / 6.0))
    T = (3.0, 0.026, 0.026)
    cycles, window = 600, 50
    runs = [(cfg, W.cold_state(cfg, counts, T, seed=i)) for i, (cfg, counts, _) in enumerate(sweep)]
    gs = W.make_discharges(api, runs, procs, capacity_factor=6, n_floor=N)
    hist, _, energy = W.run_windows(api, gs, cycles, window, snapshots=3)
    for g in gs:
        g.close()
    ref = [0.5 * (hist[-1][i] + hist[-2][i]) for i in range(len(sweep))]
    X = np.stack([W.features(sweep[i][0]) for i in range(n_train)])
    Y = np.stack([W.to_target2(ref[i], energy[i]) for i in range(n_train)])
    mlp = api.MLP([4, 256, 256, 256, 3 * W.N_CELLS + 3 * W.BINS], seed=1)
    losses = W.train(api, mlp, X, Y, steps=2000)
    assert losses[-1] < 0.05 * losses[0], losses[::10]
    import torch
    pred = mlp.forward(torch.from_numpy(np.stack([W.features(sweep[i][0]) for i in held])).cuda()).cpu().numpy()
    mlp.close()
    warm = []
    for k, i in enumerate(held):
        cells, en = W.from_target2(pred[k])
        warm.append((sweep[i][0], W.warm_state2(sweep[i][0], cells, en, seed=100 + k)))
    gw = W.make_discharges(api, warm, procs, capacity_factor=6, n_floor=N)
    hw, _, _ = W.run_windows(api, gw, cycles // 2, window)
    for g in gw:
        g.close()
    ratios = []
    for k, i in enumerate(held):
        noise = max(W.binned_error(hist[-1][i], hist[-2][i]))
        tol = max(0.05, 2.0 * noise)
        ec = [max(W.binned_error(hist[w][i], ref[i])) for w in range(len(hist) - 2)]
        ew = [max(W.binned_error(hw[w][k], ref[i])) for w in range(len(hw))]
        cc = cycles_to(ec, tol, window) or cycles
        cw = cycles_to(ew, tol, window)
        print(f"held-out {i}: tol {tol:.3f}, cold {cc} cycles, warm {cw} cycles; "
              f"cold errors {np.round(ec, 3)}, warm errors {np.round(ew, 3)}")
        assert cw is not None, (i, ew)
        ratios.append(cc / cw)
    print("cycle ratios cold/warm", ratios)
    assert np.mean(ratios) >= MIN_CYCLE_RATIO, ratios
