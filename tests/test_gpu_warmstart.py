"""Learned warm start, end to end at a small scale: cold runs of the library
give converged, cycle-averaged density and mean-energy profiles, the
library's MLP kernels learn them, and held-out discharges loaded from the
predicted profiles reach their own converged profiles in far fewer RF cycles
than their cold (uniform) start does.  The discharges are drawn where the
cold start converges within the run (U 100-300 V, p 15-50 Pa)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# a warm start must reach the tolerance at least this many times sooner (in
# RF cycles, mean over the held-out discharges) than the cold start
MIN_CYCLE_RATIO = 2.0


def cycles_to(errors, tol, window):
    return next(((w + 1) * window for w, e in enumerate(errors) if e < tol), None)


def test_warm_start_reaches_tolerance_sooner(torch_cuda):
    import torch
    from paper_0705_0497_gb300 import api, warmstart as W, xsec
    procs = xsec.oxygen_set()
    N, n_train, held = 20000, 13, [13, 14, 15]
    sweep = W.study_sweep(n_train + len(held), N, seed=77, p_range=(15.0, 50.0), U_range=(100.0, 300.0))
    T = (3.0, 0.026, 0.026)
    cycles, window = 2400, 200
    runs = [(cfg, W.cold_state(cfg, counts, T, seed=i)) for i, (cfg, counts, _) in enumerate(sweep)]
    gs = W.make_discharges(api, runs, procs, capacity_factor=20, n_floor=N)
    hist, _, energy = W.run_windows(api, gs, cycles, window, snapshots=3)
    for g in gs:
        g.close()
    ref = [0.5 * (hist[-1][i] + hist[-2][i]) for i in range(len(sweep))]
    X = np.stack([W.features(sweep[i][0]) for i in range(n_train)])
    Y = np.stack([W.to_target2(ref[i], energy[i]) for i in range(n_train)])
    mlp = api.MLP([4, 256, 256, 256, 3 * W.N_CELLS + 3 * W.BINS], seed=1)
    losses = W.train(api, mlp, X, Y, steps=2000)
    assert losses[-1] < 0.05 * losses[0], losses[::10]
    pred = mlp.forward(torch.from_numpy(np.stack([W.features(sweep[i][0]) for i in held])).cuda()).cpu().numpy()
    mlp.close()
    warm = []
    for k, i in enumerate(held):
        cells, en = W.from_target2(pred[k])
        warm.append((sweep[i][0], W.warm_state2(sweep[i][0], cells, en, seed=100 + k)))
    gw = W.make_discharges(api, warm, procs, capacity_factor=20, n_floor=N)
    hw, _, _ = W.run_windows(api, gw, cycles // 2, window)
    for g in gw:
        g.close()
    ratios = []
    for k, i in enumerate(held):
        noise = max(W.binned_error(hist[-1][i], hist[-2][i]))
        tol = max(0.08, 3.0 * noise)
        ec = [max(W.binned_error(hist[w][i], ref[i])) for w in range(len(hist) - 2)]
        ew = [max(W.binned_error(hw[w][k], ref[i])) for w in range(len(hw))]
        cc = cycles_to(ec, tol, window) or cycles
        cw = cycles_to(ew, tol, window)
        print(f"held-out {i} {({q: round(sweep[i][0][q], 3) for q in ('U', 'p', 'L', 'C_meta')})}: tol {tol:.3f}, "
              f"cold {cc} cycles, warm {cw} cycles; cold errors {np.round(ec, 3)}, warm errors {np.round(ew, 3)}")
        assert cw is not None, (i, ew)
        ratios.append(cc / cw)
    print("cycle ratios cold/warm", ratios)
    assert np.mean(ratios) >= MIN_CYCLE_RATIO, ratios
