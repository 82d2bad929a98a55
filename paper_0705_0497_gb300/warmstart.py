"""Learned warm start of a discharge (no counterpart in the paper).

A run of the method starts from uniform, Maxwellian particles and needs many
RF cycles until its cycle-averaged density profiles stop changing.  Here a
small MLP (`api.MLP`: the library's own forward, backward and Adam kernels)
learns, from runs the method itself produced, the map

    (U, p, L, C)  ->  cycle-averaged log densities of e, O-, O2+ on the cells,

and a new run is loaded from the predicted profiles instead of uniformly.
The cold start stays the fallback and the judge of the result: a warm-started
run is still the method, only its initial condition differs.

Functions here do argument marshalling and bookkeeping; the discharge steps,
the training and the inference run in the library's CUDA kernels.  Particle
positions are drawn on the host (input generation, like `inputs.py`).
"""
import math

import numpy as np

from . import inputs

N_CELLS = 256
LOG_FLOOR = 1.0e12          # m^-3: densities below are clipped before the log
LOG_SHIFT = 35.0            # log(n) - LOG_SHIFT keeps the targets near O(1)


def features(cfg):
    """Normalized inputs of the network: U, log p, L, C."""
    return np.array([(cfg["U"] - 300.0) / 200.0,
                     (math.log(cfg["p"]) - math.log(math.sqrt(5.0 * 50.0))) / math.log(math.sqrt(10.0)),
                     (cfg["L"] - 0.025) / 0.005,
                     cfg["C_meta"] * 6.0 - 0.5], np.float32)


def cell_profiles(node_density):
    """Cell-centre densities [3][Nc] from node densities [3][Nc + 1]."""
    d = np.asarray(node_density, np.float64)
    return 0.5 * (d[:, :-1] + d[:, 1:])


def to_target(cells):
    return (np.log(np.maximum(cells, LOG_FLOOR)) - LOG_SHIFT).astype(np.float32).ravel()


def from_target(y):
    return np.exp(np.asarray(y, np.float64).reshape(3, -1) + LOG_SHIFT)


def cold_state(cfg, counts, T_eV, seed):
    return inputs.initial_state(cfg, counts, T_eV, seed=seed)


def warm_state(cfg, cells, T_eV, seed):
    """Particles of the three species drawn from cell densities [3][Nc]:
    per cell round(n dx A / w) particles (stochastic rounding), uniform in
    the cell, Maxwellian at T_eV.  Ids 0..N-1 per species."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Nc = cells.shape[1]
    dx = cfg["L"] / Nc
    out = []
    for s in range(3):
        mean = cells[s] * dx * cfg["area"] / cfg["weight"]
        k = np.floor(mean + rng.random(Nc)).astype(np.int64)
        n = int(k.sum())
        c = np.repeat(np.arange(Nc), k)
        x = ((c + rng.random(n)) * dx).astype(np.float32)
        x = np.minimum(x, np.float32(cfg["L"]) * np.float32(1 - 2 ** -23))
        sig = math.sqrt(T_eV[s] * inputs.QE / inputs.species_mass(cfg, s))
        v = (rng.standard_normal((3, n)) * sig).astype(np.float32)
        out.append(dict(x=x, vx=v[0].copy(), vy=v[1].copy(), vz=v[2].copy(), id=np.arange(n, dtype=np.uint32)))
    return out


def make_discharges(api, runs, procs, capacity_factor=8, compact_check=200):
    """Library contexts for [(cfg, state)] (all processes set, particles loaded)."""
    gs = []
    for cfg, st in runs:
        n = [len(p["x"]) for p in st]
        g = api.Discharge(cfg, tuple(capacity_factor * max(k, 1000) + 65536 for k in n), compact_check=compact_check)
        g.set_processes(procs)
        g.load_state(st)
        gs.append(g)
    return gs


def run_cycles(api, gs, cycles, window, steps_per_launch=200, tune=True, progress=None):
    """Advance the discharges together by `cycles` RF cycles (one batch graph;
    launch shapes from the library's autotuner first, whose replays are real
    steps counted in `cycles`) and return per discharge the cell densities
    averaged over the last `window` cycles, plus per-window profiles
    [windows][discharge][3][Nc]."""
    spc = gs[0].cfg["steps_per_cycle"]
    per_cycle = spc // steps_per_launch
    b = api.Batch(gs, steps_per_launch)
    if tune:
        b.autotune()
        b.synchronize()
    hist = []
    for w0 in range(0, cycles, window):
        for g in gs:
            g.moments(reset=True)
        b.step(per_cycle * min(window, cycles - w0))
        b.synchronize()
        hist.append([cell_profiles(g.moments()[0]) for g in gs])
        if progress:
            progress(w0 + min(window, cycles - w0), hist)
    b.close()
    return hist[-1], hist


def train(api, mlp, X, Y, steps, lr=2e-3, lr_end=2e-4):
    """Adam on all samples at once (full batch), learning rate decayed
    geometrically; returns the losses."""
    import torch
    Xd = torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda()
    Yd = torch.from_numpy(np.ascontiguousarray(Y, np.float32)).cuda()
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    out = []
    for k in range(steps):
        a = lr * (lr_end / lr) ** (k / max(1, steps - 1))
        mlp.train_step(Xd, Yd, a, loss=loss)
        if k % 50 == 0 or k == steps - 1:
            out.append(float(loss.item()))
    return out


def predict(mlp, cfgs):
    import torch
    X = torch.from_numpy(np.stack([features(c) for c in cfgs])).cuda()
    return [from_target(y) for y in mlp.forward(X).cpu().numpy()]


def profile_error(cells, ref):
    """rms over the inner 3/4 of the cells of (n - n_ref) / mean(n_ref), per species."""
    Nc = ref.shape[1]
    inner = slice(Nc // 8, Nc - Nc // 8)
    return [float(np.sqrt(np.mean((cells[s][inner] - ref[s][inner]) ** 2)) / max(ref[s][inner].mean(), 1.0))
            for s in range(3)]


def experiment(n_train=64, n_held=8, N=20000, cycles=1200, window=100, eval_cycles=600, eval_window=20,
               train_steps=4000, seed=2024, log=print):
    """The warm-start study: cold runs of n_train + n_held discharges of the
    batched sweep's (U, p) ranges (N e + N O- + 2N O2+ each) for `cycles`
    RF cycles give the reference profiles (average of the last `window`
    cycles); the MLP learns the first n_train; each held-out discharge is
    then started warm (predicted profiles) and cold (uniform, new seed) and
    run for `eval_cycles`.  A run has converged once its `eval_window`-cycle
    profile is within tol of the reference, tol = max(0.1, 2 x the
    reference run's own change between its last two windows) (rms over the
    inner cells, per species, largest species).  Returns a summary dict."""
    import time
    import torch
    from . import api, xsec
    procs = xsec.oxygen_set()
    T = (3.0, 0.026, 0.026)
    sweep = inputs.batch_sweep(n_train + n_held, seed=seed, count_range=(N, N))
    runs = [(cfg, cold_state(cfg, counts, T, seed=seed + i)) for i, (cfg, counts, _) in enumerate(sweep)]
    gs = make_discharges(api, runs, procs)
    t0 = time.time()
    ref, hist = run_cycles(api, gs, cycles, window,
                           progress=lambda c, h: log(f"  reference: {c} cycles, {time.time() - t0:.0f} s"))
    t_ref = time.time() - t0
    noise = [max(profile_error(hist[-1][i], hist[-2][i])) for i in range(len(gs))]
    for g in gs:
        g.close()
    log(f"reference runs: {len(gs)} discharges x {cycles} cycles in {t_ref:.1f} s; "
        f"last-window change median {np.median(noise):.3f}")
    train_idx, held = list(range(n_train)), list(range(n_train, n_train + n_held))
    X = np.stack([features(sweep[i][0]) for i in train_idx])
    Y = np.stack([to_target(ref[i]) for i in train_idx])
    mlp = api.MLP([4, 256, 256, 256, 768], seed=seed)
    t0 = time.time()
    losses = train(api, mlp, X, Y, steps=train_steps)
    torch.cuda.synchronize()
    t_train = time.time() - t0
    t0 = time.time()
    pred = predict(mlp, [sweep[i][0] for i in held])
    t_pred = time.time() - t0
    pred_err = [max(profile_error(pred[k], ref[i])) for k, i in enumerate(held)]
    log(f"training {train_steps} Adam steps in {t_train:.2f} s, loss {losses[0]:.3g} -> {losses[-1]:.3g}; "
        f"held-out prediction error median {np.median(pred_err):.3f}")
    cases = []
    for k, i in enumerate(held):
        cfg, counts, _ = sweep[i]
        cases.append((cfg, warm_state(cfg, pred[k], T, seed=seed + 1000 + k)))
        cases.append((cfg, cold_state(cfg, counts, T, seed=seed + 2000 + k)))
    gs = make_discharges(api, cases, procs)
    t0 = time.time()
    _, eh = run_cycles(api, gs, eval_cycles, eval_window,
                       progress=lambda c, h: log(f"  evaluation: {c} cycles, {time.time() - t0:.0f} s"))
    t_eval = time.time() - t0
    for g in gs:
        g.close()
    per = []
    for k, i in enumerate(held):
        tol = max(0.1, 2.0 * noise[i])
        ew = [max(profile_error(eh[w][2 * k], ref[i])) for w in range(len(eh))]
        ec = [max(profile_error(eh[w][2 * k + 1], ref[i])) for w in range(len(eh))]
        first = lambda e: next(((w + 1) * eval_window for w, v in enumerate(e) if v < tol), None)
        per.append({"U": sweep[i][0]["U"], "p": sweep[i][0]["p"], "tol": tol, "warm_cycles": first(ew),
                    "cold_cycles": first(ec), "warm_err": ew, "cold_err": ec, "pred_err": pred_err[k]})
    done = [r for r in per if r["warm_cycles"] and r["cold_cycles"]]
    ratio = [r["cold_cycles"] / r["warm_cycles"] for r in done]
    summary = {"n_train": n_train, "n_held": n_held, "N": N, "cycles": cycles, "window": window,
               "eval_cycles": eval_cycles, "eval_window": eval_window, "train_steps": train_steps,
               "t_reference_s": t_ref, "t_train_s": t_train, "t_predict_s": t_pred, "t_eval_s": t_eval,
               "loss_first": losses[0], "loss_last": losses[-1], "held_out": per,
               "cycle_saving_median": float(np.median(ratio)) if ratio else None,
               "converged_warm": sum(1 for r in per if r["warm_cycles"]),
               "converged_cold": sum(1 for r in per if r["cold_cycles"])}
    log(f"held-out: warm converged {summary['converged_warm']}/{n_held}, cold {summary['converged_cold']}/{n_held}, "
        f"median cycle saving {summary['cycle_saving_median']}")
    mlp.close()
    return summary


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser(description="learned warm start study")
    ap.add_argument("--train", type=int, default=64)
    ap.add_argument("--held", type=int, default=8)
    ap.add_argument("--N", type=int, default=20000)
    ap.add_argument("--cycles", type=int, default=1200)
    ap.add_argument("--window", type=int, default=100)
    ap.add_argument("--eval-cycles", type=int, default=600)
    ap.add_argument("--eval-window", type=int, default=20)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    s = experiment(a.train, a.held, a.N, a.cycles, a.window, a.eval_cycles, a.eval_window, a.steps,
                   log=lambda m: print(m, flush=True))
    if a.out:
        with open(a.out, "w") as f:
            json.dump(s, f, indent=1)
