"""Learned warm start of a discharge (no counterpart in the paper).

A run of the method starts from uniform, Maxwellian particles and needs many
RF cycles until its cycle-averaged density profiles stop changing.  Here a
small MLP (`api.MLP`: the library's own forward, backward and Adam kernels)
learns, from runs the method itself produced, the map

    (U, p, L, C)  ->  cycle-averaged log densities of e, O-, O2+ on the cells
                      and their log mean energies on 32 bins,

and a new run is loaded from the predicted profiles instead of uniformly
(positions from the densities, Maxwellian velocities at two thirds of the
local mean energy).  The cold start stays the fallback and the reference
for the error: a warm-started run is still the method, only its initial
condition differs.

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


def make_discharges(api, runs, procs, capacity_factor=8, compact_check=200, n_floor=1000):
    """Library contexts for [(cfg, state)] (all processes set, particles
    loaded); capacity_factor slots per loaded particle, counted as at least
    n_floor (a warm start may load few of a species that then grows)."""
    gs = []
    for cfg, st in runs:
        n = [len(p["x"]) for p in st]
        g = api.Discharge(cfg, tuple(capacity_factor * max(k, n_floor) + 65536 for k in n),
                          compact_check=compact_check)
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


BINS = 32
E_FLOOR = 1.0e-3            # eV: mean energies below are clipped before the log


def binned(cells, bins=BINS):
    """Bin averages [3][bins] of cell profiles [3][Nc]."""
    c = np.asarray(cells, np.float64)
    return c.reshape(c.shape[0], bins, -1).mean(axis=2)


def binned_error(cells, ref, bins=BINS):
    """rms over the inner 3/4 of the bins of (n - n_ref) / mean(n_ref), per species."""
    a, b = binned(cells, bins), binned(ref, bins)
    inner = slice(bins // 8, bins - bins // 8)
    return [float(np.sqrt(np.mean((a[s][inner] - b[s][inner]) ** 2)) / max(b[s][inner].mean(), 1.0))
            for s in range(3)]


def energy_profiles(g, cfg, bins=BINS):
    """Mean kinetic energy [eV] of each species on the bins, from the live
    particles of a discharge (a snapshot)."""
    out = np.zeros((3, bins))
    for s in range(3):
        p = g.particles(s)
        if len(p["x"]) == 0:
            continue
        m = inputs.species_mass(cfg, s)
        e = 0.5 * m * (p["vx"].astype(np.float64) ** 2 + p["vy"] ** 2 + p["vz"] ** 2) / inputs.QE
        k = np.minimum((p["x"] / cfg["L"] * bins).astype(np.int64), bins - 1)
        cnt = np.bincount(k, minlength=bins)
        out[s] = np.bincount(k, weights=e, minlength=bins) / np.maximum(cnt, 1)
    return out


def to_target2(cells, energy):
    return np.concatenate([to_target(cells),
                           np.log(np.maximum(np.asarray(energy, np.float64), E_FLOOR)).astype(np.float32).ravel()])


def from_target2(y, n_cells=N_CELLS, bins=BINS):
    y = np.asarray(y, np.float64)
    return from_target(y[:3 * n_cells]), np.exp(y[3 * n_cells:]).reshape(3, bins)


def warm_state2(cfg, cells, energy, seed, T_floor=(0.05, 0.026, 0.026)):
    """Particles drawn from cell densities [3][Nc] (stochastic rounding per
    cell, uniform within the cell) with isotropic Maxwellian velocities at
    the local temperature (2/3) <E> of their bin."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Nc = cells.shape[1]
    bins = energy.shape[1]
    dx = cfg["L"] / Nc
    out = []
    for s in range(3):
        mean = cells[s] * dx * cfg["area"] / cfg["weight"]
        k = np.floor(mean + rng.random(Nc)).astype(np.int64)
        n = int(k.sum())
        c = np.repeat(np.arange(Nc), k)
        x = ((c + rng.random(n)) * dx).astype(np.float32)
        x = np.minimum(x, np.float32(cfg["L"]) * np.float32(1 - 2 ** -23))
        T = np.maximum(2.0 / 3.0 * energy[s][np.minimum(c * bins // Nc, bins - 1)], T_floor[s])
        sig = np.sqrt(T * inputs.QE / inputs.species_mass(cfg, s))
        v = (rng.standard_normal((3, n)) * sig).astype(np.float32)
        out.append(dict(x=x, vx=v[0].copy(), vy=v[1].copy(), vz=v[2].copy(), id=np.arange(n, dtype=np.uint32)))
    return out


def run_windows(api, gs, cycles, window, steps_per_launch=200, tune=True, snapshots=0, live=None):
    """Advance the discharges together; per `window` cycles the cycle-averaged
    cell densities of each, the wall time at the end of each window, and (if
    snapshots) the mean-energy profiles averaged over that many snapshots in
    the last window; `live` (a list), if given, gets the live particle counts
    of each discharge at the end of each window."""
    import time
    spc = gs[0].cfg["steps_per_cycle"]
    per_cycle = spc // steps_per_launch
    b = api.Batch(gs, steps_per_launch)
    if tune:
        b.autotune()
        b.synchronize()
    hist, walls, en = [], [], None
    t0 = time.perf_counter()
    nwin = (cycles + window - 1) // window
    for w in range(nwin):
        c = min(window, cycles - w * window)
        for g in gs:
            g.moments(reset=True)
        if snapshots and w == nwin - 1:
            en = [np.zeros((3, BINS)) for _ in gs]
            per = max(1, c // snapshots)
            done = 0
            while done < c:
                k = min(per, c - done)
                b.step(per_cycle * k)
                b.synchronize()
                for i, g in enumerate(gs):
                    en[i] += energy_profiles(g, g.cfg) / snapshots
                done += k
        else:
            b.step(per_cycle * c)
        b.synchronize()
        walls.append(time.perf_counter() - t0)
        hist.append([cell_profiles(g.moments()[0]) for g in gs])
        if live is not None:
            live.append([[g.count(sp) for sp in range(3)] for g in gs])
    b.close()
    return hist, walls, en


def study_sweep(total, N, seed, p_range=(5.0, 50.0), C_range=(0.05, 1.0 / 6.0), U_range=(100.0, 500.0)):
    """Discharges with U uniform on U_range, p log-uniform on p_range, L
    uniform on [2, 3] cm and C uniform on C_range, N particles per species
    loaded at 1e15 m^-3 (the batched sweep's other settings)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sweep = inputs.batch_sweep(total, seed=seed, count_range=(N, N))
    for cfg, counts, _ in sweep:
        cfg["U"] = float(rng.uniform(*U_range))
        cfg["L"] = float(rng.uniform(0.02, 0.03))
        cfg["C_meta"] = float(rng.uniform(*C_range))
        cfg["p"] = float(math.exp(rng.uniform(math.log(p_range[0]), math.log(p_range[1]))))
        cfg["weight"] = 1.0e15 * cfg["L"] / N
        cfg["dt"] = 1.0 / (cfg["f"] * cfg["steps_per_cycle"])
    return sweep


def cold_survey(api, sweep, idx, N, cycles, window, seed, capacity_factor=20, log=print):
    """Cold runs of the discharges sweep[idx] for `cycles` RF cycles: per
    window the binned density profiles [windows][runs][3][BINS] and live
    counts, the change between the last two windows, and the training
    targets (log densities of the mean of the last two windows, log mean
    energies from snapshots of the last one)."""
    import time
    from . import xsec
    T = (3.0, 0.026, 0.026)
    t0 = time.perf_counter()
    runs = [(sweep[i][0], cold_state(sweep[i][0], sweep[i][1], T, seed=seed + i)) for i in idx]
    gs = make_discharges(api, runs, xsec.oxygen_set(), capacity_factor=capacity_factor, n_floor=N)
    live = []
    h, _, en = run_windows(api, gs, cycles, window, snapshots=5, live=live)
    for g in gs:
        g.close()
    sec = time.perf_counter() - t0
    n = len(idx)
    ref = [0.5 * (h[-1][k] + h[-2][k]) for k in range(n)]
    out = {"idx": np.array(idx), "seconds": sec,
           "X": np.stack([features(sweep[i][0]) for i in idx]),
           "Y": np.stack([to_target2(ref[k], en[k]) for k in range(n)]),
           "binned": np.array([[binned(h[w][k]) for k in range(n)] for w in range(len(h))]),
           "live": np.array(live), "change": np.array([max(binned_error(h[-1][k], h[-2][k])) for k in range(n)])}
    log(f"cold survey: {n} runs x {cycles} cycles in {sec:.0f} s; last-window change median "
        f"{np.median(out['change']):.4f}, below 0.02: {int((out['change'] < 0.02).sum())}")
    return out


def study2(n0=48, n1=96, n_held=32, N=100000, ref_cycles=4000, boot_cycles=1000, eval_cycles=1000, window=200,
           tol=0.02, accept=None, train_steps=6000, seed=4242, p_range=(5.0, 50.0), C_range=(0.05, 1.0 / 6.0),
           U_range=(100.0, 500.0), capacity_factor=20, phase1=None, log=print, save=None):
    """The warm-start study at the 2 % criterion.

    1. n0 discharges of the sweep (`study_sweep`) started cold run ref_cycles
       (`cold_survey`; or its saved result `phase1`, a dict of arrays); the
       mean of the last two windows (`window` cycles each) is the reference,
       kept for training if the change between the two is below `accept`
       (default tol; the windows' own noise sets how low it can be), with
       mean-energy profiles from snapshots.
    2. The network (4 -> 256 x 3 -> 3 x 256 log densities + 3 x 32 log mean
       energies) learns them; n1 more discharges start warm from it and run
       boot_cycles; the converged ones join the training set (the method
       produces them, faster); the network learns all.
    3. n_held held-out discharges start warm (batched) and cold (batched: the
       same results as single runs, bit for bit) and run eval_cycles and
       ref_cycles; the mean of the cold run's last two windows is the
       reference; a run has converged at the first window within tol of it
       (rms over the inner bins, the largest of the three species).
    4. Wall time: the plain cold start on its own (a one-discharge step graph)
       is timed per cycle on a few held-out discharges; a cold run's wall time
       = its cycles to converge x that; a warm run's = its cycles to converge
       x the warm batch's wall time per cycle / its discharges, plus its share
       of training, inference and loading.

    `save(summary, arrays)` (optional) is called after every phase with the
    results so far (arrays: the phase-1 survey)."""
    import time
    import torch
    from . import api, xsec
    procs = xsec.oxygen_set()
    T = (3.0, 0.026, 0.026)
    total = n0 + n1 + n_held
    sweep = study_sweep(total, N, seed, p_range, C_range, U_range)
    summary = {"n0": n0, "n1": n1, "n_held": n_held, "N": N, "ref_cycles": ref_cycles, "boot_cycles": boot_cycles,
               "eval_cycles": eval_cycles, "window": window, "tol": tol, "bins": BINS, "p_range": list(p_range),
               "C_range": list(C_range), "U_range": list(U_range), "capacity_factor": capacity_factor}

    def converged_change(h, i):
        return max(binned_error(h[-1][i], h[-2][i]))

    # 1. cold references
    if phase1 is None:
        phase1 = cold_survey(api, sweep, list(range(n0)), N, ref_cycles, window, seed, capacity_factor, log)
    arrays = phase1

    def checkpoint():
        if save:
            save(summary, arrays)

    if accept is None:
        accept = tol
    summary["accept"] = accept
    ch0 = np.asarray(phase1["change"])
    keep = np.nonzero(ch0 < accept)[0]
    summary["phase1_all_used"] = len(keep) < 4   # too few converged: learn from all (short test runs)
    if summary["phase1_all_used"]:
        keep = np.arange(len(ch0))
    train_X = [phase1["X"][k] for k in keep]
    train_Y = [phase1["Y"][k] for k in keep]
    summary.update(phase1_s=float(phase1["seconds"]), phase1_kept=int((ch0 < accept).sum()),
                   phase1_change_median=float(np.median(ch0)), phase1_changes=[float(v) for v in ch0])
    log(f"phase 1: kept {summary['phase1_kept']} of {len(ch0)} (change < {accept})")
    checkpoint()
    mlp = api.MLP([4, 256, 256, 256, 3 * N_CELLS + 3 * BINS], seed=seed)
    t1 = time.perf_counter()
    train(api, mlp, np.stack(train_X), np.stack(train_Y), steps=train_steps)
    torch.cuda.synchronize()
    t_train1 = time.perf_counter() - t1

    def predict2(cfgs):
        # no extrapolation beyond the training targets: each output is held
        # to the range it took in the training set (a wild log density or
        # energy would load a discharge far from any the method produced)
        X = torch.from_numpy(np.stack([features(c) for c in cfgs])).cuda()
        Ts = np.stack(train_Y)
        lo, hi = Ts.min(axis=0), Ts.max(axis=0)
        return [from_target2(np.clip(y, lo, hi)) for y in mlp.forward(X).cpu().numpy()]

    # 2. bootstrapped runs, started warm
    t0 = time.perf_counter()
    idx1 = list(range(n0, n0 + n1))
    pred = predict2([sweep[i][0] for i in idx1])
    runs = [(sweep[i][0], warm_state2(sweep[i][0], pred[k][0], pred[k][1], seed=seed + i)) for k, i in enumerate(idx1)]
    gs = make_discharges(api, runs, procs, capacity_factor=capacity_factor, n_floor=N)
    h1, w1, en1 = run_windows(api, gs, boot_cycles, window, snapshots=5)
    for g in gs:
        g.close()
    t_boot = time.perf_counter() - t0
    ch1 = [converged_change(h1, k) for k in range(n1)]
    kept1 = 0
    for k in range(n1):
        if ch1[k] < accept:
            train_X.append(features(sweep[idx1[k]][0]))
            train_Y.append(to_target2(0.5 * (h1[-1][k] + h1[-2][k]), en1[k]))
            kept1 += 1
    log(f"phase 2: {n1} warm runs x {boot_cycles} cycles in {t_boot:.0f} s; converged {kept1}; "
        f"training set {len(train_X)}")
    summary.update(phase2_s=t_boot, phase2_kept=kept1, n_train=len(train_X), phase2_changes=[float(v) for v in ch1])
    checkpoint()
    mlp.close()
    mlp = api.MLP([4, 256, 256, 256, 3 * N_CELLS + 3 * BINS], seed=seed + 1)
    t1 = time.perf_counter()
    losses = train(api, mlp, np.stack(train_X), np.stack(train_Y), steps=train_steps)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    summary.update(train_s=t_train + t_train1, loss_first=losses[0], loss_last=losses[-1])
    log(f"training: {train_steps} Adam steps x 2 in {t_train + t_train1:.1f} s, loss {losses[0]:.3g} -> {losses[-1]:.3g}")

    # 3. held-out: warm (batched) and cold (batched == single), references from the cold runs
    held = list(range(n0 + n1, total))
    t1 = time.perf_counter()
    pred = predict2([sweep[i][0] for i in held])
    t_pred = time.perf_counter() - t1
    t1 = time.perf_counter()
    wruns = [(sweep[i][0], warm_state2(sweep[i][0], pred[k][0], pred[k][1], seed=seed + 10000 + k))
             for k, i in enumerate(held)]
    gw = make_discharges(api, wruns, procs, capacity_factor=capacity_factor, n_floor=N)
    t_load = time.perf_counter() - t1
    log(f"held-out warm loads: {[sum(len(p['x']) for p in st) for _, st in wruns]} particles")
    lw = []
    hw, ww, _ = run_windows(api, gw, eval_cycles, window, live=lw)
    log(f"held-out warm runs: {eval_cycles} cycles in {ww[-1]:.0f} s; largest live count {int(np.max(lw))}")
    summary.update(held_warm_s=ww[-1], held_warm_live_max=int(np.max(lw)))
    checkpoint()
    for g in gw:
        g.close()
    cruns = [(sweep[i][0], cold_state(sweep[i][0], sweep[i][1], T, seed=seed + 20000 + k)) for k, i in enumerate(held)]
    gc = make_discharges(api, cruns, procs, capacity_factor=capacity_factor, n_floor=N)
    hc, wc, _ = run_windows(api, gc, ref_cycles, window)
    log(f"held-out cold runs: {ref_cycles} cycles in {wc[-1]:.0f} s")
    for g in gc:
        g.close()
    # 4. the plain cold start alone: seconds per RF cycle of a one-discharge graph
    single = []
    for k in range(min(3, n_held)):
        i = held[k]
        g = make_discharges(api, [(sweep[i][0], cold_state(sweep[i][0], sweep[i][1], T, seed=seed + 30000 + k))],
                            procs, capacity_factor=capacity_factor, n_floor=N)[0]
        b = api.Batch([g], sweep[i][0]["steps_per_cycle"])
        b.step(2)
        b.synchronize()
        ta = time.perf_counter()
        b.step(20)
        b.synchronize()
        single.append((time.perf_counter() - ta) / 20)
        b.close()
        g.close()
    s_cycle_single = float(np.median(single))
    s_cycle_warm = ww[-1] / eval_cycles / len(held)      # per discharge, in the warm batch
    overhead = (t_train + t_train1 + t_pred + t_load) / len(held)
    per = []
    for k, i in enumerate(held):
        ref = 0.5 * (hc[-1][k] + hc[-2][k])
        ref_change = max(binned_error(hc[-1][k], hc[-2][k]))
        ew = [max(binned_error(hw[w][k], ref)) for w in range(len(hw))]
        ec = [max(binned_error(hc[w][k], ref)) for w in range(len(hc) - 2)]
        first = lambda e: next(((w + 1) * window for w, v in enumerate(e) if v < tol), None)
        cw, cc = first(ew), first(ec)
        rec = {"U": sweep[i][0]["U"], "p": sweep[i][0]["p"], "L": sweep[i][0]["L"], "C": sweep[i][0]["C_meta"],
               "ref_change": ref_change, "pred_err": max(binned_error(pred[k][0], ref)), "warm_cycles": cw,
               "cold_cycles": cc, "warm_err": ew, "cold_err": ec}
        if cw and cc:
            rec["wall_cold_single_s"] = cc * s_cycle_single
            rec["wall_warm_batched_s"] = cw * s_cycle_warm + overhead
            rec["wall_ratio"] = rec["wall_cold_single_s"] / rec["wall_warm_batched_s"]
            rec["cycle_ratio"] = cc / cw
        per.append(rec)
    ok = [r for r in per if "wall_ratio" in r]
    summary.update(held_out=per, s_cycle_single=s_cycle_single, s_cycle_warm_batched=s_cycle_warm,
                   overhead_per_run_s=overhead, predict_s=t_pred, load_s=t_load,
                   converged_warm=sum(1 for r in per if r["warm_cycles"]),
                   converged_cold=sum(1 for r in per if r["cold_cycles"]),
                   wall_ratio_median=float(np.median([r["wall_ratio"] for r in ok])) if ok else None,
                   cycle_ratio_median=float(np.median([r["cycle_ratio"] for r in ok])) if ok else None,
                   ref_change_median=float(np.median([r["ref_change"] for r in per])))
    checkpoint()
    log(f"held-out: warm converged {summary['converged_warm']}/{n_held}, cold {summary['converged_cold']}/{n_held}; "
        f"median cycles cold/warm {summary['cycle_ratio_median']}, wall cold-single/warm-batched "
        f"{summary['wall_ratio_median']}")
    mlp.close()
    return summary


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser(description="learned warm start study at the 2 % criterion")
    ap.add_argument("--n0", type=int, default=48, help="cold reference runs (phase 1)")
    ap.add_argument("--n1", type=int, default=96, help="warm bootstrapped runs (phase 2)")
    ap.add_argument("--held", type=int, default=32, help="held-out discharges")
    ap.add_argument("--N", type=int, default=100000, help="particles loaded per species (cold start)")
    ap.add_argument("--cycles", type=int, default=4000, help="RF cycles of the cold runs")
    ap.add_argument("--boot-cycles", type=int, default=1000)
    ap.add_argument("--eval-cycles", type=int, default=1000, help="RF cycles of the warm held-out runs")
    ap.add_argument("--window", type=int, default=200, help="RF cycles per averaging window")
    ap.add_argument("--steps", type=int, default=6000, help="Adam steps per training")
    ap.add_argument("--accept", type=float, default=None,
                    help="largest change between the last two windows of a run kept for training (default 0.02)")
    ap.add_argument("--p-range", type=float, nargs=2, default=(5.0, 50.0))
    ap.add_argument("--C-range", type=float, nargs=2, default=(0.05, 1.0 / 6.0))
    ap.add_argument("--U-range", type=float, nargs=2, default=(100.0, 500.0))
    ap.add_argument("--survey-only", action="store_true", help="phase 1 only (the cold survey)")
    ap.add_argument("--phase1", default=None, help="phase-1 arrays (.npz) from an earlier run")
    ap.add_argument("--out", default=None, help="JSON summary (rewritten after every phase) and <out>.npz")
    a = ap.parse_args()

    def save(summary, arrays=None):
        if a.out:
            with open(a.out, "w") as f:
                json.dump(summary, f, indent=1)
            if arrays is not None:
                np.savez(a.out.rsplit(".", 1)[0] + ".npz", **arrays)

    log = lambda m: print(m, flush=True)
    if a.survey_only:
        from . import api as _api
        sw = study_sweep(a.n0, a.N, 4242, tuple(a.p_range), tuple(a.C_range), tuple(a.U_range))
        out = cold_survey(_api, sw, list(range(a.n0)), a.N, a.cycles, a.window, 4242, log=log)
        save({"n0": a.n0, "N": a.N, "cycles": a.cycles, "window": a.window, "seconds": out["seconds"],
              "configs": [{k: sw[i][0][k] for k in ("U", "p", "L", "C_meta")} for i in range(a.n0)],
              "change": out["change"].tolist(), "live_last": out["live"][-1].tolist()}, out)
    else:
        ph1 = dict(np.load(a.phase1)) if a.phase1 else None
        study2(n0=a.n0, n1=a.n1, n_held=a.held, N=a.N, ref_cycles=a.cycles, boot_cycles=a.boot_cycles,
               eval_cycles=a.eval_cycles, window=a.window, train_steps=a.steps, p_range=tuple(a.p_range),
               C_range=tuple(a.C_range), U_range=tuple(a.U_range), accept=a.accept, phase1=ph1, log=log,
               save=save)
