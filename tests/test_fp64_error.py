"""Error of the FP32 particle path against the FP64 oracle (CPU only).

The library runs FP32 particles with FP64 field arithmetic and reproduces the
FP32 oracle bit for bit (GPU parity tests), so the error of every library
result against FP64 is the FP32 oracle's error against the FP64 oracle,
measured here on the parity workload (L = 2 cm, 128 cells, 1e4 e + 2e3 O- +
1e4 O2+, the oxygen process set):

* per particle after 100 steps: the same collision events in both precisions,
  relative differences of x, v with median <= 1e-5 and 99th percentile
  <= 2e-3 (the tail: particles whose velocity passes close to zero);
* RF-cycle-averaged densities over the last 5 of 20 cycles: once single
  trajectories have decorrelated (the discharge is chaotic), FP32 and FP64
  are two realizations of the same process, so their difference is compared
  with the seed-to-seed spread of the FP64 oracle itself.
"""
import numpy as np

from paper_0705_0497_gb300 import inputs, xsec


def _oracle(oracle_mod, cfg, st, procs, precision):
    o = oracle_mod.Oracle(cfg, precision)
    o.set_processes(procs)
    for s, p in enumerate(st):
        o.load(s, p["x"], p["vx"], p["vy"], p["vz"], p["id"])
    return o


def test_fp32_vs_fp64_per_particle_100_steps(oracle_mod):
    cfg, counts, T, _ = inputs.workload("parity_128")
    st = inputs.initial_state(cfg, counts, T)
    procs = xsec.oxygen_set()
    o32 = _oracle(oracle_mod, cfg, st, procs, 32)
    o64 = _oracle(oracle_mod, cfg, st, procs, 64)
    o32.step(100)
    o64.step(100)
    c32, c64 = o32.counters(), o64.counters()
    for k in c32:
        assert np.array_equal(np.asarray(c32[k]), np.asarray(c64[k])), k
    for s in range(3):
        a, b = o32.particles(s), o64.particles(s)
        assert np.array_equal(a["id"], b["id"]), s
        for k in ("x", "vx", "vy", "vz"):
            x, y = a[k].astype(np.float64), b[k]
            scale = np.maximum(np.abs(y), np.abs(y).max() * 1e-3 + 1e-30)
            rel = np.abs(x - y) / scale
            med, p99 = float(np.median(rel)), float(np.quantile(rel, 0.99))
            print(f"species {s} {k}: FP32 vs FP64 relative error median {med:.2e}, p99 {p99:.2e}, "
                  f"max {rel.max():.2e}")
            assert med <= 1e-5, (s, k, med)
            assert p99 <= 2e-3, (s, k, p99)


def _cycle_profiles(oracle_mod, precision, seed):
    cfg, counts, T, cycles = inputs.workload("parity_128", seed=seed)
    st = inputs.initial_state(cfg, counts, T, seed=seed)
    o = _oracle(oracle_mod, cfg, st, xsec.oxygen_set(), precision)
    spc = cfg["steps_per_cycle"]
    n = cycles * spc
    warm = n - 5 * spc
    o.step(warm)
    o.reset_moments()
    o.step(n - warm)
    _, Qa, steps = o.charge()
    Ng = cfg["n_cells"] + 1
    dx = cfg["L"] / cfg["n_cells"]
    vol = np.full(Ng, dx * cfg["area"])
    vol[0] = vol[-1] = dx * cfg["area"] / 2
    return Qa / (65536.0 * steps) * cfg["weight"] / vol


def test_fp32_vs_fp64_cycle_averaged_profiles(oracle_mod):
    a32 = _cycle_profiles(oracle_mod, 32, 0)
    a64 = _cycle_profiles(oracle_mod, 64, 0)
    b64 = _cycle_profiles(oracle_mod, 64, 1)
    Ng = a32.shape[1]
    inner = slice(Ng // 8, Ng - Ng // 8)
    for s in range(3):
        scale = a64[s][inner].mean()
        rms = lambda u, v: float(np.sqrt(np.mean((u[s][inner] - v[s][inner]) ** 2)) / scale)
        e_prec, e_seed = rms(a32, a64), rms(b64, a64)
        print(f"species {s}: rms |FP32 - FP64| / mean = {e_prec:.3f}; FP64 seed-to-seed = {e_seed:.3f}")
        assert e_prec <= e_seed, (s, e_prec, e_seed)
    c = Ng // 2
    alpha = [d[1][c - 4:c + 5].mean() / d[0][c - 4:c + 5].mean() for d in (a32, a64, b64)]
    print("centre electronegativity: FP32 %.4f, FP64 %.4f, FP64 other seed %.4f" % tuple(alpha))
    assert abs(alpha[0] - alpha[1]) <= 2 * abs(alpha[2] - alpha[1]) + 0.02
