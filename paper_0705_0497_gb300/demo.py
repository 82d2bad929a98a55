"""The discharge of the paper's Sec. 3 (Figs. 3-5): L = 2.5 cm, f = 13.6 MHz,
p = 13.8 Pa, U = 250 V, without associative detachment (C = 0) and with a
metastable fraction C = 1/6.

With this library's placeholder cross sections (the paper's set is not
published) the result is qualitative only: it is not a reproduction of the
paper's figures and nothing checks it against them.  Both discharges run
together through the batched stepper; the script prints the cycle-averaged
density profiles (coarse table), the centre electronegativity n_O-/n_e, the
current densities of five RF cycles and the power <U j> A.

    python -m paper_0705_0497_gb300.demo --cycles 3000 --N 100000 --out demo.json
"""
import argparse
import json
import math
import time

import numpy as np

from . import api, inputs, xsec


def configs(N, seed=0):
    out = []
    for k, C in enumerate((0.0, 1.0 / 6.0)):
        cfg = inputs.base_config(L=0.025, n_cells=256, f=13.6e6, steps_per_cycle=1000, U=250.0, p=13.8,
                                 C_meta=C, ion_subcycle=10, weight=1.0e15 * 0.025 / N, seed=seed + k)
        out.append((cfg, (N, N, 2 * N), (3.0, 0.026, 0.026)))
    return out


def run(N=100000, cycles=3000, avg_cycles=200, seed=0, log=print):
    procs = xsec.oxygen_set()
    gs = []
    for cfg, counts, T in configs(N, seed):
        g = api.Discharge(cfg, tuple(6 * n + (1 << 20) for n in counts), compact_check=20)
        g.set_processes(procs)
        g.load_state(inputs.initial_state(cfg, counts, T, seed=cfg["seed"]))
        gs.append(g)
    spc, K = 1000, 200
    b = api.Batch(gs, K)
    b.autotune()
    t0 = time.time()
    b.step((cycles - avg_cycles) * spc // K)
    b.synchronize()
    for g in gs:
        g.moments(reset=True)
    b.step(avg_cycles * spc // K)
    b.synchronize()
    wall = time.time() - t0
    res = []
    for g, (cfg, _, _) in zip(gs, configs(N, seed)):
        dens, steps = g.moments()
        n = g.stats()["step"]
        J = g.currents(n - 5 * spc, 5 * spc)
        t_half = (np.arange(n - 5 * spc, n) + 0.5) * cfg["dt"]
        V = cfg["U"] * np.sin(2.0 * math.pi * cfg["f"] * t_half)
        power = float(np.mean(V * J[:, 4]) * cfg["area"])
        c = dens.shape[1] // 2
        alpha = float(dens[1][c - 4:c + 5].mean() / max(dens[0][c - 4:c + 5].mean(), 1.0))
        res.append({"C_meta": cfg["C_meta"], "density_m3": dens.tolist(), "centre_electronegativity": alpha,
                    "centre_density_m3": [float(dens[s][c - 4:c + 5].mean()) for s in range(3)],
                    "current_density_A_m2": J[::10].tolist(), "power_W": power,
                    "live": [g.count(s) for s in range(3)]})
        log(f"C = {cfg['C_meta']:.3f}: centre n_e {res[-1]['centre_density_m3'][0]:.3e}, "
            f"n_O- {res[-1]['centre_density_m3'][1]:.3e}, n_O2+ {res[-1]['centre_density_m3'][2]:.3e} m^-3, "
            f"alpha {alpha:.2f}, <U j> A = {power:.3g} W")
    b.close()
    return {"N": N, "cycles": cycles, "avg_cycles": avg_cycles, "wall_s": wall, "runs": res}


def table(res, cols=16):
    """Coarse text table of the cycle-averaged profiles (m^-3)."""
    lines = []
    for r in res["runs"]:
        d = np.asarray(r["density_m3"])
        idx = np.linspace(0, d.shape[1] - 1, cols).astype(int)
        lines.append(f"C = {r['C_meta']:.3f}")
        for s, name in enumerate(("e", "O-", "O2+")):
            lines.append(f"  {name:4s}" + " ".join(f"{d[s][i]:8.2e}" for i in idx))
    return "\n".join(lines)


if __name__ == "__main__":
    ap = argparse.ArgumentParser(description="the paper's discharge, C = 0 and C = 1/6")
    ap.add_argument("--N", type=int, default=100000)
    ap.add_argument("--cycles", type=int, default=3000)
    ap.add_argument("--avg", type=int, default=200)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    r = run(a.N, a.cycles, a.avg)
    print(table(r))
    if a.out:
        with open(a.out, "w") as f:
            json.dump(r, f)
