"""Host-side pieces of the learned warm start (no GPU): the profile error that
defines convergence at 2 %, the network's target encoding, the sweep of the
study and the particles loaded from a predicted profile."""
import math

import numpy as np

from paper_0705_0497_gb300 import inputs, warmstart as W


def test_binned_error_is_relative_rms_of_the_inner_bins():
    # flat reference: a uniform 2 % excess is an error of exactly 0.02 in
    # that species; the largest species is what the study compares
    ref = np.full((3, W.N_CELLS), 1.0e15)
    a = ref.copy()
    a[1] *= 1.02
    e = W.binned_error(a, ref)
    assert e[0] == 0.0 and e[2] == 0.0
    assert abs(e[1] - 0.02) < 1e-12
    # the outer eighth on each side (the sheaths) does not count
    b = ref.copy()
    b[0, : W.N_CELLS // 8] *= 10.0
    b[0, -(W.N_CELLS // 8):] *= 10.0
    assert max(W.binned_error(b, ref)) == 0.0
    # one inner bin off by 24 %: rms over 24 inner bins = 0.24 / sqrt(24)
    c = ref.copy()
    k = W.N_CELLS // W.BINS
    c[2, 10 * k:11 * k] *= 1.24
    assert abs(W.binned_error(c, ref)[2] - 0.24 / math.sqrt(24)) < 1e-12


def test_targets_round_trip():
    rng = np.random.default_rng(3)
    cells = 10 ** rng.uniform(13, 16, (3, W.N_CELLS))
    energy = rng.uniform(0.03, 20.0, (3, W.BINS))
    c2, e2 = W.from_target2(W.to_target2(cells, energy))
    assert np.allclose(c2, cells, rtol=1e-5) and np.allclose(e2, energy, rtol=1e-5)
    # densities below the floor are clipped, not lost to log(0)
    z = cells.copy()
    z[0, :5] = 0.0
    c3, _ = W.from_target2(W.to_target2(z, energy))
    assert np.allclose(c3[0, :5], W.LOG_FLOOR, rtol=1e-5)


def test_study_sweep_ranges():
    sw = W.study_sweep(200, 1000, seed=9, p_range=(30.0, 50.0), C_range=(0.1, 1 / 6), U_range=(100.0, 300.0))
    U = np.array([c["U"] for c, _, _ in sw])
    p = np.array([c["p"] for c, _, _ in sw])
    L = np.array([c["L"] for c, _, _ in sw])
    C = np.array([c["C_meta"] for c, _, _ in sw])
    assert U.min() >= 100 and U.max() <= 300 and p.min() >= 30 and p.max() <= 50
    assert L.min() >= 0.02 and L.max() <= 0.03 and C.min() >= 0.1 and C.max() <= 1 / 6
    # p log-uniform: its log has the mean of the log range
    assert abs(np.log(p).mean() - 0.5 * (math.log(30) + math.log(50))) < 0.03
    for cfg, counts, _ in sw:
        assert tuple(counts)[:1] == (1000,)
        assert abs(cfg["dt"] * cfg["f"] * cfg["steps_per_cycle"] - 1.0) < 1e-12
    X = np.stack([W.features(c) for c, _, _ in sw])
    assert np.all(np.abs(X) <= 1.0 + 1e-6)


def test_warm_state_follows_the_profile():
    cfg = W.study_sweep(1, 1000, seed=1)[0][0]
    Nc = cfg["n_cells"]
    x_c = (np.arange(Nc) + 0.5) / Nc
    dens = np.stack([2e15 * np.sin(np.pi * x_c) + 1e13, 5e14 * np.ones(Nc), 3e15 * np.sin(np.pi * x_c) + 1e13])
    energy = np.stack([np.full(W.BINS, 3.0), np.full(W.BINS, 0.03), np.full(W.BINS, 0.6)])
    st = W.warm_state2(cfg, dens, energy, seed=5)
    dx = cfg["L"] / Nc
    for s in range(3):
        p = st[s]
        want = dens[s].sum() * dx * cfg["area"] / cfg["weight"]
        n = len(p["x"])
        assert abs(n - want) < 5 * math.sqrt(want) + 1
        assert p["x"].min() >= 0 and p["x"].max() < cfg["L"]
        assert np.array_equal(p["id"], np.arange(n, dtype=np.uint32))
        # velocities: Maxwellian at T = max(2/3 <E>, the species' floor), so
        # <m v^2 / 2> = 3/2 T (the floor lifts the O- at 0.03 eV to 0.026 eV)
        T = max(2.0 / 3.0 * energy[s][0], (0.05, 0.026, 0.026)[s])
        m = inputs.species_mass(cfg, s)
        e = 0.5 * m * (p["vx"].astype(np.float64) ** 2 + p["vy"] ** 2 + p["vz"] ** 2) / inputs.QE
        assert abs(e.mean() / (1.5 * T) - 1.0) < 5 * math.sqrt(2 / 3 / n) + 0.01
