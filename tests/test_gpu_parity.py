"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs.  Tolerance: 1e-5 relative per particle (expected and
usually found bit-exact, since both sides round the same FP32 operations in
the same order), identical event counts, integer charge bit-exact."""
import math

import numpy as np
import pytest

from paper_0705_0497_gb300 import inputs, xsec
from helpers import (capacity_for, compare_counters, compare_particles, curand_ref_lib, make_pair, nproc_of)

pytestmark = pytest.mark.gpu

QE, KB, ME, AMU = inputs.QE, inputs.KB, inputs.ME, inputs.AMU


def test_philox_matches_oracle_and_curand(torch_cuda):
    import oracle
    from paper_0705_0497_gb300 import api
    torch = torch_cuda
    rng = np.random.default_rng(0)
    n = 1 << 20
    ctr = rng.integers(0, 2 ** 32, (n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, (n, 2), dtype=np.uint64).astype(np.uint32)
    dc = torch.from_numpy(ctr.view(np.int32)).cuda()
    dk = torch.from_numpy(key.view(np.int32)).cuda()
    out = api.philox(dc, dk).cpu().numpy().view(np.uint32)
    ref = torch.empty_like(dc)
    L = curand_ref_lib()
    assert L.curand_ref_philox(dc.data_ptr(), dk.data_ptr(), ref.data_ptr(), n) == 0
    assert np.array_equal(out, ref.cpu().numpy().view(np.uint32))
    for i in range(0, n, n // 64):
        assert np.array_equal(out[i], oracle.philox(ctr[i], key[i]))


def test_ln_series_bitexact_and_bounded(torch_cuda):
    import oracle
    from paper_0705_0497_gb300 import api
    torch = torch_cuda
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.random(200000).astype(np.float32), np.float32([1.0, 0.5, 2.0 ** -46, 0.7071068])])
    x = x[x > 0]
    got = api.ln_f32(torch.from_numpy(x).cuda()).cpu().numpy()
    for i in range(0, len(x), 997):
        assert got[i] == np.float32(oracle.ln_f32(float(x[i])))
    ref = np.log(x.astype(np.float64))
    tol = 2.0 * np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64) + 2.0 ** -24
    assert np.all(np.abs(got - ref) <= tol)
    # and within the bound of CUDA's own logf (called through torch)
    cu = torch.log(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - cu) <= 2 * tol)


def test_initial_charge_and_field(torch_cuda):
    cfg, counts, T, _ = inputs.workload("parity_128")
    procs = xsec.oxygen_set()
    g, o, st = make_pair(cfg, counts, T, procs)
    Qg, _, _ = g.charge()
    Qo, _, _ = o.charge()
    assert np.array_equal(Qg, Qo)
    phig, Eg = g.field()
    phio, Eo, Ego = o.field()
    assert np.allclose(phig, phio, rtol=0, atol=1e-11 * np.abs(phio).max())
    assert np.allclose(Eg, Ego.astype(np.float32), rtol=2e-6, atol=1e-6 * np.abs(Ego).max())


def test_parity_100_steps(torch_cuda):
    """Parity case (2 cm, 128 cells, 2.2e4 particles), 100 coupled steps."""
    cfg, counts, T, _ = inputs.workload("parity_128")
    procs = xsec.oxygen_set()
    g, o, _ = make_pair(cfg, counts, T, procs)
    for chunk in (1, 9, 40, 50):
        g.step(chunk)
        o.step(chunk)
        compare_particles(g, o)
        compare_counters(g.stats(), o.counters(), nproc_of(procs))
        Qg, _, _ = g.charge()
        Qo, _, _ = o.charge()
        assert np.array_equal(Qg, Qo)
    gs = g.stats()
    assert sum(gs[f"born_{s}"] for s in range(3)) > 0
    assert gs["step"] == 100


@pytest.mark.parametrize("caps,violations", [((2.0, 0.5, 0.5), True), ((None, 600.0, 600.0), False)])
def test_parity_majorant_cap(torch_cuda, caps, violations):
    """Capped majorants: nu_max from the grid points up to the cap on both
    sides, the same candidates, collisions and warn_numax counts; caps far
    below the particles' energies give violations, caps above them none."""
    cfg, counts, T, _ = inputs.workload("parity_128", ion_subcycle=2)
    procs = xsec.oxygen_set()
    g, o, _ = make_pair(cfg, counts, T, procs, caps=caps)
    for chunk in (1, 20, 39):
        g.step(chunk)
        o.step(chunk)
        compare_particles(g, o)
        compare_counters(g.stats(), o.counters(), nproc_of(procs))
    assert (g.stats()["warn_numax"] > 0) == violations


@pytest.mark.parametrize("n", [0, 1, 3, 1023, 1025, 8191, 8193, 20001])
def test_parity_ragged_sizes(torch_cuda, n):
    """Empty, single, ragged and multi-tile particle counts (tiles of 8192,
    chunks of 1024, 4 particles per thread), with ion subcycling."""
    cfg, _, T, _ = inputs.workload("parity_128", ion_subcycle=3)
    counts = (n, n // 3, n)
    procs = xsec.oxygen_set()
    g, o, _ = make_pair(cfg, counts, T, procs, capacity=capacity_for(counts, 3.0, 64))
    g.step(7)
    o.step(7)
    compare_particles(g, o)
    compare_counters(g.stats(), o.counters(), nproc_of(procs))


@pytest.mark.parametrize("Nc", [97, 8192])
def test_parity_grid_sizes(torch_cuda, Nc):
    """A cell count that is not a power of two (the solve divides by N, where
    a power of two multiplies by the exact 1/N) and the largest grid (8192
    cells, 8193 nodes): 30 coupled steps with ion subcycling; particles,
    counters and charge against the oracle, then the field against the
    oracle's closed-form solve of the GPU's charge, bit for bit."""
    import oracle
    cfg, _, T, _ = inputs.workload("parity_128", n_cells=Nc, ion_subcycle=3)
    counts = (6000, 1500, 7500)
    procs = xsec.oxygen_set()
    g, o, _ = make_pair(cfg, counts, T, procs)
    for chunk in (1, 29):
        g.step(chunk)
        o.step(chunk)
        compare_particles(g, o)
        compare_counters(g.stats(), o.counters(), nproc_of(procs))
        Qg, _, _ = g.charge()
        Qo, _, _ = o.charge()
        assert np.array_equal(Qg, Qo)
    Rnet = Qg[2].astype(np.int64) - Qg[0].astype(np.int64) - Qg[1].astype(np.int64)
    V0 = cfg["U"] * math.sin(2.0 * math.pi * cfg["f"] * g.stats()["step"] * cfg["dt"])
    phi64, E64 = oracle.solve_field(Nc, cfg["L"] / Nc, cfg["weight"], cfg["area"], V0, Rnet)
    phi, E = g.field()
    assert np.array_equal(E, E64.astype(np.float32))
    assert np.array_equal(phi, phi64)


def test_parity_walls_and_edges(torch_cuda):
    """Particles exactly at x = 0, just below L and at cell boundaries."""
    cfg, counts, T, _ = inputs.workload("parity_128")
    st = inputs.initial_state(cfg, (3000, 300, 3000), T)
    L = np.float32(cfg["L"])
    dx = cfg["L"] / cfg["n_cells"]
    for p in st:
        k = min(len(p["x"]), 200)
        p["x"][:k:4] = 0.0
        p["x"][1:k:4] = np.nextafter(L, np.float32(0))
        p["x"][2:k:4] = np.float32(dx * 17)
        p["x"][3:k:4] = np.float32(dx * 64)
    procs = xsec.oxygen_set()
    g, o, _ = make_pair(cfg, None, None, procs, state=st)
    g.step(20)
    o.step(20)
    compare_particles(g, o)
    compare_counters(g.stats(), o.counters(), nproc_of(procs))


@pytest.mark.parametrize("n_om,n_op", [(30000, 26000), (26000, 30000), (9000, 8192)])
def test_neutralization_parity(torch_cuda, n_om, n_op):
    """Many (17) reactions: a large constant rate coefficient, ions at rest in
    a few cells, the library's pairing against the oracle's, pair for pair.
    Cases with more O- than O2+ per cell, fewer, and ragged tiles."""
    Nc = 32
    cfg = inputs.base_config(L=0.02, n_cells=Nc, U=0.0, p=10.0, C_meta=0.0, ion_subcycle=2, weight=2e9, seed=3,
                             steps_per_cycle=400)
    dx = cfg["L"] / Nc
    mu = cfg["m_OM"] * cfg["m_OP"] / (cfg["m_OM"] + cfg["m_OP"])
    K0 = 1e-4 * cfg["area"] * dx / (cfg["weight"] * cfg["dt"] * 2)
    procs = [xsec.constant_rate_process(1, xsec.NEUTRALIZE, K0, 1.0, mu, target=xsec.T_ION)]
    rng = np.random.default_rng(7)
    st = []
    for s, n in enumerate((500, n_om, n_op)):
        x = ((rng.integers(0, Nc, n) + 0.05 + 0.9 * rng.random(n)) * dx).astype(np.float32)
        v = (rng.standard_normal((3, n)) * (1e5 if s == 0 else 300.0)).astype(np.float32)
        st.append(dict(x=x, vx=v[0].copy(), vy=v[1].copy(), vz=v[2].copy(), id=np.arange(n, dtype=np.uint32)))
    g, o, _ = make_pair(cfg, None, None, procs, state=st)
    for _ in range(3):
        g.step(2)
        o.step(2)
        compare_particles(g, o)
        compare_counters(g.stats(), o.counters(), nproc_of(procs))
    assert o.counters()["neutralized"] > 0.01 * min(n_om, n_op)


def test_compaction_keeps_order(torch_cuda):
    """A strong field empties slots quickly; the periodic stable compaction
    must keep the array order the method defines."""
    cfg, counts, T, _ = inputs.workload("parity_128", U=2000.0, ion_subcycle=2)
    procs = xsec.oxygen_set()
    g, o, _ = make_pair(cfg, (20000, 5000, 20000), T, procs, compact_check=2)
    for _ in range(6):
        g.step(5)
        o.step(5)
        compare_particles(g, o)
    st = g.stats()
    assert st["slots_0"] < 20000 + st["born_0"]    # compaction happened
    compare_counters(st, o.counters(), nproc_of(procs))


def test_capacity_overflow_is_reported(torch_cuda):
    from paper_0705_0497_gb300 import api
    cfg, counts, T, _ = inputs.workload("parity_128", U=600.0)
    procs = xsec.oxygen_set()
    st = inputs.initial_state(cfg, counts, T)
    g = api.Discharge(cfg, (counts[0], counts[1], counts[2]))
    g.set_processes(procs)
    g.load_state(st)
    with pytest.raises(api.O2picError) as ei:
        g.step(200)
        g.synchronize()
    assert ei.value.code == -2


def test_invalid_load_rejected(torch_cuda):
    from paper_0705_0497_gb300 import api
    cfg, counts, T, _ = inputs.workload("parity_128")
    g = api.Discharge(cfg, (100, 100, 100))
    x = np.full(10, cfg["L"] * 1.5, np.float32)
    z = np.zeros(10, np.float32)
    with pytest.raises(api.O2picError) as ei:
        g.load(0, x, z, z, z, np.arange(10))
    assert ei.value.code == -1
    import torch
    with pytest.raises(api.O2picError) as ei:
        g.load(0, torch.from_numpy(x).cuda(), *(torch.from_numpy(z).cuda() for _ in range(3)),
               torch.arange(10, dtype=torch.int32).cuda())
    assert ei.value.code == -1
    # a non-finite velocity from host memory; the species stays empty and a
    # valid load afterwards is accepted
    xs = np.full(10, cfg["L"] * 0.5, np.float32)
    vbad = z.copy()
    vbad[7] = np.inf
    with pytest.raises(api.O2picError) as ei:
        g.load(0, xs, z, vbad, z, np.arange(10))
    assert ei.value.code == -1
    assert g.count(0) == 0
    g.load(0, xs, z, z, z, np.arange(10))
    assert g.count(0) == 10


def test_long_run_profiles(torch_cuda):
    """Parity case over its full 20 RF cycles: cycle-averaged density profiles
    and the centre electronegativity n_O-/n_e within 2% of the oracle; the
    deviation of the FP32 path from the FP64 oracle is reported."""
    import oracle
    cfg, counts, T, cycles = inputs.workload("parity_128")
    procs = xsec.oxygen_set()
    g, o, st = make_pair(cfg, counts, T, procs)
    o64 = oracle.Oracle(cfg, 64)
    o64.set_processes(procs)
    for s, p in enumerate(st):
        o64.load(s, p["x"], p["vx"], p["vy"], p["vz"], p["id"])
    spc = cfg["steps_per_cycle"]
    nsteps = cycles * spc
    warm = nsteps - 5 * spc
    g.step(warm)
    o.step(warm)
    o64.step(warm)
    g.moments(reset=True)
    o.reset_moments()
    o64.reset_moments()
    g.step(nsteps - warm)
    o.step(nsteps - warm)
    o64.step(nsteps - warm)
    # same arithmetic on both sides: the whole run stays particle-for-particle equal
    compare_particles(g, o)
    dg, ng = g.moments()
    _, Qa, no = o.charge()
    _, Qa64, no64 = o64.charge()
    assert ng == no == no64 == nsteps - warm
    Ng = cfg["n_cells"] + 1
    dx = cfg["L"] / cfg["n_cells"]
    vol = np.full(Ng, dx * cfg["area"])
    vol[0] = vol[-1] = dx * cfg["area"] / 2
    do = Qa / (65536.0 * no) * cfg["weight"] / vol
    d64 = Qa64 / (65536.0 * no64) * cfg["weight"] / vol
    inner = slice(Ng // 8, Ng - Ng // 8)
    for s in range(3):
        scale = do[s].max()
        if scale == 0:
            continue
        err = np.abs(dg[s] - do[s])[inner].max() / scale
        assert err < 0.02, (s, err)
        err64 = np.abs(dg[s] - d64[s])[inner].max() / scale
        print(f"species {s}: max |GPU - oracle32| / max = {err:.3e}, vs FP64 oracle = {err64:.3e}")
    c = Ng // 2
    alpha_g = dg[1][c - 4:c + 5].mean() / dg[0][c - 4:c + 5].mean()
    alpha_o = do[1][c - 4:c + 5].mean() / do[0][c - 4:c + 5].mean()
    alpha_64 = d64[1][c - 4:c + 5].mean() / d64[0][c - 4:c + 5].mean()
    print(f"centre electronegativity: GPU {alpha_g:.4f}, oracle32 {alpha_o:.4f}, oracle64 {alpha_64:.4f}")
    assert abs(alpha_g / alpha_o - 1) < 0.02


def _expected_currents(cfg, sums, first):
    """Current densities from the oracle's exact sums, with the library's
    FP64 expressions (conduction: q_s e w sum / (256 A L); displacement:
    eps0 (V(t_{n+1}) - V(t_n)) / (L dt) with V = U sin(2 pi f t))."""
    EPS0 = inputs.EPS0
    unit = QE * cfg["weight"] / (256.0 * cfg["area"] * cfg["L"])
    out = np.zeros((len(sums), 5))
    for i, row in enumerate(sums):
        k = first + i
        tot = 0.0
        for s, q in enumerate((-1, -1, 1)):
            out[i, s] = (float(q) * unit) * float(row[s])
            tot += out[i, s]
        v0 = cfg["U"] * math.sin(2.0 * math.pi * cfg["f"] * (k * cfg["dt"]))
        v1 = cfg["U"] * math.sin(2.0 * math.pi * cfg["f"] * ((k + 1) * cfg["dt"]))
        out[i, 3] = EPS0 * (v1 - v0) / (cfg["L"] * cfg["dt"])
        out[i, 4] = tot + out[i, 3]
    return out


@pytest.mark.parametrize("S", [1, 3])
def test_current_densities_match_oracle(torch_cuda, S):
    """Fig. 5 diagnostics: per-step conduction-current sums of every species
    bit-exact with the oracle (ions repeating between their pushes when
    subcycled), the displacement current from the prescribed voltage, and
    the total."""
    cfg, counts, T, _ = inputs.workload("parity_128", ion_subcycle=S)
    procs = xsec.oxygen_set()
    g, o, _ = make_pair(cfg, counts, T, procs)
    g.step(60)
    o.step(60)
    J = g.currents(0, 60)
    E = _expected_currents(cfg, o.current_sums(0, 60), 0)
    assert np.array_equal(J[:, :3], E[:, :3])
    assert np.allclose(J[:, 3:], E[:, 3:], rtol=1e-12, atol=0)
    if S > 1:
        assert J[1, 1] == J[0, 1] and J[1, 2] == J[0, 2]
    # window: the last 8191 steps since the load
    from paper_0705_0497_gb300 import api
    with pytest.raises(api.O2picError):
        g.currents(55, 10)


@pytest.mark.parametrize("n_e,n_op", [(30000, 26000), (20000, 30000)])
def test_recombination_parity(torch_cuda, n_e, n_op):
    """(16) e + O2+ with a large constant rate coefficient, run before (17)
    on the same ion steps: the library's pairing against the oracle's, pair
    for pair, and both counters.  (A small weight keeps the space-charge
    field negligible; the acceptance probability does not depend on it.)"""
    Nc = 32
    cfg = inputs.base_config(L=0.02, n_cells=Nc, U=0.0, p=10.0, C_meta=0.0, ion_subcycle=2, weight=1e3, seed=5,
                             steps_per_cycle=400)
    dx = cfg["L"] / Nc
    mur = cfg["m_e"] * cfg["m_OP"] / (cfg["m_e"] + cfg["m_OP"])
    mun = cfg["m_OM"] * cfg["m_OP"] / (cfg["m_OM"] + cfg["m_OP"])
    K0 = 1e-4 * cfg["area"] * dx / (cfg["weight"] * cfg["dt"] * 2)
    procs = [xsec.constant_rate_process(0, xsec.RECOMBINE, K0, 1.0, mur, target=xsec.T_ION),
             xsec.constant_rate_process(1, xsec.NEUTRALIZE, K0, 1.0, mun, target=xsec.T_ION)]
    rng = np.random.default_rng(9)
    st = []
    for s, n in enumerate((n_e, 8000, n_op)):
        x = ((rng.integers(0, Nc, n) + 0.05 + 0.9 * rng.random(n)) * dx).astype(np.float32)
        v = (rng.standard_normal((3, n)) * (3e4 if s == 0 else 300.0)).astype(np.float32)
        st.append(dict(x=x, vx=v[0].copy(), vy=v[1].copy(), vz=v[2].copy(), id=np.arange(n, dtype=np.uint32)))
    g, o, _ = make_pair(cfg, None, None, procs, state=st)
    for _ in range(3):
        g.step(2)
        o.step(2)
        compare_particles(g, o)
        compare_counters(g.stats(), o.counters(), nproc_of(procs))
    c = o.counters()
    assert c["recombined"] > 0.01 * min(n_e, n_op) and c["neutralized"] > 0


@pytest.mark.parametrize("n_e,n_om", [(30000, 26000), (20000, 30000)])
def test_edetach_parity(torch_cuda, n_e, n_om):
    """(22) e + O- -> O + 2e with a large constant rate coefficient, before
    (16) and (17) on the same ion steps: pairs, kinematics and newborns (their
    order and free flights) against the oracle, particle for particle, and
    every counter.  A threshold-carrying (22) runs in the second case."""
    Nc = 32
    cfg = inputs.base_config(L=0.02, n_cells=Nc, U=0.0, p=10.0, C_meta=0.0, ion_subcycle=2, weight=1e3, seed=7,
                             steps_per_cycle=400)
    dx = cfg["L"] / Nc
    mud = cfg["m_e"] * cfg["m_OM"] / (cfg["m_e"] + cfg["m_OM"])
    mur = cfg["m_e"] * cfg["m_OP"] / (cfg["m_e"] + cfg["m_OP"])
    mun = cfg["m_OM"] * cfg["m_OP"] / (cfg["m_OM"] + cfg["m_OP"])
    K0 = 1e-4 * cfg["area"] * dx / (cfg["weight"] * cfg["dt"] * 2)
    thr = 0.0 if n_e > n_om else xsec.O_AFFINITY_EV
    procs = [xsec.constant_rate_process(1, xsec.EDETACH, K0, 1.0, mud, target=xsec.T_ELECTRON, thr=thr),
             xsec.constant_rate_process(0, xsec.RECOMBINE, K0, 1.0, mur, target=xsec.T_ION),
             xsec.constant_rate_process(1, xsec.NEUTRALIZE, K0, 1.0, mun, target=xsec.T_ION)]
    rng = np.random.default_rng(11)
    st = []
    for s, n in enumerate((n_e, n_om, 8000)):
        x = ((rng.integers(0, Nc, n) + 0.05 + 0.9 * rng.random(n)) * dx).astype(np.float32)
        v = (rng.standard_normal((3, n)) * (1e6 if s == 0 else 300.0)).astype(np.float32)
        st.append(dict(x=x, vx=v[0].copy(), vy=v[1].copy(), vz=v[2].copy(), id=np.arange(n, dtype=np.uint32)))
    g, o, _ = make_pair(cfg, None, None, procs, state=st)
    for _ in range(3):
        g.step(2)
        o.step(2)
        compare_particles(g, o)
        compare_counters(g.stats(), o.counters(), nproc_of(procs))
    c = o.counters()
    assert c["edetached"] > 0.005 * min(n_e, n_om) and c["recombined"] > 0 and c["neutralized"] > 0


def test_oxygen_set_with_edetach_100_steps(torch_cuda):
    """The full process set with (16) and (22) added: 100 steps of the parity
    case, per particle and every counter."""
    cfg, counts, T, _ = inputs.workload("parity_128", ion_subcycle=2)
    procs = xsec.oxygen_set(include_rec=True, include_edet=True)
    g, o, _ = make_pair(cfg, counts, T, procs)
    g.step(100)
    o.step(100)
    compare_particles(g, o)
    compare_counters(g.stats(), o.counters(), nproc_of(procs))
    assert o.counters()["edet_candidates"] > 0


def test_oxygen_set_with_recombination_100_steps(torch_cuda):
    """The full process set with (16) added: 100 steps of the parity case,
    per particle and every counter."""
    cfg, counts, T, _ = inputs.workload("parity_128", ion_subcycle=2)
    procs = xsec.oxygen_set(include_rec=True)
    g, o, _ = make_pair(cfg, counts, T, procs)
    g.step(100)
    o.step(100)
    compare_particles(g, o)
    compare_counters(g.stats(), o.counters(), nproc_of(procs))
    assert o.counters()["rec_candidates"] > 0


@pytest.mark.parametrize("save_at,S,check", [(40, 2, 16), (41, 10, 16), (43, 10, 7)])
def test_checkpoint_and_resume_bit_for_bit(torch_cuda, save_at, S, check):
    """Saving the particles, step and next ids after `save_at` steps and
    resuming them in a new context gives, 40 steps later, exactly the
    uninterrupted run (the random streams are keyed by id and step only):
    also when the save falls between two ion steps (the resumed context
    re-deposits the ions' charge, which must equal the charge the
    uninterrupted run kept) and between two compaction checks."""
    from paper_0705_0497_gb300 import api
    cfg, counts, T, _ = inputs.workload("parity_128", ion_subcycle=S)
    procs = xsec.oxygen_set(include_rec=True)
    st = inputs.initial_state(cfg, counts, T)
    cap = capacity_for(counts)
    a = api.Discharge(cfg, cap, compact_check=check)
    a.set_processes(procs)
    a.load_state(st)
    a.step(save_at)
    saved = [a.particles(s, flight=True) for s in range(3)]
    s40 = a.stats()
    a.step(40)
    b = api.Discharge(cfg, cap, compact_check=check)
    b.set_processes(procs)
    b.load_state(saved)
    b.set_step(s40["step"])
    for s in range(3):
        b.set_next_id(s, s40[f"next_id_{s}"])
    b.step(40)
    for s in range(3):
        pa, pb = a.particles(s, flight=True), b.particles(s, flight=True)
        for k in ("x", "vx", "vy", "vz", "id", "tc"):
            assert np.array_equal(pa[k], pb[k]), (s, k)
    assert np.array_equal(a.field()[1], b.field()[1])
