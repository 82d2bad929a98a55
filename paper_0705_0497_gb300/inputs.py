"""Seeded synthetic workloads: discharge configurations and initial particles.

Input generation only — this module holds none of the method's arithmetic
(no push, no collisions, no field solve).  The CUDA path and the CPU oracle
both take their inputs from here.

The configurations follow the paper's discharge conditions (Sec. 3: L = 2.5 cm,
f = 13.6 MHz, p = 13.8 Pa, U = 250 V; O2 background at T = 300 K, Sec. 2) and
the sizes of the workloads this library is measured on.  Fields the paper
leaves open (macro-particle weight, ion subcycling, initial temperatures,
metastable fraction of the scale runs) are stated with each configuration.
"""
import math

import numpy as np

# CODATA 2018 (SI)
QE = 1.602176634e-19
KB = 1.380649e-23
EPS0 = 8.8541878128e-12
ME = 9.1093837015e-31
AMU = 1.66053906660e-27

E, OM, OP = 0, 1, 2
SPECIES = ("e", "O-", "O2+")


def base_config(**kw):
    """Physical configuration as a plain dict (SI units, energies in eV)."""
    c = dict(L=0.025, f=13.56e6, U=300.0, p=20.0, T_gas=300.0, C_meta=0.05,
             dt=None, weight=1.0e7, area=1.0,
             m_e=ME, m_OM=16.0 * AMU, m_OP=32.0 * AMU, M_gas=32.0 * AMU,
             n_cells=512, ion_subcycle=1, seed=0, steps_per_cycle=1000)
    c.update(kw)
    if c["dt"] is None:
        c["dt"] = 1.0 / (c["f"] * c["steps_per_cycle"])
    return c


# Workloads.  counts = initial macro-particles per species (e, O-, O2+);
# T_eV = initial temperatures (e, O-, O2+); cycles = RF cycles of a full run.
WORKLOADS = {
    # Small parity case: 2 cm gap, 128 cells, 400 steps per RF cycle, 20 cycles.
    # Counts as given: 1e4 e + 2e3 O- + 1e4 O2+ (net charge -2e3 macro-particles);
    # weight 2e9 m^-2 puts n_e at 1e15 m^-3.  No ion subcycling.
    "parity_128": dict(
        cfg=dict(L=0.02, n_cells=128, f=13.56e6, steps_per_cycle=400, U=200.0, p=10.0,
                 C_meta=0.05, ion_subcycle=1, weight=2.0e9, seed=0),
        counts=(10_000, 2_000, 10_000), T_eV=(3.0, 0.026, 0.026), cycles=20),
    # Scale case: 2.5 cm gap, 512 cells, 1000 steps per RF cycle, ions subcycled
    # x10, metastable fraction 5%, 200 cycles, 4e6 electrons and 4e6 O-.
    # Loaded quasi-neutral: O2+ = e + O- = 8e6 (16e6 macro-particles in all);
    # weight 6.25e6 m^-2 gives n_e = n_O- = 1e15 m^-3.
    "scale_512": dict(
        cfg=dict(L=0.025, n_cells=512, f=13.56e6, steps_per_cycle=1000, U=300.0, p=20.0,
                 C_meta=0.05, ion_subcycle=10, weight=6.25e6, seed=0),
        counts=(4_000_000, 4_000_000, 8_000_000), T_eV=(3.0, 0.026, 0.026), cycles=200),
    # Stress case: 3 cm gap, 2048 cells, 2000 steps per cycle, metastable
    # fraction 10%, no subcycling, 3e7 e + 3e7 O- + 6e7 O2+ (quasi-neutral).
    "stress_2048": dict(
        cfg=dict(L=0.03, n_cells=2048, f=13.56e6, steps_per_cycle=2000, U=500.0, p=50.0,
                 C_meta=0.10, ion_subcycle=1, weight=1.0e6, seed=0),
        counts=(30_000_000, 30_000_000, 60_000_000), T_eV=(3.0, 0.026, 0.026), cycles=100),
}


def workload(name, scale=1.0, **over):
    """Configuration + counts of a named workload; `scale` multiplies the
    particle counts and divides the weight (same densities)."""
    w = WORKLOADS[name]
    cfg = base_config(**{**w["cfg"], **over})
    counts = tuple(int(round(n * scale)) for n in w["counts"])
    if scale != 1.0 and "weight" not in over:
        cfg["weight"] = cfg["weight"] / scale
    return cfg, counts, w["T_eV"], w["cycles"]


def batch_sweep(n=64, seed=0, scale=1.0, count_range=(1.0e5, 2.0e6)):
    """A parameter sweep of `n` discharges for the batched stepper: U uniform
    on [100, 500] V, p log-uniform on [5, 50] Pa, and one particle count N per
    discharge, log-uniform on `count_range` (times `scale`), loaded
    quasi-neutral as N e + N O- + 2N O2+.  Fixed: L = 2.5 cm, 256 cells,
    metastable fraction 5%, 1000 steps per RF cycle, ions subcycled x10;
    weight n0 L / N with n0 = 1e15 m^-3; seed of discharge i = seed + i.
    Returns a list of (cfg, counts, T_eV)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lo, hi = count_range
    out = []
    for i in range(n):
        U = float(rng.uniform(100.0, 500.0))
        p = float(math.exp(rng.uniform(math.log(5.0), math.log(50.0))))
        N = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi))) * scale))
        N = max(N, 1)
        cfg = base_config(L=0.025, n_cells=256, steps_per_cycle=1000, U=U, p=p, C_meta=0.05,
                          ion_subcycle=10, weight=1.0e15 * 0.025 / N, seed=seed + i)
        out.append((cfg, (N, N, 2 * N), (3.0, 0.026, 0.026)))
    return out


def majorant_caps(cfg):
    """Majorant caps (eV) of the null-collision method per species (see
    o2pic_set_majorant_cap): none for the electrons; 2 |U| + 50 eV for the
    ions.  An ion's energy relative to a gas molecule stays below e times the
    largest potential difference in the gap (|U| plus the plasma potential,
    a few electron temperatures above the highest electrode) plus its thermal
    energy, so the cap is twice that bound; a candidate above it would be
    counted (warn_numax)."""
    cap = 2.0 * abs(float(cfg["U"])) + 50.0
    return (None, cap, cap)


def species_mass(cfg, s):
    return (cfg["m_e"], cfg["m_OM"], cfg["m_OP"])[s]


def initial_particles(cfg, species, n, T_eV, seed=None, id0=0):
    """n particles of one species: x uniform on [0, L), velocities Maxwellian at
    T_eV (all three components), ids id0..id0+n-1.  float32 arrays."""
    seed = cfg["seed"] if seed is None else seed
    rng = np.random.Generator(np.random.PCG64([int(seed), 1000 + int(species)]))
    L = cfg["L"]
    x = (rng.random(n) * L).astype(np.float32)
    x = np.minimum(x, np.nextafter(np.float32(L), np.float32(0)))
    sig = math.sqrt(QE * T_eV / species_mass(cfg, species))
    v = (rng.standard_normal((3, n)) * sig).astype(np.float32)
    ids = np.arange(id0, id0 + n, dtype=np.uint32)
    return dict(x=x, vx=v[0].copy(), vy=v[1].copy(), vz=v[2].copy(), id=ids)


def initial_state(cfg, counts, T_eV, seed=None):
    """Initial particles of all three species."""
    return [initial_particles(cfg, s, counts[s], T_eV[s], seed) for s in range(3)]


def debye_length(n, T_eV):
    return math.sqrt(EPS0 * T_eV / (n * QE))


def plasma_frequency(n, m=ME):
    return math.sqrt(n * QE * QE / (EPS0 * m))
