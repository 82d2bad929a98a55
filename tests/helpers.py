"""Shared helpers of the GPU tests: run the same seeded workload through the
CUDA library and the oracle and compare."""
import os
import subprocess

import numpy as np

from paper_0705_0497_gb300 import inputs, xsec

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
COUNTERS_COMPARED = ("neutralized", "pair_candidates", "particle_steps", "warn_emax", "warn_tries", "warn_pair_gt1",
                     "recombined", "rec_candidates", "id_overflow", "edetached", "edet_candidates",
                     "coulomb_pairs", "warn_numax")


def capacity_for(counts, factor=2.0, extra=4096):
    return tuple(int(n * factor) + extra for n in counts)


def make_pair(cfg, counts, T_eV, procs, capacity=None, compact_check=0, state=None, caps=None):
    """A library context and an FP32 oracle loaded with the same particles
    (caps: majorant caps per species in eV, or None)."""
    import oracle
    from paper_0705_0497_gb300 import api
    st = state if state is not None else inputs.initial_state(cfg, counts, T_eV)
    g = api.Discharge(cfg, capacity or capacity_for([len(p["x"]) for p in st]), compact_check=compact_check)
    o = oracle.Oracle(cfg, 32)
    if caps is not None:
        g.set_majorant_cap(caps)
        o.set_majorant_cap(caps)
    g.set_processes(procs)
    g.load_state(st)
    o.set_processes(procs)
    for s, p in enumerate(st):
        o.load(s, p["x"], p["vx"], p["vy"], p["vz"], p["id"])
    return g, o, st


def compare_particles(g, o, rtol=1e-5, atol_x=None, atol_v=1e-3):
    """Per-particle comparison in array order (ids and free flights exactly);
    returns the max relative differences."""
    worst = {}
    for s in range(3):
        a = g.particles(s, flight=True)
        b = o.particles(s)
        assert len(a["id"]) == len(b["id"]), (s, len(a["id"]), len(b["id"]))
        assert np.array_equal(a["id"], b["id"]), s
        assert np.array_equal(a["tc"], o.flight(s)), s
        for k in ("x", "vx", "vy", "vz"):
            x, y = a[k].astype(np.float64), b[k]
            if len(x) == 0:
                continue
            scale = np.maximum(np.abs(y), np.abs(y).max() * 1e-3 + 1e-30)
            rel = np.abs(x - y) / scale
            worst[(s, k)] = float(rel.max())
            assert rel.max() <= rtol, (s, k, rel.max(), int(rel.argmax()))
    return worst


def compare_counters(gs, oc, nproc):
    for s in range(3):
        for k in range(nproc[s]):
            assert gs[f"events_{s}_{k}"] == oc[f"events_{s}_{k}"], (s, k, gs[f"events_{s}_{k}"], oc[f"events_{s}_{k}"])
        for w in range(2):
            assert gs[f"absorbed_{s}_{w}"] == oc[f"absorbed_{s}_{w}"], (s, w)
        assert gs[f"born_{s}"] == oc[f"born_{s}"], s
    for n in COUNTERS_COMPARED:
        assert gs[n] == oc[n], (n, gs[n], oc[n])


def nproc_of(procs):
    return [sum(1 for p in procs if p["species"] == s and p["kind"] not in (xsec.NEUTRALIZE, xsec.RECOMBINE,
                                                                            xsec.EDETACH))
            for s in range(3)]


def curand_ref_lib():
    """Build (once) and load the cuRAND reference helper."""
    import ctypes
    src = os.path.join(ROOT, "tests", "cuda", "curand_ref.cu")
    out_dir = os.path.join(ROOT, "tests", "_build")
    os.makedirs(out_dir, exist_ok=True)
    so = os.path.join(out_dir, "libcurand_ref.so")
    if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared", "-Xcompiler", "-fPIC",
                        src, "-o", so], check=True)
    L = ctypes.CDLL(so)
    L.curand_ref_philox.restype = ctypes.c_int
    L.curand_ref_philox.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_ulonglong]
    return L
