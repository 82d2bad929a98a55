"""The oracle's multi-threaded particle loop (the all-core CPU baseline)
gives the single-threaded results bit for bit: particles with their free
flights, charge, field and every counter (CPU only)."""
import numpy as np

from paper_0705_0497_gb300 import inputs, xsec


def test_threads_do_not_change_results(oracle_mod):
    cfg, counts, T, _ = inputs.workload("parity_128", ion_subcycle=2)
    counts = (40000, 8000, 40000)
    st = inputs.initial_state(cfg, counts, T)
    procs = xsec.oxygen_set(include_rec=True, include_edet=True)
    runs = []
    for threads in (1, 4):
        o = oracle_mod.Oracle(cfg, 32)
        assert o.set_threads(threads) >= 1
        o.set_processes(procs)
        for s, p in enumerate(st):
            o.load(s, p["x"], p["vx"], p["vy"], p["vz"], p["id"])
        o.step(30)
        runs.append(o)
    a, b = runs
    assert a.counters() == b.counters()
    assert a.counters()["born_0"] > 0
    for s in range(3):
        pa, pb = a.particles(s), b.particles(s)
        for k in ("x", "vx", "vy", "vz", "id"):
            assert np.array_equal(pa[k], pb[k]), (s, k)
        assert np.array_equal(a.flight(s), b.flight(s))
    Qa, Aa, _ = a.charge()
    Qb, Ab, _ = b.charge()
    assert np.array_equal(Qa, Qb) and np.array_equal(Aa, Ab)
    assert np.array_equal(a.field()[1], b.field()[1])
