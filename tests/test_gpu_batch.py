"""Batched stepping: several discharges advanced by one CUDA graph give, per
discharge, exactly what stepping it alone gives (and what the oracle gives);
results do not depend on the particle kernels' launch shape; the autotuner
keeps that property."""
import numpy as np
import pytest

from paper_0705_0497_gb300 import inputs, xsec
from helpers import capacity_for, compare_counters, compare_particles, make_pair, nproc_of

pytestmark = pytest.mark.gpu

CC = 10     # compaction check period of these tests (steps per launch must be a multiple of it and of S)


def _sweep(n, scale=0.02, seed=5):
    return inputs.batch_sweep(n, seed=seed, scale=scale)


def _discharge(cfg, counts, T, procs):
    from paper_0705_0497_gb300 import api
    st = inputs.initial_state(cfg, counts, T)
    g = api.Discharge(cfg, capacity_for(counts), compact_check=CC)
    g.set_processes(procs)
    g.load_state(st)
    return g


def _same(a, b):
    for s in range(3):
        pa, pb = a.particles(s, flight=True), b.particles(s, flight=True)
        for k in ("x", "vx", "vy", "vz", "id", "tc"):
            assert np.array_equal(pa[k], pb[k]), (s, k)
    sa, sb = a.stats(), b.stats()
    for k in sa:
        assert sa[k] == sb[k], (k, sa[k], sb[k])
    fa, fb = a.field(), b.field()
    assert np.array_equal(fa[0], fb[0]) and np.array_equal(fa[1], fb[1])
    n = sa["step"]
    k = min(n, 40)
    assert np.array_equal(a.currents(n - k, k), b.currents(n - k, k))


@pytest.mark.parametrize("branches", [False, True])
def test_batch_equals_single_runs(torch_cuda, monkeypatch, branches):
    """Fused batched launches (the default for a shared schedule) and one
    graph branch per discharge both give the single runs bit for bit."""
    from paper_0705_0497_gb300 import api
    if branches:
        monkeypatch.setenv("O2PIC_BATCH_BRANCHES", "1")
    procs = xsec.oxygen_set(include_rec=True, include_edet=True)
    sweep = _sweep(4)
    batched = [_discharge(c, n, T, procs) for c, n, T in sweep]
    alone = [_discharge(c, n, T, procs) for c, n, T in sweep]
    b = api.Batch(batched, steps_per_launch=40)
    b.step(3)
    b.synchronize()
    for g in alone:
        g.step(120)
    for x, y in zip(batched, alone):
        assert x.stats()["step"] == 120
        _same(x, y)
    b.close()


def test_batch_member_matches_oracle(torch_cuda):
    from paper_0705_0497_gb300 import api
    procs = xsec.oxygen_set(include_rec=True, include_edet=True)
    (c0, n0, T0), (c1, n1, T1) = _sweep(2, scale=0.01, seed=11)
    g0, o0, _ = make_pair(c0, n0, T0, procs, compact_check=CC)
    g1 = _discharge(c1, n1, T1, procs)
    b = api.Batch([g0, g1], steps_per_launch=20)
    b.step(2)
    b.synchronize()
    o0.step(40)
    compare_particles(g0, o0)
    compare_counters(g0.stats(), o0.counters(), nproc_of(procs))
    b.close()


def test_launch_shape_does_not_change_results(torch_cuda):
    procs = xsec.oxygen_set()
    (cfg, counts, T), = _sweep(1, scale=0.05, seed=3)
    a = _discharge(cfg, counts, T, procs)
    b = _discharge(cfg, counts, T, procs)
    default = a.launch_shape()
    b.set_launch_shape((3, 1, 7))
    assert b.launch_shape() == (3, 1, 7) and a.launch_shape() == default
    a.step(60)
    b.step(60)
    _same(a, b)


def test_autotune_keeps_results(torch_cuda):
    from paper_0705_0497_gb300 import api
    procs = xsec.oxygen_set()
    sweep = _sweep(3, seed=9)
    batched = [_discharge(c, n, T, procs) for c, n, T in sweep]
    alone = [_discharge(c, n, T, procs) for c, n, T in sweep]
    b = api.Batch(batched, steps_per_launch=20)
    rep = b.autotune()
    assert len(rep["ms"]) == 7 and rep["particles_per_warp"][0] == 0
    assert 0 <= rep["chosen"] < len(rep["ms"]) and all(m > 0 for m in rep["ms"])
    b.step(2)
    b.synchronize()
    steps = batched[0].stats()["step"]
    assert all(g.stats()["step"] == steps for g in batched) and steps % 20 == 0
    for g in alone:
        g.step(steps)
    for x, y in zip(batched, alone):
        _same(x, y)
    b.close()


def test_batch_refuses_stale_graph(torch_cuda):
    from paper_0705_0497_gb300 import api
    procs = xsec.oxygen_set()
    sweep = _sweep(2, seed=2)
    gs = [_discharge(c, n, T, procs) for c, n, T in sweep]
    b = api.Batch(gs, steps_per_launch=20)
    gs[1].step(10)     # out of the graph's phase
    with pytest.raises(api.O2picError) as e:
        b.step(1)
    assert e.value.code == -7
    with pytest.raises(api.O2picError):
        api.Batch(gs, steps_per_launch=15)   # not a multiple of S = 10
    b.close()


def test_batch_of_different_schedules(torch_cuda):
    """Discharges with different ion subcycles cannot share batched launches:
    the batch falls back to one branch each and still matches single runs."""
    from paper_0705_0497_gb300 import api
    procs = xsec.oxygen_set()
    (c0, n0, T0), (c1, n1, T1) = _sweep(2, seed=13)
    c1 = dict(c1, ion_subcycle=5)
    gs = [_discharge(c0, n0, T0, procs), _discharge(c1, n1, T1, procs)]
    alone = [_discharge(c0, n0, T0, procs), _discharge(c1, n1, T1, procs)]
    b = api.Batch(gs, steps_per_launch=20)
    b.step(2)
    b.synchronize()
    for g in alone:
        g.step(40)
    for x, y in zip(gs, alone):
        _same(x, y)
    b.close()
