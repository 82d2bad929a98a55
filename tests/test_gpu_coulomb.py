"""Coulomb collisions (1)-(6) on the GPU against the oracle, particle for
particle: the cell sort, the pairing and the Takizuka-Abe scattering."""
import numpy as np
import pytest

from paper_0705_0497_gb300 import inputs, xsec
from helpers import compare_counters, compare_particles, make_pair, nproc_of

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("Nc,mask", [(32, 63), (97, 63), (64, 1 | 8)])
def test_coulomb_parity(torch_cuda, Nc, mask):
    """All six reactions (and a subset) with a weight that makes the
    deflections large, three Coulomb steps (ion subcycle 2), ragged cell
    occupations (one cell count odd-sized for the padded sort rows)."""
    cfg = inputs.base_config(L=0.02, n_cells=Nc, U=50.0, p=10.0, C_meta=0.0, ion_subcycle=2, weight=3e10, seed=9,
                             steps_per_cycle=400)
    procs = xsec.oxygen_set()
    rng = np.random.default_rng(41)
    st = []
    for s, n in enumerate((20000, 6000, 26000)):
        x = (rng.random(n) ** 1.5 * cfg["L"]).astype(np.float32)   # uneven cell occupations
        sig = (1.0e6 if s == 0 else 500.0)
        v = (rng.standard_normal((3, n)) * sig).astype(np.float32)
        st.append(dict(x=x, vx=v[0].copy(), vy=v[1].copy(), vz=v[2].copy(), id=np.arange(n, dtype=np.uint32)))
    g, o, _ = make_pair(cfg, None, None, procs, state=st)
    g.set_coulomb(mask, 10.0)
    o.set_coulomb(mask, 10.0)
    for _ in range(3):
        g.step(2)
        o.step(2)
        compare_particles(g, o)
        compare_counters(g.stats(), o.counters(), nproc_of(procs))
    assert o.counters()["coulomb_pairs"] > 10000


def test_oxygen_set_with_coulomb_100_steps(torch_cuda):
    """The parity case with every reaction of Table 1: (1)-(22), 100 steps,
    per particle and every counter."""
    cfg, counts, T, _ = inputs.workload("parity_128", ion_subcycle=2)
    procs = xsec.oxygen_set(include_rec=True, include_edet=True)
    g, o, _ = make_pair(cfg, counts, T, procs)
    g.set_coulomb(63, 10.0)
    o.set_coulomb(63, 10.0)
    g.step(100)
    o.step(100)
    compare_particles(g, o)
    compare_counters(g.stats(), o.counters(), nproc_of(procs))
    assert o.counters()["coulomb_pairs"] > 0


def test_coulomb_in_a_batch(torch_cuda):
    """Contexts with Coulomb collisions run in a batch (one graph branch
    each) exactly as alone."""
    from paper_0705_0497_gb300 import api
    from test_gpu_batch import _discharge, _same, _sweep
    procs = xsec.oxygen_set()
    sweep = _sweep(2)
    batched = [_discharge(c, n, T, procs) for c, n, T in sweep]
    alone = [_discharge(c, n, T, procs) for c, n, T in sweep]
    for g in batched + alone:
        g.set_coulomb(63, 10.0)
    b = api.Batch(batched, steps_per_launch=40)
    b.step(2)
    b.synchronize()
    for g in alone:
        g.step(80)
    for x, y in zip(batched, alone):
        _same(x, y)
    assert batched[0].stats()["coulomb_pairs"] > 0
    b.close()
