"""Failure detection on the GPU, with no GPU fault: a bounded device wait that
runs out on a flag nothing sets, id overflow counted per birth exactly as the
oracle counts it, and the host-side guards of next_id and the launch shape.
Every failure here is an error status the host reads; the context stays
usable afterwards."""
import ctypes

import numpy as np
import pytest

from paper_0705_0497_gb300 import inputs, xsec
from helpers import capacity_for, compare_counters, make_pair, nproc_of

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_returns(torch_cuda):
    """The look-back wait of the compaction kernels, waiting for a
    predecessor tile that never publishes, gives up after its spin limit,
    records O2PIC_E_TIMEOUT and returns; the device keeps working."""
    from paper_0705_0497_gb300 import api
    secs = ctypes.c_double()
    rc = api.lib().o2pic_check_bounded_wait(ctypes.byref(secs), None)
    assert rc == -6, rc
    assert 0.0 < secs.value < 30.0, secs.value
    # the context is still usable: a short run matches the oracle
    cfg, counts, T, _ = inputs.workload("parity_128")
    g, o, _ = make_pair(cfg, (2000, 400, 2000), T, xsec.oxygen_set())
    g.step(5)
    o.step(5)
    for s in range(3):
        assert np.array_equal(g.particles(s)["id"], o.particles(s)["id"])


def _stats_any(g):
    """o2pic_get_stats, accepting a latched device error (returned too)."""
    from paper_0705_0497_gb300 import api
    st = api.Stats()
    rc = api.lib().o2pic_get_stats(g.h, ctypes.byref(st))
    return rc, st.as_dict()


def _ids_any(g, s):
    from paper_0705_0497_gb300 import api
    n = ctypes.c_uint64()
    api.lib().o2pic_read_particles(g.h, s, None, None, None, None, None, 0, ctypes.byref(n), api.HOST)
    out = {k: np.zeros(n.value, np.float32) for k in ("x", "vx", "vy", "vz")}
    out["id"] = np.zeros(n.value, np.uint32)
    m = ctypes.c_uint64()
    rc = api.lib().o2pic_read_particles(g.h, s, *[out[k].ctypes.data_as(ctypes.c_void_p)
                                                  for k in ("x", "vx", "vy", "vz", "id")],
                                        n.value, ctypes.byref(m), api.HOST)
    return rc, out


def test_id_overflow_matches_oracle(torch_cuda):
    """Next ids set 3 below 2^32 on both sides: births past 2^32 - 1 are
    counted one by one (id_overflow), keep the low 32 bits of their id, and
    the step reports O2PIC_E_ID_OVERFLOW; ids, particles and every counter
    equal the oracle's."""
    cfg, counts, T, _ = inputs.workload("parity_128", ion_subcycle=2)
    procs = xsec.oxygen_set(include_rec=True)
    g, o, _ = make_pair(cfg, counts, T, procs)
    start = 0xFFFFFFFF - 3
    for s in range(3):
        g.set_next_id(s, start)
        o.set_next_id(s, start)
    g.step(40)
    o.step(40)
    rc, gs = _stats_any(g)
    oc = o.counters()
    assert rc == -3, rc
    assert oc["id_overflow"] > 0
    assert gs["id_overflow"] == oc["id_overflow"]
    expected = sum(max(0, oc[f"born_{s}"] - 4) for s in range(3))
    assert oc["id_overflow"] == expected
    for s in range(3):
        assert gs[f"next_id_{s}"] == o.next_id(s) == start + oc[f"born_{s}"]
        rc, a = _ids_any(g, s)
        b = o.particles(s)
        assert np.array_equal(a["id"], b["id"]), s
        for k in ("x", "vx", "vy", "vz"):
            assert np.array_equal(a[k].astype(np.float64), b[k]), (s, k)
    compare_counters(gs, oc, nproc_of(procs))


def test_set_next_id_rejects_ids_in_use(torch_cuda):
    """After a load the next id is the largest loaded id + 1: a smaller one
    would give newborns live ids (and shared random streams) and is
    rejected; equal or larger is accepted."""
    from paper_0705_0497_gb300 import api
    cfg, counts, T, _ = inputs.workload("parity_128")
    st = inputs.initial_state(cfg, (500, 100, 500), T)
    g = api.Discharge(cfg, capacity_for((500, 100, 500)))
    g.set_processes(xsec.oxygen_set())
    g.load_state(st)
    with pytest.raises(api.O2picError) as ei:
        g.set_next_id(0, 499)
    assert ei.value.code == -1
    g.set_next_id(0, 500)
    g.set_next_id(0, 10_000)
    with pytest.raises(api.O2picError):
        g.set_next_id(0, 9_999)
    assert g.stats()["next_id_0"] == 10_000


def test_launch_shape_keeps_the_deposit_count_in_range(torch_cuda):
    """A block's shared-memory deposit counts fewer than 2^24 particles per
    cell, so a species needs at least capacity / 2^23 blocks: fewer are
    rejected, and the defaults and the autotuner's shapes respect it."""
    from paper_0705_0497_gb300 import api
    cfg, counts, T, _ = inputs.workload("parity_128")
    cap = (1 << 25, 1000, 1000)
    g = api.Discharge(cfg, cap)
    g.set_processes(xsec.oxygen_set())
    assert g.launch_shape()[0] >= 4
    with pytest.raises(api.O2picError) as ei:
        g.set_launch_shape((3, 1, 1))
    assert ei.value.code == -1
    g.set_launch_shape((4, 1, 1))
    assert g.launch_shape() == (4, 1, 1)
