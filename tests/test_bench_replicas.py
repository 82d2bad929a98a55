"""Multi-GPU runs of bench.py are independent replicas (one discharge per
rank); the host-side reduction (slowest rank's time, summed particle-steps)
and the rank handling of the reference arm run here as two gloo ranks on the
CPU."""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, _ = bench.dist_setup()
    assert (w, r) == (world, rank) and dist.get_backend() == "gloo"
    # rank r: 10 + r ms, (r + 1) * 1e9 particle-steps
    agg = bench.aggregate(10.0 + rank, (rank + 1) * 1e9, (rank + 1) * 5e8, 7.0 * (rank + 1), 2.0 + rank)
    bench.barrier()
    out.put((rank, agg))
    dist.destroy_process_group()


def test_two_replicas_reduce_max_time_and_summed_work():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        agg = res[r]
        assert agg["t_max_ms"] == 11.0 and agg["e2e_t_max"] == 3.0
        assert agg["ps_sum"] == 3e9 and agg["pe_sum"] == 1.5e9 and agg["e2e_ps_sum"] == 21.0


def test_single_process_aggregate_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    agg = bench.aggregate(5.0, 1e9, 4e8, 3.0, 1.5)
    assert agg == {"t_max_ms": 5.0, "e2e_t_max": 1.5, "ps_sum": 1e9, "pe_sum": 4e8, "e2e_ps_sum": 3.0}


def test_reference_arm_line_on_the_cpu():
    """`bench.py --impl reference` (the oracle on the host cores) prints one
    JSON line with the contract's keys: the same metric and unit as the GPU
    arm, the cores it used, and an end-to-end figure equal to its value with
    no host-device bytes."""
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "parity_128", "--steps", "2", "--warmup", "3"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    sys.path.insert(0, ROOT)
    import bench
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 3 and d["higher_is_better"] is True
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "parity_128"
