"""Host logic of bench.py that needs no GPU: the cross-rank reduction used for
N > 1 replicas (max of times, sum of units) on two gloo ranks, and the JSON
line of the CPU reference arm."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, u = bench.reduce_job(1.0 + rank, 10.0 * (rank + 1), world)
    bench.barrier(world)
    # one rank saw a throttled clock: both ranks re-measure
    again = bench.any_rank(rank == 1, world)
    assert again and not bench.any_rank(False, world)
    q.put((rank, t, u))
    dist.destroy_process_group()


def test_reduce_job_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == [(0, 2.0, 30.0), (1, 2.0, 30.0)]


def test_reference_arm_json_line():
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=600,
                         cwd=ROOT)
    assert res.returncode == 0, res.stderr
    line = json.loads(res.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"


def test_clock_records_that_invalidate_a_measurement():
    import importlib.util
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(root, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    ok = {"sm_mhz": 2020.0, "sm_max_mhz": 2032.0, "reasons": ["sw_power_cap"]}
    assert not b.clocks_rejected(ok)
    assert b.clocks_rejected(dict(ok, reasons=["hw_slowdown"]))
    assert b.clocks_rejected(dict(ok, reasons=["sw_thermal_slowdown", "sw_power_cap"]))
    assert b.clocks_rejected({"sm_mhz": 1100.0, "sm_max_mhz": 2032.0, "reasons": []})  # locked low
    assert not b.clocks_rejected({"sm_mhz": 1100.0, "sm_max_mhz": 2032.0, "reasons": ["sw_power_cap"]})
    assert not b.clocks_rejected({"sm_mhz": None, "sm_max_mhz": None, "reasons": []})


def test_committed_dram_profile_matches_the_kernel_source():
    """The bench's roofline `traffic` comes from the DRAM bytes per update in
    profiles/sweep_large_cube.md, used only while the hash recorded there
    matches the current forward kernel source: a kernel change needs a new
    capture before the bench reports traffic again."""
    import bench
    t = bench.profiled_traffic("large_cube", 257575)
    assert t is not None, "profiles/sweep_large_cube.md was taken on other kernel source (%s)" % (
        bench.kernel_source_sha())
    # DRAM bytes per update within the algorithmic model's range (1,303 B at this size)
    assert 0.8 * 1303 <= t / 257575 <= 1.1 * 1303
