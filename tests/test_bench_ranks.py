"""The N > 1 bench path on CPU: two gloo ranks run the replica protocol
(barrier, max over ranks of the timed region, whole-job throughput) that
bench.py runs over NCCL, one process per GPU."""
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, os, sys
sys.path.insert(0, sys.argv[1])
import bench
dist, world, rank, local = bench.dist_init("gloo")
assert (world, rank) == (2, int(os.environ["RANK"]))
bench.rank_barrier(dist)
ms = 10.0 * (rank + 1)                      # rank 1 is the slow one
tot = bench.max_over_ranks(ms, dist, "cpu")
value = bench.job_value(world, 1000, 5, tot)
print(json.dumps({"rank": rank, "tot": tot, "value": value}), flush=True)
dist.destroy_process_group()
"""


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _spawn(code, world, extra_args=()):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, WORLD_SIZE=str(world), RANK=str(r), LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", code, ROOT, *extra_args], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=120) for p in procs]
    return [(p.returncode, o, e) for p, (o, e) in zip(procs, outs)]


def test_two_gloo_ranks_take_the_max_and_sum_the_work():
    import json

    res = _spawn(CHILD, 2)
    for rc, out, err in res:
        assert rc == 0, err
    lines = [json.loads(o.strip().splitlines()[-1]) for _, o, _ in res]
    for d in lines:
        assert d["tot"] == 20.0
        # 2 ranks x 1000 units x 5 steps in the slowest rank's 20 ms
        assert abs(d["value"] - 2 * 1000 * 5 / 0.020) < 1e-6


def test_reference_arm_runs_on_rank_zero_only():
    code = r"""
import sys
root = sys.argv.pop(1)
sys.path.insert(0, root)
import bench
args = bench.parse()
args.impl = "reference"
bench.run_reference(args)
"""
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, "-c", code, ROOT], env=env, capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""


def test_clock_summary_keeps_the_timed_window():
    """Samples outside the marked host-time window are dropped; reasons are the
    union over the window; the median SM clock is over the window."""
    import bench

    c = bench.ClockSampler(0)
    c.nvml = object()  # summary label only
    c.rows = [(0.0, 1000.0, 2070.0, 100.0, ["sw_power_cap"]),
              (1.0, 2070.0, 2070.0, 900.0, []),
              (1.5, 2060.0, 2070.0, 950.0, ["hw_slowdown"]),
              (3.0, 500.0, 2070.0, 50.0, [])]
    c.mark(0.9, 2.0)
    s = c.summary()
    assert s["samples"] == 2 and s["sm_mhz"] == 2065.0 and s["reasons"] == ["hw_slowdown"]
    assert s["sm_max_mhz"] == 2070.0 and s["power_w_max"] == 950.0
