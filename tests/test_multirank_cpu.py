"""Host logic of the multi-rank runs, on CPU with two `gloo` ranks (no GPU): the batched
workload's instances are split across ranks with every instance on exactly one rank, and
the job time is the slowest rank's (an all-reduce MAX, the only collective; the sweep runs
as replicas with the same timing reduction)."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, %r)
import torch.distributed as dist
rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d", rank=rank, world_size=world)
import bench
mine = bench.shard_instances(256, rank, world)
t = bench.max_over_ranks(1.5 * (rank + 1), world)
dist.barrier()
dist.destroy_process_group()
print(json.dumps({"rank": rank, "mine": mine, "t": t}))
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_batched_sharding_and_max_time_two_gloo_ranks():
    world, port = 2, _free_port()
    procs = []
    for rank in range(world):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER % (ROOT, port)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err[-2000:]
        outs.append(json.loads(out.strip().splitlines()[-1]))
    outs.sort(key=lambda o: o["rank"])
    sets = [set(o["mine"]) for o in outs]
    assert sets[0].isdisjoint(sets[1])
    assert sets[0] | sets[1] == set(range(256))
    assert abs(len(sets[0]) - len(sets[1])) <= 1
    assert all(o["t"] == 3.0 for o in outs)


def test_single_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.shard_instances(5, 0, 1) == [0, 1, 2, 3, 4]
    assert bench.max_over_ranks(2.5, 1) == 2.5


def test_clock_samples_summary():
    """The clocks record of the bench line: median SM clock under load, the maximum, and the
    throttle reasons seen active in any sample (malformed samples are skipped)."""
    import bench
    lines = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1995, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.5, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage",
        "0, 1800, 2070, 1400.0, 0x40, Not Active, Active, Not Active, Not Active",
    ]
    s = bench.summarize_clocks(lines)
    assert s["samples"] == 4 and s["sm_max_mhz"] == 2070.0
    assert s["sm_mhz"] == (1995.0 + 2070.0) / 2                  # median of 4 samples
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert bench.summarize_clocks([])["samples"] == 0
