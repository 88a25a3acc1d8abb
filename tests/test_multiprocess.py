"""The N > 1 host logic of the benchmark on CPU: two ranks over gloo (127.0.0.1).  The path
runs replicas only (one problem per rank, no data-path collective): the ranks meet at a
barrier around the timed region, the reported time is the maximum over ranks, and the
reference arm runs on rank 0 alone."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank, port):
    env = dict(os.environ)
    env.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": "2", "MASTER_ADDR": "127.0.0.1",
                "MASTER_PORT": str(port), "SP2_BENCH_GLOO": "1", "CUDA_VISIBLE_DEVICES": ""})
    return env


_HELPERS = r"""
import json, sys
sys.path.insert(0, {root!r})
import bench
ws, rank, local = bench.dist_setup()
bench.barrier(ws)
m = bench.max_over_ranks(1.5 + 10.0 * rank, ws)
bench.barrier(ws)
import torch.distributed as dist
dist.destroy_process_group()
print(json.dumps({{"ws": ws, "rank": rank, "local": local, "max": m}}))
"""


def test_rank_helpers_two_ranks_gloo():
    port = _free_port()
    code = _HELPERS.format(root=ROOT)
    procs = [subprocess.Popen([sys.executable, "-c", code], env=_env(r, port), stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True) for r in range(2)]
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    assert sorted(o["rank"] for o in outs) == [0, 1]
    for o in outs:
        assert o["ws"] == 2 and o["local"] == o["rank"]
        assert o["max"] == 11.5                        # the slowest rank's time, on every rank


def test_reference_arm_prints_on_rank_zero_only():
    port = _free_port()
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--N", "400",
           "--steps", "1", "--warmup", "0", "--cpu-sample-s", "0.5"]
    procs = [subprocess.Popen(cmd, env=_env(r, port), stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True,
                              cwd=ROOT) for r in range(2)]
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=300)
        assert p.returncode == 0, err
        outs.append(out.strip())
    assert outs[1] == ""                               # rank 1 exits without work
    line = json.loads(outs[0].splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    # the same metric, unit and direction as the GPU arm, and an e2e entry with no copies
    sys.path.insert(0, ROOT)
    import bench
    assert line["metric"] == bench.METRIC and line["unit"] == "ms" and line["higher_is_better"] is False
    assert line["e2e"] == {"value": line["value"], "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert line["cpu_baseline"]["value"] == line["value"] and line["cpu_baseline"]["cores"] >= 1
