"""The multi-GPU mode of bench.py is N independent replicas of the workload
(the transform does not shard on a one-GPU pool): the whole-job step time is
the maximum over the ranks and the value counts the units of every rank.
These tests run that host logic as two `gloo` ranks on CPU, and check that
the reference arm leaves ranks other than 0 without work and prints the
contract's line on rank 0."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_RANK_CHILD = r"""
import json, os, sys
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
dist.init_process_group("gloo")
import bench
rank, world = dist.get_rank(), dist.get_world_size()
t, v = bench.aggregate_over_ranks(1.0 + rank, 1000, world, "cpu")
print(json.dumps({"rank": rank, "t": t, "value": v}))
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_replicas_take_max_time_and_count_all_units():
    pytest.importorskip("torch")
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", _RANK_CHILD, ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=180)
        assert p.returncode == 0, err[-2000:]
        outs.append(json.loads(out.strip().splitlines()[-1]))
    for r in outs:
        # rank 0 took 1 ms, rank 1 took 2 ms: the job's step is 2 ms for 2 x 1000 units
        assert r["t"] == 2.0
        assert r["value"] == pytest.approx(2 * 1000 / 2e-3)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", CUDA_VISIBLE_DEVICES="")
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                          "--steps", "3", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120)
    assert res.returncode == 0, res.stderr[-2000:]
    assert res.stdout.strip() == ""


def test_reference_arm_line_on_rank_0():
    """The reference arm (the oracle on the host cores) prints one JSON line
    with the contract's keys, the same metric, unit and workload as the GPU
    arm, and an end-to-end entry without host transfers."""
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr[-2000:]
    line = json.loads(res.stdout.strip().splitlines()[-1])
    sys.path.insert(0, ROOT)
    import bench
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["config"]["workload"] == bench.DEFAULT_CONFIG
    for key in ("value", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling", "dtype",
                "data", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["value"] > 0 and line["steps"] == 1 and line["warmup"] == 3
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    # the same workload object as the GPU arm's line (same sample size for the oracle in both)
    d, M, m = (bench.CONFIGS[bench.DEFAULT_CONFIG][k] for k in (0, 1, 2))
    assert line["config"] == bench.workload_config(bench.DEFAULT_CONFIG, bench.default_beta(m), 1)
    assert line["cpu_baseline"]["cores"] >= 1
    assert f"first {bench.ORACLE_SAMPLE[d]} of the" in line["cpu_baseline"]["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
