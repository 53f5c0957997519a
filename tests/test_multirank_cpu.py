"""The bench's multi-rank path on CPU: two gloo ranks on 127.0.0.1.  Each
rank's timed total enters a max over ranks; the whole-job rate is all units
over the slowest rank's time; the reference arm prints on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


WORKER = r"""
import os, sys, json
sys.path.insert(0, os.environ["UCP_ROOT"])
import torch.distributed as dist
import bench
rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", init_method="env://")
local = 1.5 + 2.0 * rank            # seconds this rank spent
m = bench.max_over_ranks(local, world)
rate = bench.whole_job_rate(world, 3, m)
dist.barrier()
print(json.dumps({"rank": rank, "max": m, "rate": rate}))
dist.destroy_process_group()
"""


def test_max_over_ranks_and_rate_with_two_gloo_ranks(tmp_path):
    port = _free_port()
    script = tmp_path / "worker.py"
    script.write_text(WORKER)
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), UCP_ROOT=ROOT)
        procs.append(subprocess.Popen([sys.executable, str(script)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                      text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(out.strip().splitlines()[-1])
    import json
    res = [json.loads(o) for o in outs]
    for r in res:
        assert r["max"] == 3.5                      # the slower rank's time
        assert abs(r["rate"] - 2 * 3 / 3.5) < 1e-12  # 6 units over 3.5 s


def test_single_rank_aggregation_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.25, 1) == 2.25
    assert bench.whole_job_rate(1, 4, 2.0) == 2.0


def test_reference_arm_prints_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl",
                        "reference", "--steps", "1", "--warmup", "0"], env=env,
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_product_path_fails_loudly_without_the_library(monkeypatch):
    sys.path.insert(0, ROOT)
    from paper_1908_04489_gb300 import binding
    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding, "lib_path", lambda: "/nonexistent/libucp.so")
    with pytest.raises(RuntimeError, match="not built"):
        binding.load()


def test_instances_are_partitioned_by_work_for_several_gpus():
    """The batched workload's split over GPUs: every instance on exactly one
    rank, deterministic, and no rank above the ideal share by more than the
    largest instance (longest-first greedy)."""
    sys.path.insert(0, ROOT)
    from paper_1908_04489_gb300 import workloads as W
    ps = W.c3()
    est = [W.work_estimate(p) for p in ps]
    for world in (1, 2, 3, 8):
        parts = W.partition(ps, world)
        assert sorted(k for part in parts for k in part) == list(range(len(ps)))
        assert parts == W.partition(ps, world)
        load = [sum(est[k] for k in part) for part in parts]
        assert max(load) <= sum(est) / world + max(est) + 1e-9
        assert all(part == sorted(part) for part in parts)
