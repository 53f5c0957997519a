"""One instance's sweep split over processes (Section IV-A: the x0 points are
independent for a fixed controller), through the C ABI: ranks search their
ranges (ucp_sweep_part), all-gather the new values over a gloo group, and
finish the sweep (ucp_sweep_finish).  Here the ranks are processes sharing
one GPU; their kernels never wait on each other (the exchange is on the
host), so the test needs one GPU.  The result must be bit-equal to one
process sweeping alone: f, u1 and J after every sweep."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

from paper_1908_04489_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import os, sys, json
sys.path.insert(0, os.environ["UCP_ROOT"])
import numpy as np
import torch
import torch.distributed as dist
from paper_1908_04489_gb300 import binding, shard
dist.init_process_group("gloo", init_method="env://")
torch.cuda.set_device(0)
binding.load()
p = json.loads(os.environ["UCP_PARAMS"])
stream = torch.cuda.Stream()
with binding.Instance(p, stream=stream) as inst:
    shard.sweep(inst, p["sweeps"])
    st = inst.get_controllers(want=("f", "U"))
    Jh = inst.J_history()
np.savez(os.environ["UCP_OUT"], f=st["f"], U=st["U"], J=Jh)
dist.destroy_process_group()
"""


@pytest.fixture(scope="module")
def binding():
    import torch
    assert torch.cuda.is_available()
    from paper_1908_04489_gb300 import binding as b, build
    build.build()
    b.load()
    return b


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def run_ranks(tmp_path, p, world):
    script = tmp_path / "worker.py"
    script.write_text(WORKER)
    port = _free_port()
    procs, outs = [], []
    for rank in range(world):
        out = tmp_path / f"rank{rank}.npz"
        outs.append(out)
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(world),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), UCP_ROOT=ROOT,
                   UCP_PARAMS=json.dumps(p), UCP_OUT=str(out))
        procs.append(subprocess.Popen([sys.executable, str(script)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                      text=True))
    for pr in procs:
        _, err = pr.communicate(timeout=600)
        assert pr.returncode == 0, err[-3000:]
    return [np.load(o) for o in outs]


@pytest.mark.parametrize("precision,world,sweeps", [(1, 2, 5), (1, 3, 3), (0, 2, 2)])
def test_split_sweeps_equal_one_process(binding, tmp_path, precision, world, sweeps):
    import torch
    p = dict(W.c1(), precision=precision, sweeps=sweeps)
    with binding.Instance(p, stream=torch.cuda.Stream()) as inst:
        inst.sweep(sweeps)
        ref = inst.get_controllers(want=("f", "U"))
        ref_J = inst.J_history()
    for res in run_ranks(tmp_path, p, world):
        np.testing.assert_array_equal(res["f"], ref["f"])
        np.testing.assert_array_equal(res["U"], ref["U"])
        np.testing.assert_array_equal(res["J"], ref_J)


def test_part_over_every_point_then_finish_is_one_sweep(binding):
    p = dict(W.small(), precision=1)
    with binding.Instance(p) as a, binding.Instance(p) as b:
        a.sweep(2)
        for _ in range(2):
            b.sweep_finish(b.sweep_part(0, b.n_x))
        np.testing.assert_array_equal(a.get_controllers()["f"], b.get_controllers()["f"])
        np.testing.assert_array_equal(a.J_history(), b.J_history())
        with pytest.raises(binding.UcpError):
            b.sweep_part(5, 2)
        with pytest.raises(binding.UcpError):
            b.sweep_finish(np.zeros(3))
