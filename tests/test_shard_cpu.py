"""The split of one instance's sweep over ranks (Section IV-A's independence
of the x0 points for a fixed controller), host logic on CPU: x0 ranges, and
two gloo ranks exchanging their parts around a stand-in instance whose
per-point update is a Jacobi map of its neighbours -- the sharded result
must equal the single-process one bit for bit.  (The same exchange around
the GPU library is tested in test_gpu_shard.py.)"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
from paper_1908_04489_gb300 import shard  # noqa: E402


@pytest.mark.parametrize("n,world", [(10, 1), (10, 3), (1001, 2), (7, 8), (0, 2)])
def test_x_ranges_cover_the_grid_in_order(n, world):
    r = shard.x_ranges(n, world)
    assert len(r) == world and r[0][0] == 0 and r[-1][1] == n
    for (a, b), (c, d) in zip(r, r[1:]):
        assert b == c
    sizes = [b - a for a, b in r]
    assert max(sizes) - min(sizes) <= 1


class Toy:
    """A stand-in with the library's part/finish calls: the new value of point
    i is a Jacobi map of the pre-sweep values of i and its neighbours."""

    def __init__(self, n):
        self.n_x = n
        self.f = np.sin(np.arange(n) * 0.37)

    def new(self, i):
        f = self.f
        left, right = f[max(i - 1, 0)], f[min(i + 1, self.n_x - 1)]
        return 0.25 * left + 0.5 * f[i] + 0.25 * right + 1e-3 * i

    def sweep_part(self, i0, i1):
        return np.array([self.new(i) for i in range(i0, i1)])

    def sweep_finish(self, f):
        assert len(f) == self.n_x
        self.f = np.array(f)


WORKER = r"""
import os, sys, json
sys.path.insert(0, os.environ["UCP_ROOT"]); sys.path.insert(0, os.environ["UCP_TESTS"])
import numpy as np
import torch.distributed as dist
from paper_1908_04489_gb300 import shard
from test_shard_cpu import Toy
dist.init_process_group("gloo", init_method="env://")
t = Toy(int(os.environ["TOY_N"]))
shard.sweep(t, 5)
print(json.dumps(t.f.tolist()))
dist.destroy_process_group()
"""


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


@pytest.mark.parametrize("n", [101, 3])
def test_two_gloo_ranks_equal_one_process(tmp_path, n):
    script = tmp_path / "worker.py"
    script.write_text(WORKER)
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), UCP_ROOT=ROOT, TOY_N=str(n),
                   UCP_TESTS=os.path.dirname(os.path.abspath(__file__)))
        procs.append(subprocess.Popen([sys.executable, str(script)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                      text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(np.array(json.loads(out.strip().splitlines()[-1])))
    ref = Toy(n)
    for _ in range(5):
        ref.sweep_finish(ref.sweep_part(0, n))
    for f in outs:
        np.testing.assert_array_equal(f, ref.f)
