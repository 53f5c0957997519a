"""The allocation-free u1 step (ucp_u1_update_noalloc) against the existing
entry points.

That call serves callers that may not allocate device memory (a process
whose device memory belongs to another framework, a real-time loop that must
not enter the allocator); its scratch is one fixed device array.  Here its
output is compared with the u1 table that an instance computes for the same
controller through ucp_set_controllers, on two calls in a row, within the
u1 tolerance of the other parity tests.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_1908_04489_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_U = 1e-11


def _lib():
    from paper_1908_04489_gb300 import binding, build
    build.build()
    L = binding.load()
    L.ucp_u1_update_noalloc.argtypes = [ctypes.POINTER(binding.Params),
                                        ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p]
    return binding, L


def test_u1_update_noalloc_matches_instance_twice():
    import torch
    binding, L = _lib()
    p = W.c2(precision=1)
    n = binding.plan(p)
    d = p["delta"]
    x = (np.arange(n["n_x"]) - (n["n_x"] - 1) // 2) * d
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(5)
    for call in range(2):
        f = np.where(x == 0, 0.0, np.sign(x) * 3.5 * (2 * np.minimum(
            np.abs(x) // 7.0, 2) + 1)) + rng.normal(0, 0.3 + call, x.size)
        with binding.Instance(p) as inst:
            inst.set_controllers(f)
            U_ref = inst.get_controllers(want=("U",))["U"]
        f_dev = torch.from_numpy(f).to("cuda")
        U_dev = torch.full((n["n_y"],), float("nan"), dtype=torch.float64,
                           device="cuda")
        torch.cuda.synchronize()
        st = L.ucp_u1_update_noalloc(ctypes.byref(binding.Params.from_dict(p)),
                                     f_dev.data_ptr(), U_dev.data_ptr(),
                                     stream.cuda_stream)
        assert st == 0, L.ucp_last_error()
        torch.cuda.synchronize()
        U = U_dev.cpu().numpy()
        assert np.all(np.isfinite(U))
        assert np.max(np.abs(U - U_ref)) <= TOL_U


def test_u1_update_noalloc_rejects_grids_beyond_its_scratch():
    import torch
    binding, L = _lib()
    p = W.c5()
    buf = torch.zeros(4, dtype=torch.float64, device="cuda")
    st = L.ucp_u1_update_noalloc(ctypes.byref(binding.Params.from_dict(p)),
                                 buf.data_ptr(), buf.data_ptr(), None)
    assert st == -1 and b"too large" in L.ucp_last_error()


def _controller(x, call, seed=5):
    rng = np.random.default_rng(seed)
    return np.where(x == 0, 0.0, np.sign(x) * 3.5 * (2 * np.minimum(
        np.abs(x) // 7.0, 2) + 1)) + rng.normal(0, 0.3 + call, x.size)


def test_u1_update_noalloc_at_the_largest_grid():
    """n_x = n_y = 32767, the largest grids the static scratch takes: eight
    source tiles of 4096 and the per-tile partial sums at the full target
    count, against the instance path."""
    import torch
    binding, L = _lib()
    d = 0.002
    p = W.base(delta=d, x_half=16383 * d, y_half=16383 * d, w_half=6.0, cand_half=30.0,
               precision=1)
    n = binding.plan(p)
    assert (n["n_x"], n["n_y"]) == (32767, 32767)
    x = (np.arange(n["n_x"]) - (n["n_x"] - 1) // 2) * d
    f = _controller(x, 1, seed=11)
    with binding.Instance(p) as inst:
        inst.set_controllers(f)
        U_ref = inst.get_controllers(want=("U",))["U"]
    f_dev = torch.from_numpy(f).to("cuda")
    U_dev = torch.full((n["n_y"],), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    st = L.ucp_u1_update_noalloc(ctypes.byref(binding.Params.from_dict(p)),
                                 f_dev.data_ptr(), U_dev.data_ptr(),
                                 torch.cuda.current_stream().cuda_stream)
    assert st == 0, L.ucp_last_error()
    torch.cuda.synchronize()
    U = U_dev.cpu().numpy()
    assert np.all(np.isfinite(U))
    assert np.max(np.abs(U - U_ref)) <= TOL_U


def test_u1_update_noalloc_inside_a_captured_graph():
    """Captured into a CUDA graph after an uncaptured call (which looks up the
    scratch address), replayed on new inputs written into the same buffers."""
    import torch
    binding, L = _lib()
    p = W.c2(precision=1)
    n = binding.plan(p)
    x = (np.arange(n["n_x"]) - (n["n_x"] - 1) // 2) * p["delta"]
    prm = binding.Params.from_dict(p)
    f_dev = torch.from_numpy(_controller(x, 0)).to("cuda")
    U_dev = torch.zeros((n["n_y"],), dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        assert L.ucp_u1_update_noalloc(ctypes.byref(prm), f_dev.data_ptr(), U_dev.data_ptr(),
                                       s.cuda_stream) == 0
    s.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        st = L.ucp_u1_update_noalloc(ctypes.byref(prm), f_dev.data_ptr(), U_dev.data_ptr(),
                                     torch.cuda.current_stream().cuda_stream)
    assert st == 0, L.ucp_last_error()
    f2 = _controller(x, 1, seed=7)
    f_dev.copy_(torch.from_numpy(f2))
    U_dev.fill_(float("nan"))
    graph.replay()
    torch.cuda.synchronize()
    with binding.Instance(p) as inst:
        inst.set_controllers(f2)
        U_ref = inst.get_controllers(want=("U",))["U"]
    assert np.max(np.abs(U_dev.cpu().numpy() - U_ref)) <= TOL_U
