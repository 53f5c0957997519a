"""The C-ABI library loads and exports every symbol include/ucp.h declares;
host-side validation works without a GPU (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1908_04489_gb300 import binding, build
    build.build()
    return binding.load()


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"UCP_API\s+[\w\s\*]+?\b(ucp2?_\w+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert "ucp_create" in names and "ucp_sweep" in names and "ucp2_sweep" in names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"


def test_version_and_status_strings(lib):
    assert b"sm_103a" in lib.ucp_version()
    assert lib.ucp_status_str(0) == b"ok"
    assert lib.ucp_status_str(-7) == b"unknown ticket"


def test_plan_sizes_match_the_configs(lib):
    from paper_1908_04489_gb300 import binding, workloads
    s = binding.plan(workloads.c1())
    assert (s["n_x"], s["n_w"], s["n_y"], s["n_cand"]) == (1001, 241, 1401, 133)
    s = binding.plan(workloads.c2())
    assert (s["n_x"], s["n_w"], s["n_y"]) == (10001, 2401, 14001)
    s = binding.plan(workloads.c5())
    assert (s["n_x"], s["n_w"], s["n_y"], s["n_cand"]) == (100001, 14001, 120001,
                                                           1 + 4 + 64 + 96)
    # c5's largest buffer is the tensor-core table partials (3 tables x 111 tap
    # chunks x 106k positions, double-float)
    assert 0 < s["device_bytes"] < 512 << 20


def test_plan_of_a_table_start(lib):
    """A start from a host table (init_kind 2) is planned with its table; the
    sizes are those of the same grids, and a table of the wrong length or no
    table is rejected."""
    import numpy as np
    from paper_1908_04489_gb300 import binding, workloads
    p = workloads.c1()
    n = binding.plan(p)["n_x"]
    q = dict(p, init_kind=2)
    s = binding.plan(q, np.linspace(-25.0, 25.0, n))
    assert (s["n_x"], s["n_y"]) == (1001, 1401)
    for bad in (None, np.zeros(n - 1)):
        with pytest.raises(binding.UcpError) as e:
            binding.plan(q, bad)
        assert e.value.status == -1


@pytest.mark.parametrize("field,value,msg", [
    ("k", 0.0, "k must"), ("sigma", -1.0, "sigma"), ("delta", 0.0, "delta"),
    ("x_half", 25.02, "x_half"), ("w_half", 0.0, "w_half"),
    ("n_refine", 12, "n_refine"), ("n_levels", 9, "n_levels"),
    ("n_coarse", 1, "n_coarse"), ("n_nbr", -1, "n_nbr"),
    ("precision", 2, "precision"), ("init_kind", 5, "init_kind"),
    ("flags", 1, "flags"), ("problem", 2, "problem"),
])
def test_plan_rejects_invalid_fields(lib, field, value, msg):
    from paper_1908_04489_gb300 import binding, workloads
    p = workloads.c1()
    p[field] = value
    with pytest.raises(binding.UcpError) as e:
        binding.plan(p)
    assert e.value.status == -1 and msg in str(e.value)


def test_source_channel_problem_is_planned_on_both_modes(lib):
    """Problem 1 (Section V-B): its plan has the grids of its parameters on
    the plain path and in its fast mode (precision 1: the three tables and the
    f values, no tensor-core buffers)."""
    from paper_1908_04489_gb300 import binding, workloads
    p = workloads.source_channel()
    s = binding.plan(p)
    assert (s["n_x"], s["n_w"], s["n_y"], s["n_cand"]) == (501, 101, 701, 133)
    f = binding.plan(dict(p, precision=1))
    assert (f["n_x"], f["n_w"], f["n_y"], f["n_cand"]) == (501, 101, 701, 133)
    extra = f["device_bytes"] - s["device_bytes"]
    assert 0 < extra <= 8 * 3 * (701 + 101 + 2) + 8 * 501 + 3 * 256   # tables, f values


def test_create_validates_before_touching_the_device(lib):
    from paper_1908_04489_gb300 import binding, workloads
    p = binding.Params.from_dict(dict(workloads.c1(), k=-1.0))
    h = ctypes.c_void_p()
    assert lib.ucp_create(None, ctypes.byref(p), None, ctypes.byref(h)) == -1
    assert b"k must" in lib.ucp_last_error()
    p = binding.Params.from_dict(workloads.c1())
    assert lib.ucp_create(None, ctypes.byref(p), None, ctypes.byref(h)) == -1
    assert b"context" in lib.ucp_last_error()
    p = binding.Params.from_dict(dict(workloads.c1(), init_kind=2))
    assert lib.ucp_create(None, ctypes.byref(p), None, ctypes.byref(h)) == -1
    assert b"init_table" in lib.ucp_last_error()


def test_plan_of_the_2d_problem_matches_the_oracle(lib):
    """Section V-D's problem: the library's sizes are the 2-D oracle's, and
    invalid parameters are refused on the host (no context is created)."""
    import oracle
    from paper_1908_04489_gb300 import binding
    p = dict(k=0.2, sigma=5.0, delta=0.3125, x_half=25.0, w_half=5.0, y_half=35.0,
             cand_half=30.0, n_coarse=13, n_levels=8, n_nbr=2)
    s = binding.plan2(p)
    o = oracle.Oracle2D(p)
    assert (s["n_x"], s["n_w"], s["n_y"], s["n_cand"]) == (o.n_x, o.n_w, o.n_y, o.n_cand)
    assert (s["n_x"], s["n_cand"]) == (161, 25 + 169 + 64)
    for bad, msg in ((dict(p, x_half=25.1), "multiples of delta"),
                     (dict(p, n_coarse=65), "n_coarse"), (dict(p, n_levels=41), "n_levels"),
                     (dict(p, n_nbr=9), "n_nbr"), (dict(p, sigma=0.0), "> 0"),
                     (dict(p, delta=0.05), "too large")):
        with pytest.raises(binding.UcpError) as e:
            binding.plan2(bad)
        assert e.value.status == -1 and msg in str(e.value), (bad, str(e.value))
    h = ctypes.c_void_p()
    pp = binding.Params2.from_dict(p)
    assert lib.ucp2_create(None, ctypes.byref(pp), None, None, ctypes.byref(h)) == -1
    assert b"context" in lib.ucp_last_error()
