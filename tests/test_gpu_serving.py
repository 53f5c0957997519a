"""Serving (ucp_submit / ucp_poll): continuous batching of requests of
different sizes and sweep counts; every result equals the same request
solved alone, and admission honours slots and the HBM budget."""
import time

import numpy as np
import pytest

from paper_1908_04489_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def binding():
    import torch
    assert torch.cuda.is_available()
    from paper_1908_04489_gb300 import binding as b, build
    build.build()
    b.load()
    return b


def small_requests(n, seed=21):
    rng = W.SplitMix64(seed, 1)
    reqs = []
    for k in range(n):
        p = W.random_instance(rng, (0.1, 0.05), 2 + (k % 4), 1)
        reqs.append(p)
    return reqs


def solve_alone(binding, p):
    with binding.Instance(p) as inst:
        inst.sweep(p["sweeps"])
        st = inst.get_controllers(want=("f", "U"))
        st["J"] = inst.eval_J()
    return st


def wait_all(srv, tickets, timeout=120.0):
    out, t0 = {}, time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                r = srv.poll(t)
                if r is not None:
                    out[t] = r
        assert time.time() - t0 < timeout, "server did not finish in time"
        time.sleep(0.001)
    return out


def test_served_results_equal_standalone_solves(binding):
    reqs = small_requests(9)
    with binding.Server(max_slots=4) as srv:
        tickets = []
        for k, p in enumerate(reqs):
            tickets.append(srv.submit(p))
            if k == 4:
                time.sleep(0.01)      # later requests arrive while others run
        res = wait_all(srv, tickets)
        st = srv.stats()
    assert st["max_active"] >= 2 and st["completed"] == len(reqs)
    for t, p in zip(tickets, reqs):
        ref = solve_alone(binding, p)
        np.testing.assert_array_equal(res[t]["f"], ref["f"])
        np.testing.assert_array_equal(res[t]["U"], ref["U"])
        assert res[t]["J"] == ref["J"]
        assert res[t]["t_submit"] <= res[t]["t_admit"] <= res[t]["t_done"]


def test_requests_join_while_others_run(binding):
    """A request submitted after others started is admitted before they
    finish (it shares their steps) and still gets its standalone result."""
    long_req = dict(small_requests(1, seed=5)[0], sweeps=2000)
    late = dict(small_requests(1, seed=6)[0], sweeps=2)
    with binding.Server(max_slots=8) as srv:
        t1 = srv.submit(long_req)
        while srv.stats()["steps"] < 3:
            time.sleep(0.0005)
        t2 = srv.submit(late)
        res = wait_all(srv, [t1, t2])
    assert res[t2]["t_admit"] < res[t1]["t_done"]
    assert res[t2]["t_done"] < res[t1]["t_done"]
    ref = solve_alone(binding, late)
    np.testing.assert_array_equal(res[t2]["f"], ref["f"])


def test_served_table_starts_equal_standalone_solves(binding):
    """Requests started from host tables (copied at submission, set up by the
    batched set-up kernels at admission) equal the same solves alone."""
    reqs = small_requests(4, seed=23)
    tables = []
    for k, p in enumerate(reqs):
        n = binding.plan(p)["n_x"]
        x = (np.arange(n) - (n - 1) // 2) * p["delta"]
        tables.append(0.9 * x + 0.4 * np.sin(0.5 * x))
        reqs[k] = dict(p, init_kind=2)
    with binding.Server(max_slots=8) as srv:
        tickets = [srv.submit(p, table=t) for p, t in zip(reqs, tables)]
        res = wait_all(srv, tickets)
    for p, t, tk in zip(reqs, tables, tickets):
        with binding.Instance(p, table=t) as inst:
            inst.sweep(p["sweeps"])
            ref = inst.get_controllers(want=("f", "U"))
            J = inst.eval_J()
        np.testing.assert_array_equal(res[tk]["f"], ref["f"])
        np.testing.assert_array_equal(res[tk]["U"], ref["U"])
        assert res[tk]["J"] == J


def test_budget_admission_and_rejection(binding):
    reqs = small_requests(3, seed=8)
    needs = sorted(binding.plan(p)["device_bytes"] for p in reqs)
    # the largest fits alone, no two fit together
    budget = min(needs[-1] + (1 << 16), needs[0] + needs[1] - 1)
    assert budget >= needs[-1]
    with binding.Server(hbm_budget_bytes=budget, max_slots=8) as srv:
        with pytest.raises(binding.UcpError) as e:
            srv.submit(W.c2())
        assert e.value.status == -3                      # UCP_E_BUDGET
        tickets = [srv.submit(p) for p in reqs]
        res = wait_all(srv, tickets)
        assert srv.stats()["max_active"] == 1            # one fits at a time
    assert len(res) == 3


def test_unknown_and_collected_tickets(binding):
    with binding.Server() as srv:
        with pytest.raises(binding.UcpError) as e:
            srv.poll(12345)
        assert e.value.status == -7
        t = srv.submit(small_requests(1)[0])
        wait_all(srv, [t])
        with pytest.raises(binding.UcpError) as e:
            srv.poll(t)
        assert e.value.status == -7


def test_injected_step_failure_reaches_every_request(binding):
    """Failure drill on the host: a failing step ends every request with
    UCP_E_CUDA and the server refuses new work; the GPU is untouched."""
    with binding.Server(max_slots=2) as srv:
        tickets = [srv.submit(dict(p, sweeps=50)) for p in small_requests(4)]
        srv.fail_next_step()
        statuses = []
        t0 = time.time()
        for t in tickets:
            while True:
                try:
                    r = srv.poll(t)
                except binding.UcpError as e:
                    statuses.append(e.status)
                    break
                if r is not None:
                    statuses.append(0)
                    break
                assert time.time() - t0 < 60
                time.sleep(0.001)
        assert all(s == -4 for s in statuses)
        with pytest.raises(binding.UcpError) as e:
            srv.submit(small_requests(1)[0])
        assert e.value.status == -6
