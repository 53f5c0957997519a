"""The bounded waits of the tensor-core table kernel turn into a status, not a
hang.  Test hook 1 keeps the kernel from issuing its filter-slice copy, so
the wait that copy would complete runs out (nothing is in flight behind it);
hook 2 stops the builder warps after the first filter tile, so the MMA
thread's wait for the second runs out while the first slice group's MMAs are
in flight, and the kernel waits for them before freeing tensor memory.
Either way the kernel waits for its other copies, writes zero partials and
frees its tensor memory; the next synchronising call reports UCP_E_TIMEOUT,
the instance is poisoned, and the context keeps working: a new instance on it
solves exactly as before."""
import ctypes

import pytest

from paper_1908_04489_gb300 import workloads as W

pytestmark = pytest.mark.gpu

UCP_E_TIMEOUT, UCP_E_STATE = -5, -6


@pytest.mark.parametrize("hook", [1, 2])
def test_tensor_core_wait_runs_out_and_reports_a_timeout(hook):
    import torch
    from paper_1908_04489_gb300 import binding
    L = binding.load()
    L.ucp_test_tc_skip_copy.argtypes = [ctypes.c_void_p, ctypes.c_int32]
    p = dict(W.c1(), precision=1, sweeps=3)
    with binding.Instance(p) as ref:
        ref.sweep(3)
        J_ref = ref.J_history()
    inst = binding.Instance(p)
    inst.sweep(1)
    assert L.ucp_test_tc_skip_copy(inst.h, hook) == 0
    with pytest.raises(binding.UcpError) as e:
        inst.sweep(1)
        inst.eval_J()
    assert e.value.status == UCP_E_TIMEOUT, str(e.value)
    assert b"timed out" in L.ucp_last_error()
    with pytest.raises(binding.UcpError) as e:
        inst.eval_J()
    assert e.value.status == UCP_E_STATE
    inst.close()
    torch.cuda.synchronize()
    with binding.Instance(p) as again:
        again.sweep(3)
        assert (again.J_history() == J_ref).all()
