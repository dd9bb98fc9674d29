"""Failure detection on the GPU without a fault: a bounded device wait that runs out is
reported as JTFS_ERR_TIMEOUT by the next jtfs_sync_status (and the status word is cleared,
the context stays usable), and the opt-in output check reports a NaN in the input as
JTFS_ERR_NUMERIC.  The timeout is made by jtfs_diagnose_wait_timeout: one block waits, with
the contraction kernels' own bounded wait and a 100 us budget, on a barrier that nothing
completes.  Through the C ABI."""
import ctypes

import numpy as np
import pytest

import synth_signals as SS

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CFG = dict(N=2 ** 12, J=6, Q=8, J_fr=3, Q_fr=1, T=2 ** 6, F=8)
OK, INVALID, TIMEOUT, NUMERIC = 0, 1, 5, 6


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_08269_gb300 import build, jtfs
    build.build()
    torch.cuda.set_device(0)
    return jtfs


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("prec", ["fp32", "fp32_simt"])
def test_wait_timeout_is_reported_and_cleared(L, prec):
    plan = L.JTFSPlan(**CFG, precision=prec)
    lib = L.lib()
    x = torch.from_numpy(SS.workload_signals(1, 2, CFG["N"])).cuda()
    before = plan.forward(x)
    assert lib.jtfs_sync_status(plan._h, _stream()) == OK
    assert lib.jtfs_diagnose_wait_timeout(plan._h, 100_000, _stream()) == OK
    assert lib.jtfs_sync_status(plan._h, _stream()) == TIMEOUT
    assert b"gave up" in lib.jtfs_last_error()
    assert lib.jtfs_sync_status(plan._h, _stream()) == OK      # the word was cleared
    after = plan.forward(x)                                      # the context is usable
    plan.sync()
    for a, b in zip(before, after):
        assert torch.equal(a, b)


def test_wait_budget_arguments_are_validated(L):
    plan = L.JTFSPlan(**CFG, precision="fp32")
    lib = L.lib()
    assert lib.jtfs_diagnose_wait_timeout(plan._h, 0, _stream()) == INVALID
    assert lib.jtfs_diagnose_wait_timeout(plan._h, 2_000_000_000, _stream()) == INVALID
    assert lib.jtfs_plan_set_wait_budget(plan._h, 10) == INVALID
    assert lib.jtfs_plan_set_wait_budget(plan._h, 500_000_000) == OK
    x = torch.from_numpy(SS.workload_signals(1, 2, CFG["N"])).cuda()
    plan.forward(x)
    assert lib.jtfs_sync_status(plan._h, _stream()) == OK


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_non_finite_output_is_reported_when_checked(L, prec):
    plan = L.JTFSPlan(**CFG, precision=prec)
    lib = L.lib()
    xs = SS.workload_signals(1, 2, CFG["N"])
    bad = xs.copy()
    bad[1, 1000] = np.nan
    xb = torch.from_numpy(bad).cuda()
    # unchecked: nothing is reported
    plan.forward(xb)
    assert lib.jtfs_sync_status(plan._h, _stream()) == OK
    plan.check_finite(True)
    plan.forward(xb)
    assert lib.jtfs_sync_status(plan._h, _stream()) == NUMERIC
    assert b"non-finite" in lib.jtfs_last_error()
    # finite input: clean; the fused call's gradient is checked too
    x = torch.from_numpy(xs).cuda()
    sh = plan.shapes
    g = [torch.ones(f(2), device="cuda") for f in (sh.s0, sh.s1, sh.s2)]
    plan.forward_backward(x, *g)
    assert lib.jtfs_sync_status(plan._h, _stream()) == OK
    plan.forward_backward(xb, *g)
    with pytest.raises(L.JTFSError) as e:
        plan.sync()
    assert e.value.status == NUMERIC
    plan.check_finite(False)
