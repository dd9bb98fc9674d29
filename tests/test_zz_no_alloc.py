"""jtfs_first_order_static: the first-order transform for callers that cannot allocate device
memory while they run (a real-time audio callback, a plug-in inside a host that owns all
device memory).  Its scratch is a fixed array inside the library, so its results must equal
those of the ordinary entry point, call after call, and oversized batches must be refused.
Called through the C ABI."""
import ctypes

import numpy as np
import pytest

import synth_signals as SS
from oracle import jtfs_oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-4   # the FP32 per-order tolerance of the parity tests


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_08269_gb300 import build, jtfs
    build.build()
    torch.cuda.set_device(0)
    return jtfs


def _rel(a, b):
    return float((a - b).norm() / b.norm())


@pytest.mark.parametrize("cfg,B,workload", [
    (dict(N=2 ** 12, J=6, Q=8, J_fr=3, Q_fr=1, T=2 ** 6, F=8), 3, 1),
    (dict(N=2 ** 16, J=12, Q=16, J_fr=4, Q_fr=2, T=2 ** 12, F=16), 2, 2),
])
def test_static_scratch_matches_forward_twice(L, cfg, B, workload):
    plan = L.JTFSPlan(**cfg, precision="fp32")
    x = torch.from_numpy(SS.workload_signals(workload, B, cfg["N"])).cuda()
    ref0, ref1, _, _ = plan.forward(x)
    lib = L.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        s0 = torch.full_like(ref0, float("nan"))
        s1 = torch.full_like(ref1, float("nan"))
        st = lib.jtfs_first_order_static(plan._h, L._ptr(x), B, L._ptr(s0), L._ptr(s1), stream)
        assert st == 0, lib.jtfs_last_error().decode()
        torch.cuda.synchronize()
        assert _rel(s0, ref0) <= TOL, call
        assert _rel(s1, ref1) <= TOL, call
        assert torch.isfinite(s1).all()


def test_static_scratch_rejects_oversized_batch(L):
    cfg = dict(N=2 ** 16, J=12, Q=16, J_fr=4, Q_fr=2, T=2 ** 12, F=16)
    plan = L.JTFSPlan(**cfg, precision="fp32")
    B = 64
    x = torch.zeros((B, cfg["N"]), device="cuda")
    s0 = torch.empty(plan.shapes.s0(B), device="cuda")
    s1 = torch.empty(plan.shapes.s1(B), device="cuda")
    lib = L.lib()
    st = lib.jtfs_first_order_static(plan._h, L._ptr(x), B, L._ptr(s0), L._ptr(s1), None)
    assert st == 3   # JTFS_ERR_WORKSPACE
    assert b"fixed array" in lib.jtfs_last_error()


def test_static_scratch_matches_oracle(L):
    """S0 and S1 of the fixed-scratch path against the FP64 oracle (not only against the
    ordinary entry point, which runs the same first-order kernels)."""
    oc = O.WORKLOADS[1]
    cfg = dict(N=oc.N, J=oc.J, Q=oc.Q, J_fr=oc.J_fr, Q_fr=oc.Q_fr, T=oc.T, F=oc.F)
    plan = L.JTFSPlan(**cfg, precision="fp32")
    B = 3
    xs = SS.workload_signals(1, B, cfg["N"])
    x = torch.from_numpy(xs).cuda()
    s0 = torch.empty(plan.shapes.s0(B), device="cuda")
    s1 = torch.empty(plan.shapes.s1(B), device="cuda")
    lib = L.lib()
    st = lib.jtfs_first_order_static(plan._h, L._ptr(x), B, L._ptr(s0), L._ptr(s1),
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, lib.jtfs_last_error().decode()
    torch.cuda.synchronize()
    op = O.Plan(oc)
    sc = O.Schedule(op, 0)
    for b in range(B):
        ref = O.forward_one(xs[b].astype(np.float64), op, sc)
        assert O.relative_l2(s0[b].double().cpu().numpy(), ref["S0"]) <= TOL
        assert O.relative_l2(s1[b].double().cpu().numpy(), ref["S1"]) <= TOL


def test_static_scratch_largest_batch_that_fits(L):
    """At the benchmark's signal length the largest accepted batch fills most of the fixed
    array; one more signal is refused, and the accepted batch matches jtfs_forward."""
    cfg = dict(N=2 ** 16, J=12, Q=16, J_fr=4, Q_fr=2, T=2 ** 12, F=16)
    plan = L.JTFSPlan(**cfg, precision="fp32")
    lib = L.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    xs = torch.from_numpy(SS.workload_signals(2, 16, cfg["N"])).cuda()
    best = None
    for B in range(16, 0, -1):
        s0 = torch.empty(plan.shapes.s0(B), device="cuda")
        s1 = torch.empty(plan.shapes.s1(B), device="cuda")
        st = lib.jtfs_first_order_static(plan._h, L._ptr(xs[:B]), B, L._ptr(s0), L._ptr(s1),
                                         stream)
        if st == 0:
            best = (B, s0, s1)
            break
        assert st == 3
    assert best is not None and best[0] >= 4
    B, s0, s1 = best
    torch.cuda.synchronize()
    ref0, ref1, _, _ = plan.forward(xs[:B].contiguous())
    assert _rel(s0, ref0) <= TOL and _rel(s1, ref1) <= TOL
