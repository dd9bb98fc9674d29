"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same seeded
inputs, element by element.  Tolerances: per-order relative L2 <= 1e-4 for the FP32 forms,
<= 2e-2 for BF16, gradients <= 1e-3 relative L2."""
import numpy as np
import pytest

import synth_signals as SS
from oracle import jtfs_oracle as O
from parity_checks import check_orders

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = {"fp32": 1e-4, "fp32_simt": 1e-4, "tf32": 1e-3, "bf16": 2e-2}
# TF32: unit roundoff 2^-11 on each contraction operand; its backward is the FP32-grade one
GTOL = {"fp32": 1e-3, "fp32_simt": 1e-3, "tf32": 1e-3, "bf16": 5e-2}
PRECS = ["fp32_simt", "fp32", "bf16", "tf32"]

SMALL_CFGS = [
    dict(N=512, J=5, Q=4, J_fr=3, Q_fr=1, T=32, F=4),
    dict(N=512, J=5, Q=4, J_fr=3, Q_fr=1, T=32, F=4, average_fr=False),
    dict(N=256, J=4, Q=3, J_fr=2, Q_fr=2, T=16, F=3),
    dict(N=1024, J=6, Q=2, J_fr=2, Q_fr=1, T=1024, F=1),      # T = N: one frame
    dict(N=2048, J=7, Q=12, J_fr=3, Q_fr=2, T=128, F=12, oversampling=1),
    dict(N=1024, J=6, Q=16, J_fr=3, Q_fr=2, T=64, F=16),      # the gradient-check slice
    dict(N=1024, J=6, Q=8, J_fr=3, Q_fr=1, T=32, F=8),        # 32 frames
]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_08269_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _plans(cfg, precision):
    from paper_2204_08269_gb300 import JTFSPlan
    from paper_2204_08269_gb300.jtfs import JTFSError
    kw = dict(cfg)
    try:
        return JTFSPlan(**kw, precision=precision)
    except JTFSError as e:
        # the TF32 contraction exists in the 16-frame form only
        if precision == "tf32" and e.status == 2:
            pytest.skip("TF32 contraction needs 16 pooled frames")
        raise


def _oracle(cfg):
    kw = dict(cfg)
    N = kw.pop("N")
    o = kw.pop("oversampling", 0)
    avg = kw.pop("average_fr", True)
    oc = O.Config(N=N, average_fr=avg, oversampling=o, **kw)
    p = O.Plan(oc)
    return p, O.Schedule(p, o)


def _workload_cfg(w):
    c = O.WORKLOADS[w]
    return dict(N=c.N, J=c.J, Q=c.Q, J_fr=c.J_fr, Q_fr=c.Q_fr, T=c.T, F=c.F)


def _rel(a, b):
    return O.relative_l2(a, b)


@pytest.mark.parametrize("w", [1, 2, 3, 4, 5])
def test_plan_counts_and_schedule_match_oracle(w):
    cfg = _workload_cfg(w)
    plan = _plans(cfg, "fp32_simt")
    op, sc = _oracle(cfg)
    sh = plan.shapes
    assert (sh.n1, sh.n2, sh.n_fr, sh.C, sh.n_t, sh.n_lam_out, sh.N_fr, sh.s_F) == (
        op.n1, op.n2, op.n_fr, op.C, op.n_t, op.n_lam_out, op.N_fr, op.s_F)
    s1, s2, lm = plan.schedule()
    np.testing.assert_array_equal(s1, sc.s1)
    np.testing.assert_array_equal(np.where(sc.skip2, 0, sc.s2), s2)
    np.testing.assert_array_equal(lm, sc.lam_min)
    assert sh.u1_len == int(sc.L1.sum())


def _check_forward(plan, x, op, sc, tol, idx=None):
    xd = torch.from_numpy(x).cuda()
    s0, s1, s2, u1 = plan.forward(xd)
    torch.cuda.synchronize()
    idx = range(x.shape[0]) if idx is None else idx
    worst = {}
    for b in idx:
        ref = O.forward_one(x[b].astype(np.float64), op, sc)
        got = {"S0": s0[b].cpu().numpy(), "S1": s1[b].cpu().numpy(), "S2": s2[b].cpu().numpy()}
        for name, e in check_orders(got, ref, tol, label=f"signal {b}").items():
            worst[name] = max(worst.get(name, 0.0), e)
    return s0, s1, s2, u1, worst


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("ci", range(len(SMALL_CFGS)))
def test_forward_small_configs(ci, prec):
    cfg = SMALL_CFGS[ci]
    plan = _plans(cfg, prec)
    op, sc = _oracle(cfg)
    x = SS.white_noise_batch(3, cfg["N"], 100 + ci)
    _check_forward(plan, x, op, sc, TOL[prec])


@pytest.mark.parametrize("prec", PRECS)
def test_forward_workload1(prec):
    cfg = _workload_cfg(1)
    plan = _plans(cfg, prec)
    op, sc = _oracle(cfg)
    x = SS.workload_signals(1, 4, cfg["N"])
    _check_forward(plan, x, op, sc, TOL[prec])


@pytest.mark.parametrize("prec", PRECS)
def test_forward_workload2_full_batch_sampled(prec):
    """The benchmark's launch configuration (B = 64, N = 2^16); two signals re-computed by
    the oracle."""
    cfg = _workload_cfg(2)
    plan = _plans(cfg, prec)
    op, sc = _oracle(cfg)
    x = SS.workload_signals(2, 64, cfg["N"])
    _check_forward(plan, x, op, sc, TOL[prec], idx=[0, 37])


@pytest.mark.parametrize("prec", PRECS)
def test_forward_workload4_sampled(prec):
    cfg = _workload_cfg(4)
    plan = _plans(cfg, prec)
    op, sc = _oracle(cfg)
    x = SS.workload_signals(4, 32, cfg["N"])
    _check_forward(plan, x, op, sc, TOL[prec], idx=[5])


def _check_backward(plan, x, op, sc, gtol, idx=None, seed=0):
    xd = torch.from_numpy(x).cuda()
    s0, s1, s2, u1 = plan.forward(xd)
    rng = np.random.default_rng(seed)
    g = [rng.standard_normal(tuple(t.shape)).astype(np.float32) for t in (s0, s1, s2)]
    gx = plan.backward(xd, u1, *[torch.from_numpy(v).cuda() for v in g]).cpu().numpy()
    idx = range(x.shape[0]) if idx is None else idx
    worst = 0.0
    for b in idx:
        ref = O.backward_one(x[b].astype(np.float64), g[0][b], g[1][b], g[2][b], op, sc)
        worst = max(worst, _rel(gx[b], ref))
    assert worst <= gtol, worst
    return worst


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("ci", [0, 1, 2, 4, 5, 6])
def test_backward_small_configs(ci, prec):
    cfg = SMALL_CFGS[ci]
    plan = _plans(cfg, prec)
    op, sc = _oracle(cfg)
    x = SS.white_noise_batch(2, cfg["N"], 200 + ci)
    _check_backward(plan, x, op, sc, GTOL[prec])


@pytest.mark.parametrize("prec", PRECS)
def test_backward_workload1(prec):
    cfg = _workload_cfg(1)
    plan = _plans(cfg, prec)
    op, sc = _oracle(cfg)
    x = SS.workload_signals(1, 2, cfg["N"])
    _check_backward(plan, x, op, sc, GTOL[prec])


@pytest.mark.parametrize("prec", PRECS)
def test_backward_workload2_sampled(prec):
    cfg = _workload_cfg(2)
    plan = _plans(cfg, prec)
    op, sc = _oracle(cfg)
    x = SS.workload_signals(2, 64, cfg["N"])
    _check_backward(plan, x, op, sc, GTOL[prec], idx=[11])


# 32 pooled frames over several 64-sample tiles per rate: the spin-pair contraction with its
# 32-frame pooling; at J = 11 the rates with lam_min = 0 (K1 = 144) take the three-atom
# backward (BF16 planes) or the channel-row one (the FP32-grade split)
FRAMES32 = [dict(N=2 ** 13, J=8, Q=16, J_fr=3, Q_fr=2, T=2 ** 8, F=16),
            dict(N=2 ** 15, J=11, Q=16, J_fr=4, Q_fr=2, T=2 ** 10, F=16)]


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("ci", range(len(FRAMES32)))
def test_thirty_two_frames_forward_and_backward(ci, prec):
    cfg = FRAMES32[ci]
    plan = _plans(cfg, prec)
    assert plan.shapes.n_t == 32
    op, sc = _oracle(cfg)
    x = SS.white_noise_batch(3, cfg["N"], 300 + ci)
    _check_forward(plan, x, op, sc, TOL[prec])
    _check_backward(plan, x, op, sc, GTOL[prec], idx=[0, 2], seed=ci)


@pytest.mark.parametrize("prec", ["fp32", "bf16", "tf32"])
def test_tensor_core_matches_cuda_core_form(prec):
    """The tcgen05 contraction and the CUDA-core FP32 form agree on the same input."""
    cfg = _workload_cfg(2)
    a = _plans(cfg, "fp32_simt")
    b = _plans(cfg, prec)
    x = torch.from_numpy(SS.workload_signals(2, 8, cfg["N"])).cuda()
    ra = a.forward(x)
    rb = b.forward(x)
    for u, v in zip(ra[:3], rb[:3]):
        e = float((u - v).norm() / u.norm())
        assert e <= TOL[prec], e
    b.sync()


def test_partial_cotangents_and_zero_input():
    cfg = SMALL_CFGS[0]
    plan = _plans(cfg, "fp32_simt")
    op, sc = _oracle(cfg)
    x = SS.white_noise_batch(2, cfg["N"], 7)
    xd = torch.from_numpy(x).cuda()
    s0, s1, s2, u1 = plan.forward(xd)
    g1 = torch.randn_like(s1)
    gx = plan.backward(xd, u1, None, g1, None).cpu().numpy()
    ref = O.backward_one(x[0].astype(np.float64), np.zeros(op.n_t), g1[0].cpu().numpy(),
                         np.zeros((op.n2, op.C, op.n_lam_out, op.n_t)), op, sc)
    assert _rel(gx[0], ref) < 1e-3
    # x = 0: every wavelet coefficient is 0 and its modulus gradient is taken as 0
    z = torch.zeros_like(xd)
    s0, s1, s2, u1 = plan.forward(z)
    assert float(s1.abs().max()) == 0.0 and float(s2.abs().max()) == 0.0
    g0 = torch.randn_like(s0)
    gx = plan.backward(z, u1, g0, torch.randn_like(s1), torch.randn_like(s2)).cpu().numpy()
    ref = O.Operators(op, sc).pool_T_T(g0[0].cpu().numpy().astype(np.float64), 1)
    assert _rel(gx[0], ref) < 1e-5


def test_empty_batch_is_noop():
    cfg = SMALL_CFGS[0]
    plan = _plans(cfg, "fp32_simt")
    x = torch.zeros((0, cfg["N"]), device="cuda")
    s0, s1, s2, u1 = plan.forward(x)
    assert s0.shape[0] == 0 and s2.shape[0] == 0


def test_deterministic_replay():
    cfg = _workload_cfg(1)
    plan = _plans(cfg, "fp32_simt")
    x = torch.from_numpy(SS.workload_signals(1, 3, cfg["N"])).cuda()
    a = plan.forward(x)
    b = plan.forward(x)
    for u, v in zip(a, b):
        assert torch.equal(u, v)
    g = [torch.ones_like(t) for t in a[:3]]
    assert torch.equal(plan.backward(x, a[3], *g), plan.backward(x, a[3], *g))


def test_workspace_too_small_is_reported():
    from paper_2204_08269_gb300 import jtfs
    cfg = SMALL_CFGS[0]
    plan = _plans(cfg, "fp32_simt")
    x = torch.zeros((2, cfg["N"]), device="cuda")
    s0 = torch.empty(plan.shapes.s0(2), device="cuda")
    s1 = torch.empty(plan.shapes.s1(2), device="cuda")
    s2 = torch.empty(plan.shapes.s2(2), device="cuda")
    ws = torch.empty(16, dtype=torch.uint8, device="cuda")
    st = jtfs.lib().jtfs_forward(plan._h, jtfs._ptr(x), 2, jtfs._ptr(s0), jtfs._ptr(s1),
                                 jtfs._ptr(s2), None, jtfs._ptr(ws), 16, None)
    assert st == 3


def test_autograd_function_and_host_step():
    from paper_2204_08269_gb300 import JTFS
    cfg = _workload_cfg(1)
    m = JTFS(**cfg, precision="fp32_simt")
    xh = SS.workload_signals(1, 2, cfg["N"])
    x = torch.from_numpy(xh).cuda().requires_grad_(True)
    s0, s1, s2 = m(x)
    loss = (s0 ** 2).sum() + (s1 ** 2).sum() + (s2 ** 2).sum()
    loss.backward()
    g = [2 * t.detach() for t in (s0, s1, s2)]
    ref = m.plan.backward(x.detach(), m.plan.forward(x.detach())[3], *g)
    assert torch.allclose(x.grad, ref, rtol=0, atol=1e-6 * float(ref.abs().max()))
    # end-to-end host entry point reproduces the device path
    gh = [t.cpu().contiguous() for t in g]
    o0, o1, o2, gxh = m.plan.forward_backward_host(torch.from_numpy(xh), *gh)
    assert torch.allclose(o2, s2.detach().cpu(), rtol=0, atol=1e-6 * float(s2.abs().max()))
    assert torch.allclose(gxh, ref.cpu(), rtol=0, atol=1e-6 * float(ref.abs().max()))


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("ci", [0, 5])
def test_fused_step_matches_separate_calls(ci, prec):
    """jtfs_forward_backward keeps the forward's spectra for the backward half: its outputs
    equal jtfs_forward followed by jtfs_backward (the same arithmetic, up to the rounding
    order of the first-order spectra), and its gradient matches the oracle's."""
    cfg = SMALL_CFGS[ci]
    plan = _plans(cfg, prec)
    sh = plan.shapes
    x = torch.from_numpy(SS.white_noise_batch(3, cfg["N"], 77 + ci)).cuda()
    gen = torch.Generator(device="cuda").manual_seed(5 + ci)
    g = [torch.randn(f(3), device="cuda", generator=gen) for f in (sh.s0, sh.s1, sh.s2)]
    s0, s1, s2, u1 = plan.forward(x)
    gx = plan.backward(x, u1, *g)
    f0, f1, f2, fgx, fu1 = plan.forward_backward(x, *g, keep_checkpoint=True)
    torch.cuda.synchronize()
    for a, b in ((s0, f0), (s1, f1), (s2, f2), (u1, fu1)):
        assert torch.equal(a, b)
    assert (fgx - gx).norm().item() <= 1e-6 * gx.norm().item()
    op, sc = _oracle(cfg)
    xs = x.double().cpu().numpy()
    gs = [t.double().cpu().numpy() for t in g]
    got = fgx.double().cpu().numpy()
    for b in range(3):
        ref = O.backward_one(xs[b], gs[0][b], gs[1][b], gs[2][b], op, sc)
        assert _rel(got[b], ref) <= GTOL[prec]


@pytest.mark.parametrize("T", [1, 2, 4])
def test_short_pooling_windows_cuda_cores(T):
    """T <= 2: the lowpass spectrum reaches the Nyquist bin and aliases across the first-order
    rows, so the frequency-domain S1 / S0 pooling and adjoints take their every-bin forms and
    the S0 adjoint its time-domain form (CUDA-core contraction, which has no frame limit)."""
    cfg = dict(N=256, J=4, Q=3, J_fr=2, Q_fr=2, T=T, F=3)
    plan = _plans(cfg, "fp32_simt")
    op, sc = _oracle(cfg)
    x = SS.white_noise_batch(2, cfg["N"], 300 + T)
    _check_forward(plan, x, op, sc, TOL["fp32_simt"])
    _check_backward(plan, x, op, sc, GTOL["fp32_simt"], seed=T)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_fused_step_full_batch_sampled(prec):
    """The benchmark's call (jtfs_forward_backward, B = 64, N = 2^16): one signal's S and g_x
    re-computed by the oracle, and the step is bit-for-bit repeatable."""
    cfg = _workload_cfg(2)
    plan = _plans(cfg, prec)
    op, sc = _oracle(cfg)
    sh = plan.shapes
    xs = SS.workload_signals(2, 64, cfg["N"])
    x = torch.from_numpy(xs).cuda()
    rng = np.random.default_rng(64)
    g = [rng.standard_normal((64,) + tuple(f(1)[1:])).astype(np.float32) for f in (sh.s0, sh.s1, sh.s2)]
    gd = [torch.from_numpy(v).cuda() for v in g]
    s0, s1, s2, gx = plan.forward_backward(x, *gd)
    r0, r1, r2, rgx = plan.forward_backward(x, *gd)
    torch.cuda.synchronize()
    for a, b in ((s0, r0), (s1, r1), (s2, r2), (gx, rgx)):
        assert torch.equal(a, b)
    b = 23
    ref = O.forward_one(xs[b].astype(np.float64), op, sc)
    check_orders({"S0": s0[b].cpu().numpy(), "S1": s1[b].cpu().numpy(),
                  "S2": s2[b].cpu().numpy()}, ref, TOL[prec], label=f"signal {b}")
    refg = O.backward_one(xs[b].astype(np.float64), g[0][b], g[1][b], g[2][b], op, sc)
    assert _rel(gx[b].double().cpu().numpy(), refg) <= GTOL[prec]


def test_largest_supported_length_and_refusal_beyond():
    """Q = 16: the top first-order row has stride 8, so N = 2^17 is the longest signal whose
    rows fit the 2^14-sample shared-memory FFT; N = 2^18 is refused as unsupported (status 2)
    before any device work, and N = 2^17 plans build (the parity at that size is in
    test_gpu_parity_large)."""
    from paper_2204_08269_gb300 import JTFSPlan
    from paper_2204_08269_gb300.jtfs import JTFSError
    cfg = dict(J=13, Q=16, J_fr=4, Q_fr=2, T=2 ** 13, F=16)
    p = JTFSPlan(N=2 ** 17, **cfg, precision="fp32")
    s1, s2, lm = p.schedule()
    assert (2 ** 17) // int(s1.min()) == 2 ** 14
    with pytest.raises(JTFSError) as e:
        JTFSPlan(N=2 ** 18, **cfg, precision="fp32")
    assert e.value.status == 2


def test_launch_count_of_the_fused_step():
    """The profiler's launch counter matches the kernels the fused FP32-grade step issues at
    the benchmark's workload: 8 in the forward (x FFT 2, S0, scalogram, Y producer, two
    contraction forms, phi_F pooling) and 10 in the backward (G1, four contraction forms,
    gY spectra, second-order backward, first-order backward, g_x 2)."""
    cfg = _workload_cfg(2)
    plan = _plans(cfg, "fp32")
    sh = plan.shapes
    x = torch.from_numpy(SS.workload_signals(2, 4, cfg["N"])).cuda()
    g = [torch.ones(f(4), device="cuda") for f in (sh.s0, sh.s1, sh.s2)]
    plan.forward_backward(x, *g)
    plan.profile_read()
    plan.forward_backward(x, *g)
    _, launches = plan.profile_read()
    assert launches == 18
