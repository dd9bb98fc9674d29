"""Uneven-length batches (jtfs_varlen_*): every signal's packed outputs equal the fixed-length
transform of its zero-padded copy restricted to the kept frames, the captured CUDA graph
replays the same step bit for bit, and one padded signal matches the oracle.  Through the C
ABI via the binding."""
import numpy as np
import pytest

import synth_signals as SS
from oracle import jtfs_oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CFG = dict(J=6, Q=8, J_fr=3, Q_fr=1, T=64, F=8)
LENGTHS = [300, 512, 700, 1024, 1500, 2048, 3000, 64]


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_08269_gb300 import build, jtfs
    build.build()
    torch.cuda.set_device(0)
    return jtfs


def _rel(a, b):
    a = torch.as_tensor(a, dtype=torch.float64)
    b = torch.as_tensor(b, dtype=torch.float64)
    d = float(b.norm())
    return float((a - b).norm()) / (d if d > 0 else 1.0)


def _packed_inputs(v, seed):
    rng = np.random.default_rng(seed)
    x = torch.from_numpy(rng.standard_normal(int(v.x_off[-1])).astype(np.float32)).cuda()
    g = [torch.from_numpy(rng.standard_normal(int(o[-1])).astype(np.float32)).cuda()
         for o in (v.s0_off, v.s1_off, v.s2_off)]
    return x, g


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp32_simt"])
def test_varlen_matches_padded_fixed_length(L, prec):
    v = L.JTFSVarlen(LENGTHS, **CFG, precision=prec, chunk=3)
    x, g = _packed_inputs(v, 5)
    s0, s1, s2, gx = v.forward_backward(x, g)
    torch.cuda.synchronize()
    plans = {}
    for i, n in enumerate(LENGTHS):
        Np = L.varlen_padded_length(n, J=CFG["J"])
        assert Np == max(1 << int(np.ceil(np.log2(n))), 1 << (CFG["J"] + 3))
        p = plans.setdefault(Np, L.JTFSPlan(N=Np, **CFG, precision=prec))
        sh = p.shapes
        fr = -(-n // CFG["T"])
        xi = torch.zeros((1, Np), device="cuda")
        xi[0, :n] = x[int(v.x_off[i]):int(v.x_off[i]) + n]
        r0, r1, r2, u1 = p.forward(xi)
        got0 = s0[int(v.s0_off[i]):int(v.s0_off[i + 1])].view(fr)
        got1 = s1[int(v.s1_off[i]):int(v.s1_off[i + 1])].view(sh.n1, fr)
        got2 = s2[int(v.s2_off[i]):int(v.s2_off[i + 1])].view(sh.n2, sh.C, sh.n_lam_out, fr)
        assert _rel(got0, r0[0, :fr]) <= 1e-6
        assert _rel(got1, r1[0, :, :fr]) <= 1e-6
        assert _rel(got2, r2[0, ..., :fr]) <= 1e-6
        # cotangents of the kept frames, zero elsewhere
        g0 = torch.zeros_like(r0)
        g1 = torch.zeros_like(r1)
        g2 = torch.zeros_like(r2)
        g0[0, :fr] = g[0][int(v.s0_off[i]):int(v.s0_off[i + 1])]
        g1[0, :, :fr] = g[1][int(v.s1_off[i]):int(v.s1_off[i + 1])].view(sh.n1, fr)
        g2[0, ..., :fr] = g[2][int(v.s2_off[i]):int(v.s2_off[i + 1])].view(
            sh.n2, sh.C, sh.n_lam_out, fr)
        ref_gx = p.backward(xi, u1, g0, g1, g2)
        assert _rel(gx[int(v.x_off[i]):int(v.x_off[i]) + n], ref_gx[0, :n]) <= 1e-6


def test_varlen_graph_replay_is_deterministic(L):
    v = L.JTFSVarlen(LENGTHS, **CFG, precision="fp32")
    x, g = _packed_inputs(v, 9)
    direct = [t.clone() for t in v.forward_backward(x, g)]
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        outs = v.capture(x, g)
        for t in outs:
            t.fill_(float("nan"))
        v.replay()
        first = [t.clone() for t in outs]
        for t in outs:
            t.fill_(float("nan"))
        v.replay()
    side.synchronize()
    for a, b, c in zip(direct, first, outs):
        assert torch.equal(a, b)
        assert torch.equal(b, c)


def test_varlen_signal_matches_oracle(L):
    cfg = O.Config(N=1024, **CFG)
    plan, sched = O.Plan(cfg), None
    sched = O.Schedule(plan, 0)
    n = 700
    v = L.JTFSVarlen([n], **CFG, precision="fp32")
    x = SS.white_noise_batch(1, n, 77)[0].astype(np.float32)
    xt = torch.from_numpy(x).cuda()
    s0, s1, s2, _ = v.forward_backward(xt)
    torch.cuda.synchronize()
    xp = np.zeros(1024)
    xp[:n] = x
    ref = O.forward_one(xp, plan, sched)
    fr = -(-n // CFG["T"])
    assert _rel(s0.cpu().view(fr), ref["S0"][:fr]) <= 1e-4
    assert _rel(s1.cpu().view(plan.n1, fr), ref["S1"][:, :fr]) <= 1e-4
    assert _rel(s2.cpu().view(plan.n2, plan.C, plan.n_lam_out, fr), ref["S2"][..., :fr]) <= 1e-4


def test_autotune_keeps_results(L):
    cfg = dict(N=2048, J=7, Q=12, J_fr=3, Q_fr=2, T=128, F=12)
    for prec in ("fp32", "fp32_simt"):
        plan = L.JTFSPlan(**cfg, precision=prec)
        x = torch.from_numpy(SS.white_noise_batch(3, cfg["N"], 31)).cuda()
        before = plan.forward(x)
        g = [torch.ones_like(t) for t in before[:3]]
        gx0 = plan.backward(x, before[3], *g)
        choice = plan.autotune(3)
        assert choice["threads"] in (256, 512)
        assert choice["samples_per_cta"] in (4096, 8192, 16384)
        after = plan.forward(x)
        for a, b in zip(before, after):
            assert torch.equal(a, b)
        assert torch.equal(gx0, plan.backward(x, after[3], *g))


def test_varlen_autotune_then_graph(L):
    v = L.JTFSVarlen(LENGTHS, **CFG, precision="bf16")
    x, g = _packed_inputs(v, 13)
    direct = [t.clone() for t in v.forward_backward(x, g)]
    v.autotune()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        outs = v.capture(x, g)
        v.replay()
    side.synchronize()
    for a, b in zip(direct, outs):
        assert torch.equal(a, b)


def test_schedule_tuner_keeps_results(L):
    """jtfs_varlen_tune_schedule times sub-batches of 16, 32, ... up to the creation's size
    and keeps the fastest; every split gives the same outputs, bit for bit, and the graph
    captured afterwards replays them."""
    lengths = LENGTHS * 5
    v = L.JTFSVarlen(lengths, **CFG, precision="fp32", chunk=64)
    x, g = _packed_inputs(v, 17)
    direct = [t.clone() for t in v.forward_backward(x, g)]
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        chosen = v.tune_schedule(x, g)
        after = [t.clone() for t in v.forward_backward(x, g)]
        outs = v.capture(x, g)
        v.replay()
    side.synchronize()
    assert chosen in (16, 32, 64)
    for a, b, c in zip(direct, after, outs):
        assert torch.equal(a, b)
        assert torch.equal(a, c)
