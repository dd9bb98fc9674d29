"""GPU parity at the largest signal lengths: N = 2^17 with the resynthesis workload's
parameters (J = 13, Q = 16, J_fr = 4, Q_fr = 2, T = 2^13, F = 16; click-train inputs), and an
uneven-length batch with one signal in each padded length of the 2^13..2^17 mix (2^15, 2^16,
2^17 at J = 12).  The CUDA path runs in the launch configuration of its workload (B = 16 at
N = 2^17; one uneven-length call) and the FP64 oracle recomputes sampled signals: per-order
relative L2 and every visible S1 row and S2 (alpha, c) slice, g_x to 1e-3 (5e-2 for BF16).

Gradients are compared on inputs with a white-noise floor 40 dB down: on bare click trains
(and in a zero-padded tail) some first-order rows hold no energy, the modulus Jacobian z / |z|
there is set by rounding, and the FP64 oracle's own gradient moves by order one under a 1e-7
perturbation of the input (pinned on the CPU by test_gradient_conditioning_needs_a_noise_floor).
The forward outputs are well conditioned and are compared on the bare inputs."""
import numpy as np
import pytest

import synth_signals as SS
from oracle import jtfs_oracle as O
from parity_checks import check_orders, relative_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = {"fp32": 1e-4, "tf32": 1e-3, "bf16": 2e-2}
GTOL = {"fp32": 1e-3, "tf32": 1e-3, "bf16": 5e-2}


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_08269_gb300 import build, jtfs
    build.build()
    torch.cuda.set_device(0)
    return jtfs


@pytest.fixture(scope="module")
def oracle3():
    oc = O.WORKLOADS[3]
    p = O.Plan(oc)
    return oc, p, O.Schedule(p, 0)


@pytest.mark.parametrize("prec", ["fp32", "bf16", "tf32"])
def test_workload3_fused_step_sampled(L, oracle3, prec):
    """B = 16 click trains of N = 2^17 through jtfs_forward_backward; signal 9 recomputed by
    the oracle (S per order and per slice, g_x)."""
    oc, op, sc = oracle3
    cfg = dict(N=oc.N, J=oc.J, Q=oc.Q, J_fr=oc.J_fr, Q_fr=oc.Q_fr, T=oc.T, F=oc.F)
    plan = L.JTFSPlan(**cfg, precision=prec)
    sh = plan.shapes
    assert (sh.n1, sh.n2, sh.C, sh.n_lam_out, sh.n_t) == (op.n1, op.n2, op.C, op.n_lam_out,
                                                          op.n_t)
    B = 16
    rng = np.random.default_rng(2 ** 17)
    g = [rng.standard_normal((B,) + tuple(f(1)[1:])).astype(np.float32)
         for f in (sh.s0, sh.s1, sh.s2)]
    gd = [torch.from_numpy(v).cuda() for v in g]
    b = 9
    # forward on the bare click trains
    xs = SS.workload_signals(3, B, oc.N)
    s0, s1, s2, _ = plan.forward_backward(torch.from_numpy(xs).cuda(), *gd)
    torch.cuda.synchronize()
    ref = O.forward_one(xs[b].astype(np.float64), op, sc)
    check_orders({"S0": s0[b].cpu().numpy(), "S1": s1[b].cpu().numpy(),
                  "S2": s2[b].cpu().numpy()}, ref, TOL[prec], label=f"N=2^17 signal {b}")
    # gradient on the click trains with a -40 dB floor
    xn = SS.click_train_batch(B, oc.N, SS.BASE_SEED + 3, noise_db=-40.0)
    _, _, _, gx = plan.forward_backward(torch.from_numpy(xn).cuda(), *gd)
    gref = O.backward_one(xn[b].astype(np.float64), g[0][b], g[1][b], g[2][b], op, sc)
    assert relative_l2(gx[b].cpu().numpy(), gref) <= GTOL[prec]


def test_workload3_separate_calls_match_fused(L):
    """At N = 2^17 the separate jtfs_forward / jtfs_backward calls (the autograd path, which
    rebuilds the spectra from the U1 checkpoint) agree with the fused call."""
    oc = O.WORKLOADS[3]
    cfg = dict(N=oc.N, J=oc.J, Q=oc.Q, J_fr=oc.J_fr, Q_fr=oc.Q_fr, T=oc.T, F=oc.F)
    plan = L.JTFSPlan(**cfg, precision="fp32")
    sh = plan.shapes
    B = 4
    x = torch.from_numpy(SS.workload_signals(3, B, oc.N)).cuda()
    gen = torch.Generator(device="cuda").manual_seed(17)
    g = [torch.randn(f(B), device="cuda", generator=gen) for f in (sh.s0, sh.s1, sh.s2)]
    s0, s1, s2, u1 = plan.forward(x)
    gx = plan.backward(x, u1, *g)
    f0, f1, f2, fgx = plan.forward_backward(x, *g)
    torch.cuda.synchronize()
    for a, b in ((s0, f0), (s1, f1), (s2, f2)):
        assert torch.equal(a, b)
    assert float((fgx - gx).norm()) <= 1e-6 * float(gx.norm())


# one signal per padded length of the uneven-length workload (J = 12: N_i >= 2^15)
VARLEN_CFG = dict(J=12, Q=16, J_fr=4, Q_fr=2, T=2 ** 12, F=16)
VARLEN_LENGTHS = [9001, 40000, 100003]


def _varlen_parts(lengths, floor):
    gens = [SS.amfm_batch, lambda B, n, seed: SS.click_train_batch(B, n, seed, noise_db=floor),
            SS.amfm_batch]
    return [gen(1, n, SS.BASE_SEED + 500 + i)[0] for i, (gen, n) in
            enumerate(zip(gens, lengths))]


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_varlen_workload_lengths_match_oracle(L, prec):
    """An uneven-length batch (lengths 9001, 40000, 100003: padded to 2^15, 2^16, 2^17; an
    AM/FM tone, a click train, an AM/FM tone) in one jtfs_varlen_forward_backward call.  Each
    signal's S on the kept frames is checked against the oracle on its zero-padded copy."""
    parts = _varlen_parts(VARLEN_LENGTHS, None)
    v = L.JTFSVarlen(VARLEN_LENGTHS, **VARLEN_CFG, precision=prec)
    x = torch.from_numpy(np.concatenate(parts).astype(np.float32)).cuda()
    rng = np.random.default_rng(31)
    g = [rng.standard_normal(int(o[-1])).astype(np.float32) for o in (v.s0_off, v.s1_off,
                                                                       v.s2_off)]
    s0, s1, s2, gx = [t.cpu().numpy() for t in v.forward_backward(
        x, [torch.from_numpy(a).cuda() for a in g])]
    T = VARLEN_CFG["T"]
    padded = []
    for i, n in enumerate(VARLEN_LENGTHS):
        Np = L.varlen_padded_length(n, J=VARLEN_CFG["J"])
        padded.append(Np)
        op = O.Plan(O.Config(N=Np, **VARLEN_CFG))
        sc = O.Schedule(op, 0)
        fr = -(-n // T)
        xp = np.zeros(Np)
        xp[:n] = parts[i]
        ref = O.forward_one(xp, op, sc)
        got = {"S0": s0[v.s0_off[i]:v.s0_off[i + 1]].reshape(fr),
               "S1": s1[v.s1_off[i]:v.s1_off[i + 1]].reshape(op.n1, fr),
               "S2": s2[v.s2_off[i]:v.s2_off[i + 1]].reshape(op.n2, op.C, op.n_lam_out, fr)}
        kept = {"S0": ref["S0"][:fr], "S1": ref["S1"][:, :fr], "S2": ref["S2"][..., :fr]}
        check_orders(got, kept, TOL[prec], label=f"len {n} (N = {Np})")
    assert padded == [2 ** 15, 2 ** 16, 2 ** 17]


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_varlen_workload_gradients_match_oracle(L, prec):
    """g_x of an uneven-length batch of one signal per padded length, each filling it (2^15,
    2^16, 2^17 samples: no zero tail, whose empty rows would leave the gradient set by
    rounding), the click train with a -40 dB floor; cotangents on every kept frame.  Checked
    against the oracle per signal.  Zero-padded signals' gradients are compared with the
    fixed-length transform of the padded copy in the uneven-length tests."""
    lengths = [2 ** 15, 2 ** 16, 2 ** 17]
    parts = _varlen_parts(lengths, -40.0)
    v = L.JTFSVarlen(lengths, **VARLEN_CFG, precision=prec)
    x = torch.from_numpy(np.concatenate(parts).astype(np.float32)).cuda()
    rng = np.random.default_rng(37)
    g = [rng.standard_normal(int(o[-1])).astype(np.float32) for o in (v.s0_off, v.s1_off,
                                                                       v.s2_off)]
    gx = v.forward_backward(x, [torch.from_numpy(a).cuda() for a in g])[3].cpu().numpy()
    T = VARLEN_CFG["T"]
    for i, n in enumerate(lengths):
        op = O.Plan(O.Config(N=n, **VARLEN_CFG))
        sc = O.Schedule(op, 0)
        fr = n // T
        g0 = np.zeros(op.n_t)
        g1 = np.zeros((op.n1, op.n_t))
        g2 = np.zeros((op.n2, op.C, op.n_lam_out, op.n_t))
        g0[:fr] = g[0][v.s0_off[i]:v.s0_off[i + 1]]
        g1[:, :fr] = g[1][v.s1_off[i]:v.s1_off[i + 1]].reshape(op.n1, fr)
        g2[..., :fr] = g[2][v.s2_off[i]:v.s2_off[i + 1]].reshape(op.n2, op.C, op.n_lam_out, fr)
        gref = O.backward_one(parts[i].astype(np.float64), g0, g1, g2, op, sc)
        assert relative_l2(gx[v.x_off[i]:v.x_off[i] + n], gref) <= GTOL[prec], n
