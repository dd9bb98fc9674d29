"""GPU parity of the phi_t paths (phi_T x psi_{beta,+1}, phi_T x phi_F; jtfs_config.branches)
and of the 2-D output layout (out_3d = 0), through the C ABI against the FP64 oracle.  The
phi_t paths run on CUDA cores in FP32 for every precision (only the psi_t contraction changes
with it), so they are held to the FP32 tolerances; the psi_t paths keep their precision's."""
import numpy as np
import pytest

import synth_signals as SS
from oracle import jtfs_oracle as O
from parity_checks import check_orders, relative_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = {"fp32": 1e-4, "fp32_simt": 1e-4, "bf16": 2e-2}
GTOL = {"fp32": 1e-3, "fp32_simt": 1e-3, "bf16": 5e-2}
ALL = ("phi_psi", "phi_phi")
CFGS = [
    dict(N=512, J=5, Q=4, J_fr=3, Q_fr=1, T=32, F=4),
    dict(N=512, J=5, Q=4, J_fr=3, Q_fr=1, T=32, F=4, average_fr=False),
    dict(N=2 ** 12, J=6, Q=8, J_fr=3, Q_fr=1, T=2 ** 6, F=8),
    dict(N=2 ** 16, J=12, Q=16, J_fr=4, Q_fr=2, T=2 ** 12, F=16),
]


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_08269_gb300 import build, jtfs
    build.build()
    torch.cuda.set_device(0)
    return jtfs


def _oracle(cfg, branches):
    kw = dict(cfg)
    N = kw.pop("N")
    avg = kw.pop("average_fr", True)
    mask = 3 | sum(O.__dict__[b.upper()] for b in branches)
    p = O.Plan(O.Config(N=N, average_fr=avg, branches=mask, **kw))
    return p, O.Schedule(p, 0)


def _split(s2, op):
    """GPU S2 [s2_paths, n_lo, n_t] -> (psi_t paths as [n2, C, n_lo, n_t], phi_t paths)."""
    k = op.n2 * op.C
    return s2[:k].reshape(op.n2, op.C, op.n_lam_out, op.n_t), s2[k:]


@pytest.mark.parametrize("prec", ["fp32_simt", "fp32", "bf16"])
@pytest.mark.parametrize("ci", range(len(CFGS)))
@pytest.mark.parametrize("branches", [ALL, ("phi_phi",)])
def test_phi_paths_forward_and_gradient(L, ci, prec, branches):
    cfg = CFGS[ci]
    if ci == 3 and (prec == "fp32_simt" or branches != ALL):
        pytest.skip("the full-size case runs the tensor-core forms with both phi_t paths")
    plan = L.JTFSPlan(**cfg, precision=prec, branches=branches)
    op, sc = _oracle(cfg, branches)
    sh = plan.shapes
    assert sh.n_phi == op.n_phi and sh.s2_paths == op.n2 * op.C + op.n_phi
    B = 3 if ci < 3 else 8
    idx = [0, 2] if ci < 3 else [5]
    if cfg["N"] >= 2 ** 12:
        xs = SS.click_train_batch(B, cfg["N"], SS.BASE_SEED + 40 + ci, noise_db=-40.0)
    else:
        xs = SS.white_noise_batch(B, cfg["N"], 400 + ci)
    rng = np.random.default_rng(41 + ci)
    g = [rng.standard_normal(f(B)).astype(np.float32) for f in (sh.s0, sh.s1, sh.s2)]
    s0, s1, s2, gx = plan.forward_backward(torch.from_numpy(xs).cuda(),
                                           *[torch.from_numpy(v).cuda() for v in g])
    s0, s1, s2, gx = (t.cpu().numpy() for t in (s0, s1, s2, gx))
    for b in idx:
        ref = O.forward_one(xs[b].astype(np.float64), op, sc)
        psi, phi = _split(s2[b], op)
        check_orders({"S0": s0[b], "S1": s1[b], "S2": psi}, ref, TOL[prec], label=f"signal {b}")
        assert relative_l2(phi, ref["S2phi"]) <= TOL["fp32"]
        for q in range(op.n_phi):
            assert relative_l2(phi[q], ref["S2phi"][q]) <= 10 * TOL["fp32"], q
        gpsi, gphi = _split(g[2][b], op)
        gref = O.backward_one(xs[b].astype(np.float64), g[0][b], g[1][b], gpsi, op, sc,
                              gS2phi=gphi)
        assert relative_l2(gx[b], gref) <= GTOL[prec]


@pytest.mark.parametrize("prec", ["fp32_simt", "fp32"])
def test_phi_paths_separate_calls_rebuild_s1(L, prec):
    """jtfs_backward without the forward in the same call rebuilds S1 from the checkpoint for
    the phi_t paths' adjoint; it agrees with the fused call."""
    cfg = CFGS[2]
    plan = L.JTFSPlan(**cfg, precision=prec, branches=ALL)
    sh = plan.shapes
    x = torch.from_numpy(SS.white_noise_batch(3, cfg["N"], 61)).cuda()
    gen = torch.Generator(device="cuda").manual_seed(62)
    g = [torch.randn(f(3), device="cuda", generator=gen) for f in (sh.s0, sh.s1, sh.s2)]
    s0, s1, s2, u1 = plan.forward(x)
    gx = plan.backward(x, u1, *g)
    f0, f1, f2, fgx = plan.forward_backward(x, *g)
    torch.cuda.synchronize()
    assert torch.equal(s2, f2)
    assert float((fgx - gx).norm()) <= 1e-5 * float(gx.norm())


@pytest.mark.parametrize("branches", [None, ALL])
def test_two_dimensional_layout(L, branches):
    """out_3d = 0: one [B, 1 + n1 + s2_paths n_lam_out, n_t] output per call holding S0, the
    S1 rows and the S2 paths in that order, bit for bit the 3-D outputs; its cotangent in the
    same layout gives the same gradient; the host entry point takes it too."""
    cfg = CFGS[2]
    p3 = L.JTFSPlan(**cfg, precision="fp32", branches=branches)
    p2 = L.JTFSPlan(**cfg, precision="fp32", branches=branches, out_3d=False)
    sh = p2.shapes
    assert sh.out_rows == 1 + sh.n1 + sh.s2_paths * sh.n_lam_out
    B = 3
    xh = SS.white_noise_batch(B, cfg["N"], 71)
    x = torch.from_numpy(xh).cuda()
    a0, a1, a2, u1 = p3.forward(x)
    out, none1, none2, u1b = p2.forward(x)
    assert none1 is None and none2 is None and out.shape == sh.out_2d(B)
    flat = torch.cat([a0.reshape(B, 1, -1), a1.reshape(B, sh.n1, -1),
                      a2.reshape(B, -1, sh.n_t)], dim=1)
    assert torch.equal(out, flat)
    gen = torch.Generator(device="cuda").manual_seed(72)
    g = [torch.randn(f(B), device="cuda", generator=gen) for f in (sh.s0, sh.s1, sh.s2)]
    gflat = torch.cat([g[0].reshape(B, 1, -1), g[1].reshape(B, sh.n1, -1),
                       g[2].reshape(B, -1, sh.n_t)], dim=1).contiguous()
    gx3 = p3.backward(x, u1, *g)
    gx2 = p2.backward(x, u1b, gflat)
    assert torch.equal(gx3, gx2)
    o2, _, _, fgx = p2.forward_backward(x, gflat)
    assert torch.equal(o2, out)
    h0, h1, h2, hgx = p2.forward_backward_host(torch.from_numpy(xh), gflat.cpu())
    assert h1 is None and h2 is None
    assert torch.equal(h0, out.cpu()) and torch.equal(hgx, fgx.cpu())
    # the module form returns the single tensor
    m = L.JTFS(**cfg, precision="fp32", out_3d=False, branches=branches)
    xr = x.clone().requires_grad_(True)
    y = m(xr)
    assert torch.equal(y.detach(), out)
    (y * gflat).sum().backward()
    assert torch.equal(xr.grad, gx2)


def test_phi_paths_need_oversampling_zero(L):
    cfg = dict(CFGS[2], oversampling=1)
    with pytest.raises(L.JTFSError) as e:
        L.JTFSPlan(**cfg, precision="fp32_simt", branches=ALL)
    assert e.value.status == 2
