"""Texture resynthesis through the autograd form (JTFSFunction: U1 checkpoint, hand-written
adjoints) on the resynthesis workload: N = 2^17, J = 13, Q = 16, J_fr = 4, Q_fr = 2, T = 2^13,
F = 16, click-train targets.  The normalised error E falls over three Adam and three
bold-driver steps, and the gradient of E at the white-noise start matches the FP64 oracle's
to 1e-3.  On the N = 2^10 gradient slice (J = 6, Q = 16, J_fr = 3, Q_fr = 2, T = 2^6, F = 16)
the gradient also matches central finite differences of E."""
import numpy as np
import pytest

import synth_signals as SS
from oracle import jtfs_oracle as O
from parity_checks import relative_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

W3 = O.WORKLOADS[3]
CFG3 = dict(J=W3.J, Q=W3.Q, J_fr=W3.J_fr, Q_fr=W3.Q_fr, T=W3.T, F=W3.F)
SLICE = dict(N=2 ** 10, J=6, Q=16, J_fr=3, Q_fr=2, T=2 ** 6, F=16)


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_08269_gb300 import build, resynth
    build.build()
    torch.cuda.set_device(0)
    return resynth


def _oracle_grad_E(x, y, op, sc):
    """dE/dy of E = ||S y - S x|| / ||S x|| in FP64: the cotangent of S(y) is
    (S y - S x) / (||S x|| ||S y - S x||), pulled back by the oracle's adjoint chain."""
    rx = O.forward_one(x, op, sc)
    ry = O.forward_one(y, op, sc)
    nx = np.sqrt(sum(np.sum(rx[k] ** 2) for k in ("S0", "S1", "S2")))
    nd = np.sqrt(sum(np.sum((ry[k] - rx[k]) ** 2) for k in ("S0", "S1", "S2")))
    g = {k: (ry[k] - rx[k]) / (nx * nd) for k in ("S0", "S1", "S2")}
    return O.backward_one(y, g["S0"], g["S1"], g["S2"], op, sc), nd / nx


@pytest.mark.parametrize("method", ["adam", "bold"])
def test_resynthesis_steps_at_N_2_17(R, method):
    B = 2
    xs = SS.workload_signals(3, B, W3.N)
    x = torch.from_numpy(xs).cuda()
    r = R.Resynthesis(x, method=method, seed=3, precision="fp32", **CFG3)
    y0 = r.signal().clone()
    E0, g0 = r._eval(y0)
    out = r.run(3)
    E = out["E"]
    assert len(E) == 3 and all(np.isfinite(E))
    assert float(out["E_last"].mean()) < float(E0.mean())
    if method == "bold":
        assert all(b <= a + 1e-7 for a, b in zip(E, E[1:]))     # only decreases are kept
    # the gradient of E at the white-noise start against the oracle, signal 1
    op = O.Plan(W3)
    sc = O.Schedule(op, 0)
    y64 = y0[1].double().cpu().numpy()
    gref, Eref = _oracle_grad_E(xs[1].astype(np.float64), y64, op, sc)
    assert abs(float(E0[1]) - Eref) <= 1e-4 * Eref
    assert relative_l2(g0[1].double().cpu().numpy(), gref) <= 1e-3


@pytest.mark.parametrize("prec", ["fp32_simt", "fp32"])
def test_gradient_slice_finite_differences_and_oracle(R, prec):
    B = 2
    N = SLICE["N"]
    cfg = {k: v for k, v in SLICE.items() if k != "N"}
    xs = SS.click_train_batch(B, N, SS.BASE_SEED + 3)
    x = torch.from_numpy(xs).cuda()
    r = R.Resynthesis(x, method="adam", seed=11, precision=prec, **cfg)
    y = r.signal().clone()
    E, g = r._eval(y)
    op = O.Plan(O.Config(N=N, **cfg))
    sc = O.Schedule(op, 0)
    for b in range(B):
        gref, _ = _oracle_grad_E(xs[b].astype(np.float64), y[b].double().cpu().numpy(), op, sc)
        assert relative_l2(g[b].double().cpu().numpy(), gref) <= 1e-3
    # central differences of E along a seeded direction, per signal
    gen = torch.Generator(device="cuda").manual_seed(5)
    v = torch.randn(y.shape, device="cuda", generator=gen)
    v /= v.norm(dim=1, keepdim=True)
    h = 1e-2 * float(y.norm(dim=1).min())
    with torch.no_grad():
        Ep = R.normalised_error(R._flat(*r.model(y + h * v)), r.s_x).double()
        Em = R.normalised_error(R._flat(*r.model(y - h * v)), r.s_x).double()
    fd = (Ep - Em) / (2 * h)
    an = (g.double() * v.double()).sum(dim=1)
    assert torch.allclose(fd, an, rtol=2e-3, atol=1e-3 * float(g.norm(dim=1).max())), (fd, an)
