"""mu-log compression (Sec. 4.3, Eq. 6-7) through the C ABI against the oracle, on the S2
paths of a transform (P = n2 C, M = n_lam_out n_t) and on arbitrary [B, P, M] arrays; its
gradient against the derivative of Eq. 7 with mu fixed."""
import numpy as np
import pytest

import synth_signals as SS
from oracle import jtfs_oracle as O
from parity_checks import relative_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_08269_gb300 import build, jtfs
    build.build()
    torch.cuda.set_device(0)
    return jtfs


def test_mulog_on_transform_paths(L):
    cfg = dict(N=2 ** 12, J=6, Q=8, J_fr=3, Q_fr=1, T=2 ** 6, F=8)
    plan = L.JTFSPlan(**cfg, precision="fp32")
    x = torch.from_numpy(SS.workload_signals(1, 6, cfg["N"])).cuda()
    s2 = plan.forward(x)[2]
    B, P = s2.shape[0], s2.shape[1] * s2.shape[2]
    s = s2.reshape(B, P, -1).contiguous()
    mu = L.mulog_mean(s)
    out = L.mulog(s, mu, eps=0.1)
    sh = s.double().cpu().numpy()
    mref = O.mu_log_mean(sh)
    assert relative_l2(mu.cpu().numpy(), mref) <= 1e-6
    assert relative_l2(out.cpu().numpy(), O.mu_log(sh, mu.double().cpu().numpy(), 0.1)) <= 1e-6


@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 17, 5), (2, 300, 1000)])
def test_mulog_arrays_and_gradient(L, shape):
    gen = torch.Generator(device="cuda").manual_seed(sum(shape))
    s = torch.rand(shape, device="cuda", generator=gen) * 3.0
    mu = L.mulog_mean(s)
    ref_mu = s.double().sum(dim=2).mean(dim=0)
    assert torch.allclose(mu.double(), ref_mu, rtol=1e-6, atol=0)
    out = L.mulog(s, mu, eps=0.1)
    assert torch.allclose(out.double(), torch.log1p(s.double() / (0.1 * mu.double()[None, :, None])),
                          rtol=1e-6, atol=1e-7)
    g = torch.randn(shape, device="cuda", generator=gen)
    gs = L.mulog_backward(s, mu, g, eps=0.1)
    ref = g.double() / (0.1 * mu.double()[None, :, None] + s.double())
    assert torch.allclose(gs.double(), ref, rtol=1e-6, atol=1e-7)


def test_mulog_rejects_bad_arguments(L):
    lib = L.lib()
    s = torch.ones((2, 3, 4), device="cuda")
    mu = torch.ones(3, device="cuda")
    assert lib.jtfs_mulog(L._ptr(s), 2, 3, 4, L._ptr(mu), 0.0, L._ptr(s), None) == 1
    assert lib.jtfs_mulog_mean(L._ptr(s), 0, 3, 4, L._ptr(mu), None) == 1
    assert lib.jtfs_mulog(None, 2, 3, 4, L._ptr(mu), 0.1, L._ptr(s), None) == 1
