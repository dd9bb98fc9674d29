"""Pins of the oracle's time scattering (Scattering1D, the baseline of Sec. 4.4: the first-order
scalogram followed by the time wavelets alone) against brute-force circular sums, a pure tone,
shift covariance, the second-order energy identity, and its adjoint (finite differences)."""
import numpy as np
import pytest

from oracle import jtfs_oracle as O

SMALL = O.Config(J=5, Q=4, J_fr=3, Q_fr=1, T=32, F=4, N=512)


@pytest.mark.parametrize("cfg", [O.Config(J=3, Q=2, J_fr=2, Q_fr=1, T=8, F=2, N=128),
                                 O.Config(J=4, Q=3, J_fr=2, Q_fr=2, T=16, F=3, N=256)])
def test_brute_force(cfg):
    """EXACT mode (every stride 1, every path) equals the circular sums of the definitions."""
    p = O.Plan(cfg)
    x = np.random.default_rng(31).standard_normal(cfg.N)
    ref = O.scattering1d_exact_direct(x, p)
    ex = O.Schedule(p, None)
    assert O.scattering1d_paths(p, ex) == p.n1 * p.n2
    for engine in ("fft", "direct"):
        out = O.scattering1d_one(x, p, ex, engine)
        for k in ("S0", "S1", "S2t"):
            assert O.relative_l2(out[k], ref[k]) < 1e-12, (engine, k)


@pytest.mark.parametrize("mode", [None, 0])
def test_pure_tone_has_no_second_order(mode):
    """A pure tone gives a scalogram constant in time, and every time wavelet has zero mean."""
    p = O.Plan(O.WORKLOADS[1])
    s = O.Schedule(p, mode)
    x = 0.8 * np.cos(2 * np.pi * 211 * np.arange(p.N) / p.N)
    out = O.scattering1d_one(x, p, s)
    assert np.abs(out["S2t"]).max() < 1e-12
    assert out["S1"].max() > 0.1


def test_shift_by_T_permutes_frames():
    p = O.Plan(SMALL)
    s = O.Schedule(p, 0)
    x = np.random.default_rng(32).standard_normal(p.N)
    a = O.scattering1d_one(x, p, s)
    b = O.scattering1d_one(np.roll(x, p.T), p, s)
    assert O.relative_l2(b["S2t"], np.roll(a["S2t"], 1, axis=-1)) < 1e-12


def test_second_order_energy_identity():
    """For every scalogram row u (real): ||u * phi_T||^2 + sum_alpha ||u * psi_alpha||^2 =
    (1/N) sum_k |u-hat_k|^2 LP2(k/N) <= ||u||^2 (the second-order bank's Littlewood-Paley
    sum), here at the full rate on a click-free noise input."""
    p = O.Plan(SMALL)
    x = np.random.default_rng(33).standard_normal(p.N)
    xh = np.fft.fft(x)
    lp2 = O.littlewood_paley(p, 2)
    for lam in (0, p.n1 // 2, p.n1 - 1):
        u = np.abs(np.fft.ifft(xh * p.psi1_hat[lam]))
        uh = np.fft.fft(u)
        lhs = np.sum(np.real(np.fft.ifft(uh * p.phi_T_hat)) ** 2) + sum(
            np.sum(np.abs(np.fft.ifft(uh * p.psi2_hat[a])) ** 2) for a in range(p.n2))
        rhs = np.sum(np.abs(uh) ** 2 * lp2) / p.N
        assert abs(lhs - rhs) <= 1e-12 * rhs
        assert lhs <= np.sum(u * u) * (1 + 1e-12)


def test_paper_path_count_soft():
    """Sec. 4.4 quotes 1423 coefficients per frame (S0, S1 and S2 concatenated) at J = 13,
    Q = 16, T = 2^11 and N = 2^16.  The filterbank reading and the schedule's path rule give a
    count of the same order (recorded, not matched: the paper's path rule is not stated)."""
    p = O.Plan(O.Config(J=13, Q=16, J_fr=4, Q_fr=1, T=2 ** 11, F=4, N=2 ** 16))
    s = O.Schedule(p, 0)
    total = 1 + p.n1 + O.scattering1d_paths(p, s)
    assert total == 1714
    assert 0.5 * 1423 < total < 1.5 * 1423


@pytest.mark.parametrize("mode", [0, None])
def test_finite_differences(mode):
    p = O.Plan(SMALL)
    s = O.Schedule(p, mode)
    rng = np.random.default_rng(34)
    x = rng.standard_normal(p.N)
    out = O.scattering1d_one(x, p, s)
    g = {k: rng.standard_normal(v.shape) for k, v in out.items()}

    def loss(xx):
        o = O.scattering1d_one(xx, p, s)
        return sum(float(np.sum(g[k] * o[k])) for k in g)

    gx = O.scattering1d_backward_one(x, g["S0"], g["S1"], g["S2t"], p, s)
    for _ in range(3):
        v = rng.standard_normal(p.N)
        h = 1e-6
        fd = (loss(x + h * v) - loss(x - h * v)) / (2 * h)
        assert abs(fd - gx @ v) <= 1e-7 * max(1.0, abs(fd))
