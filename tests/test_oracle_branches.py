"""Pins of the oracle's phi_t paths (Eq. 3 with the time lowpass phi_T in place of the time
wavelet: phi_T x psi_{beta,+1} and phi_T x phi_F) against brute force, a pure-tone closed
form, the linearity of the phi_T x phi_F path on the non-negative scalogram, the spin symmetry
that lets one spin stand for both, shift covariance, and the adjoint (dot products and finite
differences)."""
import numpy as np
import pytest

from oracle import jtfs_oracle as O

ALL = O.PSI_PSI | O.PSI_PHI | O.PHI_PSI | O.PHI_PHI
TINY = O.Config(J=3, Q=2, J_fr=2, Q_fr=1, T=8, F=2, N=128, branches=ALL)
SMALL = O.Config(J=5, Q=4, J_fr=3, Q_fr=1, T=32, F=4, N=512, branches=ALL)


def _rel(a, b):
    return O.relative_l2(a, b)


def test_path_counts_and_rejected_masks():
    p = O.Plan(SMALL)
    assert p.n_phi == p.n_fr + 1
    assert p.phi_channels == list(range(p.n_fr)) + [2 * p.n_fr]
    q = O.Plan(O.Config(**{**SMALL.__dict__, "branches": 3 | O.PHI_PHI}))
    assert q.n_phi == 1 and q.phi_channels == [2 * q.n_fr]
    assert O.Plan(O.Config(**{**SMALL.__dict__, "branches": 3})).n_phi == 0
    for bad in (1, 2, 5, 16 | 3):
        with pytest.raises(ValueError):
            O.Plan(O.Config(**{**SMALL.__dict__, "branches": bad}))


@pytest.mark.parametrize("cfg", [TINY, O.Config(**{**TINY.__dict__, "average_fr": False}),
                                 O.Config(J=4, Q=3, J_fr=2, Q_fr=2, T=16, F=3, N=256,
                                          branches=ALL)])
def test_phi_paths_brute_force(cfg):
    """EXACT mode: time-domain circular sums (X * phi_T, then the lambda convolution, modulus,
    phi_T and phi_F) equal the oracle's operator form; the scheduled machinery with every
    stride forced to 1 does too."""
    p = O.Plan(cfg)
    x = np.random.default_rng(21).standard_normal(cfg.N)
    ref = O.forward_exact_direct(x, p)
    for sched in (O.Schedule(p, None), O.Schedule(p, 50)):
        out = O.forward_one(x, p, sched)
        assert _rel(out["S2phi"], ref["S2phi"]) < 1e-12
        assert _rel(out["S2"], ref["S2"]) < 1e-12


@pytest.mark.parametrize("mode", [None, 0])
def test_phi_paths_pure_tone_closed_form(mode):
    """x = A cos(2 pi k0 n / N): the scalogram row lambda is the constant
    c_lambda = (A/2) psi-hat_lambda(k0/N), phi_T keeps it (unit DC gain), so every phi_t path is
    constant in time and equals sum_lambda PhiF[lo, lambda] |sum_lambda' h_c[lambda - lambda']
    c_lambda'| (the filters' lambda-domain taps, wrapped on the N_fr grid)."""
    cfg = O.Config(J=6, Q=8, J_fr=3, Q_fr=1, T=64, F=8, N=4096, branches=ALL)
    p = O.Plan(cfg)
    s = O.Schedule(p, mode)
    A, k0 = 1.3, 517
    x = A * np.cos(2 * np.pi * k0 * np.arange(p.N) / p.N)
    out = O.forward_one(x, p, s)
    c = 0.5 * A * p.psi1_hat[:, k0]
    lam = np.arange(p.n1)
    taps = np.fft.ifft(p.fr_hat, axis=-1)
    for q, ch in enumerate(p.phi_channels):
        H = taps[ch][(lam[:, None] - lam[None, :]) % p.N_fr]
        prof = np.abs(H @ c)
        expect = p.PhiF @ prof
        np.testing.assert_allclose(out["S2phi"][q], np.repeat(expect[:, None], p.n_t, 1),
                                   rtol=1e-10, atol=1e-12 * A)


def test_phi_phi_path_is_linear_in_s1():
    """phi_T and phi_F are positive and the scalogram is non-negative, so the modulus of the
    phi_T x phi_F path acts on a non-negative signal and drops out: the path is the linear map
    PhiF (H_phi S1) P_T^T of S1 (at oversampling 0 the phi_t paths' input is S1 itself)."""
    p = O.Plan(SMALL)
    s = O.Schedule(p, 0)
    assert s.s_phi == p.T
    x = np.random.default_rng(22).standard_normal(p.N)
    out = O.forward_one(x, p, s)
    lam = np.arange(p.n1)
    taps = np.fft.ifft(p.fr_hat[2 * p.n_fr])
    assert np.max(np.abs(taps.imag)) < 1e-15 and taps.real.min() > 0
    H = taps.real[(lam[:, None] - lam[None, :]) % p.N_fr]
    t = np.arange(p.n_t)
    PT = p.T * p.phi_T[((t[:, None] - t[None, :]) * p.T) % p.N]
    assert PT.min() > 0
    np.testing.assert_allclose(out["S2phi"][-1], p.PhiF @ (H @ out["S1"]) @ PT.T, rtol=1e-12)


def test_spin_down_phi_path_equals_spin_up():
    """The phi_t paths' input X * phi_T is real and the spin-down filters are the conjugates
    of the spin-up ones, so their Z are conjugate and their moduli equal: one spin suffices."""
    p = O.Plan(SMALL)
    s = O.Schedule(p, 0)
    ops = O.Operators(p, s)
    x = np.random.default_rng(23).standard_normal(p.N)
    out = O.forward_one(x, p, s, keep=True)
    Yp = out["Yphi"]
    for beta in range(p.n_fr):
        up = ops.pool_F(ops.pool_T(np.abs(ops.wfr(Yp, beta)), int(s.s_phi)))
        down = ops.pool_F(ops.pool_T(np.abs(ops.wfr(Yp, beta + p.n_fr)), int(s.s_phi)))
        assert _rel(down, up) < 1e-13
        assert _rel(out["S2phi"][beta], up) < 1e-15


def test_phi_paths_shift_by_T_permutes_frames():
    p = O.Plan(SMALL)
    s = O.Schedule(p, 0)
    x = np.random.default_rng(24).standard_normal(p.N)
    a = O.forward_one(x, p, s)
    b = O.forward_one(np.roll(x, p.T), p, s)
    assert _rel(b["S2phi"], np.roll(a["S2phi"], 1, axis=-1)) < 1e-12


@pytest.mark.parametrize("mode", [0, None])
def test_lowpass_operator_adjoint(mode):
    p = O.Plan(SMALL)
    s = O.Schedule(p, mode)
    ops = O.Operators(p, s)
    rng = np.random.default_rng(25)
    sp = int(s.s_phi)
    for lam in (0, p.n1 // 2, p.n1 - 1):
        sl = int(s.s1[lam])
        u = rng.standard_normal(p.N // sl)
        g = rng.standard_normal(p.N // sp)
        assert abs(ops.lowpass_to(u, sl, sp) @ g - u @ ops.lowpass_to_T(g, sl, sp)) < 1e-12


@pytest.mark.parametrize("cfg,mode", [(TINY, 0), (SMALL, 0), (SMALL, None),
                                      (O.Config(**{**SMALL.__dict__, "average_fr": False}), 0)])
def test_phi_paths_finite_differences(cfg, mode):
    p = O.Plan(cfg)
    s = O.Schedule(p, mode)
    rng = np.random.default_rng(26)
    x = rng.standard_normal(p.N)
    out = O.forward_one(x, p, s)
    g = {k: rng.standard_normal(v.shape) for k, v in out.items()}

    def loss(xx):
        o = O.forward_one(xx, p, s)
        return sum(float(np.sum(g[k] * o[k])) for k in g)

    gx = O.backward_one(x, g["S0"], g["S1"], g["S2"], p, s, gS2phi=g["S2phi"])
    for _ in range(3):
        v = rng.standard_normal(p.N)
        h = 1e-6
        fd = (loss(x + h * v) - loss(x - h * v)) / (2 * h)
        assert abs(fd - gx @ v) <= 1e-7 * max(1.0, abs(fd))
