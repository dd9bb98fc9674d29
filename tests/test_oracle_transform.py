"""Pins of the oracle's forward transform (Sec. 2, Eq. 2-4) against brute force, energy
identities, closed forms for tones, and exact symmetries of the definition."""
import numpy as np
import pytest

import synth_signals as SS
from oracle import jtfs_oracle as O

TINY = O.Config(J=3, Q=2, J_fr=2, Q_fr=1, T=8, F=2, N=128)
SMALL = O.Config(J=5, Q=4, J_fr=3, Q_fr=1, T=32, F=4, N=512)
SMALL4 = O.Config(J=5, Q=4, J_fr=3, Q_fr=1, T=32, F=4, N=512, average_fr=False)
KEYS = ("S0", "S1", "S2")


def _rel(a, b):
    return O.relative_l2(a, b)


@pytest.mark.parametrize("cfg", [TINY, O.Config(J=4, Q=3, J_fr=2, Q_fr=2, T=16, F=3, N=256),
                                 O.Config(J=3, Q=2, J_fr=2, Q_fr=1, T=8, F=2, N=128,
                                          average_fr=False)])
def test_brute_force_time_domain_equals_fft_engines(cfg):
    """EXACT mode: circular sums of the time-domain filters == spectral products (numpy FFT
    and the explicit DFT matrices)."""
    p = O.Plan(cfg)
    x = np.random.default_rng(1).standard_normal(cfg.N)
    ref = O.forward_exact_direct(x, p)
    ex = O.Schedule(p, None)
    for engine in ("fft", "direct"):
        out = O.forward_one(x, p, ex, engine)
        for k in KEYS:
            assert _rel(out[k], ref[k]) < 1e-12, (engine, k)


def test_schedule_with_unit_strides_is_exact():
    """The SCHEDULED machinery (periodisation, row skipping, Riemann pooling) with every
    stride forced to 1 reproduces the brute-force definition."""
    p = O.Plan(O.Config(J=4, Q=3, J_fr=2, Q_fr=2, T=16, F=3, N=256))
    s = O.Schedule(p, 50)
    assert s.s1.max() == 1 and s.s2.max() == 1
    x = np.random.default_rng(2).standard_normal(p.N)
    ref = O.forward_exact_direct(x, p)
    out = O.forward_one(x, p, s)
    for k in KEYS:
        assert _rel(out[k], ref[k]) < 1e-12


def test_stage1_parseval_identity():
    """For real x: ||x * phi_T||^2 + sum_lambda ||x * psi_lambda||^2 = (1/N) sum_k |x-hat_k|^2 LP(k/N),
    which is at most ||x||^2 by the Littlewood-Paley bound."""
    for w in (1, 2):
        p = O.Plan(O.WORKLOADS[w])
        x = SS.workload_signals(w, 1, p.N)[0].astype(np.float64)
        low, z = O.stage1_full_rate(x, p)
        lhs = np.sum(low ** 2) + np.sum(np.abs(z) ** 2)
        xh = np.fft.fft(x)
        rhs = np.sum(np.abs(xh) ** 2 * O.littlewood_paley(p, 1)) / p.N
        assert abs(lhs - rhs) / rhs < 1e-12
        assert lhs <= np.sum(x ** 2) * (1 + 1e-12)


@pytest.mark.parametrize("mode", [None, 0])
def test_pure_tone_closed_forms(mode):
    """x = A cos(2 pi k0 n / N): |x * psi_lambda| = (A/2) psi-hat_lambda(k0/N) at every n, so
    S1 is that constant; S0[t] = A phi-hat_T(k0/N) cos(2 pi k0 t T / N); and the scalogram is
    constant in time, so every time wavelet (zero mean) gives S2 = 0."""
    p = O.Plan(O.WORKLOADS[1])
    s = O.Schedule(p, mode)
    A, k0 = 1.7, 301
    n = np.arange(p.N)
    x = A * np.cos(2 * np.pi * k0 * n / p.N)
    out = O.forward_one(x, p, s)
    s1 = 0.5 * A * p.psi1_hat[:, k0]
    np.testing.assert_allclose(out["S1"], np.repeat(s1[:, None], p.n_t, 1), rtol=1e-12,
                               atol=1e-13 * A)
    t = np.arange(p.n_t) * p.T
    s0 = A * p.phi_T_hat[k0] * np.cos(2 * np.pi * k0 * t / p.N)
    np.testing.assert_allclose(out["S0"], s0, atol=1e-13 * A)
    assert np.abs(out["S2"]).max() < 1e-12 * A


def test_homogeneity():
    p = O.Plan(SMALL)
    s = O.Schedule(p, 0)
    x = np.random.default_rng(4).standard_normal(p.N)
    a = O.forward_one(x, p, s)
    b = O.forward_one(-2.5 * x, p, s)
    for k in ("S1", "S2"):
        assert _rel(b[k], 2.5 * a[k]) < 1e-13
    assert _rel(b["S0"], -2.5 * a["S0"]) < 1e-13


@pytest.mark.parametrize("cfg", [SMALL, SMALL4])
def test_shift_by_T_permutes_frames(cfg):
    """A circular shift by T samples shifts every output by one frame, exactly, in SCHEDULED
    mode too (every stride divides T)."""
    p = O.Plan(cfg)
    s = O.Schedule(p, 0)
    x = np.random.default_rng(5).standard_normal(p.N)
    a = O.forward_one(x, p, s)
    b = O.forward_one(np.roll(x, p.T), p, s)
    for k in KEYS:
        assert _rel(b[k], np.roll(a[k], 1, axis=-1)) < 1e-12


def test_approximate_shift_invariance_below_T():
    """Shifts tau < T change S1 and S2 only a little, and the change grows with tau."""
    p = O.Plan(O.WORKLOADS[1])
    s = O.Schedule(p, 0)
    x = SS.workload_signals(1, 1, p.N)[0].astype(np.float64)
    a = O.forward_one(x, p, s)
    errs = []
    for tau in (1, 4, 16):
        b = O.forward_one(np.roll(x, tau), p, s)
        errs.append(_rel(b["S1"], a["S1"]))
    assert errs[0] < errs[1] < errs[2] < 0.2
    assert errs[0] < 0.02


@pytest.mark.parametrize("cfg", [SMALL, SMALL4])
def test_time_reversal_swaps_spin(cfg):
    """Real psi-hat gives psi(-t) = conj psi(t); hence reversing x reverses the scalogram,
    conjugates Y, and maps h_{beta,theta} to conj = h_{beta,-theta}:
    S2(x(-n))[alpha, beta, theta, :, t] = S2(x)[alpha, beta, -theta, :, -t mod n_t]."""
    p = O.Plan(cfg)
    s = O.Schedule(p, 0)
    x = np.random.default_rng(6).standard_normal(p.N)
    xr = x[(-np.arange(p.N)) % p.N]
    a = O.forward_one(x, p, s)
    b = O.forward_one(xr, p, s)
    tr = (-np.arange(p.n_t)) % p.n_t
    nf = p.n_fr
    perm = np.r_[np.arange(nf, 2 * nf), np.arange(nf), 2 * nf]
    assert _rel(b["S0"], a["S0"][tr]) < 1e-12
    assert _rel(b["S1"], a["S1"][:, tr]) < 1e-12
    assert _rel(b["S2"], a["S2"][:, perm][..., tr]) < 1e-12
    # and the two spins are genuinely different for this input
    assert _rel(a["S2"][:, :nf], a["S2"][:, nf:2 * nf]) > 1e-3


@pytest.mark.parametrize("fc,fm,gamma", [(1000.0, 8.0, 4.0), (2000.0, 16.0, 2.0),
                                         (700.0, 4.0, 3.0)])
def test_up_chirp_energy_on_theta_minus_one(fc, fm, gamma):
    """Sec. 2 / Fig. 1(a): for an upward AM chirp the JTFS energy concentrates on theta = -1;
    its time reversal (downward) puts it on theta = +1.  Input: the paper's Eq. 5 generator."""
    cfg = O.Config(J=10, Q=8, J_fr=4, Q_fr=1, T=2 ** 10, F=8, N=2 ** 14)
    p = O.Plan(cfg)
    s = O.Schedule(p, 0)
    for g, sign in ((gamma, -1), (-gamma, +1)):
        x = SS.chirp_eq5(p.N, fc, fm, g).astype(np.float64)
        S2 = O.forward_one(x, p, s)["S2"]
        e_plus = np.sum(S2[:, : p.n_fr] ** 2)
        e_minus = np.sum(S2[:, p.n_fr: 2 * p.n_fr] ** 2)
        if sign == -1:
            assert e_minus > 2.5 * e_plus
        else:
            assert e_plus > 2.5 * e_minus


def test_scheduled_approaches_exact_with_oversampling():
    """Measured, not pinned: the schedule's aliasing shrinks as the oversampling grows."""
    p = O.Plan(O.WORKLOADS[1])
    x = SS.workload_signals(1, 1, p.N)[0].astype(np.float64)
    ex = O.forward_one(x, p, O.Schedule(p, None))
    errs = []
    for o in (0, 1, 2):
        sc = O.forward_one(x, p, O.Schedule(p, o))
        assert _rel(sc["S0"], ex["S0"]) < 1e-14
        errs.append((_rel(sc["S1"], ex["S1"]), _rel(sc["S2"], ex["S2"])))
    assert errs[0][1] > errs[1][1] > errs[2][1]
    assert errs[0][1] < 1e-2 and errs[2][1] < 2e-4


@pytest.mark.parametrize("cfg", [SMALL, O.WORKLOADS[1]])
def test_time_pooling_is_a_product_on_the_aliased_lowpass_spectrum(cfg):
    """The phi_T Riemann sums at stride s (L = N / s samples) and their adjoint, written from
    the definition phi_T[n] = (1/N) sum_q phi-hat[q] e^{2 pi i q n / N}.  With T / s an
    integer, the sums fold the spectrum onto L bins:
      S[t] = (1/L) sum_k Phi[k] U[k] e^{2 pi i k t / n_t},  Phi[k] = sum_r phi-hat[k + r L],
    and the adjoint is the inverse L-point DFT of Phi[k] G[k mod n_t] (G the n_t-point DFT of
    the cotangent; phi-hat is real and even).  Keeping only the bins |q| <= ceil(12 sigma_T N)
    (phi-hat < e^-72 beyond) changes neither.  The oracle keeps the time-domain sums."""
    p = O.Plan(cfg)
    rng = np.random.default_rng(7)
    N, n_t = p.N, p.n_t
    q = np.where(np.arange(N) <= N // 2, np.arange(N), np.arange(N) - N)
    kmax = int(np.ceil(12.0 * p.sigma_T * N))
    ph_trunc = np.where(np.abs(q) <= kmax, p.phi_T_hat, 0.0)
    assert np.max(np.abs(p.phi_T_hat - ph_trunc)) < np.exp(-72.0)
    s = 1
    while s <= p.T:
        L = N // s
        Phi = p.pool_T_matrix(s)
        u = rng.standard_normal(L)
        g = rng.standard_normal(n_t)
        for ph in (p.phi_T_hat, ph_trunc):
            fold = ph.reshape(N // L, L).sum(axis=0)               # Phi[k], k < L
            k = np.arange(L)
            S = (fold * np.fft.fft(u)) @ np.exp(2j * np.pi * np.outer(k, np.arange(n_t)) / n_t) / L
            assert np.max(np.abs(S.imag)) < 1e-12 * np.max(np.abs(S.real))
            assert _rel(S.real, Phi @ u) < 1e-12, s
            gu = np.fft.ifft(fold * np.fft.fft(g)[k % n_t])
            assert np.max(np.abs(gu.imag)) < 1e-12 * np.max(np.abs(gu.real))
            assert _rel(gu.real, g @ Phi) < 1e-12, s
        s *= 2


def test_mu_log_definitions():
    """Eq. 6-7: mu is the mean over examples of each path's sum over (lambda, t) (checked by an
    explicit loop); the compression is invariant to one scale factor applied to the whole
    dataset (mu scales with it), increasing in S, and 0 where S = 0."""
    rng = np.random.default_rng(40)
    S = rng.gamma(2.0, 1.0, size=(5, 7, 3, 4))
    mu = O.mu_log_mean(S)
    for p in range(7):
        assert abs(mu[p] - sum(S[n, p].sum() for n in range(5)) / 5) < 1e-12 * mu[p]
    a = O.mu_log(S, mu)
    b = O.mu_log(3.7 * S, O.mu_log_mean(3.7 * S))
    assert np.max(np.abs(a - b)) < 1e-14
    assert np.all(O.mu_log(S + 1.0, mu) > a)
    assert np.all(O.mu_log(np.zeros_like(S), mu) == 0.0)


def test_schedule_measurement_script():
    """oracle.measure_schedule reports SCHEDULED against EXACT per order; on a small workload
    the departure shrinks with the oversampling and vanishes once every stride is 1."""
    from oracle import measure_schedule as MS
    O.WORKLOADS[99] = O.Config(J=4, Q=3, J_fr=2, Q_fr=2, T=16, F=3, N=256)
    try:
        import synth_signals as SS
        orig = SS.workload_signals
        SS.workload_signals = lambda c, B, N: SS.white_noise_batch(B, N, 99)
        res = MS.measure(99, 2, [0, 1, 50])
    finally:
        SS.workload_signals = orig
        del O.WORKLOADS[99]
    r = res["oversampling"]
    assert r[0]["S2"] >= r[1]["S2"] and r[0]["S1"] >= r[1]["S1"]
    assert r[50]["S1"] < 1e-12 and r[50]["S2"] < 1e-12
    assert r[50]["L1_max"] == 256
