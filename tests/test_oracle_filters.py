"""Pins of the oracle's filterbanks (Sec. 2, Eq. 1, Sec. 4.2) against facts that do not
come from the oracle's own formulas: closed-form properties, an independent count
derivation, the Littlewood-Paley bound and energy identities."""
import json
import math
import os

import numpy as np
import pytest

from oracle import jtfs_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TINY = O.Config(J=3, Q=2, J_fr=2, Q_fr=1, T=8, F=2, N=128)


def _count_closed_form(J, Q):
    """Filter count derived independently: the constant-Q part stops when
    rho xi_0 2^{-k/Q} < sigma_min, i.e. k > Q log2(rho xi_0 / sigma_min); the linear part
    keeps xi_last - m Delta >= Delta, i.e. m <= xi_last / Delta - 1."""
    rho = (1 - 2 ** (-1 / Q)) / (2 * math.sqrt(2 * math.log(2)))
    xi0 = min(0.35, 0.5 / (1 + 4 * rho))
    smin = 0.1 / 2 ** J
    n_cq = math.floor(Q * math.log2(rho * xi0 / smin)) + 1
    xi_last = xi0 * 2 ** (-(n_cq - 1) / Q)
    delta = 2 * math.sqrt(2 * math.log(2)) * smin
    n_lin = max(0, math.floor(xi_last / delta) - 1)
    return n_cq + n_lin


@pytest.mark.parametrize("w", sorted(O.WORKLOADS))
def test_counts_closed_form_and_locked(w):
    cfg = O.WORKLOADS[w]
    p = O.Plan(cfg)
    assert p.n1 == _count_closed_form(cfg.J, cfg.Q)
    assert p.n2 == _count_closed_form(cfg.J, cfg.Q2)
    assert p.n_fr == _count_closed_form(cfg.J_fr, cfg.Q_fr)
    locked = json.load(open(os.path.join(GOLDEN, "counts.json")))[str(w)]
    for k, v in p.shapes().items():
        assert locked[k] == v, k
    s = O.Schedule(p, cfg.oversampling)
    np.testing.assert_array_equal(s.s1, locked["s1"])
    np.testing.assert_array_equal(s.s2, locked["s2"])
    np.testing.assert_array_equal(s.lam_min, locked["lam_min"])


@pytest.mark.parametrize("w", sorted(O.WORKLOADS))
def test_locked_schedule_samples_each_band_critically(w):
    """The stored strides are the sampling rule of the schedule, checked as properties of the
    sampled bands rather than by re-evaluating its formula: each first-order row's stride s is
    a power of two whose Nyquist 1/(2s) covers the envelope band |w| <= 8 sigma (no aliasing)
    while 2s would not (critical), unless s is capped at T; each kept second-order rate's
    stride covers its band width [xi - 4 sigma, xi + 4 sigma] clipped to the finest
    first-order Nyquist, critically or capped at T; a rate whose clipped band is empty is
    skipped; lam_min is the first first-order row whose Nyquist lies above the band's low
    edge (rows below it are identically zero after the time wavelet)."""
    cfg = O.WORKLOADS[w]
    p = O.Plan(cfg)
    lk = json.load(open(os.path.join(GOLDEN, "counts.json")))[str(w)]
    s1 = np.array(lk["s1"])
    for sig, s in zip(p.sigma1, s1):
        assert s >= 1 and (s & (s - 1)) == 0 and s <= p.T
        assert 1.0 / (2 * s) >= 8 * sig or s == 1
        assert s == p.T or 1.0 / (4 * s) < 8 * sig
    nyq = 0.5 / s1.min()
    for a, (xi, sig) in enumerate(zip(p.xi2, p.sigma2)):
        lo, hi = max(0.0, xi - 4 * sig), min(xi + 4 * sig, nyq)
        s = lk["s2"][a]
        if lo >= hi:
            assert lk["lam_min"][a] == p.n1
            continue
        assert (s & (s - 1)) == 0 and s <= p.T
        assert 1.0 / (2 * s) >= hi - lo or s == 1
        assert s == p.T or 1.0 / (4 * s) < hi - lo
        above = [lam for lam in range(p.n1) if 0.5 / s1[lam] > lo]
        assert lk["lam_min"][a] == (above[0] if above else p.n1)
        assert all(0.5 / s1[lam] <= lo for lam in range(lk["lam_min"][a]))


def test_paper_frame_count():
    """Sec. 4.2: N = 2^16 and T = 2^11 give 32 frames along time."""
    facts = json.load(open(os.path.join(GOLDEN, "paper_facts.json")))
    p = O.Plan(O.Config(J=13, Q=16, J_fr=6, Q_fr=1, T=2 ** 11, F=4, N=2 ** 16))
    assert p.n_t == facts["frames_N65536_T2048"]["value"]
    # J = 13 second-order bank: one filter per octave plus one linear filter
    assert p.n2 == 14


@pytest.mark.parametrize("w", [1, 2])
def test_analytic_and_nyquist(w):
    """Sec. 2: psi-hat(omega) = 0 for omega < 0; the grid's omega = 0 and 1/2 bins are 0 too."""
    p = O.Plan(O.WORKLOADS[w])
    N = p.N
    for bank in (p.psi1_hat, p.psi2_hat):
        assert np.all(bank[:, 0] == 0.0)
        assert np.all(bank[:, N // 2:] == 0.0)
        assert np.all(bank[:, 1:N // 2].max(axis=1) > 0.5)
    Nf = p.N_fr
    up, down = p.fr_hat[: p.n_fr], p.fr_hat[p.n_fr: 2 * p.n_fr]
    assert np.all(up[:, Nf // 2:] == 0.0) and np.all(up[:, 0] == 0.0)
    assert np.all(down[:, : Nf // 2 + 1] == 0.0)


def test_zero_mean_is_continuous_at_dc():
    """The Morlet's DC correction makes psi-hat(omega) -> 0 as omega -> 0+ (zero mean in
    time), linearly with slope kappa xi / sigma^2; without the correction the limit would
    be kappa > 0.  Checked where kappa is not negligible: the lowest first-order filters
    and every Q2 = 1 second-order filter."""
    p = O.Plan(O.WORKLOADS[2])
    checked = 0
    pairs = list(zip(p.xi1[:20], p.sigma1[:20])) + list(zip(p.xi2, p.sigma2))
    for xi, s in pairs:
        kappa = math.exp(-xi * xi / (2 * s * s))
        if kappa < 1e-12:
            continue
        checked += 1
        assert abs(float(O.morlet_hat(np.array([1e-9]), xi, s)[0])) < 1e-3 * kappa
        for eps in (1e-9, 1e-10):
            v = float(O.morlet_hat(np.array([eps]), xi, s)[0])
            assert abs(v) <= 1.01 * kappa * xi / s ** 2 * eps + 1e-18
    assert checked >= 10
    # time-domain mean of every filter is 0 (psi-hat at DC)
    psi_t = np.fft.ifft(p.psi1_hat, axis=-1)
    assert np.max(np.abs(psi_t.sum(axis=-1))) < 1e-12


def test_eq1_dilation_of_constant_q_part():
    """Eq. 1: psi_k(t) = 2^{-k/Q} psi_0(2^{-k/Q} t), i.e. psi-hat_k(omega) = psi-hat_0(2^{k/Q} omega),
    for every constant-Q filter, at arbitrary (off-grid) frequencies."""
    cfg = O.WORKLOADS[2]
    xi, sg = O.morlet_bank(cfg.J, cfg.Q)
    rho = (1 - 2 ** (-1 / cfg.Q)) / (2 * math.sqrt(2 * math.log(2)))
    rng = np.random.default_rng(0)
    n_cq = int(np.sum(np.isclose(sg, rho * xi, rtol=1e-12)))
    assert n_cq == 129
    for k in range(0, n_cq, 7):
        d = 2.0 ** (k / cfg.Q)
        om = rng.uniform(xi[k] - 5 * sg[k], xi[k] + 5 * sg[k], size=64)
        om = om[(om > 0) & (om * d < 0.5)]
        a = O.morlet_hat(om, xi[k], sg[k])
        b = O.morlet_hat(om * d, xi[0], sg[0])
        np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-300)


def test_eq1_equal_l1_norms_in_time():
    """Eq. 1's 2^alpha factor keeps the L1 norm of every dilation equal: the time-domain
    L1 norms of well-resolved constant-Q filters agree (discretisation error only)."""
    p = O.Plan(O.WORKLOADS[2])
    psi_t = np.fft.ifft(p.psi1_hat / p.c1, axis=-1)
    l1 = np.abs(psi_t).sum(axis=-1)
    # constant-Q filters away from both ends of the bank (resolved in time and frequency)
    cq = slice(p.n1 - 100, p.n1 - 10)
    v = l1[cq]
    assert np.max(np.abs(v / v.mean() - 1.0)) < 1e-3


def test_half_maximum_crossing():
    """rho is chosen from the half-maximum rule: the half-widths at half maximum of two
    neighbours add up to their spacing.  With sigma proportional to xi, two Gaussians
    a ratio r = 2^{-1/Q} apart then cross at 2^{-4 / (1 + r)^2}, which tends to 1/2 as Q grows."""
    for Q in (1, 2, 8, 12, 16):
        xi, sg = O.morlet_bank(10, Q)
        r = 2.0 ** (-1.0 / Q)
        expect = 2.0 ** (-4.0 / (1.0 + r) ** 2)
        for k in range(0, 4):
            a, b = xi[k + 1], xi[k]
            om = np.linspace(a, b, 400001)
            d = np.abs(O.morlet_hat(om, xi[k], sg[k]) - O.morlet_hat(om, xi[k + 1], sg[k + 1]))
            v = float(O.morlet_hat(om[np.argmin(d)], xi[k], sg[k]))
            assert abs(v - expect) < 1e-4, (Q, k, v, expect)
            if Q >= 8:
                assert 0.45 <= v <= 0.55


@pytest.mark.parametrize("Q", [1, 2, 8, 16])
def test_top_band_fits_below_nyquist(Q):
    xi, sg = O.morlet_bank(8, Q)
    assert xi[0] <= 0.35 + 1e-15
    assert xi[0] + 4 * sg[0] <= 0.5 + 1e-15


@pytest.mark.parametrize("w", [1, 2, 4])
@pytest.mark.parametrize("order", [1, 2, 3])
def test_littlewood_paley_bound(w, order):
    """LP(omega) <= 1 on every bin, = 1 at DC, and tight (= 1) at one bin inside the band."""
    p = O.Plan(O.WORKLOADS[w])
    lp = O.littlewood_paley(p, order)
    assert lp.max() <= 1.0 + 1e-12
    assert abs(lp[0] - 1.0) < 1e-15
    G = lp.shape[0]
    assert abs(lp[1:G // 2].max() - 1.0) < 1e-12
    assert lp[1:G // 2].min() > 0.0


def test_lp_lower_bound_locked():
    b = json.load(open(os.path.join(GOLDEN, "lp_bounds.json")))
    for w in (1, 2, 4):
        p = O.Plan(O.WORKLOADS[w])
        lp = O.littlewood_paley(p, 1)
        om = O.grid_freqs(p.N)
        band = (om >= p.xi1.min()) & (om <= p.xi1.max())
        assert abs(lp[band].min() - b[str(w)]["A1"]) < 1e-12
        assert abs(p.c1 - b[str(w)]["c1"]) < 1e-12
        assert 0.3 < b[str(w)]["A1"] < 1.0


def test_spin_down_is_mirror():
    """Eq. 1: psi_{beta,-1}(lambda) = psi_{beta,+1}(-lambda), so its spectrum is mirrored."""
    p = O.Plan(O.WORKLOADS[2])
    Nf = p.N_fr
    j = np.arange(Nf)
    for b in range(p.n_fr):
        np.testing.assert_array_equal(p.fr_hat[p.n_fr + b], p.fr_hat[b][(-j) % Nf])
    np.testing.assert_allclose(p.h[p.n_fr:2 * p.n_fr], p.h[:p.n_fr][:, (-j) % Nf], atol=1e-15)


def test_lambda_axis_energy_identity():
    """Frame identity of the frequential bank on its circular grid: for any complex v,
    sum_c ||h_c (*) v||^2 = (1/N_fr) sum_j |v-hat_j|^2 (phi_F^2 + sum_beta psi_beta(w)^2 + psi_beta(-w)^2).
    This ties the time-domain lambda filters h (used by the contraction) to their spectra."""
    p = O.Plan(O.WORKLOADS[2])
    Nf = p.N_fr
    rng = np.random.default_rng(3)
    v = np.zeros(Nf, dtype=complex)
    v[: p.n1] = rng.standard_normal(p.n1) + 1j * rng.standard_normal(p.n1)
    n = np.arange(Nf)
    lhs = 0.0
    for c in range(p.C):
        Hc = p.h[c][(n[:, None] - n[None, :]) % Nf]
        lhs += np.sum(np.abs(Hc @ v) ** 2)
    vh = np.fft.fft(v)
    ps = p.fr_hat[: p.n_fr]
    frame = p.phi_F_hat ** 2 + np.sum(ps ** 2 + ps[:, (-n) % Nf] ** 2, axis=0)
    rhs = np.sum(np.abs(vh) ** 2 * frame) / Nf
    assert abs(lhs - rhs) / rhs < 1e-12


@pytest.mark.parametrize("w", sorted(O.WORKLOADS))
def test_spin_down_is_conjugate(w):
    """The spin-down filter is the complex conjugate of the spin-up one (real spectra that
    vanish at DC and Nyquist), so W_{c + n_fr} = conj(W_c); the contractions build both spins
    from the four real products of the spin-up rows (Sec. 2, spin pairs)."""
    p = O.Plan(O.WORKLOADS[w])
    nf = p.n_fr
    for b in range(nf):
        assert p.fr_hat[b][p.N_fr // 2] == 0.0 and p.fr_hat[b][0] == 0.0
    np.testing.assert_allclose(p.h[nf:2 * nf], np.conj(p.h[:nf]), rtol=0, atol=1e-15)
    np.testing.assert_allclose(p.W[nf:2 * nf], np.conj(p.W[:nf]), rtol=0, atol=1e-15)


def test_spin_pair_products_and_adjoint():
    """The spin-pair algebra on the oracle's W: with W_up = Wr + i Wi,
    Z_up = (Wr Yr - Wi Yi) + i (Wr Yi + Wi Yr) and Z_dn = (Wr Yr + Wi Yi) + i (Wr Yi - Wi Yr)
    equal W_up Y and W_dn Y; and W_up^H gZ_up + W_dn^H gZ_dn = Wr^T S + Wi^T T with
    S = gZ_up + gZ_dn, T = (Im gZ_up - Im gZ_dn) + i (Re gZ_dn - Re gZ_up)."""
    p = O.Plan(O.WORKLOADS[2])
    rng = np.random.default_rng(16)
    Y = rng.standard_normal((p.n1, 7)) + 1j * rng.standard_normal((p.n1, 7))
    for b in range(p.n_fr):
        Wu, Wd = p.W[b], p.W[b + p.n_fr]
        Wr, Wi = Wu.real, Wu.imag
        P1, P2, P3, P4 = Wr @ Y.real, Wi @ Y.imag, Wr @ Y.imag, Wi @ Y.real
        np.testing.assert_allclose(P1 - P2 + 1j * (P3 + P4), Wu @ Y, atol=1e-13)
        np.testing.assert_allclose(P1 + P2 + 1j * (P3 - P4), Wd @ Y, atol=1e-13)
        gu = rng.standard_normal((p.n1, 7)) + 1j * rng.standard_normal((p.n1, 7))
        gd = rng.standard_normal((p.n1, 7)) + 1j * rng.standard_normal((p.n1, 7))
        S = gu + gd
        T = (gu.imag - gd.imag) + 1j * (gd.real - gu.real)
        np.testing.assert_allclose(Wr.T @ S + Wi.T @ T,
                                   Wu.conj().T @ gu + Wd.conj().T @ gd, atol=1e-13)


@pytest.mark.parametrize("w", [1, 2, 4])
def test_band_support_bound_of_the_time_wavelets(w):
    """The GPU keeps each time wavelet psi-hat on |omega - xi| <= 8 sigma (first order) and
    folds psi_alpha-hat up to xi_alpha + 8 sigma_alpha.  Outside those bands both Morlet terms
    (the Gaussian at xi and the zero-mean correction kappa e^{-omega^2 / 2 sigma^2}) stay below
    e^-32 of the filter's peak, on every bin of the N-point grid."""
    p = O.Plan(O.WORKLOADS[w])
    om = np.arange(1, p.N // 2) / float(p.N)
    bound = math.exp(-32.0) * (1.0 + 1e-9)
    for xi, sig, both in ((p.xi1, p.sigma1, True), (p.xi2, p.sigma2, False)):
        for x, s in zip(xi, sig):
            h = np.abs(O.morlet_hat(om, float(x), float(s)))
            peak = h.max()
            out = om > x + 8.0 * s
            if both:
                out |= om < x - 8.0 * s
            if out.any():
                assert h[out].max() <= bound * peak, (w, x, s)
