"""FP64 CPU oracle for the joint time-frequency scattering (JTFS) transform.

TEST INFRASTRUCTURE ONLY.  This module is the independent, plain, slow reference that
the CUDA path is checked against.  Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it; the product path never does.  It
shares no code with the CUDA library (no kernels, headers, tables or helpers).

What it computes (paper: "Differentiable time-frequency scattering on GPU", DAFx 2022):

* Sec. 2: first-order scalogram X(t, lambda) = |x * psi_lambda|(t) with analytic Morlet
  wavelets (psi-hat = 0 for omega < 0), S0 = x * phi_T and S1 = X * phi_T sampled every
  T samples (no frequential averaging on S1, Sec. 4.2).
* Eq. 1: dilations psi_alpha(t) = 2^alpha psi(2^alpha t) (time rates) and
  psi_{beta,theta}(lambda) = 2^beta psi(theta 2^beta lambda) (frequential scales, spin
  theta = +-1; theta = -1 is the positive slope).
* Eq. 2: the joint wavelet is the separable outer product psi_alpha(t) psi_{beta,theta}(lambda).
* Eq. 3: S2 = (|X *_{t,lambda} Psi_{alpha,beta,theta}| *_{t,lambda} Phi_{T,F}) subsampled by
  (T, 2^floor(log2 F)); Eq. 4: the variant with time-only averaging.
* Sec. 5: gradients by reverse-ordered adjoints of the forward operators.

Where the paper is silent the oracle follows these readings (all of them restated in the
design notes of the repository):

* Filterbank rule FB-P.  For a bank (J, Q): rho = (1 - 2^{-1/Q}) / (2 sqrt(2 ln 2)) (half-maximum
  crossing of neighbours), xi_0 = min(0.35, 0.5 / (1 + 4 rho)), sigma_min = 0.1 * 2^-J.  Constant-Q
  filters xi_k = xi_0 2^{-k/Q}, sigma_k = rho xi_k while sigma_k >= sigma_min; then linearly spaced
  filters xi = xi_last - m * Delta, Delta = 2 sqrt(2 ln 2) sigma_min, sigma = sigma_min, while xi >= Delta.
  Morlet: psi-hat(w) = c [exp(-(w-xi)^2 / 2 sigma^2) - kappa exp(-w^2 / 2 sigma^2)] on 0 < w < 1/2,
  kappa = exp(-xi^2 / 2 sigma^2) (zero mean), 0 elsewhere.  Lowpass phi-hat(w) = exp(-w^2 / 2 sigma_phi^2),
  sigma_phi = 0.1 / T (time) or 0.1 / F (log-frequency).  One scalar c per bank makes the
  Littlewood-Paley sum phi-hat^2 + (c^2/2) sum |psi-hat(w)|^2 + |psi-hat(-w)|^2 <= 1 with equality
  at its tightest grid bin.
* The log-frequency axis lambda increases with frequency; the frequential convolution is
  zero-padded (linear) on a grid of N_fr = 2 * 2^ceil(log2 n1) bins; everything along time is
  periodic on the N-sample grid.
* EXACT mode evaluates the definitions at the full sampling rate.  SCHEDULED mode (rule S-P,
  the GPU's schedule) computes every first-order row at its own stride
  s_lambda = min(T, 2^max(0, floor(log2(1 / (16 sigma_lambda))) - o)) by periodising the spectrum
  (exact sampling), computes Y_alpha at a common stride s_alpha from the width of psi_alpha's
  band [xi - 4 sigma, xi + 4 sigma] clipped to the finest first-order Nyquist, skips rows whose
  Nyquist lies below the band, and pools with Riemann sums of phi_T at each stride.  With
  every stride 1 it reduces to EXACT.

Parity status: every function here is pinned by the CPU tests (closed-form filter facts,
Littlewood-Paley bound, Parseval, brute-force time-domain convolution, tone, shift, time
reversal / spin, finite differences and dot-product adjoint tests).  The paper's printed
shape counts (44/45 log-frequency bins, 195 channels at J=13, Q=16) are not reproduced by
FB-P and are recorded as unpinned counts; the frame count 32 = 2^16 / 2^11 is reproduced.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

PSI_PSI, PSI_PHI, PHI_PSI, PHI_PHI = 1, 2, 4, 8
FWHM_PER_SIGMA = 2.0 * math.sqrt(2.0 * math.log(2.0))
XI_CAP = 0.35
SIGMA0 = 0.1
BAND_SIGMAS = 4.0      # half-width, in sigmas, of a band-pass filter's band for the schedule


# ----------------------------------------------------------------------------------------
# configuration
# ----------------------------------------------------------------------------------------
@dataclass(frozen=True)
class Config:
    """Sec. 4.2 parameters: J octaves, Q filters per octave (first order), Q2 at second
    order, J_fr / Q_fr for the frequential bank, temporal support T, frequential support F,
    signal length N.  ``average_fr`` selects Eq. 3 (True) or Eq. 4 (False).
    ``oversampling`` o >= 0 divides every schedule stride by 2^o.  ``branches`` is a bit mask
    of the second-order joint wavelets (Eq. 3 with either factor replaced by its lowpass):
    1 psi_t x psi_f, 2 psi_t x phi_f (both always on), 4 phi_t x psi_f, 8 phi_t x phi_f."""
    J: int
    Q: int
    J_fr: int
    Q_fr: int
    T: int
    F: int
    N: int
    Q2: int = 1
    average_fr: bool = True
    oversampling: int = 0
    branches: int = 3


WORKLOADS = {
    # the five benchmark workloads (T and F default to 2^J and Q where unspecified)
    1: Config(J=6, Q=8, J_fr=3, Q_fr=1, T=2 ** 6, F=8, N=2 ** 12),
    2: Config(J=12, Q=16, J_fr=4, Q_fr=2, T=2 ** 12, F=16, N=2 ** 16),
    3: Config(J=13, Q=16, J_fr=4, Q_fr=2, T=2 ** 13, F=16, N=2 ** 17),
    4: Config(J=11, Q=12, J_fr=4, Q_fr=1, T=2 ** 11, F=12, N=2 ** 15),
    5: Config(J=12, Q=16, J_fr=4, Q_fr=2, T=2 ** 12, F=16, N=2 ** 17),
}


def _is_pow2(v: int) -> bool:
    return v > 0 and (v & (v - 1)) == 0


# ----------------------------------------------------------------------------------------
# filters (Sec. 2, Eq. 1; FB-P reading)
# ----------------------------------------------------------------------------------------
def morlet_bank(J: int, Q: int):
    """Centre frequencies and widths (cycles/sample) of a (J, Q) Morlet bank, highest
    frequency first.  Constant-Q part: dilations by 2^{1/Q} (Eq. 1); then a linearly
    spaced tail of width sigma_min so that no filter is wider in time than scale 2^J."""
    rho = (1.0 - 2.0 ** (-1.0 / Q)) / FWHM_PER_SIGMA
    xi0 = min(XI_CAP, 0.5 / (1.0 + 4.0 * rho))
    sigma_min = SIGMA0 * 2.0 ** (-J)
    xi, sigma = [], []
    k = 0
    while True:
        xk = xi0 * 2.0 ** (-k / Q)
        if rho * xk < sigma_min:
            break
        xi.append(xk)
        sigma.append(rho * xk)
        k += 1
    if not xi:
        raise ValueError(f"bank (J={J}, Q={Q}) has no constant-Q filter")
    delta = FWHM_PER_SIGMA * sigma_min
    xlast = xi[-1]
    m = 1
    while True:
        xm = xlast - m * delta
        if xm < delta:
            break
        xi.append(xm)
        sigma.append(sigma_min)
        m += 1
    return np.array(xi), np.array(sigma)


def grid_freqs(G: int):
    """Frequency (cycles/sample) of bin k on a G-point DFT grid: k/G up to G/2, then negative."""
    k = np.arange(G)
    return np.where(k <= G // 2, k, k - G) / float(G)


def morlet_hat(omega, xi: float, sigma: float):
    """Un-normalised analytic Morlet: unit-amplitude Gaussian at xi minus its DC
    correction (so the value tends to 0 at omega -> 0+); zero for omega <= 0 and omega >= 1/2."""
    omega = np.asarray(omega, dtype=np.float64)
    kappa = math.exp(-xi * xi / (2.0 * sigma * sigma))
    g = np.exp(-((omega - xi) ** 2) / (2.0 * sigma * sigma)) - kappa * np.exp(
        -(omega ** 2) / (2.0 * sigma * sigma))
    return np.where((omega > 0.0) & (omega < 0.5), g, 0.0)


def lowpass_hat(omega, sigma_phi: float):
    omega = np.asarray(omega, dtype=np.float64)
    return np.exp(-(omega ** 2) / (2.0 * sigma_phi * sigma_phi))


def lp_scale(xi, sigma, sigma_phi: float, G: int) -> float:
    """Bank scalar c: the largest c with phi^2 + (c^2/2) sum_k psi_k(w)^2 <= 1 on every
    grid bin 0 < w < 1/2 of a G-point grid (the Littlewood-Paley bound)."""
    om = np.arange(1, G // 2) / float(G)
    P = np.zeros_like(om)
    for x, s in zip(xi, sigma):
        P += morlet_hat(om, x, s) ** 2
    P *= 0.5
    phi2 = lowpass_hat(om, sigma_phi) ** 2
    ok = P > 0.0
    return math.sqrt(float(np.min((1.0 - phi2[ok]) / P[ok])))


# ----------------------------------------------------------------------------------------
# transforms (engines)
# ----------------------------------------------------------------------------------------
def dft(v, engine: str = "fft"):
    """V[k] = sum_n v[n] exp(-2 pi i k n / L) along the last axis."""
    v = np.asarray(v)
    if engine == "fft":
        return np.fft.fft(v, axis=-1)
    L = v.shape[-1]
    n = np.arange(L)
    E = np.exp(-2j * np.pi * (np.outer(n, n) % L) / L)
    return v @ E.T


def idft_sum(V, engine: str = "fft"):
    """v[n] = sum_k V[k] exp(+2 pi i k n / L) along the last axis (no 1/L)."""
    V = np.asarray(V)
    if engine == "fft":
        return np.fft.ifft(V, axis=-1) * V.shape[-1]
    L = V.shape[-1]
    n = np.arange(L)
    E = np.exp(2j * np.pi * (np.outer(n, n) % L) / L)
    return V @ E.T


def circconv_direct(x, f):
    """Circular convolution by its definition: y[n] = sum_m x[m] f[(n - m) mod N]."""
    N = x.shape[-1]
    n = np.arange(N)
    C = f[(n[:, None] - n[None, :]) % N]
    return C @ x


# ----------------------------------------------------------------------------------------
# plan: filters on their grids
# ----------------------------------------------------------------------------------------
class Plan:
    """All filters of one configuration, sampled on their grids (Sec. 2, Eq. 1-3)."""

    def __init__(self, cfg: Config):
        if not (_is_pow2(cfg.N) and _is_pow2(cfg.T) and cfg.T <= cfg.N):
            raise ValueError("N and T must be powers of two with T <= N")
        if cfg.F < 1 or cfg.Q < 1 or cfg.Q2 < 1 or cfg.Q_fr < 1:
            raise ValueError("F, Q, Q2, Q_fr must be >= 1")
        if cfg.branches & (PSI_PSI | PSI_PHI) != (PSI_PSI | PSI_PHI) or cfg.branches & ~15:
            raise ValueError("branches must hold psi_t x psi_f and psi_t x phi_f (bits 1, 2)")
        self.cfg = cfg
        N, T = cfg.N, cfg.T
        self.N, self.T = N, T
        self.n_t = N // T
        # first order: lambda increases with frequency (generated high -> low, flipped)
        xi1, sg1 = morlet_bank(cfg.J, cfg.Q)
        self.xi1, self.sigma1 = xi1[::-1].copy(), sg1[::-1].copy()
        self.n1 = len(xi1)
        # second order (time rates), alpha = 0 is the highest rate
        self.xi2, self.sigma2 = morlet_bank(cfg.J, cfg.Q2)
        self.n2 = len(self.xi2)
        # frequential scales, beta = 0 is the finest scale (highest quefrency)
        self.xi_fr, self.sigma_fr = morlet_bank(cfg.J_fr, cfg.Q_fr)
        self.n_fr = len(self.xi_fr)
        self.N_fr = 2 * (1 << int(math.ceil(math.log2(self.n1))))
        self.C = 2 * self.n_fr + 1
        self.s_F = 1 << int(math.floor(math.log2(cfg.F)))
        self.n_lam_out = -(-self.n1 // self.s_F) if cfg.average_fr else self.n1

        self.sigma_T = SIGMA0 / T
        self.sigma_F = SIGMA0 / cfg.F
        self.c1 = lp_scale(self.xi1, self.sigma1, self.sigma_T, N)
        self.c2 = lp_scale(self.xi2, self.sigma2, self.sigma_T, N)
        self.c_fr = lp_scale(self.xi_fr, self.sigma_fr, self.sigma_F, self.N_fr)

        om = grid_freqs(N)
        self.psi1_hat = np.stack([self.c1 * morlet_hat(om, x, s)
                                  for x, s in zip(self.xi1, self.sigma1)])
        self.psi2_hat = np.stack([self.c2 * morlet_hat(om, x, s)
                                  for x, s in zip(self.xi2, self.sigma2)])
        self.phi_T_hat = lowpass_hat(om, self.sigma_T)
        # phi_T[n]: the time-domain lowpass (inverse DFT on the N grid; real and even)
        self.phi_T = np.real(np.fft.ifft(self.phi_T_hat))

        omf = grid_freqs(self.N_fr)
        up = [self.c_fr * morlet_hat(omf, x, s) for x, s in zip(self.xi_fr, self.sigma_fr)]
        down = [self.c_fr * morlet_hat(-omf, x, s) for x, s in zip(self.xi_fr, self.sigma_fr)]
        self.phi_F_hat = lowpass_hat(omf, self.sigma_F)
        # channel c: (beta, theta=+1) for c < n_fr, (beta, theta=-1) for n_fr <= c < 2 n_fr,
        # and the phi_F (psi_t x phi_f) branch last
        self.fr_hat = np.stack(up + down + [self.phi_F_hat])
        self.h = np.fft.ifft(self.fr_hat, axis=-1)          # [C, N_fr] complex
        self.phi_F = np.real(np.fft.ifft(self.phi_F_hat))
        lam = np.arange(self.n1)
        idx = (lam[:, None] - lam[None, :]) % self.N_fr
        self.W = self.h[:, idx]                               # [C, n1, n1] Toeplitz
        lo = np.arange(self.n_lam_out)
        self.PhiF = self.phi_F[(lo[:, None] * self.s_F - lam[None, :]) % self.N_fr]
        # phi_t paths (time lowpass phi_T in place of psi_alpha): the spin-up scales beta, then
        # the phi_F channel.  Their input U1 * phi_T is real, so the spin-down channel gives the
        # conjugate Z and the same modulus: one spin is kept.
        self.phi_channels = (list(range(self.n_fr)) if cfg.branches & PHI_PSI else []) + (
            [2 * self.n_fr] if cfg.branches & PHI_PHI else [])
        self.n_phi = len(self.phi_channels)

    # -- pooling matrices ------------------------------------------------------------
    def pool_T_matrix(self, s: int):
        """Phi[t, m] = s * phi_T[(t T - m s) mod N]: Riemann sum of phi_T at stride s."""
        L = self.N // s
        t = np.arange(self.n_t)
        m = np.arange(L)
        return s * self.phi_T[(t[:, None] * self.T - m[None, :] * s) % self.N]

    def pool_T_matrix_at(self, s_in: int, s_out: int):
        """Phi[m, n] = s_in * phi_T[(m s_out - n s_in) mod N]: the Riemann sum of phi_T taking a
        row at stride s_in to every s_out-th sample (s_out = T gives pool_T_matrix)."""
        m = np.arange(self.N // s_out)
        n = np.arange(self.N // s_in)
        return s_in * self.phi_T[(m[:, None] * s_out - n[None, :] * s_in) % self.N]

    def shapes(self):
        out = dict(n1=self.n1, n2=self.n2, n_fr=self.n_fr, C=self.C, n_t=self.n_t,
                   n_lam_out=self.n_lam_out, N_fr=self.N_fr, s_F=self.s_F)
        if self.n_phi:
            out["n_phi"] = self.n_phi
        return out


# ----------------------------------------------------------------------------------------
# schedule (S-P reading)
# ----------------------------------------------------------------------------------------
def _pow2_stride(v: float, o: int, cap: int) -> int:
    e = int(math.floor(math.log2(v))) if v > 0 else 0
    return min(cap, 1 << max(0, e - o))


class Schedule:
    """Strides of SCHEDULED mode; ``oversampling=None`` gives EXACT (every stride 1)."""

    def __init__(self, plan: Plan, oversampling):
        n1, n2, N, T = plan.n1, plan.n2, plan.N, plan.T
        self.exact = oversampling is None
        if self.exact:
            self.s1 = np.ones(n1, dtype=np.int64)
        else:
            o = int(oversampling)
            self.s1 = np.array([_pow2_stride(1.0 / (16.0 * s), o, T) for s in plan.sigma1],
                               dtype=np.int64)
        nyq = 0.5 / float(self.s1.min())
        self.s2 = np.ones(n2, dtype=np.int64)
        self.skip2 = np.zeros(n2, dtype=bool)
        self.lo2 = np.zeros(n2)
        self.lam_min = np.zeros(n2, dtype=np.int64)
        for a in range(n2):
            lo = max(0.0, plan.xi2[a] - BAND_SIGMAS * plan.sigma2[a])
            hi = min(plan.xi2[a] + BAND_SIGMAS * plan.sigma2[a], nyq)
            self.lo2[a] = lo
            if lo >= hi:
                self.skip2[a] = True
                self.lam_min[a] = n1
                continue
            if not self.exact:
                self.s2[a] = _pow2_stride(1.0 / (2.0 * (hi - lo)), int(oversampling), T)
            keep = 0.5 / self.s1 > lo
            self.lam_min[a] = int(np.argmax(keep)) if keep.any() else n1
        self.L1 = N // self.s1
        self.L2 = N // self.s2
        # phi_t paths: the band [0, 4 sigma_T] of phi_T, sampled like a time wavelet's band
        self.s_phi = 1 if self.exact else _pow2_stride(
            1.0 / (2.0 * BAND_SIGMAS * plan.sigma_T), int(oversampling), T)


# ----------------------------------------------------------------------------------------
# linear operators and their adjoints (SCHEDULED; stride 1 everywhere is EXACT)
# ----------------------------------------------------------------------------------------
class Operators:
    def __init__(self, plan: Plan, sched: Schedule, engine: str = "fft"):
        self.p, self.s, self.engine = plan, sched, engine
        self._phiT = {}

    def PhiT(self, s: int):
        if s not in self._phiT:
            self._phiT[s] = self.p.pool_T_matrix(s)
        return self._phiT[s]

    # x -> x_hat
    def x_hat(self, x):
        return dft(x, self.engine)

    def x_hat_T(self, g_xh):
        return np.real(idft_sum(g_xh, self.engine))

    # first order: x_hat -> z_lambda sampled at stride s_lambda (Sec. 2)
    def psi1(self, xh, lam):
        N = self.p.N
        L = int(self.s.L1[lam])
        P = xh * self.p.psi1_hat[lam]
        return idft_sum(P.reshape(N // L, L).sum(axis=0), self.engine) / N

    def psi1_T(self, gz, lam):
        N = self.p.N
        L = int(self.s.L1[lam])
        gF = dft(gz, self.engine) / N
        return self.p.psi1_hat[lam] * np.tile(gF, N // L)

    # phi_T pooling at stride s (S0 with s=1 on x, S1 on U1 rows, S2 on |Z|)
    def pool_T(self, u, s):
        return u @ self.PhiT(s).T

    def pool_T_T(self, g, s):
        return g @ self.PhiT(s)

    # U1 row at stride s_in -> U1 * phi_T at stride s_out (the phi_t paths' time filter)
    def lowpass_to(self, u, s_in, s_out):
        key = (s_in, s_out)
        if key not in self._phiT:
            self._phiT[key] = self.p.pool_T_matrix_at(s_in, s_out)
        return u @ self._phiT[key].T

    def lowpass_to_T(self, g, s_in, s_out):
        self.lowpass_to(np.zeros(self.p.N // s_in), s_in, s_out)
        return g @ self._phiT[(s_in, s_out)]

    # second order, time: U1 row lambda' -> Y_alpha row at stride s_alpha (Eq. 3, t axis)
    def psi2(self, u, lam, a):
        N = self.p.N
        Lr = int(self.s.L1[lam])
        La = int(self.s.L2[a])
        Uh = dft(u, self.engine)
        k = np.arange(1, Lr // 2)
        G = np.zeros(La, dtype=np.complex128)
        np.add.at(G, k % La, Uh[k] * self.p.psi2_hat[a][k])
        return idft_sum(G, self.engine) / Lr

    def psi2_T(self, gy, lam, a):
        Lr = int(self.s.L1[lam])
        La = int(self.s.L2[a])
        gG = dft(gy, self.engine) / Lr
        k = np.arange(1, Lr // 2)
        gUh = np.zeros(Lr, dtype=np.complex128)
        gUh[k] = self.p.psi2_hat[a][k] * gG[k % La]
        return np.real(idft_sum(gUh, self.engine))

    # second order, log-frequency: Z_c = W_c Y (zero-padded convolution along lambda, Eq. 2-3)
    def wfr(self, Y, c, lam_min=0):
        return self.p.W[c][:, lam_min:] @ Y[lam_min:]

    def wfr_T(self, gZ, c, lam_min=0):
        return self.p.W[c][:, lam_min:].conj().T @ gZ

    # phi_F pooling along lambda with stride s_F (Eq. 3); identity for Eq. 4
    def pool_F(self, v):
        return self.p.PhiF @ v if self.p.cfg.average_fr else v

    def pool_F_T(self, g):
        return self.p.PhiF.T @ g if self.p.cfg.average_fr else g


def _safe_phase(z):
    a = np.abs(z)
    out = np.zeros_like(z)
    nz = a > 0
    out[nz] = z[nz] / a[nz]
    return out


# ----------------------------------------------------------------------------------------
# forward / backward
# ----------------------------------------------------------------------------------------
def forward_one(x, plan: Plan, sched: Schedule, engine: str = "fft", keep: bool = False):
    """S0 [n_t], S1 [n1, n_t], S2 [n2, C, n_lam_out, n_t] of one signal (Eq. 3 or Eq. 4)."""
    ops = Operators(plan, sched, engine)
    x = np.asarray(x, dtype=np.float64)
    assert x.shape == (plan.N,)
    xh = ops.x_hat(x)
    S0 = ops.pool_T(x, 1)
    z = [ops.psi1(xh, lam) for lam in range(plan.n1)]
    U1 = [np.abs(v) for v in z]
    S1 = np.stack([ops.pool_T(U1[lam], int(sched.s1[lam])) for lam in range(plan.n1)])
    S2 = np.zeros((plan.n2, plan.C, plan.n_lam_out, plan.n_t))
    Ys = {}
    for a in range(plan.n2):
        if sched.skip2[a]:
            continue
        lm = int(sched.lam_min[a])
        La = int(sched.L2[a])
        Y = np.zeros((plan.n1, La), dtype=np.complex128)
        for lam in range(lm, plan.n1):
            Y[lam] = ops.psi2(U1[lam], lam, a)
        if keep:
            Ys[a] = Y
        sa = int(sched.s2[a])
        for c in range(plan.C):
            Z = ops.wfr(Y, c, lm)
            S2[a, c] = ops.pool_F(ops.pool_T(np.abs(Z), sa))
    out = dict(S0=S0, S1=S1, S2=S2)
    if plan.n_phi:
        # phi_t x psi_f and phi_t x phi_f: Eq. 3 with the time lowpass as the time filter
        sp = int(sched.s_phi)
        Yp = np.stack([ops.lowpass_to(U1[lam], int(sched.s1[lam]), sp) for lam in range(plan.n1)])
        S2phi = np.zeros((plan.n_phi, plan.n_lam_out, plan.n_t))
        for q, c in enumerate(plan.phi_channels):
            S2phi[q] = ops.pool_F(ops.pool_T(np.abs(ops.wfr(Yp, c)), sp))
        out["S2phi"] = S2phi
        if keep:
            out["Yphi"] = Yp
    if keep:
        out.update(z=z, U1=U1, Y=Ys)
    return out


def forward(x, plan: Plan, sched: Schedule, engine: str = "fft"):
    """Batched forward: x [B, N] -> dict of S0 [B, n_t], S1 [B, n1, n_t], S2 [B, n2, C, n_lo, n_t]
    (and S2phi [B, n_phi, n_lo, n_t] when phi_t paths are selected)."""
    X = np.atleast_2d(np.asarray(x, dtype=np.float64))
    outs = [forward_one(xb, plan, sched, engine) for xb in X]
    return {k: np.stack([o[k] for o in outs]) for k in outs[0]}


def backward_one(x, gS0, gS1, gS2, plan: Plan, sched: Schedule, engine: str = "fft",
                 gS2phi=None):
    """Gradient w.r.t. x of <gS0, S0> + <gS1, S1> + <gS2, S2> (+ <gS2phi, S2phi>) (Sec. 5:
    reverse-ordered adjoints).  Modulus Jacobian: d|z| = Re(conj(z) dz) / |z|, taken as 0 at
    z = 0."""
    ops = Operators(plan, sched, engine)
    x = np.asarray(x, dtype=np.float64)
    xh = ops.x_hat(x)
    z = [ops.psi1(xh, lam) for lam in range(plan.n1)]
    U1 = [np.abs(v) for v in z]
    gU1 = [np.zeros_like(u) for u in U1]
    if plan.n_phi and gS2phi is not None:
        # phi_t paths: Y = U1 * phi_T is real, so its cotangent is Re(W^H gZ)
        sp = int(sched.s_phi)
        Yp = np.stack([ops.lowpass_to(U1[lam], int(sched.s1[lam]), sp) for lam in range(plan.n1)])
        gYp = np.zeros_like(Yp)
        for q, c in enumerate(plan.phi_channels):
            Z = ops.wfr(Yp, c)
            g_abs = ops.pool_T_T(ops.pool_F_T(gS2phi[q]), sp)
            gYp += np.real(ops.wfr_T(g_abs * _safe_phase(Z), c))
        for lam in range(plan.n1):
            gU1[lam] += ops.lowpass_to_T(gYp[lam], int(sched.s1[lam]), sp)
    for a in range(plan.n2):
        if sched.skip2[a]:
            continue
        lm = int(sched.lam_min[a])
        La = int(sched.L2[a])
        sa = int(sched.s2[a])
        Y = np.zeros((plan.n1, La), dtype=np.complex128)
        for lam in range(lm, plan.n1):
            Y[lam] = ops.psi2(U1[lam], lam, a)
        gY = np.zeros((plan.n1 - lm, La), dtype=np.complex128)
        for c in range(plan.C):
            Z = ops.wfr(Y, c, lm)
            g_abs = ops.pool_T_T(ops.pool_F_T(gS2[a, c]), sa)
            gY += ops.wfr_T(g_abs * _safe_phase(Z), c, lm)
        for lam in range(lm, plan.n1):
            gU1[lam] += ops.psi2_T(gY[lam - lm], lam, a)
    g_xh = np.zeros(plan.N, dtype=np.complex128)
    for lam in range(plan.n1):
        g = gU1[lam] + ops.pool_T_T(gS1[lam], int(sched.s1[lam]))
        g_xh += ops.psi1_T(g * _safe_phase(z[lam]), lam)
    return ops.x_hat_T(g_xh) + ops.pool_T_T(gS0, 1)


def backward(x, gS0, gS1, gS2, plan: Plan, sched: Schedule, engine: str = "fft",
             gS2phi=None):
    X = np.atleast_2d(np.asarray(x, dtype=np.float64))
    return np.stack([backward_one(X[b], gS0[b], gS1[b], gS2[b], plan, sched, engine,
                                  None if gS2phi is None else gS2phi[b])
                     for b in range(X.shape[0])])


# ----------------------------------------------------------------------------------------
# EXACT mode written directly from the definitions (time-domain convolutions)
# ----------------------------------------------------------------------------------------
def forward_exact_direct(x, plan: Plan):
    """Eq. 3 / Eq. 4 at the full sampling rate with every time convolution computed as a
    circular sum y[n] = sum_m x[m] f[(n-m) mod N] of the time-domain filters (inverse DFTs
    of the filters, by direct sums).  O(N^2): tiny inputs only."""
    N = plan.N
    x = np.asarray(x, dtype=np.float64)
    psi1 = idft_sum(plan.psi1_hat, "direct") / N
    psi2 = idft_sum(plan.psi2_hat, "direct") / N
    phiT = np.real(idft_sum(plan.phi_T_hat, "direct")) / N
    t = np.arange(plan.n_t) * plan.T
    S0 = circconv_direct(x, phiT)[t]
    U1 = np.stack([np.abs(circconv_direct(x, psi1[lam])) for lam in range(plan.n1)])
    S1 = np.stack([circconv_direct(U1[lam], phiT)[t] for lam in range(plan.n1)])
    h = idft_sum(plan.fr_hat, "direct") / plan.N_fr
    phiF = np.real(idft_sum(plan.phi_F_hat, "direct")) / plan.N_fr
    S2 = np.zeros((plan.n2, plan.C, plan.n_lam_out, plan.n_t))
    lam = np.arange(plan.n1)
    for a in range(plan.n2):
        Y = np.stack([circconv_direct(U1[l], psi2[a]) for l in range(plan.n1)])
        for c in range(plan.C):
            Z = np.zeros_like(Y)
            for l in range(plan.n1):           # zero-padded convolution along lambda
                for lp in range(plan.n1):
                    Z[l] += h[c][(l - lp) % plan.N_fr] * Y[lp]
            pooled_t = np.stack([circconv_direct(np.abs(Z[l]), phiT)[t] for l in range(plan.n1)])
            if plan.cfg.average_fr:
                lo = np.arange(plan.n_lam_out) * plan.s_F
                for o in range(plan.n_lam_out):
                    S2[a, c, o] = sum(phiF[(lo[o] - l) % plan.N_fr] * pooled_t[l] for l in lam)
            else:
                S2[a, c] = pooled_t
    out = dict(S0=S0, S1=S1, S2=S2)
    if plan.n_phi:
        Y = np.stack([circconv_direct(U1[l], phiT) for l in range(plan.n1)])
        S2phi = np.zeros((plan.n_phi, plan.n_lam_out, plan.n_t))
        for q, c in enumerate(plan.phi_channels):
            Z = np.zeros(Y.shape, dtype=np.complex128)
            for l in range(plan.n1):
                for lp in range(plan.n1):
                    Z[l] += h[c][(l - lp) % plan.N_fr] * Y[lp]
            pooled_t = np.stack([circconv_direct(np.abs(Z[l]), phiT)[t] for l in range(plan.n1)])
            if plan.cfg.average_fr:
                lo = np.arange(plan.n_lam_out) * plan.s_F
                for o in range(plan.n_lam_out):
                    S2phi[q, o] = sum(phiF[(lo[o] - l) % plan.N_fr] * pooled_t[l] for l in lam)
            else:
                S2phi[q] = pooled_t
        out["S2phi"] = S2phi
    return out


# ----------------------------------------------------------------------------------------
# time scattering (Scattering1D): the baseline of Sec. 4.4, the second order without the
# log-frequency stage, on the same filterbanks and schedule
# ----------------------------------------------------------------------------------------
def scattering1d_one(x, plan: Plan, sched: Schedule, engine: str = "fft"):
    """S0 [n_t], S1 [n1, n_t] as the transform, and S2t [n2, n1, n_t]:
    S2t[alpha, lambda] = (|U1[lambda] * psi_alpha| * phi_T) sampled every T, on the paths of a
    kept rate with lambda >= lam_min[alpha] (the rows whose Y_alpha the schedule computes),
    0 elsewhere."""
    ops = Operators(plan, sched, engine)
    x = np.asarray(x, dtype=np.float64)
    xh = ops.x_hat(x)
    U1 = [np.abs(ops.psi1(xh, lam)) for lam in range(plan.n1)]
    S0 = ops.pool_T(x, 1)
    S1 = np.stack([ops.pool_T(U1[lam], int(sched.s1[lam])) for lam in range(plan.n1)])
    S2t = np.zeros((plan.n2, plan.n1, plan.n_t))
    for a in range(plan.n2):
        if sched.skip2[a]:
            continue
        sa = int(sched.s2[a])
        for lam in range(int(sched.lam_min[a]), plan.n1):
            S2t[a, lam] = ops.pool_T(np.abs(ops.psi2(U1[lam], lam, a)), sa)
    return dict(S0=S0, S1=S1, S2t=S2t)


def scattering1d_backward_one(x, gS0, gS1, gS2t, plan: Plan, sched: Schedule,
                              engine: str = "fft"):
    """Gradient w.r.t. x of <gS0, S0> + <gS1, S1> + <gS2t, S2t> (reverse-ordered adjoints,
    d|z| taken as 0 at z = 0)."""
    ops = Operators(plan, sched, engine)
    x = np.asarray(x, dtype=np.float64)
    xh = ops.x_hat(x)
    z = [ops.psi1(xh, lam) for lam in range(plan.n1)]
    U1 = [np.abs(v) for v in z]
    gU1 = [ops.pool_T_T(gS1[lam], int(sched.s1[lam])) for lam in range(plan.n1)]
    for a in range(plan.n2):
        if sched.skip2[a]:
            continue
        sa = int(sched.s2[a])
        for lam in range(int(sched.lam_min[a]), plan.n1):
            Y = ops.psi2(U1[lam], lam, a)
            gY = ops.pool_T_T(gS2t[a, lam], sa) * _safe_phase(Y)
            gU1[lam] = gU1[lam] + ops.psi2_T(gY, lam, a)
    g_xh = np.zeros(plan.N, dtype=np.complex128)
    for lam in range(plan.n1):
        g_xh += ops.psi1_T(gU1[lam] * _safe_phase(z[lam]), lam)
    return ops.x_hat_T(g_xh) + ops.pool_T_T(gS0, 1)


def scattering1d_exact_direct(x, plan: Plan):
    """EXACT time scattering from the definitions: circular sums of the time-domain filters
    at the full rate, every (alpha, lambda) pair.  O(N^2): tiny inputs only."""
    N = plan.N
    x = np.asarray(x, dtype=np.float64)
    psi1 = idft_sum(plan.psi1_hat, "direct") / N
    psi2 = idft_sum(plan.psi2_hat, "direct") / N
    phiT = np.real(idft_sum(plan.phi_T_hat, "direct")) / N
    t = np.arange(plan.n_t) * plan.T
    U1 = [np.abs(circconv_direct(x, psi1[lam])) for lam in range(plan.n1)]
    S2t = np.zeros((plan.n2, plan.n1, plan.n_t))
    for a in range(plan.n2):
        for lam in range(plan.n1):
            S2t[a, lam] = circconv_direct(np.abs(circconv_direct(U1[lam], psi2[a])), phiT)[t]
    return dict(S0=circconv_direct(x, phiT)[t],
                S1=np.stack([circconv_direct(u, phiT)[t] for u in U1]), S2t=S2t)


def scattering1d_paths(plan: Plan, sched: Schedule) -> int:
    """Number of second-order (alpha, lambda) paths the schedule computes."""
    return int(sum(plan.n1 - sched.lam_min[a] for a in range(plan.n2) if not sched.skip2[a]))


# ----------------------------------------------------------------------------------------
# mu-log compression (Sec. 4.3, Eq. 6-7)
# ----------------------------------------------------------------------------------------
def mu_log_mean(S):
    """Eq. 6: mu(lambda_2) = (1/N) sum_n sum_{lambda, t} S x_n(lambda_2, lambda, t), the path's
    integral over its other axes (a sum on the grid), averaged over the N examples.
    S: [examples, paths, ...]."""
    S = np.asarray(S, dtype=np.float64)
    return S.reshape(S.shape[0], S.shape[1], -1).sum(axis=2).mean(axis=0)


def mu_log(S, mu, eps: float = 0.1):
    """Eq. 7: log(1 + S / (eps mu(lambda_2))), path by path (axis 1)."""
    S = np.asarray(S, dtype=np.float64)
    shape = (1, -1) + (1,) * (S.ndim - 2)
    return np.log1p(S / (eps * np.asarray(mu, dtype=np.float64).reshape(shape)))


def stage1_full_rate(x, plan: Plan):
    """x * phi_T and x * psi_lambda at every sample (for the energy identity)."""
    xh = np.fft.fft(np.asarray(x, dtype=np.float64))
    low = np.real(np.fft.ifft(xh * plan.phi_T_hat))
    z = np.fft.ifft(xh[None, :] * plan.psi1_hat, axis=-1)
    return low, z


def littlewood_paley(plan: Plan, order: int = 1):
    """LP(w) = phi^2 + (1/2) sum |psi(w)|^2 + |psi(-w)|^2 on the bank's grid."""
    if order == 1:
        ph, ps = plan.phi_T_hat, plan.psi1_hat
        return ph ** 2 + 0.5 * np.sum(ps ** 2 + np.roll(ps[:, ::-1], 1, axis=-1) ** 2, axis=0)
    if order == 2:
        ph, ps = plan.phi_T_hat, plan.psi2_hat
        return ph ** 2 + 0.5 * np.sum(ps ** 2 + np.roll(ps[:, ::-1], 1, axis=-1) ** 2, axis=0)
    ps = plan.fr_hat[: plan.n_fr]
    return plan.phi_F_hat ** 2 + 0.5 * np.sum(ps ** 2 + np.roll(ps[:, ::-1], 1, axis=-1) ** 2,
                                              axis=0)


def relative_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / den) if den > 0 else float(np.linalg.norm(a - b))
