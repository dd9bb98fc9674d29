"""Seeded synthetic audio generators shared by the tests, the benchmark and the oracle checks.

This module holds no arithmetic of the scattering transform: it only draws signals.
The paper's recordings (bird calls, Medley-solos-DB, dizi glissandi) are not available,
so these generators stand in for them with the same lengths and the same kinds of
content (AM/FM tones, chirps, click trains).

Seeding: workload ``c`` uses base seed ``20220408 + c`` and one child stream per
signal from ``numpy.random.SeedSequence(base).spawn(B)``.  Every generator works in
float64 and returns float32 arrays (the transform's input type).
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 20220408
SR = 22050.0


def _streams(seed: int, count: int):
    return [np.random.default_rng(s) for s in np.random.SeedSequence(seed).spawn(count)]


def noise_plus_chirp(N: int, seed: int, f0: float = 0.01, f1: float = 0.4, amp: float = 0.5):
    """Unit-variance white noise plus a linear chirp sweeping f0 -> f1 cycles/sample."""
    rng = _streams(seed, 1)[0]
    n = np.arange(N, dtype=np.float64)
    phase = 2.0 * np.pi * (f0 * n + (f1 - f0) * n * n / (2.0 * N))
    x = rng.standard_normal(N) + amp * np.sin(phase)
    return x.astype(np.float32)


def amfm_batch(B: int, N: int, seed: int, sr: float = SR, noise_db: float = -30.0):
    """AM/FM tones: (1 + 0.5 sin(2 pi f_am t + p1)) * sin(phi(t)),
    phi'(t) = 2 pi f_c 2^{(e/12) sin(2 pi f_fm t + p2)}, plus white noise at
    ``noise_db`` re the tone's RMS.  f_c log-uniform in [100, 4000] Hz, f_am uniform
    in [1, 16] Hz, f_fm uniform in [1, 8] Hz, excursion e uniform in [1, 6] semitones."""
    out = np.empty((B, N), dtype=np.float32)
    t = np.arange(N, dtype=np.float64) / sr
    for b, rng in enumerate(_streams(seed, B)):
        fc = np.exp(rng.uniform(np.log(100.0), np.log(4000.0)))
        fam = rng.uniform(1.0, 16.0)
        ffm = rng.uniform(1.0, 8.0)
        e = rng.uniform(1.0, 6.0)
        p1, p2 = rng.uniform(0.0, 2.0 * np.pi, size=2)
        inst = 2.0 * np.pi * fc * 2.0 ** ((e / 12.0) * np.sin(2.0 * np.pi * ffm * t + p2))
        phi = np.cumsum(inst) / sr
        tone = (1.0 + 0.5 * np.sin(2.0 * np.pi * fam * t + p1)) * np.sin(phi)
        rms = np.sqrt(np.mean(tone * tone))
        noise = rng.standard_normal(N) * rms * 10.0 ** (noise_db / 20.0)
        out[b] = tone + noise
    return out


def _biquad_bandpass(x, fc, q, sr):
    """Second-order resonator (constant 0 dB peak gain band-pass)."""
    from scipy.signal import lfilter
    w0 = 2.0 * np.pi * fc / sr
    alpha = np.sin(w0) / (2.0 * q)
    b = np.array([alpha, 0.0, -alpha])
    a = np.array([1.0 + alpha, -2.0 * np.cos(w0), 1.0 - alpha])
    return lfilter(b, a, x)


def click_train_batch(B: int, N: int, seed: int, sr: float = SR, noise_db=None):
    """Poisson click trains (rate uniform in [5, 40] Hz); every click is an impulse
    through its own random resonator (centre uniform in [200, 6000] Hz, Q log-uniform
    in [5, 30]).  Normalised to unit RMS.  With ``noise_db`` (e.g. -40), white noise at that
    level re the unit RMS is added from the signal's own stream (after the clicks)."""
    out = np.empty((B, N), dtype=np.float32)
    for b, rng in enumerate(_streams(seed, B)):
        rate = rng.uniform(5.0, 40.0)
        n_clicks = rng.poisson(rate * N / sr)
        pos = np.sort(rng.integers(0, N, size=max(n_clicks, 1)))
        y = np.zeros(N)
        for p in pos:
            fc = rng.uniform(200.0, 6000.0)
            q = np.exp(rng.uniform(np.log(5.0), np.log(30.0)))
            # the response decays as exp(-pi fc t / q): keep it until ~1e-9 of its start
            span = int(min(N - p, np.ceil(21.0 * q * sr / (np.pi * fc))))
            imp = np.zeros(span)
            imp[0] = rng.uniform(0.5, 1.0) * (1.0 if rng.random() < 0.5 else -1.0)
            y[p:p + span] += _biquad_bandpass(imp, fc, q, sr)
        rms = np.sqrt(np.mean(y * y))
        y = y / (rms if rms > 0 else 1.0)
        if noise_db is not None:
            y = y + rng.standard_normal(N) * 10.0 ** (noise_db / 20.0)
        out[b] = y
    return out


def white_noise_batch(B: int, N: int, seed: int, std: float = 1.0):
    out = np.empty((B, N), dtype=np.float32)
    for b, rng in enumerate(_streams(seed, B)):
        out[b] = rng.standard_normal(N) * std
    return out


def chirp_eq5(N: int, fc: float, fm: float, gamma: float, sr: float = SR, w: float = 2.0):
    """The paper's AM/FM exponential chirp (Sec. 3.2, Eq. 5): a Gaussian window of
    characteristic width w (octaves) in gamma*t, times sin(2 pi f_m t), times
    sin(2 pi f_c 2^{gamma t} / (gamma ln 2)), centred in the frame."""
    t = (np.arange(N, dtype=np.float64) - N / 2) / sr
    window = np.exp(-0.5 * (gamma * t / (w / 2.0)) ** 2)
    x = window * np.sin(2.0 * np.pi * fm * t) * np.sin(
        2.0 * np.pi * fc / (gamma * np.log(2.0)) * 2.0 ** (gamma * t))
    return x.astype(np.float32)


def eq5_grid(count: int = 16):
    """The paper's Eq. 5 dataset parameters (Sec. 3.2): ``count`` values each of f_c
    (512 to 1024 Hz), f_m (4 to 32 Hz) and gamma (0.5 to 4 octaves/s) in geometric progression,
    all count^3 triplets, f_c varying slowest.  Returns an array [count^3, 3]."""
    fc = np.geomspace(512.0, 1024.0, count)
    fm = np.geomspace(4.0, 32.0, count)
    gm = np.geomspace(0.5, 4.0, count)
    g = np.stack(np.meshgrid(fc, fm, gm, indexing="ij"), axis=-1)
    return g.reshape(-1, 3)


def chirp_eq5_batch(N: int, params, sr: float = SR, w: float = 2.0):
    """Eq. 5 chirps for every (f_c, f_m, gamma) row of ``params``: [len(params), N] float32."""
    params = np.asarray(params, dtype=np.float64)
    out = np.empty((len(params), N), dtype=np.float32)
    t = (np.arange(N, dtype=np.float64) - N / 2) / sr
    for i in range(0, len(params), 64):
        fc, fm, gm = (params[i:i + 64, j][:, None] for j in range(3))
        window = np.exp(-0.5 * (gm * t / (w / 2.0)) ** 2)
        out[i:i + 64] = window * np.sin(2.0 * np.pi * fm * t) * np.sin(
            2.0 * np.pi * fc / (gm * np.log(2.0)) * 2.0 ** (gm * t))
    return out


def varlen_lengths(count: int, seed: int, lo_log2: float = 13.0, hi_log2: float = 17.0):
    """Signal lengths drawn log-uniform in [2^lo, 2^hi]."""
    rng = _streams(seed, 1)[0]
    return np.floor(2.0 ** rng.uniform(lo_log2, hi_log2, size=count)).astype(np.int64)


def varlen_batch(count: int, seed: int, lo_log2: float = 13.0, hi_log2: float = 17.0):
    """Uneven-length batch: lengths log-uniform in [2^lo, 2^hi], even-numbered signals AM/FM
    tones and odd-numbered ones click trains.  Returns (x packed back to back, lengths)."""
    lengths = varlen_lengths(count, seed, lo_log2, hi_log2)
    parts = []
    for i, n in enumerate(lengths):
        gen = amfm_batch if i % 2 == 0 else click_train_batch
        parts.append(gen(1, int(n), seed + 7919 * (i + 1))[0])
    return np.concatenate(parts).astype(np.float32), lengths


def workload_signals(config: int, B: int, N: int):
    """Inputs for the named workloads (1: noise + chirp, 2/4: AM/FM, 3: click trains)."""
    seed = BASE_SEED + config
    if config == 1:
        return np.stack([noise_plus_chirp(N, seed + 1000 * b) for b in range(B)])
    if config in (2, 4):
        return amfm_batch(B, N, seed)
    if config == 3:
        return click_train_batch(B, N, seed)
    raise ValueError(f"no generator for workload {config}")
