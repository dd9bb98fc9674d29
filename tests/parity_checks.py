"""Comparison helpers shared by the GPU parity tests (no arithmetic of the transform).

Beside the per-order relative L2 error, every slice that carries a visible share of its
order's energy is checked on its own: a wrong low-energy channel (the psi_t x phi_F branch,
a high rate alpha, the rows next to lam_min) would otherwise hide inside the order's norm.
"""
import numpy as np

SLICE_FLOOR = 1e-3      # slices whose oracle norm is below this share of the order's are skipped
SLICE_FACTOR = 10.0     # a slice may be this many times the order's tolerance


def relative_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / den) if den > 0 else float(np.linalg.norm(a - b))


def slice_errors(got, ref, lead):
    """Relative L2 error of every slice over the first ``lead`` axes (S1: one axis, the
    first-order row lambda; S2: two axes, the rate alpha and the channel c) whose oracle norm
    is at least SLICE_FLOOR of the whole order's.  Returns {index: error}."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    total = np.linalg.norm(ref)
    out = {}
    for idx in np.ndindex(*ref.shape[:lead]):
        r = ref[idx]
        n = np.linalg.norm(r)
        if total == 0 or n < SLICE_FLOOR * total:
            continue
        out[idx] = float(np.linalg.norm(got[idx] - r) / n)
    return out


def check_orders(got, ref, tol, label=""):
    """Per-order relative L2 <= tol, and every visible S1 row and S2 (alpha, c) slice
    <= SLICE_FACTOR * tol.  ``got`` / ``ref``: dicts with S0, S1, S2 of one signal."""
    worst = {}
    for name in ("S0", "S1", "S2"):
        e = relative_l2(got[name], ref[name])
        assert e <= tol, (label, name, e)
        worst[name] = e
    for name, lead in (("S1", 1), ("S2", 2)):
        errs = slice_errors(got[name], ref[name], lead)
        assert errs, (label, name, "no slice above the floor")
        bad = {k: v for k, v in errs.items() if v > SLICE_FACTOR * tol}
        assert not bad, (label, name, sorted(bad.items(), key=lambda kv: -kv[1])[:5])
        worst[name + "_slice"] = max(errs.values())
    return worst
