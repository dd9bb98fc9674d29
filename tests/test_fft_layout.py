"""The shared-memory layout of the row FFTs (csrc/fft.cuh: fft_pos): a bijection within each
row onto the padded positions, and free of bank conflicts for every access pattern the row
kernels use (8-byte elements: 16 slots of two 4-byte banks; a warp access costs as many
wavefronts as the most loaded slot holds distinct positions, two at best)."""
import collections

import pytest


def fft_pos(i, logL):
    if logL >= 9:
        i ^= (i >> (logL - 4)) & 15
    return i + (i >> 4)


def bitrev(k, n):
    return int(format(k, f"0{n}b")[::-1], 2) if n else 0


def wavefronts(addrs, logL):
    seen, load = set(), collections.Counter()
    for a in addrs:
        p = fft_pos(a, logL)
        if p not in seen:
            seen.add(p)
            load[p % 16] += 1
    return max(load.values())


def passes(logL):
    out, s0 = [], 1
    if logL & 3:
        out.append((logL & 3, s0))
        s0 += logL & 3
    while s0 + 3 <= logL:
        out.append((4, s0))
        s0 += 4
    return out


def patterns(logL, total=8192):
    """Every warp access of the kernels on a block of rows: the bit-reversed input scatter,
    the passes' strided loads and stores, natural-order reads."""
    L = 1 << logL
    G = max(1, total // L)
    n = G * L
    for base in range(0, n, 32):
        idx = range(base, min(base + 32, n))
        yield "bitrev", [((i >> logL) << logL) + bitrev(i & (L - 1), logL) for i in idx]
        yield "natural", list(idx)
    for RB, s0 in passes(logL):
        q, lgpr = 1 << (s0 - 1), logL - RB
        groups = G << lgpr
        for g0 in range(0, groups, 32):
            for m in range(1 << RB):
                addrs = []
                for g in range(g0, min(g0 + 32, groups)):
                    row, b = g >> lgpr, g & ((1 << lgpr) - 1)
                    j = b & (q - 1)
                    addrs.append((row << logL) + ((b >> (s0 - 1)) << (s0 - 1 + RB)) + j + m * q)
                yield f"pass{RB}@{s0}", addrs


@pytest.mark.parametrize("logL", range(5, 16))
def test_fft_layout_is_a_bijection_per_row(logL):
    L = 1 << logL
    for row in range(2):
        pos = [fft_pos((row << logL) + i, logL) for i in range(L)]
        base = [(row << logL) + i + (((row << logL) + i) >> 4) for i in range(L)]
        assert sorted(pos) == sorted(base)


@pytest.mark.parametrize("logL", range(5, 16))
def test_fft_layout_accesses_are_conflict_free(logL):
    worst = collections.defaultdict(int)
    for name, addrs in patterns(logL):
        worst[name] = max(worst[name], wavefronts(addrs, logL))
    assert all(w <= 2 for w in worst.values()), dict(worst)


def pass_positions(logL, s0, RB, g, G):
    """The positions the radix pass computes for its group g (fft_dit_pass's shortcut)."""
    R, q, lgpr = 1 << RB, 1 << (s0 - 1), logL - RB
    row, b = g >> lgpr, g & ((1 << lgpr) - 1)
    j = b & (q - 1)
    base = (row << logL) + ((b >> (s0 - 1)) << (s0 - 1 + RB)) + j
    pad = lambda i: i + (i >> 4)
    if logL >= 9 and RB == 4 and s0 + 3 == logL:
        c0 = (row << logL) + (row << (logL - 4)) + (j >> 4)
        return base, [c0 + (j ^ m) + m * (q + (q >> 4)) for m in range(R)]
    if logL < 9 or s0 + RB - 1 <= logL - 4:
        t = (base >> (logL - 4)) & 15 if logL >= 9 else 0
        if q >= 16:
            return base, [pad(base ^ t) + m * (q + (q >> 4)) for m in range(R)]
        return base, [pad((base + m * q) ^ t) for m in range(R)]
    return base, [fft_pos(base + m * q, logL) for m in range(R)]


@pytest.mark.parametrize("logL", range(5, 16))
def test_pass_positions_match_the_layout(logL):
    G = max(1, 8192 >> logL) if logL < 13 else 2
    for RB, s0 in passes(logL):
        q = 1 << (s0 - 1)
        for g in range(G << (logL - RB)):
            base, p = pass_positions(logL, s0, RB, g, G)
            assert p == [fft_pos(base + m * q, logL) for m in range(1 << RB)], (RB, s0, g)
