"""Pins of the oracle's hand-written adjoint (Sec. 5: reverse-ordered Hermitian adjoints):
dot-product tests of every linear stage and central finite differences of the whole map."""
import numpy as np
import pytest

from oracle import jtfs_oracle as O

SMALL = O.Config(J=5, Q=4, J_fr=3, Q_fr=1, T=32, F=4, N=512)


def _cplx(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("mode", [0, None])
def test_dot_product_adjoints(mode):
    p = O.Plan(SMALL)
    s = O.Schedule(p, mode)
    ops = O.Operators(p, s)
    rng = np.random.default_rng(7)
    N = p.N
    # x -> x-hat (real input): <A x, v>_R = <x, Re A^H v>
    x = rng.standard_normal(N)
    v = _cplx(rng, N)
    assert abs(np.real(np.vdot(ops.x_hat(x), v)) - x @ ops.x_hat_T(v)) < 1e-10 * N
    for lam in (0, p.n1 // 2, p.n1 - 1):
        L = int(s.L1[lam])
        u, w = _cplx(rng, N), _cplx(rng, L)
        lhs = np.vdot(ops.psi1(u, lam), w)
        rhs = np.vdot(u, ops.psi1_T(w, lam))
        assert abs(lhs - rhs) < 1e-12 * (1 + abs(lhs))
        ur, g = rng.standard_normal(L), rng.standard_normal(p.n_t)
        sl = int(s.s1[lam])
        assert abs(ops.pool_T(ur, sl) @ g - ur @ ops.pool_T_T(g, sl)) < 1e-12
    for a in range(p.n2):
        if s.skip2[a]:
            continue
        La = int(s.L2[a])
        for lam in range(int(s.lam_min[a]), p.n1, 5):
            Lr = int(s.L1[lam])
            ur, w = rng.standard_normal(Lr), _cplx(rng, La)
            lhs = np.real(np.vdot(ops.psi2(ur, lam, a), w))
            rhs = ur @ ops.psi2_T(w, lam, a)
            assert abs(lhs - rhs) < 1e-11 * (1 + abs(lhs))
    Y = _cplx(rng, p.n1, 16)
    G = _cplx(rng, p.n1, 16)
    for c in range(p.C):
        lhs = np.vdot(ops.wfr(Y, c), G)
        rhs = np.vdot(Y, ops.wfr_T(G, c))
        assert abs(lhs - rhs) < 1e-12 * (1 + abs(lhs))
    V = rng.standard_normal((p.n1, p.n_t))
    Gf = rng.standard_normal((p.n_lam_out, p.n_t))
    assert abs(np.sum(ops.pool_F(V) * Gf) - np.sum(V * ops.pool_F_T(Gf))) < 1e-12


@pytest.mark.parametrize("cfg,mode", [
    (O.Config(J=3, Q=2, J_fr=2, Q_fr=1, T=8, F=2, N=128), 0),
    (SMALL, 0),
    (SMALL, None),
    (O.Config(J=5, Q=4, J_fr=3, Q_fr=1, T=32, F=4, N=512, average_fr=False), 0),
])
def test_finite_differences(cfg, mode):
    p = O.Plan(cfg)
    s = O.Schedule(p, mode)
    rng = np.random.default_rng(8)
    x = rng.standard_normal(p.N)
    out = O.forward_one(x, p, s)
    g = {k: rng.standard_normal(v.shape) for k, v in out.items()}

    def loss(xx):
        o = O.forward_one(xx, p, s)
        return sum(float(np.sum(g[k] * o[k])) for k in g)

    gx = O.backward_one(x, g["S0"], g["S1"], g["S2"], p, s)
    for _ in range(3):
        v = rng.standard_normal(p.N)
        h = 1e-6
        fd = (loss(x + h * v) - loss(x - h * v)) / (2 * h)
        assert abs(fd - gx @ v) <= 1e-7 * max(1.0, abs(fd))


def test_modulus_gradient_is_zero_at_zero():
    """With x = 0 every wavelet coefficient is 0, where the reading takes d|z| = 0; only
    the (linear) S0 path carries gradient."""
    p = O.Plan(SMALL)
    s = O.Schedule(p, 0)
    rng = np.random.default_rng(9)
    out = O.forward_one(np.zeros(p.N), p, s)
    g = {k: rng.standard_normal(v.shape) for k, v in out.items()}
    gx = O.backward_one(np.zeros(p.N), g["S0"], g["S1"], g["S2"], p, s)
    ops = O.Operators(p, s)
    np.testing.assert_allclose(gx, ops.pool_T_T(g["S0"], 1), atol=1e-15)


def test_gradient_conditioning_needs_a_noise_floor():
    """The modulus Jacobian z / |z| is ill-conditioned where a first-order row holds almost
    no energy (|z| at the rounding level of the input): click trains through resonators leave
    rows empty, and there the FP64 gradient itself moves by order one under a 1e-7 relative
    perturbation of x (the size of FP32 rounding).  White noise 40 dB below the signal fills
    every row and the gradient moves by about 1e-5.  So gradient parity between an FP32 and an
    FP64 path is only defined on inputs with such a floor; the GPU gradient tests use them."""
    import synth_signals as SS
    cfg = O.WORKLOADS[1]
    p = O.Plan(cfg)
    s = O.Schedule(p, 0)
    moved = {}
    for floor in (None, -40):
        x = SS.click_train_batch(1, cfg.N, SS.BASE_SEED + 3, noise_db=floor)[0].astype(np.float64)
        out = O.forward_one(x, p, s)
        rng = np.random.default_rng(0)
        g = {k: rng.standard_normal(v.shape) for k, v in out.items()}
        g0 = O.backward_one(x, g["S0"], g["S1"], g["S2"], p, s)
        xp = x + 1e-7 * np.sqrt(np.mean(x ** 2)) * rng.standard_normal(x.shape)
        g1 = O.backward_one(xp, g["S0"], g["S1"], g["S2"], p, s)
        moved[floor] = O.relative_l2(g1, g0)
    assert moved[None] > 0.1
    assert moved[-40] < 1e-4
