"""Pins of the FP64 oracle to facts fixed by the paper and by the mathematics.

Nothing here re-types the oracle's formulas: each check reaches the same
quantity another way (brute force, dense linear algebra on the Eq. 8 normal
equations, finite differences of Eq. 1/Eq. 2, invariants, closed forms).
"""
import numpy as np
import pytest

import oracle as O
from paper_2003_07504_gb300 import synth


# ---------------------------------------------------------------- helpers (dense, from definitions)

def dense_forward_difference(H, W, axis):
    """Matrix of the periodic forward difference on row-major H*W vectors."""
    n = H * W
    D = np.zeros((n, n))
    for y in range(H):
        for x in range(W):
            i = y * W + x
            j = y * W + (x + 1) % W if axis == "x" else ((y + 1) % H) * W + x
            D[i, j] += 1.0
            D[i, i] -= 1.0
    return D


def dense_backward_difference(H, W, axis):
    n = H * W
    D = np.zeros((n, n))
    for y in range(H):
        for x in range(W):
            i = y * W + x
            j = y * W + (x - 1) % W if axis == "x" else ((y - 1) % H) * W + x
            D[i, i] += 1.0
            D[i, j] -= 1.0
    return D


def fd_dphi(x, p, eps, h=1e-6):
    """Central finite difference of Eq. 2's penalty (second-order accurate)."""
    return (O.phi_p(x + h, p, eps) - O.phi_p(x - h, p, eps)) / (2 * h)


def dense_ils(f, lam, p, eps, N, Dx, Dy):
    """Algorithm 1 with every operator a dense matrix and phi' by finite differences.

    mu = c*g - phi'(g) is the optimum condition of Eq. 3 (Appendix A); u^{n+1}
    solves the normal equations of Eq. 8: (2I + lam c (Dx^T Dx + Dy^T Dy)) u = 2f + lam (Dx^T mu_x + Dy^T mu_y).
    """
    c = p * eps ** (p / 2 - 1)
    n = f.size
    fv = f.reshape(-1)
    A = 2 * np.eye(n) + lam * c * (Dx.T @ Dx + Dy.T @ Dy)
    u = fv.copy()
    for _ in range(N):
        gx, gy = Dx @ u, Dy @ u
        mx = c * gx - fd_dphi(gx, p, eps)
        my = c * gy - fd_dphi(gy, p, eps)
        u = np.linalg.solve(A, 2 * fv + lam * (Dx.T @ mx + Dy.T @ my))
    return u.reshape(f.shape)


def small_image(H, W, seed):
    return synth.voronoi_texture(H, W, 1, K=4, A=0.05, Tmin=3, Tmax=5, sigma=0.02, seed=seed)[0].astype(np.float64)


# ---------------------------------------------------------------- DFT

def test_dft2_matches_bruteforce_quadruple_sum():
    rng = np.random.default_rng(1)
    H, W = 6, 10
    x = rng.normal(size=(H, W))
    X = np.zeros((H, W), dtype=complex)
    for l in range(H):
        for k in range(W):
            s = 0j
            for y in range(H):
                for xx in range(W):
                    s += x[y, xx] * np.exp(-2j * np.pi * (l * y / H + k * xx / W))
            X[l, k] = s
    np.testing.assert_allclose(O.dft2(x), X, atol=1e-11)
    np.testing.assert_allclose(O.idft2(X).real, x, atol=1e-12)


@pytest.mark.parametrize("H,W", [(8, 8), (15, 12), (27, 40)])
def test_dft2_matches_numpy_fft(H, W):
    rng = np.random.default_rng(H * 100 + W)
    x = rng.normal(size=(H, W)) + 1j * rng.normal(size=(H, W))
    np.testing.assert_allclose(O.dft2(x), np.fft.fft2(x), atol=1e-10)
    np.testing.assert_allclose(O.idft2(x), np.fft.ifft2(x), atol=1e-12)


def test_denominator_closed_form():
    # |F grad|^2 for the periodic [1,-1] operator is 4 sin^2(pi k / n).
    H, W, lam, c = 9, 14, 1.3, 7.0
    den = O.denominator(H, W, lam, c)
    l = np.arange(H)[:, None]
    k = np.arange(W)[None, :]
    want = 1 + (lam * c / 2) * (4 * np.sin(np.pi * k / W) ** 2 + 4 * np.sin(np.pi * l / H) ** 2)
    np.testing.assert_allclose(den.real, want, rtol=1e-13, atol=1e-12)
    assert np.abs(den.imag).max() < 1e-12


# ---------------------------------------------------------------- pieces

def test_c0_is_the_convexity_threshold():
    # Appendix B: at c = c0, g'' >= 0 everywhere; any smaller c makes g'' negative at 0.
    x = np.linspace(-2, 2, 400001)
    for p in (0.2, 0.5, 0.8, 1.0):
        eps = 1e-4
        c = O.c0(p, eps)
        assert np.min(O.g2(x, p, eps, c)) >= -1e-9 * c
        assert np.min(O.g2(x, p, eps, 0.9 * c)) < 0
        # numerical second derivative of g = c/2 x^2 - phi at a few points agrees with g''
        h = 1e-4
        xs = np.array([-0.3, -0.02, 0.004, 0.05, 0.7])
        g = lambda t: c / 2 * t * t - O.phi_p(t, p, eps)
        num = (g(xs + h) - 2 * g(xs) + g(xs - h)) / h ** 2
        np.testing.assert_allclose(O.g2(xs, p, eps, c), num, rtol=2e-4, atol=1e-3)
    assert O.c0(0.8, 1e-4) == pytest.approx(0.8 * 10 ** 2.4, rel=1e-14)


def test_mu_is_c_x_minus_numerical_derivative_of_penalty():
    x = np.concatenate([np.linspace(-1, 1, 201), [1e-5, -3e-3, 0.011]])
    for p in (0.5, 0.8, 1.0):
        eps = 1e-4
        c = O.c0(p, eps)
        np.testing.assert_allclose(O.mu_update(x, p, eps, c), c * x - fd_dphi(x, p, eps),
                                   rtol=1e-7, atol=1e-8)


def test_mu_is_the_argmin_of_the_half_quadratic_bound():
    # Eq. 3 / Appendix A: phi(t) <= 1/2 (sqrt(c) t - mu/sqrt(c))^2 + psi(mu) with equality at the
    # optimum mu = mu(x0) when t = x0.  So for that fixed mu, t -> 1/2 (sqrt(c) t - mu/sqrt(c))^2 - phi(t)
    # (which equals -psi(mu) at t = x0 and is >= -psi(mu) elsewhere) is minimal at t = x0.
    p, eps = 0.8, 1e-4
    c = O.c0(p, eps)
    for x0 in (-0.4, -0.01, 0.003, 0.2):
        mu = O.mu_update(x0, p, eps, c)
        t = x0 + np.linspace(-0.05, 0.05, 20001)
        val = 0.5 * (np.sqrt(c) * t - mu / np.sqrt(c)) ** 2 - O.phi_p(t, p, eps)
        assert abs(t[np.argmin(val)] - x0) <= 1e-5


# ---------------------------------------------------------------- the Eq. 9 solve

@pytest.mark.parametrize("H,W,lam,p", [(8, 8, 1.0, 0.8), (8, 8, 3.5, 0.5), (6, 10, 0.4, 1.0), (5, 7, 2.0, 0.8)])
def test_eq9_solves_the_eq8_least_squares_problem(H, W, lam, p):
    rng = np.random.default_rng(H * W)
    eps = 1e-4
    c = O.c0(p, eps)
    f = rng.uniform(size=(H, W))
    mx = rng.normal(size=(H, W)) * 5
    my = rng.normal(size=(H, W)) * 5
    Fdx, Fdy = O.gradient_transfer_functions(H, W)
    den = O.denominator(H, W, lam, c, Fdx, Fdy)
    u = O.solve_eq9(O.dft2(f), mx, my, lam, den, Fdx, Fdy)
    # Dense minimization of the Eq. 8 objective for these mu.
    Dx, Dy = dense_forward_difference(H, W, "x"), dense_forward_difference(H, W, "y")
    n = H * W
    A = 2 * np.eye(n) + lam * c * (Dx.T @ Dx + Dy.T @ Dy)
    b = 2 * f.reshape(-1) + lam * (Dx.T @ mx.reshape(-1) + Dy.T @ my.reshape(-1))
    u_dense = np.linalg.solve(A, b).reshape(H, W)
    np.testing.assert_allclose(u, u_dense, atol=1e-12 * max(1, np.abs(u_dense).max()))

    def J(v):
        v = v.reshape(-1)
        return (np.sum((v - f.reshape(-1)) ** 2)
                + lam * 0.5 * np.sum((np.sqrt(c) * (Dx @ v) - mx.reshape(-1) / np.sqrt(c)) ** 2)
                + lam * 0.5 * np.sum((np.sqrt(c) * (Dy @ v) - my.reshape(-1) / np.sqrt(c)) ** 2))
    j0 = J(u)
    for s in range(5):
        d = rng.normal(size=(H, W)) * 1e-3
        assert J(u + d) > j0


@pytest.mark.parametrize("H,W,lam,p,N", [(8, 8, 1.0, 0.8, 4), (4, 6, 2.0, 0.5, 3), (6, 5, 0.7, 1.0, 2)])
def test_full_algorithm_matches_dense_bruteforce(H, W, lam, p, N):
    eps = 1e-4
    f = small_image(H, W, seed=H + W)
    Dx, Dy = dense_forward_difference(H, W, "x"), dense_forward_difference(H, W, "y")
    want = dense_ils(f, lam, p, eps, N, Dx, Dy)
    got = O.ils_channel(f, lam, p, eps, N)
    np.testing.assert_allclose(got, want, atol=1e-7)   # the finite-difference phi' limits this


def test_backward_difference_reading_gives_the_same_result():
    # Sec. 3 only names the [1,-1] filter; periodic forward and backward differences give one result.
    H, W, lam, p, eps, N = 6, 8, 1.0, 0.8, 1e-4, 3
    f = small_image(H, W, seed=3)
    Bx, By = dense_backward_difference(H, W, "x"), dense_backward_difference(H, W, "y")
    np.testing.assert_allclose(O.ils_channel(f, lam, p, eps, N), dense_ils(f, lam, p, eps, N, Bx, By), atol=1e-7)


def test_p2_reduces_to_tikhonov():
    # p = 2 (outside the paper's range but the formulas hold): c0 = 2, mu == 0, so one
    # iteration is the closed-form quadratic smoother (I + lam (Dx^T Dx + Dy^T Dy))^{-1} f.
    H, W, lam = 7, 9, 1.7
    f = small_image(H, W, seed=5)
    assert O.c0(2.0, 1e-4) == pytest.approx(2.0)
    Dx, Dy = dense_forward_difference(H, W, "x"), dense_forward_difference(H, W, "y")
    want = np.linalg.solve(np.eye(H * W) + lam * (Dx.T @ Dx + Dy.T @ Dy), f.reshape(-1)).reshape(H, W)
    np.testing.assert_allclose(O.ils_channel(f, lam, 2.0, 1e-4, 1), want, atol=1e-12)
    np.testing.assert_allclose(O.ils_channel(f, lam, 2.0, 1e-4, 3), want, atol=1e-12)


# ---------------------------------------------------------------- invariants

def test_lambda_zero_returns_f():
    f = small_image(12, 10, seed=7)
    np.testing.assert_allclose(O.ils_channel(f, 0.0, 0.8, 1e-4, 4), f, atol=1e-13)


def test_constant_image_is_a_fixed_point():
    f = np.full((9, 12), 0.37)
    np.testing.assert_allclose(O.ils_channel(f, 2.0, 0.8, 1e-4, 4), f, atol=1e-13)


def test_mean_is_preserved():
    f = small_image(16, 20, seed=11)
    u = O.ils_channel(f, 1.0, 0.8, 1e-4, 4)
    assert abs(u.mean() - f.mean()) < 1e-13


def test_energy_is_non_increasing():
    # The half-quadratic majorization (Eq. 3-6, Appendix A) makes Eq. 1 monotone along the iterates.
    for p, lam in ((0.8, 1.0), (0.5, 3.0), (1.0, 0.5)):
        f = small_image(24, 20, seed=int(10 * p + lam))
        _, its = O.ils_channel(f, lam, p, 1e-4, 12, return_iterates=True)
        E = [O.energy(u, f, lam, p, 1e-4) for u in its]
        assert all(E[i + 1] <= E[i] * (1 + 1e-12) for i in range(len(E) - 1)), E
        assert E[-1] < E[0]


def test_fixed_point_is_a_stationary_point_of_eq1():
    # A limit of the iteration makes the gradient of Eq. 1 vanish; checked with a finite-difference
    # gradient of the energy itself.
    H, W, lam, p, eps = 6, 6, 0.5, 1.0, 1e-2
    f = small_image(H, W, seed=13)
    u = O.ils_channel(f, lam, p, eps, 3000)
    h = 1e-6
    grad = np.zeros_like(u)
    for i in range(H):
        for j in range(W):
            e = np.zeros_like(u)
            e[i, j] = h
            grad[i, j] = (O.energy(u + e, f, lam, p, eps) - O.energy(u - e, f, lam, p, eps)) / (2 * h)
    assert np.abs(grad).max() < 1e-6


def test_shift_and_transpose_equivariance():
    f = small_image(12, 16, seed=17)
    u = O.ils_channel(f, 1.0, 0.8, 1e-4, 4)
    us = O.ils_channel(np.roll(f, (3, -5), axis=(0, 1)), 1.0, 0.8, 1e-4, 4)
    np.testing.assert_allclose(us, np.roll(u, (3, -5), axis=(0, 1)), atol=1e-12)
    ut = O.ils_channel(f.T.copy(), 1.0, 0.8, 1e-4, 4)
    np.testing.assert_allclose(ut, u.T, atol=1e-12)


def test_colour_channels_are_independent():
    f = synth.voronoi_texture(10, 12, 3, K=3, seed=19).astype(np.float64)
    u = O.ils_smooth(f, 1.0, 0.8, 1e-4, 2)
    for ch in range(3):
        np.testing.assert_array_equal(u[ch], O.ils_channel(f[ch], 1.0, 0.8, 1e-4, 2))


# ---------------------------------------------------------------- adjoint

def test_adjoint_matches_directional_finite_differences():
    H, W, lam, p, eps, N = 8, 10, 1.0, 0.8, 1e-4, 4
    f = small_image(H, W, seed=23)
    rng = np.random.default_rng(0)
    w = rng.normal(size=(H, W))
    g = O.ils_backward(f, w, lam, p, eps, N)
    for trial in range(3):
        v = rng.normal(size=(H, W))
        h = 1e-6
        Lp = np.sum(w * O.ils_channel(f + h * v, lam, p, eps, N))
        Lm = np.sum(w * O.ils_channel(f - h * v, lam, p, eps, N))
        fd = (Lp - Lm) / (2 * h)
        assert np.sum(g * v) == pytest.approx(fd, rel=1e-6, abs=1e-7)


def test_adjoint_per_pixel_finite_differences_on_a_crop():
    H, W, lam, p, eps, N = 6, 6, 2.0, 0.5, 1e-4, 3
    f = small_image(H, W, seed=29)
    w = np.random.default_rng(1).normal(size=(H, W))
    g = O.ils_backward(f, w, lam, p, eps, N)
    h = 1e-6
    for i in range(H):
        for j in range(W):
            e = np.zeros((H, W))
            e[i, j] = h
            fd = (np.sum(w * O.ils_channel(f + e, lam, p, eps, N)) - np.sum(w * O.ils_channel(f - e, lam, p, eps, N))) / (2 * h)
            assert g[i, j] == pytest.approx(fd, rel=1e-5, abs=1e-6)


# ---------------------------------------------------------------- warm-start network helpers

def test_conv3x3_matches_loops():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(2, 5, 7))
    w = rng.normal(size=(3, 2, 3, 3))
    b = rng.normal(size=3)
    want = np.zeros((3, 5, 7))
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1)))
    for o in range(3):
        for y in range(5):
            for xx in range(7):
                want[o, y, xx] = b[o] + np.sum(w[o] * xp[:, y:y + 3, xx:xx + 3])
    np.testing.assert_allclose(O.conv3x3(x, w, b), want, atol=1e-12)


def test_golden_regression_vector():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "ils_12x10_lam1_p08_N4.txt")
    rows = [l for l in open(path) if not l.startswith("#")]
    f = np.array([float(v) for v in rows[0].split()]).reshape(12, 10)
    u = np.array([float(v) for v in rows[1].split()]).reshape(12, 10)
    np.testing.assert_allclose(O.ils_channel(f, 1.0, 0.8, 1e-4, 4), u, atol=1e-12)


def test_adjoint_split_for_a_warm_start():
    # dL/df through Eq. 9 and dL/du^0 separately, each against finite differences of the forward.
    H, W, lam, p, eps, N = 6, 7, 1.0, 0.8, 1e-4, 3
    f = small_image(H, W, seed=31)
    u0 = np.random.default_rng(3).uniform(size=(H, W))
    w = np.random.default_rng(4).normal(size=(H, W))
    gf, gu0 = O.ils_backward(f, w, lam, p, eps, N, u0=u0, split=True)
    v = np.random.default_rng(5).normal(size=(H, W))
    h = 1e-6
    L = lambda ff, uu: np.sum(w * O.ils_channel(ff, lam, p, eps, N, u0=uu))
    assert np.sum(gf * v) == pytest.approx((L(f + h * v, u0) - L(f - h * v, u0)) / (2 * h), rel=1e-6, abs=1e-7)
    assert np.sum(gu0 * v) == pytest.approx((L(f, u0 + h * v) - L(f, u0 - h * v)) / (2 * h), rel=1e-6, abs=1e-7)


def test_bf16_rounding_is_round_to_nearest_even():
    # exactly representable values pass; halfway cases go to the even neighbour
    assert O.bf16_round(1.0) == 1.0 and O.bf16_round(-2.5) == -2.5
    one_ulp = 2.0 ** -7                       # BF16 spacing in [1, 2)
    assert O.bf16_round(1.0 + one_ulp / 2) == 1.0            # tie -> even (1.0)
    assert O.bf16_round(1.0 + 3 * one_ulp / 2) == 1.0 + 2 * one_ulp  # tie -> even
    assert O.bf16_round(1.0 + 0.51 * one_ulp) == 1.0 + one_ulp
    x = np.random.default_rng(0).normal(size=1000)
    r = O.bf16_round(x)
    assert np.all(np.abs(r - x) <= np.abs(x) * 2.0 ** -8 + 1e-300)


def test_warmstart_chain_without_rounding_matches_autograd():
    # with rounding off, the oracle's forward and its hand-ordered backward (masks, flips,
    # transposes, bias sums) equal float64 autograd through conv2d + ReLU + residual
    import torch
    rng = np.random.default_rng(1)
    chans = [3, 8, 8, 3]
    ws = [rng.normal(scale=0.3, size=(chans[i + 1], chans[i], 3, 3)) for i in range(3)]
    bs = [rng.normal(scale=0.1, size=chans[i + 1]) for i in range(3)]
    f = rng.uniform(size=(2, 3, 6, 7))
    g = rng.normal(size=(2, 3, 6, 7))
    wt = [torch.tensor(w, requires_grad=True) for w in ws]
    bt = [torch.tensor(b, requires_grad=True) for b in bs]
    x = torch.tensor(f)
    h = x
    for i in range(3):
        h = torch.nn.functional.conv2d(h, wt[i], bt[i], padding=1)
        if i < 2:
            h = torch.relu(h)
    u = x + h
    u.backward(torch.tensor(g))
    u0, _ = O.warmstart_forward_bf16(f, ws, bs, rounding=False)
    np.testing.assert_allclose(u0, u.detach().numpy(), rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(O.warmstart_cnn_forward(f[1], ws, bs), u.detach().numpy()[1], rtol=1e-13, atol=1e-13)
    dW, db = O.warmstart_backward_bf16(f, ws, bs, g, rounding=False)
    for i in range(3):
        np.testing.assert_allclose(dW[i], wt[i].grad.numpy(), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(db[i], bt[i].grad.numpy(), rtol=1e-12, atol=1e-12)


def test_adam_step_closed_form_first_step():
    # at t = 1 the bias-corrected update is lr * g / (|g| + eps) (a signed step of ~lr)
    w, g = np.array([1.0, -2.0, 3.0]), np.array([0.5, -4.0, 1e-3])
    w1, m, v = O.adam_step(w, g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    np.testing.assert_allclose(w1, w - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


# ---------------------------------------------------------------- Welsch-penalty ILS (Sec. 5)

def fd_dphi_welsch(x, gamma, h=1e-7):
    return (O.phi_welsch(x + h, gamma) - O.phi_welsch(x - h, gamma)) / (2 * h)


def dense_ils_welsch(f, lam, gamma, N, Dx, Dy):
    """Algorithm 1 with the Welsch penalty, dense operators, phi_W' by finite differences, c = 2."""
    c = 2.0
    n = f.size
    fv = f.reshape(-1)
    A = 2 * np.eye(n) + lam * c * (Dx.T @ Dx + Dy.T @ Dy)
    u = fv.copy()
    for _ in range(N):
        gx, gy = Dx @ u, Dy @ u
        mx = c * gx - fd_dphi_welsch(gx, gamma)
        my = c * gy - fd_dphi_welsch(gy, gamma)
        u = np.linalg.solve(A, 2 * fv + lam * (Dx.T @ mx + Dy.T @ my))
    return u.reshape(f.shape)


def test_welsch_penalty_is_bounded_quadratic_near_zero():
    # the reading of Eq. 18: phi_W(0) = 0, phi_W ~ x^2 for |x| << gamma, phi_W -> 2 gamma^2 for |x| >> gamma
    g = 0.05
    assert O.phi_welsch(0.0, g) == 0.0
    np.testing.assert_allclose(O.phi_welsch(1e-4, g), 1e-8, rtol=1e-5)
    np.testing.assert_allclose(O.phi_welsch(10.0, g), 2 * g * g, rtol=1e-12)
    assert np.all(np.diff(O.phi_welsch(np.linspace(0, 1, 1001), g)) >= 0)


def test_welsch_mu_is_c_x_minus_numerical_derivative_of_penalty():
    x = np.concatenate([np.linspace(-1, 1, 201), [1e-5, -3e-3, 0.011]])
    for gamma in (5 / 255, 10 / 255, 0.3):
        np.testing.assert_allclose(O.mu_welsch(x, gamma, 2.0), 2.0 * x - fd_dphi_welsch(x, gamma),
                                   rtol=1e-6, atol=1e-9)


def test_welsch_c0_is_the_convexity_threshold():
    # Appendix B (Eq. 24): g = c/2 x^2 - phi_W is convex for c >= 2 and not for any smaller c.
    x = np.linspace(-1, 1, 400001)
    for gamma in (5 / 255, 10 / 255, 0.3):
        assert np.min(O.g2_welsch(x, gamma, O.C0_WELSCH)) >= -1e-12
        assert np.min(O.g2_welsch(x, gamma, 0.95 * O.C0_WELSCH)) < 0
        h = 1e-5 * gamma
        xs = np.array([-0.7, -gamma, 0.3 * gamma, 2 * gamma])
        g = lambda t: t * t - O.phi_welsch(t, gamma)
        num = (g(xs + h) - 2 * g(xs) + g(xs - h)) / h ** 2
        np.testing.assert_allclose(O.g2_welsch(xs, gamma, 2.0), num, rtol=1e-4, atol=1e-4)


@pytest.mark.parametrize("H,W,lam,gamma,N", [(8, 8, 20.0, 10 / 255, 4), (5, 7, 3.0, 0.2, 3)])
def test_welsch_algorithm_matches_dense_bruteforce(H, W, lam, gamma, N):
    f = small_image(H, W, seed=3 * H + W)
    Dx, Dy = dense_forward_difference(H, W, "x"), dense_forward_difference(H, W, "y")
    want = dense_ils_welsch(f, lam, gamma, N, Dx, Dy)
    np.testing.assert_allclose(O.ils_channel_welsch(f, lam, gamma, N), want, atol=1e-6)


def test_welsch_large_gamma_is_the_quadratic_smoother():
    # gamma -> infinity: phi_W(x) -> x^2, so mu -> 0 and one iteration gives the closed-form
    # quadratic smoother (I + lam (Dx^T Dx + Dy^T Dy))^{-1} f.
    H, W, lam = 7, 9, 1.7
    f = small_image(H, W, seed=5)
    Dx, Dy = dense_forward_difference(H, W, "x"), dense_forward_difference(H, W, "y")
    want = np.linalg.solve(np.eye(H * W) + lam * (Dx.T @ Dx + Dy.T @ Dy), f.reshape(-1)).reshape(H, W)
    np.testing.assert_allclose(O.ils_channel_welsch(f, lam, 1e4, 1), want, atol=1e-9)


def test_welsch_energy_is_non_increasing_and_invariants():
    f = small_image(24, 20, seed=17)
    for lam, gamma in ((20.0, 10 / 255), (5.0, 0.1)):
        _, its = O.ils_channel_welsch(f, lam, gamma, 12, return_iterates=True)
        E = [O.energy_welsch(u, f, lam, gamma) for u in its]
        assert all(E[i + 1] <= E[i] * (1 + 1e-12) for i in range(len(E) - 1)), E
        assert E[-1] < E[0]
        assert abs(its[-1].mean() - f.mean()) < 1e-12
    np.testing.assert_allclose(O.ils_channel_welsch(f, 0.0, 0.05, 3), f, atol=1e-13)
    np.testing.assert_allclose(O.ils_channel_welsch(np.full((6, 8), 0.4), 9.0, 0.05, 3), 0.4, atol=1e-13)


def test_welsch_adjoint_matches_finite_differences():
    H, W, lam, gamma, N = 8, 10, 6.0, 0.08, 3
    rng = np.random.default_rng(4)
    f = small_image(H, W, seed=19)
    gu = rng.normal(size=(H, W))
    got = O.ils_backward_welsch(f, gu, lam, gamma, N)
    for _ in range(3):
        d = rng.normal(size=(H, W))
        h = 1e-6
        num = (np.sum(gu * O.ils_channel_welsch(f + h * d, lam, gamma, N))
               - np.sum(gu * O.ils_channel_welsch(f - h * d, lam, gamma, N))) / (2 * h)
        assert np.sum(got * d) == pytest.approx(num, rel=1e-6, abs=1e-9)


# ---------------------------------------------------------------- luminance-only colour mode and detail enhancement

def yuv_from_rgb(f):
    # a full YUV transform (BT.601 luma; U, V scaled colour differences) and its inverse,
    # written independently of the oracle's shortcut
    R, G, B = f
    Y = 0.299 * R + 0.587 * G + 0.114 * B
    return Y, 0.492 * (B - Y), 0.877 * (R - Y)


def rgb_from_yuv(Y, U, V):
    R = Y + V / 0.877
    B = Y + U / 0.492
    G = (Y - 0.299 * R - 0.114 * B) / 0.587
    return np.stack([R, G, B])


def test_luma_mode_is_smoothing_y_in_yuv_and_converting_back():
    f = synth.voronoi_texture(20, 24, 3, K=5, A=0.05, Tmin=3, Tmax=5, sigma=0.02, seed=3).astype(np.float64)
    for k in (0.0, 3.0):
        Y, U, V = yuv_from_rgb(f)
        uY = O.ils_channel(Y, 1.0, 0.8, 1e-4, 4)
        want = rgb_from_yuv(uY + k * (Y - uY), U, V)
        np.testing.assert_allclose(O.ils_smooth_luma(f, 1.0, 0.8, 1e-4, 4, k), want, atol=1e-12)


def test_luma_mode_on_a_gray_image_equals_per_channel_smoothing():
    g = small_image(16, 20, seed=23)
    f = np.stack([g, g, g])
    np.testing.assert_allclose(O.ils_smooth_luma(f, 1.0, 0.8, 1e-4, 4), O.ils_smooth(f, 1.0, 0.8, 1e-4, 4),
                               atol=1e-12)


def test_detail_enhance_limits():
    f = small_image(10, 12, seed=29)
    u = O.ils_channel(f, 1.0, 0.8, 1e-4, 4)
    np.testing.assert_allclose(O.detail_enhance(f, u, 0.0), u, atol=0)
    np.testing.assert_allclose(O.detail_enhance(f, u, 1.0), f, atol=1e-15)
    # the detail layer is scaled by k: (out - u) = k (f - u)
    np.testing.assert_allclose(O.detail_enhance(f, u, 3.0) - u, 3.0 * (f - u), atol=1e-14)


# ---------------------------------------------------------------- HDR tone mapping (Sec. 4.2)

def hdr_image(H, W, seed, stops=12.0):
    """Linear radiance spanning 2^stops: exp2 of a scaled synthetic texture per channel."""
    g = synth.voronoi_texture(H, W, 3, K=5, A=0.05, Tmin=3, Tmax=5, sigma=0.02, seed=seed).astype(np.float64)
    return np.exp2(stops * (g - 0.5))


def test_log_luma_floor_and_value():
    f = hdr_image(6, 8, seed=41)
    f[:, 2, 3] = 0.0                      # a black pixel
    l = O.log_luma(f)
    assert l[2, 3] == pytest.approx(np.log(1e-12), abs=1e-12)
    y = 0.299 * f[0, 1, 1] + 0.587 * f[1, 1, 1] + 0.114 * f[2, 1, 1]
    assert l[1, 1] == pytest.approx(np.log(y), abs=1e-13)


def test_tonemap_identity_and_lambda_zero_closed_form():
    f = hdr_image(10, 12, seed=43)
    out, b, d = O.tonemap_log(f, s=1.0, k=1.0, o=0.0, lam=10.0, N=4)
    np.testing.assert_allclose(out, f, rtol=1e-12)
    # lambda = 0: the base is l itself (u = f for every N), so out_c = f_c Y^(s - 1) e^o
    s_, o_ = 0.4, 0.3
    Y = 0.299 * f[0] + 0.587 * f[1] + 0.114 * f[2]
    out0, b0, d0 = O.tonemap_log(f, s=s_, k=2.0, o=o_, lam=0.0, N=3)
    np.testing.assert_allclose(out0, f * np.power(Y, s_ - 1.0)[None] * np.exp(o_), rtol=1e-12)
    np.testing.assert_allclose(d0, 0.0, atol=1e-12)


def test_tonemap_output_log_luminance_is_compressed_base_plus_boosted_detail():
    # ln Y(out) = s b + k d + o, with b + d = ln Y(f): the colour scaling applies exactly the
    # intended change of log-luminance (luminance is linear in the channels)
    f = hdr_image(12, 16, seed=47)
    s_, k_, o_ = 0.35, 1.5, -0.2
    out, b, d = O.tonemap_log(f, s=s_, k=k_, o=o_, lam=10.0, N=4)
    Yf = 0.299 * f[0] + 0.587 * f[1] + 0.114 * f[2]
    Yo = 0.299 * out[0] + 0.587 * out[1] + 0.114 * out[2]
    np.testing.assert_allclose(b + d, np.log(Yf), atol=1e-12)
    np.testing.assert_allclose(np.log(Yo), s_ * b + k_ * d + o_, atol=1e-11)
    # colour ratios are kept
    np.testing.assert_allclose(out[0] / out[1], f[0] / f[1], rtol=1e-12)
    np.testing.assert_allclose(out[2] / out[1], f[2] / f[1], rtol=1e-12)
    # the smoothing keeps the mean (the DC denominator is 1), so the detail layer has zero mean
    assert abs(d.mean()) < 1e-12


def test_tonemap_exposure_equivariance():
    # ILS commutes with adding a constant (gradients ignore it; the DC denominator is 1), so
    # scaling the radiance by g scales the tone-mapped image by g^s
    f = hdr_image(8, 10, seed=53)
    s_, k_ = 0.5, 1.2
    a, _, _ = O.tonemap_log(f, s=s_, k=k_, lam=10.0, N=4)
    g = 37.0
    bb, _, _ = O.tonemap_log(g * f, s=s_, k=k_, lam=10.0, N=4)
    np.testing.assert_allclose(bb, g ** s_ * a, rtol=1e-9)


# ---------------------------------------------------------------- Gaussian pre-smoothing (Sec. 5, texture smoothing)

def test_gaussian_weights_shape():
    w = O.gaussian_weights(1.0)
    assert len(w) == 7 and abs(w.sum() - 1.0) < 1e-15
    np.testing.assert_allclose(w, w[::-1], atol=0)
    assert w[3] == w.max() and w[2] / w[3] == pytest.approx(np.exp(-0.5), rel=1e-14)
    np.testing.assert_array_equal(O.gaussian_weights(0.0), [1.0])


def test_gaussian_blur_impulse_response_and_mean():
    # the response to a unit impulse is the outer product of the taps (brute force), wrapped
    H, W, s = 9, 11, 1.3
    f = np.zeros((H, W))
    f[2, 9] = 1.0
    g = O.gaussian_blur_periodic(f, s)
    w = O.gaussian_weights(s)
    r = (len(w) - 1) // 2
    want = np.zeros((H, W))
    for a in range(-r, r + 1):
        for b in range(-r, r + 1):
            want[(2 + a) % H, (9 + b) % W] += w[a + r] * w[b + r]
    np.testing.assert_allclose(g, want, atol=1e-15)
    x = small_image(12, 10, seed=61)
    assert abs(O.gaussian_blur_periodic(x, 0.8).mean() - x.mean()) < 1e-14
    np.testing.assert_allclose(O.gaussian_blur_periodic(np.full((5, 6), 0.3), 2.0), 0.3, atol=1e-15)
    np.testing.assert_allclose(O.gaussian_blur_periodic(x, 0.0), x, atol=0)


def test_gaussian_blur_is_a_periodic_convolution():
    # equal to the product of DFTs with the wrapped kernel (numpy.fft as a library comparator)
    H, W, s = 16, 20, 1.7
    x = small_image(H, W, seed=67)
    w = O.gaussian_weights(s)
    r = (len(w) - 1) // 2
    k = np.zeros((H, W))
    for a in range(-r, r + 1):
        for b in range(-r, r + 1):
            k[(-a) % H, (-b) % W] += w[a + r] * w[b + r]   # correlation taps as a kernel
    want = np.real(np.fft.ifft2(np.fft.fft2(x) * np.fft.fft2(k)))
    np.testing.assert_allclose(O.gaussian_blur_periodic(x, s), want, atol=1e-12)


def test_texture_smooth_is_welsch_ils_of_the_blurred_input():
    x = small_image(12, 14, seed=71)
    g = O.gaussian_blur_periodic(x, 1.0)
    np.testing.assert_allclose(O.texture_smooth(x, 1.0, 30.0, 10 / 255, 3),
                               O.ils_channel_welsch(g, 30.0, 10 / 255, 3), atol=1e-14)


# ---------------------------------------------------------------- interleaved (H x W x C) images

def test_hwc_layout_by_explicit_indexing():
    H, W, C = 3, 4, 3
    x = np.arange(H * W * C, dtype=np.float64).reshape(H, W, C)
    p = O.hwc_to_planar(x)
    flat = x.ravel()
    for c in range(C):
        for y in range(H):
            for xx in range(W):
                assert p[c, y, xx] == flat[(y * W + xx) * C + c]
    np.testing.assert_array_equal(O.planar_to_hwc(p), x)


def test_ils_smooth_hwc_is_per_channel_smoothing():
    f = synth.voronoi_texture(10, 12, 3, K=5, A=0.05, Tmin=3, Tmax=5, sigma=0.02, seed=59).astype(np.float64)
    fh = np.stack([f[0], f[1], f[2]], axis=-1)
    uh = O.ils_smooth_hwc(fh, 1.0, 0.8, 1e-4, 4)
    for c in range(3):
        np.testing.assert_allclose(uh[:, :, c], O.ils_channel(f[c], 1.0, 0.8, 1e-4, 4), atol=1e-14)


# ---------------------------------------------------------------- half-quadratic splitting (Sec. 3.5)

def test_hqs_q1_is_the_argmin_and_matches_huber():
    # Q1 of Eq. 14 by brute force over mu, and Eq. 17: min_mu g_H = the Huber penalty of Eq. 16
    lam, beta = 0.25, 0.7
    mus = np.linspace(-2, 2, 400001)
    alpha = lam / (2 * beta)          # 1/(2 alpha) = beta / lam
    for x in (-0.9, -0.2, -0.05, 0.0, 0.03, 0.17, 0.6):
        obj = beta * (x - mus) ** 2 + lam * np.abs(mus)
        assert abs(mus[np.argmin(obj)] - O.hqs_shrink_l1(x, lam, beta)) <= 2e-5
        gH = (x - mus) ** 2 / (2 * alpha) + np.abs(mus)
        huber = x * x / (2 * alpha) if abs(x) <= alpha else abs(x) - alpha / 2
        assert gH.min() == pytest.approx(huber, abs=1e-9)


@pytest.mark.parametrize("H,W,lam,N", [(8, 8, 0.25, 4), (5, 7, 0.1, 3)])
def test_hqs_matches_dense_bruteforce(H, W, lam, N):
    f = small_image(H, W, seed=5 * H + W)
    Dx, Dy = dense_forward_difference(H, W, "x"), dense_forward_difference(H, W, "y")
    u = f.reshape(-1).copy()
    beta = 2 * lam
    for _ in range(N):
        gx, gy = Dx @ u, Dy @ u
        # Q1 by a per-element brute force over mu (no closed form used)
        grid = np.linspace(-1.5, 1.5, 300001)
        mx = np.array([grid[np.argmin(beta * (g - grid) ** 2 + lam * np.abs(grid))] for g in gx])
        my = np.array([grid[np.argmin(beta * (g - grid) ** 2 + lam * np.abs(grid))] for g in gy])
        A = np.eye(H * W) + beta * (Dx.T @ Dx + Dy.T @ Dy)
        u = np.linalg.solve(A, f.reshape(-1) + beta * (Dx.T @ mx + Dy.T @ my))
        beta *= 2.0
    np.testing.assert_allclose(O.hqs_channel(f, lam, N), u.reshape(H, W), atol=3e-5)


def test_hqs_limits():
    f = small_image(12, 10, seed=31)
    np.testing.assert_allclose(O.hqs_channel(f, 0.0, 4, beta0=1.0), f, atol=1e-13)  # no threshold: mu = grad f
    np.testing.assert_allclose(O.hqs_channel(np.full((6, 8), 0.3), 0.5, 3), 0.3, atol=1e-13)
    u = O.hqs_channel(f, 0.25, 4)
    assert abs(u.mean() - f.mean()) < 1e-13
    # a huge threshold (lam >> gradients) zeroes mu: one step is the quadratic smoother with weight beta0
    H, W = f.shape
    Dx, Dy = dense_forward_difference(H, W, "x"), dense_forward_difference(H, W, "y")
    b0 = 3.0
    want = np.linalg.solve(np.eye(H * W) + b0 * (Dx.T @ Dx + Dy.T @ Dy), f.reshape(-1)).reshape(H, W)
    np.testing.assert_allclose(O.hqs_channel(f, 1e3, 1, beta0=b0), want, atol=1e-12)
