"""Pins of the oracle's RBF level-set map (Eq. 2, Eq. 3 with the
renormalisation) and of its Adam step against closed forms, limits and
central finite differences."""
import numpy as np
import pytest

from oracle import rbf

H = 5e-9


def _setup(nrx=4, nry=3, box=(2, 14, 1, 10), seed=0):
    xk, yk, c = rbf.centres(20, 12, H, H, box, nrx, nry)
    xj, yj = rbf.design_nodes(20, 12, H, H, box)
    rng = np.random.default_rng(seed)
    s = rng.uniform(-20e-9, 20e-9, xk.size)
    return s, xk, yk, c, xj, yj


def test_centres_are_cell_centres_of_the_design_box():
    xk, yk, c = rbf.centres(20, 12, H, H, (2, 14, 1, 10), 4, 3)
    assert xk.size == 12
    np.testing.assert_allclose(np.unique(xk), (2 + (np.arange(4) + 0.5) * 3) * H)
    np.testing.assert_allclose(np.unique(yk), (1 + (np.arange(3) + 0.5) * 3) * H)
    assert c == pytest.approx(3 * H)


def test_single_rbf_is_the_cone_renormalised():
    # one term: [(g + dphi)^p]^(1/p) - dphi = g exactly, then Phi = g / max|g|
    xj, yj = rbf.design_nodes(20, 12, H, H, (0, 20, 0, 12))
    xk, yk, c = np.array([7 * H]), np.array([4 * H]), 2 * H
    s = np.array([30e-9])
    phi, q = rbf.phi_map(s, xk, yk, c, xj, yj, 90)
    g = 30e-9 - np.sqrt((xj - 7 * H) ** 2 + (yj - 4 * H) ** 2 + 4 * H * H)
    np.testing.assert_allclose(q["F"], g, rtol=0, atol=1e-22)
    np.testing.assert_allclose(phi, g / np.abs(g).max(), rtol=1e-13, atol=1e-13)


def test_identical_rbfs_scale_the_norm_by_k_to_the_one_over_p():
    xj, yj = rbf.design_nodes(8, 8, H, H, (0, 8, 0, 8))
    K, p = 5, 90
    xk, yk = np.full(K, 3 * H), np.full(K, 4 * H)
    s = np.full(K, 12e-9)
    _, q = rbf.phi_map(s, xk, yk, H, xj, yj, p)
    g = 12e-9 - np.sqrt((xj - 3 * H) ** 2 + (yj - 4 * H) ** 2 + H * H)
    dphi = abs(g.min())
    np.testing.assert_allclose(q["F"], (g + dphi) * K ** (1.0 / p) - dphi, rtol=1e-12, atol=1e-22)


def test_large_p_approaches_the_maximum():
    s, xk, yk, c, xj, yj = _setup()
    _, q = rbf.phi_map(s, xk, yk, c, xj, yj, 4000)
    gmax = q["G"].max(axis=1)
    U = q["u"].max(axis=1)
    gap = q["F"] - gmax                     # in [0, (K^(1/p) - 1) U]
    assert (gap >= -1e-22).all()
    assert (gap <= (xk.size ** (1 / 4000) - 1) * U + 1e-22).all()


def test_no_overflow_at_p_90_with_large_arguments():
    # u = 2e5 and 1e5: the naive sum of 90th powers overflows, the p-norm is
    # 2e5 (1 + 2^-90)^(1/90) = 2e5 to double precision
    xj, yj = np.array([0.0]), np.array([0.0])
    xk, yk = np.array([0.0, 0.0]), np.array([0.0, 0.0])
    s = np.array([2e5 + 1.0, 1e5 + 1.0])    # g = s - 1 (c = 1, centre on the node)
    _, q = rbf.phi_map(s, xk, yk, 1.0, xj, yj, 90)
    # dphi = |min g| = 1e5, u = (3e5, 2e5): ||u||_90 = 3e5 (1 + (2/3)^90)^(1/90)
    expect = 3e5 * (1 + (2 / 3) ** 90) ** (1 / 90) - 1e5
    assert np.isfinite(q["F"]).all()
    assert q["F"][0] == pytest.approx(expect, rel=1e-15)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gradient_matches_central_differences(seed):
    s, xk, yk, c, xj, yj = _setup(seed=seed)
    rng = np.random.default_rng(100 + seed)
    w = rng.standard_normal(xj.size)
    J = lambda ss: float(w @ rbf.phi_map(ss, xk, yk, c, xj, yj, 90)[0])
    g = rbf.phi_grad(s, xk, yk, c, xj, yj, 90, w)
    h = 1e-14
    scale = np.abs(g).max()
    for k in range(xk.size):
        e = np.zeros_like(s)
        e[k] = h
        fd = (J(s + e) - J(s - e)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * scale, (k, fd, g[k])


def test_gradient_includes_the_shift_and_the_renormalisation():
    # dropping either chain-rule term changes the gradient (a plausible
    # mistake the finite differences above would also catch)
    s, xk, yk, c, xj, yj = _setup(seed=3)
    w = np.random.default_rng(7).standard_normal(xj.size)
    full = rbf.phi_grad(s, xk, yk, c, xj, yj, 90, w)
    _, q = rbf.phi_map(s, xk, yk, c, xj, yj, 90)
    W = (q["u"] / q["norm"][:, None]) ** 89
    naive = (w / q["M"]) @ W
    assert np.abs(full - naive).max() > 1e-3 * np.abs(full).max()


def test_adam_first_steps_by_hand():
    s0, g0, g1 = np.array([0.5, -0.2]), np.array([2.0, -0.5]), np.array([1.0, 0.25])
    lr, b1, b2, eps = 0.01, 0.9, 0.999, 1e-8
    s1, m1, v1 = rbf.adam(s0, g0, np.zeros(2), np.zeros(2), 1, lr, b1, b2, eps)
    # first step: bias-corrected moments are g and g^2
    np.testing.assert_allclose(s1, s0 - lr * g0 / (np.abs(g0) + eps), rtol=1e-15)
    s2, m2, v2 = rbf.adam(s1, g1, m1, v1, 2, lr, b1, b2, eps)
    m = b1 * (1 - b1) * g0 + (1 - b1) * g1
    v = b2 * (1 - b2) * g0 ** 2 + (1 - b2) * g1 ** 2
    step = lr * (m / (1 - b1 ** 2)) / (np.sqrt(v / (1 - b2 ** 2)) + eps)
    np.testing.assert_allclose(s2, s1 - step, rtol=1e-14)
