"""Pins of the oracle's demagnetising tensor and demag field.

Each check compares the oracle with something other than itself: Aharoni's
closed-form prism factors (written out here, independently of Newell's
functions), exact identities of the cell-averaged tensor (trace, parity,
self term), the point-dipole limit, and the direct O(N^2) sum.
"""
import numpy as np
import pytest

from oracle import demag as dm


def aharoni_factor(a, b, c):
    """Demagnetising factor along the 2c edge of a uniformly magnetised
    2a x 2b x 2c prism (A. Aharoni, J. Appl. Phys. 83, 3432 (1998))."""
    r = np.sqrt(a * a + b * b + c * c)
    ab, bc, ac = np.sqrt(a * a + b * b), np.sqrt(b * b + c * c), np.sqrt(a * a + c * c)
    t = (b * b - c * c) / (2 * b * c) * np.log((r - a) / (r + a))
    t += (a * a - c * c) / (2 * a * c) * np.log((r - b) / (r + b))
    t += b / (2 * c) * np.log((ab + a) / (ab - a))
    t += a / (2 * c) * np.log((ab + b) / (ab - b))
    t += c / (2 * a) * np.log((bc - b) / (bc + b))
    t += c / (2 * b) * np.log((ac - a) / (ac + a))
    t += 2 * np.arctan(a * b / (c * r))
    t += (a ** 3 + b ** 3 - 2 * c ** 3) / (3 * a * b * c)
    t += (a * a + b * b - 2 * c * c) / (3 * a * b * c) * r
    t += c / (a * b) * (ac + bc)
    t -= (ab ** 3 + bc ** 3 + ac ** 3) / (3 * a * b * c)
    return t / np.pi


def test_aharoni_identities():
    # the pin itself: cube 1/3, factors sum to 1, thin plate -> 1
    assert aharoni_factor(1.0, 1.0, 1.0) == pytest.approx(1 / 3, abs=1e-14)
    for a, b, c in [(1, 2, 3), (5, 1, 0.2), (0.3, 0.7, 0.1)]:
        s = aharoni_factor(a, b, c) + aharoni_factor(b, c, a) + aharoni_factor(c, a, b)
        assert s == pytest.approx(1.0, abs=1e-12)
    assert aharoni_factor(100.0, 100.0, 0.01) > 0.999


def test_self_term_cube():
    t = dm.tensor_newell(np.array(0.0), np.array(0.0), np.array(0.0), 5e-9, 5e-9, 5e-9)
    np.testing.assert_allclose(t[:3], 1 / 3, rtol=1e-13)
    np.testing.assert_allclose(t[3:], 0.0, atol=1e-15)


@pytest.mark.parametrize("d", [(4e-9, 3e-9, 2e-9), (5e-9, 5e-9, 1e-9), (2e-9, 7e-9, 3e-9)])
def test_self_term_is_prism_factor(d):
    dx, dy, dz = d
    t = dm.demag_tensor(np.array(0), np.array(0), np.array(0), dx, dy, dz)
    assert t[0] == pytest.approx(aharoni_factor(dy / 2, dz / 2, dx / 2), rel=1e-11)
    assert t[1] == pytest.approx(aharoni_factor(dz / 2, dx / 2, dy / 2), rel=1e-11)
    assert t[2] == pytest.approx(aharoni_factor(dx / 2, dy / 2, dz / 2), rel=1e-11)


@pytest.mark.parametrize("d", [(5e-9, 5e-9, 5e-9), (4e-9, 3e-9, 2e-9)])
def test_trace_and_parity(d):
    dx, dy, dz = d
    rng = np.random.default_rng(0)
    off = rng.integers(-9, 10, size=(3, 60))
    t = dm.demag_tensor(off[0], off[1], off[2], dx, dy, dz)
    origin = (off == 0).all(axis=0)
    tr = t[0] + t[1] + t[2]
    scale = np.abs(t).max()
    np.testing.assert_allclose(tr[~origin], 0.0, atol=1e-11 * scale)
    tm = dm.demag_tensor(-off[0], -off[1], -off[2], dx, dy, dz)
    np.testing.assert_allclose(tm, t, atol=1e-11 * scale)
    # mirror in x flips xy and xz only
    tx = dm.demag_tensor(-off[0], off[1], off[2], dx, dy, dz)
    sign = np.array([1, 1, 1, -1, -1, 1])[:, None]
    np.testing.assert_allclose(tx, sign * t, atol=1e-11 * scale)


def test_far_field_is_point_dipole():
    h = 5e-9
    V = h ** 3
    for off in [(40, 0, 0), (30, 30, 0), (25, 17, 9)]:
        r = np.array(off, float) * h
        rn = np.linalg.norm(r)
        u = r / rn
        dip = V / (4 * np.pi * rn ** 3) * (np.eye(3) - 3 * np.outer(u, u))
        t = dm.demag_tensor(*[np.array(o) for o in off], h, h, h)
        full = np.array([[t[0], t[3], t[4]], [t[3], t[1], t[5]], [t[4], t[5], t[2]]])
        assert np.abs(full - dip).max() < 2e-3 * np.abs(dip).max()


def test_closed_form_meets_quadrature_at_switch():
    h = (5e-9, 4e-9, 3e-9)
    for off in [(5, 2, 1), (4, 4, 2), (6, 0, 0), (3, 5, 4)]:
        X, Y, Z = [np.array(o * s) for o, s in zip(off, h)]
        a = np.array(dm.tensor_newell(X, Y, Z, *h))
        b = np.array(dm.tensor_quadrature(X, Y, Z, *h, n=10))
        assert np.abs(a - b).max() < 1e-9 * np.abs(b).max()


@pytest.mark.parametrize("cells", [(4, 3, 2), (6, 2, 1), (3, 3, 3)])
def test_prism_average_equals_aharoni(cells):
    """The cell-averaged tensor summed over all cell pairs of a prism, divided
    by the number of cells, is the prism's demagnetising factor exactly."""
    nx, ny, nz = cells
    dx, dy, dz = 3e-9, 4e-9, 2.5e-9
    z, y, x = [a.ravel() for a in np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")]
    tot = np.zeros(6)
    for i in range(x.size):
        tot += dm.demag_tensor(x[i] - x, y[i] - y, z[i] - z, dx, dy, dz).sum(axis=1)
    tot /= x.size
    a, b, c = nx * dx / 2, ny * dy / 2, nz * dz / 2
    assert tot[0] == pytest.approx(aharoni_factor(b, c, a), rel=1e-10)
    assert tot[1] == pytest.approx(aharoni_factor(c, a, b), rel=1e-10)
    assert tot[2] == pytest.approx(aharoni_factor(a, b, c), rel=1e-10)
    np.testing.assert_allclose(tot[3:], 0.0, atol=1e-12)


def test_thin_film_limit():
    """At the centre of a large single-layer film N_zz -> 1, and the
    in-plane factors -> 0, approaching the point value at the centre of a
    prism, (2/pi) atan(ab / (c sqrt(a^2+b^2+c^2)))."""
    n = 96
    h = 5e-9
    ix, iy = np.meshgrid(np.arange(n) - n // 2, np.arange(n) - n // 2)
    t = dm.demag_tensor(ix, iy, np.zeros_like(ix), h, h, h)
    Nzz = t[2].sum()
    a = b = n * h / 2
    c = h / 2
    point = 2 / np.pi * np.arctan(a * b / (c * np.sqrt(a * a + b * b + c * c)))
    assert Nzz > 0.98
    assert Nzz == pytest.approx(point, abs=5e-3)
    assert abs(t[0].sum()) < 0.02


@pytest.mark.parametrize("shape", [(1, 4, 4), (1, 3, 5), (2, 3, 3), (1, 1, 1), (3, 2, 2)])
def test_fft_convolution_equals_direct_sum(shape):
    rng = np.random.default_rng(1)
    M = rng.standard_normal((3,) + shape) * 8e5
    h = (5e-9, 4e-9, 3e-9)
    A = dm.demag_field_direct(M, *h)
    B = dm.demag_field_fft(M, *h)
    assert np.abs(A - B).max() <= 1e-13 * np.abs(A).max()


def test_uniform_cube_cell_field_is_parallel():
    M = np.zeros((3, 1, 1, 1))
    M[:, 0, 0, 0] = [3e5, -2e5, 5e5]
    B = dm.demag_field_fft(M, 5e-9, 5e-9, 5e-9)
    np.testing.assert_allclose(B[:, 0, 0, 0], -dm.MU0 * M[:, 0, 0, 0] / 3, rtol=1e-13)


@pytest.mark.parametrize("cells", [(16, 4, 1), (20, 3, 2)])
def test_long_prism_average_equals_aharoni(cells):
    """Prisms longer than the near/far switch radius: 6 % (16 x 4 x 1) and
    11 % (20 x 3 x 2) of N_xx come from cell pairs the quadrature branch
    evaluates, so the sum pins that branch to about 1e-9."""
    nx, ny, nz = cells
    dx, dy, dz = 3e-9, 4e-9, 2.5e-9
    z, y, x = [a.ravel() for a in np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")]
    hmax = max(dx, dy, dz)
    tot = np.zeros(6)
    far_xx = 0.0
    for i in range(x.size):
        ox, oy, oz = x[i] - x, y[i] - y, z[i] - z
        t = dm.demag_tensor(ox, oy, oz, dx, dy, dz)
        tot += t.sum(axis=1)
        far = (ox * dx) ** 2 + (oy * dy) ** 2 + (oz * dz) ** 2 >= (dm.NEAR_RADIUS * hmax) ** 2
        far_xx += t[0][far].sum()
    tot /= x.size
    a, b, c = nx * dx / 2, ny * dy / 2, nz * dz / 2
    assert abs(far_xx / x.size) > 0.05 * abs(tot[0])        # the far branch carries weight here
    assert tot[0] == pytest.approx(aharoni_factor(b, c, a), rel=1e-10)
    assert tot[1] == pytest.approx(aharoni_factor(c, a, b), rel=1e-10)
    assert tot[2] == pytest.approx(aharoni_factor(a, b, c), rel=1e-10)
    np.testing.assert_allclose(tot[3:], 0.0, atol=1e-12)


def test_far_branch_equals_closed_form_elementwise():
    """Every component of the quadrature branch, off-diagonals included
    (which the prism sums cancel), against Newell's closed form just beyond
    the switch radius, where the closed form still holds ~1e-10 ((R/h)^6 eps
    cancellation)."""
    h = (5e-9, 4e-9, 3e-9)
    hmax = max(h)
    offs = np.array([(7, 2, 1), (6, -3, 2), (-5, 5, 3), (2, 7, -4), (8, 1, 0), (0, 8, 2), (-4, -6, 5)])
    for o in offs:
        X, Y, Z = [np.array(float(k) * s) for k, s in zip(o, h)]
        assert X * X + Y * Y + Z * Z >= (dm.NEAR_RADIUS * hmax) ** 2
        q = dm.demag_tensor(np.array(o[0]), np.array(o[1]), np.array(o[2]), *h)
        c = np.array(dm.tensor_newell(X, Y, Z, *h))
        assert np.abs(q - c).max() < 2e-9 * np.abs(c).max(), o
