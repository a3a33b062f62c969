"""Pins of the oracle's discrete adjoint (Eq. 6/7 in discrete form).

* exact dot-product tests <T^T u, v> = <u, T v> for each linear field map
  (exchange, demag, anisotropy), whose transposes are written separately
  (scatter over edges, same convolution of the cotangent);
* psi-derivatives of each field map against finite differences;
* dJ/dPhi and dJ/dm0 of the whole discrete map against Richardson-extrapolated
  central finite differences of J on 6x6 and 8x8 grids, 50 steps, for both
  objective kinds;
* every checkpoint schedule reproduces the store-all gradient bit for bit;
* the level-set step of Eq. 5 plus renormalisation.
"""
import numpy as np
import pytest

import workloads as W
from oracle import llg, schedule


def _model(nx=6, ny=5, nz=1, seed=2, **kw):
    inst = W.random_small(nx, ny, nz, seed=seed, **kw)
    return inst, llg.Model(inst.problem, inst.phi)


@pytest.mark.parametrize("nz", [1, 2])
def test_dot_product_field_maps(nz):
    inst, mod = _model(6, 5, nz)
    rng = np.random.default_rng(5)
    u = rng.standard_normal(inst.m0.shape)
    v = rng.standard_normal(inst.m0.shape)
    Y = inst.m0
    lhs = (mod.exchange_T(u, Y)[0] * v).sum()
    rhs = (u * mod.exchange(v)).sum()
    assert lhs == pytest.approx(rhs, rel=1e-12)
    lhs = (mod.demag_T(u, Y)[0] * v).sum()
    rhs = (u * mod.demag(v)).sum()
    assert lhs == pytest.approx(rhs, rel=1e-12)
    lhs = (mod.anisotropy_T(u) * v).sum()
    rhs = (u * mod.anisotropy(v)).sum()
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_psi_derivatives_of_field_maps():
    inst, mod = _model(6, 5, 1)
    rng = np.random.default_rng(6)
    u = rng.standard_normal(inst.m0.shape)
    q = rng.standard_normal(mod.psi.shape)
    Y = inst.m0
    ge = mod.exchange_T(u, Y)[1]
    gd = mod.demag_T(u, Y)[1]
    psi0 = mod.psi.copy()
    h = 1e-6
    vals = []
    for s in (1, -1):
        mod.psi = psi0 + s * h * q
        vals.append(((u * mod.exchange(Y)).sum(), (u * mod.demag(Y)).sum()))
    mod.psi = psi0
    fd_e = (vals[0][0] - vals[1][0]) / (2 * h)
    fd_d = (vals[0][1] - vals[1][1]) / (2 * h)
    assert (ge * q).sum() == pytest.approx(fd_e, rel=1e-7)
    assert (gd * q).sum() == pytest.approx(fd_d, rel=1e-7)


def test_stage_vjp_against_directional_derivative():
    inst, mod = _model(5, 4, 1)
    rng = np.random.default_rng(7)
    Y = inst.m0
    u = rng.standard_normal(Y.shape)
    v = rng.standard_normal(Y.shape)
    q = rng.standard_normal(mod.psi.shape)
    t = 1.7e-12
    B = mod.field(Y, t)
    g, gq = mod.stage_vjp(u, Y, B)
    psi0 = mod.psi.copy()
    h = 1e-6
    vals = []
    for s in (1, -1):
        mod.psi = psi0 + s * h * q
        Ys = Y + s * h * v
        vals.append((u * mod.rhs(Ys, mod.field(Ys, t))).sum())
    mod.psi = psi0
    fd = (vals[0] - vals[1]) / (2 * h)
    assert (g * v).sum() + (gq * q).sum() == pytest.approx(fd, rel=1e-7)


def _J(p, phi, m0):
    return llg.Model(p, phi).forward(m0, keep=False)[0]


def _fd_richardson(f, x0, idx, h):
    def d(hh):
        xp, xm = x0.copy(), x0.copy()
        xp[idx] += hh
        xm[idx] -= hh
        return (f(xp) - f(xm)) / (2 * hh)
    return (4 * d(h / 2) - d(h)) / 3


@pytest.mark.parametrize("shape,objective", [((6, 6), W.J_PORT), ((8, 8), W.J_ENERGY_AREA),
                                             ((6, 6), W.J_ENERGY_AREA), ((8, 8), W.J_PORT)])
def test_gradient_matches_finite_differences(shape, objective):
    inst = W.random_small(*shape, 1, seed=11, nsteps=50, objective=objective)
    p = inst.problem
    J, g, gm0 = llg.gradient(inst)
    rng = np.random.default_rng(12)
    scale = np.abs(g).max()
    for _ in range(5):
        idx = tuple(int(rng.integers(0, s)) for s in inst.phi.shape)
        fd = _fd_richardson(lambda ph: _J(p, ph, inst.m0), inst.phi, idx, 2e-4)
        assert abs(g[idx] - fd) <= 1e-6 * scale + 1e-6 * abs(fd)
    scale = np.abs(gm0).max()
    for _ in range(3):
        idx = tuple(int(rng.integers(0, s)) for s in inst.m0.shape)
        fd = _fd_richardson(lambda m: _J(p, inst.phi, m), inst.m0, idx, 1e-4)
        assert abs(gm0[idx] - fd) <= 1e-6 * scale + 1e-6 * abs(fd)


def test_gradient_3d_and_running_port_window():
    """nz = 2 (z exchange, 3D demag) and a port window that starts late."""
    inst = W.random_small(4, 4, 2, seed=4, nsteps=20, n_from=12)
    p = inst.problem
    J, g, _ = llg.gradient(inst)
    scale = np.abs(g).max()
    rng = np.random.default_rng(1)
    for _ in range(4):
        idx = tuple(int(rng.integers(0, s)) for s in inst.phi.shape)
        fd = _fd_richardson(lambda ph: _J(p, ph, inst.m0), inst.phi, idx, 2e-4)
        assert abs(g[idx] - fd) <= 1e-6 * scale + 1e-6 * abs(fd)


@pytest.mark.parametrize("seg", [0, 1, 3, 7, 17, 40])
def test_checkpoint_schedules_reproduce_store_all(seg):
    inst = W.random_small(5, 4, 1, seed=8, nsteps=17)
    mod = llg.Model(inst.problem, inst.phi)
    J0, g0, gm0 = llg.gradient(inst)
    fwd, rev = schedule.periodic(inst.problem.nsteps, seg)
    J1, g1, gm1 = schedule.run_adjoint(mod, inst.m0, fwd, rev)
    assert J1 == J0
    np.testing.assert_array_equal(g1, g0)
    np.testing.assert_array_equal(gm1, gm0)


@pytest.mark.parametrize("snaps", [0, 1, 2, 5])
def test_binomial_schedules_reproduce_store_all(snaps):
    inst = W.random_small(5, 4, 1, seed=8, nsteps=17)
    mod = llg.Model(inst.problem, inst.phi)
    J0, g0, gm0 = llg.gradient(inst)
    fwd, rev = schedule.binomial(inst.problem.nsteps, snaps)
    J1, g1, gm1 = schedule.run_adjoint(mod, inst.m0, fwd, rev)
    assert J1 == J0
    np.testing.assert_array_equal(g1, g0)
    np.testing.assert_array_equal(gm1, gm0)


def test_levelset_step():
    rng = np.random.default_rng(3)
    phi = rng.uniform(-1, 1, (1, 6, 7))
    grad = rng.standard_normal(phi.shape)
    mask = np.zeros(phi.shape, np.uint8)
    mask[0, 1:5, 2:6] = 1
    out = llg.levelset_step(phi, grad, mask, 0.3)
    sel = mask.astype(bool)
    np.testing.assert_array_equal(out[~sel], phi[~sel])
    raw = phi[sel] - 0.3 * grad[sel]
    np.testing.assert_allclose(out[sel], raw / np.abs(raw).max(), rtol=1e-15)
    assert np.abs(out[sel]).max() == 1.0


def test_descent_step_lowers_J():
    """A small step along -dJ/dPhi lowers J by about lr |g|^2 (Eq. 5)."""
    inst = W.random_small(6, 6, 1, seed=9, nsteps=30, objective=W.J_ENERGY_AREA)
    J0, g, _ = llg.gradient(inst)
    lr = 1e-4 / np.abs(g).max()
    J1 = _J(inst.problem, inst.phi - lr * g, inst.m0)
    assert J1 < J0
    assert (J0 - J1) == pytest.approx(lr * (g * g).sum(), rel=1e-2)
