"""Pins of the oracle's magnetisation-curve objective (Eq. 8 sampled at the
end of each field level, with the size and centre terms of Eq. 9): a damped
macrospin's closed form, hand-computed penalties of a rectangle, the
staircase field of the Stoner-Wohlfarth workload, and central finite
differences of dJ/dPhi and dJ/dm0."""
import numpy as np
import pytest

import workloads as W
from oracle import llg

from tests.test_oracle_adjoint import _J, _fd_richardson

G = llg.GAMMA


def test_damped_macrospin_curve_closed_form():
    # one cube node: its demag field is parallel to m, so m_z follows the
    # Gilbert closed form tan(th/2) = tan(th0/2) exp(-a G B t / (1 + a^2))
    B, a, dt, th0 = 0.2, 0.1, 2e-14, 1.0
    steps = (400, 1500, 3000)
    targets = (0.7, 0.9, 0.2)
    weights = (0.5, 1.5, -2.0)
    p = W.Problem(nx=1, ny=1, nz=1, Ms=8e5, A=1.3e-11, alpha=a, B_bias=(0.0, 0.0, B), dt=dt, nsteps=3000,
                  objective=W.J_CURVE, comp=2, sample_steps=steps, sample_targets=targets, sample_weights=weights,
                  penalty_w=0.0, centre_w=0.0)
    mod = llg.Model(p, np.ones((1, 1, 1)))
    J, _, _ = mod.forward(np.array([np.sin(th0), 0.0, np.cos(th0)]), keep=False)
    expect = 0.0
    for n, T, w in zip(steps, targets, weights):
        th = 2 * np.arctan(np.tan(th0 / 2) * np.exp(-a * G * B * n * dt / (1 + a * a)))
        expect += w * abs(np.cos(th) - T)
    assert J == pytest.approx(expect, rel=1e-9)
    assert len(mod.curve) == 3


def test_curve_point_is_the_psi_weighted_mean():
    inst = W.random_small(6, 5, seed=3, nsteps=4, objective=W.J_CURVE, comp=1, sample_steps=(4,),
                          sample_targets=(0.0,), sample_weights=(1.0,), penalty_w=0.0)
    mod = llg.Model(inst.problem, inst.phi)
    m = np.random.default_rng(1).standard_normal((3,) + mod.shape)
    psi = mod.psi
    # written out as a loop over nodes
    num = den = 0.0
    for z in range(1):
        for y in range(5):
            for x in range(6):
                num += psi[z, y, x] * m[1, z, y, x]
                den += psi[z, y, x]
    assert mod.curve_point(m) == pytest.approx(num / den, rel=1e-14)


def test_size_and_centre_penalties_of_a_rectangle():
    # Phi = +1 on a 3 x 2 rectangle, -1 elsewhere: psi = 1 there and ~2e-22
    # elsewhere, so the centre is the rectangle's centre and mean psi = 6/48
    nx, ny = 8, 6
    phi = -np.ones((1, ny, nx))
    phi[0, 1:3, 4:7] = 1.0                                  # x 4..6, y 1..2
    p = W.Problem(nx=nx, ny=ny, objective=W.J_CURVE, sample_steps=(1,), sample_targets=(0.0,),
                  sample_weights=(0.0,), nsteps=1, penalty_w=0.05, area_target=0.1, centre_w=1.3,
                  centre_target=(3.5, 2.5))
    mod = llg.Model(p, phi)
    assert mod.centre() == pytest.approx((5.0, 1.5), abs=1e-18)
    expect = 0.05 * (6 / 48 - 0.1) ** 2 + 1.3 * (abs(5.0 - 3.5) + abs(1.5 - 2.5))
    assert mod.penalties() == pytest.approx(expect, rel=1e-12)


def test_sw_workload_ramps_the_field_in_levels():
    inst = W.sw_particle(levels=4, hold=5)
    p = inst.problem
    mod = llg.Model(p, inst.phi)
    b_max = 4e-7 * np.pi * 0.3 * p.Ms
    assert p.nsteps == 25 and p.sample_steps == (10, 15, 20, 25)
    for n in (0, 4, 5, 9, 12, 24, 25):
        for ci in range(3):
            assert mod.drive(n, ci) == pytest.approx(b_max * min(n // 5, 4) / 4, rel=1e-15)
    np.testing.assert_allclose(p.sample_targets, [0.15, 0.3, 0.45, 0.6])
    np.testing.assert_allclose(np.array(p.sample_weights) * np.array(p.sample_targets) * 4, 1.0)


@pytest.mark.parametrize("shape", [(6, 6), (8, 5)])
def test_curve_gradient_matches_finite_differences(shape):
    nx, ny = shape
    N = 40
    drive = tuple(np.repeat(0.02 * (np.arange(N + 1) // 10), 3).tolist())
    inst = W.random_small(nx, ny, 1, seed=23, nsteps=N, objective=W.J_CURVE, comp=0, drive=drive,
                          rf_dir=(1.0, 0.0, 0.0), src=(0, nx, 0, ny), sample_steps=(10, 20, 30, 40),
                          sample_targets=(0.9, -0.8, 0.95, -0.9), sample_weights=(1.0, 0.5, 2.0, 1.0),
                          penalty_w=0.3, area_target=0.2, centre_w=0.7, centre_target=(1.2, 3.9))
    p = inst.problem
    J, g, gm0 = llg.gradient(inst)
    rng = np.random.default_rng(24)
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


def test_curve_samples_must_lie_after_step_zero():
    inst = W.random_small(4, 4, 1, seed=1, nsteps=5, objective=W.J_CURVE, sample_steps=(0,),
                          sample_targets=(0.1,), sample_weights=(1.0,))
    with pytest.raises(ValueError):
        llg.Model(inst.problem, inst.phi).forward(inst.m0)
