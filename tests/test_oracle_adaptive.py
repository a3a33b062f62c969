"""Pins of the oracle's adaptive integrator (Dormand-Prince 5(4) with step
control) and of its adjoint over a fixed schedule: the tableau's order
conditions, the Larmor and Gilbert closed forms, fifth-order convergence at a
fixed step, the controller's behaviour, and finite differences of dJ/dPhi
and dJ/dm0 over a fixed schedule."""
import numpy as np
import pytest

import workloads as W
from oracle import adaptive as AD
from oracle import llg

from tests.test_oracle_adjoint import _fd_richardson

G = llg.GAMMA


def test_tableau_order_conditions():
    c, b, bs = np.array(AD.C), np.array(AD.B5), np.array(AD.B4)
    a = np.zeros((7, 7))
    for i, row in enumerate(AD.A):
        a[i, :len(row)] = row
    np.testing.assert_allclose(a.sum(1), c, atol=1e-15)                # row sums = nodes
    np.testing.assert_allclose(a[6], b, atol=0)                         # first same as last
    for w, order in ((b, 5), (bs, 4)):
        assert w.sum() == pytest.approx(1.0, abs=1e-15)
        for q in range(1, order):                                       # quadrature conditions
            assert w @ c ** q == pytest.approx(1.0 / (q + 1), abs=1e-14)
        assert w @ a @ c == pytest.approx(1.0 / 6, abs=1e-14)
        assert w @ a @ c ** 2 == pytest.approx(1.0 / 12, abs=1e-14)
        assert (w * c) @ a @ c == pytest.approx(1.0 / 8, abs=1e-14)
        assert w @ a @ a @ c == pytest.approx(1.0 / 24, abs=1e-14)
    # fifth-order conditions of the solution weights
    assert b @ a @ c ** 3 == pytest.approx(1.0 / 20, abs=1e-14)
    assert (b * c) @ a @ c ** 2 == pytest.approx(1.0 / 15, abs=1e-14)
    assert (b * c ** 2) @ a @ c == pytest.approx(1.0 / 10, abs=1e-14)
    assert b @ (a @ c) ** 2 == pytest.approx(1.0 / 20, abs=1e-14)
    assert b @ a @ a @ a @ c == pytest.approx(1.0 / 120, abs=1e-14)
    # the embedded pair differs (its difference is the error estimate)
    assert np.abs(b - bs).max() > 1e-3


def macrospin(**kw):
    base = dict(nx=1, ny=1, nz=1, Ms=8e5, A=1.3e-11, alpha=0.0, dt=1e-13, nsteps=1,
                objective=W.J_ENERGY_AREA, penalty_w=0.0)
    base.update(kw)
    return llg.Model(W.Problem(**base), np.ones((1, 1, 1)))


def test_larmor_precession_adaptive_and_fifth_order():
    B = 0.1
    mod = macrospin(B_bias=(0.0, 0.0, B))
    w = G * B
    T = 2e-10
    exact = np.array([np.cos(w * T), np.sin(w * T), 0.0])
    mT, sched, att = AD.integrate(mod, np.array([1.0, 0.0, 0.0]), T, 1e-13, rtol=1e-9, atol=1e-12)
    assert sum(h for _, h in sched) == pytest.approx(T, rel=1e-14)
    assert np.abs(mT.ravel() - exact).max() < 1e-7
    errs = []
    for n in (40, 80):
        h = T / n
        traj = AD.replay(mod, np.array([1.0, 0.0, 0.0]), [(k * h, h) for k in range(n)])
        errs.append(np.abs(traj[-1].ravel() - exact).max())
    assert 26 < errs[0] / errs[1] < 38                                  # 2^5 = 32


def test_gilbert_damping_adaptive_closed_form_and_growing_steps():
    B, a, th0 = 0.2, 0.1, 1.0
    mod = macrospin(B_bias=(0.0, 0.0, B), alpha=a)
    T = 1e-9
    mT, sched, att = AD.integrate(mod, np.array([np.sin(th0), 0.0, np.cos(th0)]), T, 1e-13, rtol=1e-10,
                                  atol=1e-13)
    th = 2 * np.arctan(np.tan(th0 / 2) * np.exp(-a * G * B * T / (1 + a * a)))
    ph = G * B * T / (1 + a * a)
    exact = np.array([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
    assert np.abs(mT.ravel() - exact).max() < 1e-7
    hs = [h for _, h in sched]
    assert hs[len(hs) // 2] > 3 * hs[0]                                  # the step grows from dt
    looser = AD.integrate(mod, np.array([np.sin(th0), 0.0, np.cos(th0)]), T, 1e-13, rtol=1e-6, atol=1e-9)[1]
    assert len(looser) < len(sched)


def test_controller_rejects_an_oversized_step():
    mod = macrospin(B_bias=(0.0, 0.0, 1.0))
    _, sched, att = AD.integrate(mod, np.array([1.0, 0.0, 0.0]), 5e-11, 5e-11, rtol=1e-10, atol=1e-12)
    assert att[0][2] is False and att[0][3] > 1.0                       # one step over the horizon fails
    assert all(ok == (err <= 1.0) for _, _, ok, err in att)
    assert att[1][1] < att[0][1]                                         # and the next try is shorter


def _case(nx, ny, seed):
    inst = W.random_small(nx, ny, 1, seed=seed, nsteps=30, objective=W.J_ENERGY_AREA)
    return inst, llg.Model(inst.problem, inst.phi)


@pytest.mark.parametrize("shape", [(6, 6), (8, 5)])
def test_adjoint_over_a_fixed_schedule_matches_finite_differences(shape):
    inst, mod = _case(*shape, seed=41)
    p = inst.problem
    T = p.nsteps * p.dt
    _, sched, _ = AD.integrate(mod, inst.m0, T, p.dt, rtol=1e-5, atol=1e-8)
    assert 3 < len(sched) < p.nsteps                                    # adaptive: fewer steps than fixed
    J, g, gm0 = AD.adjoint(mod, inst.m0, sched)

    def Jof(phi, m0):
        md = llg.Model(p, phi)
        return AD.objective(md, AD.replay(md, m0, sched)[-1])

    assert J == pytest.approx(Jof(inst.phi, inst.m0), rel=1e-14)
    rng = np.random.default_rng(42)
    scale = np.abs(g).max()
    for _ in range(5):
        idx = tuple(int(rng.integers(0, s)) for s in inst.phi.shape)
        fd = _fd_richardson(lambda ph: Jof(ph, inst.m0), inst.phi, idx, 2e-4)
        assert abs(g[idx] - fd) <= 1e-6 * scale + 1e-6 * abs(fd)
    scale = np.abs(gm0).max()
    for _ in range(3):
        idx = tuple(int(rng.integers(0, s)) for s in inst.m0.shape)
        fd = _fd_richardson(lambda m: Jof(inst.phi, m), inst.m0, idx, 1e-4)
        assert abs(gm0[idx] - fd) <= 1e-6 * scale + 1e-6 * abs(fd)
