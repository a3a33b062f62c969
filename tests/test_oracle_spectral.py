"""Pins of the oracle's spectral port objective (Eq. 10 in discrete form:
sum_b w_b sum_q |DFT of the port-mean series at f_q|): a closed form for a
precessing macrospin, finite differences of the per-step weights, and
central finite differences of the full gradient dJ/dPhi, dJ/dm0."""
import numpy as np
import pytest

import workloads as W
from oracle import llg

from tests.test_oracle_adjoint import _J, _fd_richardson


def test_larmor_macrospin_spectrum_closed_form():
    # m = (cos wt, sin wt, 0) for B along z, alpha = 0: the port series is
    # sin(w n dt) and X(f) = sum_n sin(w n dt) exp(-2 pi i f n dt)
    B, dt, N, n0 = 0.1, 1e-13, 400, 100
    w = llg.GAMMA * B
    f0 = w / (2 * np.pi)
    freqs = (f0, f0 + 0.3e9, f0 - 0.5e9)
    p = W.Problem(nx=1, ny=1, nz=1, Ms=8e5, A=1.3e-11, alpha=0.0, B_bias=(0.0, 0.0, B), dt=dt, nsteps=N,
                  objective=W.J_SPECTRAL, comp=1, boxes=((0, 1, 0, 1), (0, 0, 0, 0)), weights=(1.0, 0.0),
                  n_from=n0, freqs=freqs)
    J, _, _ = llg.Model(p, np.ones((1, 1, 1))).forward(np.array([1.0, 0.0, 0.0]), keep=False)
    n = np.arange(n0, N + 1)
    expect = sum(abs((np.sin(w * n * dt) * np.exp(-2j * np.pi * f * n * dt)).sum()) for f in freqs)
    assert J == pytest.approx(expect, rel=1e-9)


def test_spectral_weights_are_the_derivative_of_the_spectral_sum():
    p = W.Problem(nx=4, ny=4, dt=1e-13, nsteps=30, objective=W.J_SPECTRAL, weights=(1.0, -0.7), n_from=5,
                  boxes=((0, 2, 0, 2), (2, 4, 2, 4)), freqs=(3e9, 7e9, 11e9))
    mod = llg.Model(p, np.ones((1, 4, 4)))
    rng = np.random.default_rng(2)
    series = rng.standard_normal((p.nsteps - p.n_from + 1, 2))
    Wt = mod.spectral_weights(series)
    h = 1e-6
    for n, b in [(0, 0), (7, 1), (25, 0), (13, 1)]:
        sp, sm = series.copy(), series.copy()
        sp[n, b] += h
        sm[n, b] -= h
        fd = (mod.spectral_value(sp) - mod.spectral_value(sm)) / (2 * h)
        assert Wt[n, b] == pytest.approx(fd, rel=1e-7, abs=1e-9)


@pytest.mark.parametrize("shape", [(6, 6), (8, 5)])
def test_spectral_gradient_matches_finite_differences(shape):
    inst = W.random_small(*shape, 1, seed=21, nsteps=50, objective=W.J_SPECTRAL, freqs=(8e9, 9.5e9), n_from=10)
    p = inst.problem
    J, g, gm0 = llg.gradient(inst)
    rng = np.random.default_rng(22)
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


def test_spectral_objective_needs_a_window_after_step_zero():
    inst = W.random_small(4, 4, 1, seed=1, nsteps=5, objective=W.J_SPECTRAL, freqs=(1e9,), n_from=0)
    with pytest.raises(ValueError):
        llg.Model(inst.problem, inst.phi).forward(inst.m0)
