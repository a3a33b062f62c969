"""Pins of the oracle's field terms and LLG time stepping.

Closed forms: Larmor precession, Gilbert damping of a macrospin, the
anisotropy-shifted precession frequency, Kittel's formula (with Aharoni's
prism factors for the demag of a single platelet cell and, at a few percent,
of the 32x32 film), the discrete Neumann-Laplacian eigenvalue of exchange.
Invariants: fields are minus the energy gradient, monotone energy decay at
alpha > 0, |m| = 1 up to the RK4 truncation order.
"""
import numpy as np
import pytest

import workloads as W
from oracle import llg
from tests.test_oracle_demag import aharoni_factor

G = llg.GAMMA
MU0 = llg.MU0


def macrospin(dx=5e-9, dy=5e-9, dz=5e-9, **kw):
    base = dict(nx=1, ny=1, nz=1, dx=dx, dy=dy, dz=dz, Ms=8e5, A=1.3e-11,
                alpha=0.0, dt=1e-13, nsteps=1, objective=W.J_PORT, weights=(0.0, 0.0))
    base.update(kw)
    p = W.Problem(**base)
    return llg.Model(p, np.ones((1, 1, 1)))


def run(model, m0, nsteps):
    m = np.array(m0, float).reshape(3, 1, 1, 1)
    out = [m]
    for n in range(nsteps):
        m = model.step(m, n)
        out.append(m)
    return np.array(out)[:, :, 0, 0, 0]


def test_material_map():
    phi = np.array([-1.0, -0.1, 0.0, 0.02, 1.0])
    psi = llg.psi_map(phi, 50.0)
    assert psi[2] == 0.5
    np.testing.assert_allclose(psi + llg.psi_map(-phi, 50.0), 1.0, rtol=1e-15)
    h = 1e-7
    fd = (llg.psi_map(phi + h, 50.0) - llg.psi_map(phi - h, 50.0)) / (2 * h)
    np.testing.assert_allclose(50.0 * psi * (1 - psi), fd, rtol=1e-7, atol=1e-25)


def test_larmor_precession_and_rk4_order():
    B = 0.1
    errs = []
    for dt in (2e-12, 1e-12):
        mod = macrospin(B_bias=(0.0, 0.0, B), dt=dt)
        T = 2e-10
        n = int(round(T / dt))
        traj = run(mod, [1.0, 0.0, 0.0], n)
        t = np.arange(n + 1) * dt
        exact = np.stack([np.cos(G * B * t), np.sin(G * B * t), 0 * t], axis=1)
        errs.append(np.abs(traj - exact).max())
    assert errs[1] < 1e-6
    assert 14.0 < errs[0] / errs[1] < 18.0       # fourth order


def test_gilbert_damping_closed_form():
    B, a = 0.2, 0.1
    mod = macrospin(B_bias=(0.0, 0.0, B), alpha=a, dt=2e-14)
    th0 = 1.0
    n = 5000
    traj = run(mod, [np.sin(th0), 0.0, np.cos(th0)], n)
    t = n * 2e-14
    th = 2 * np.arctan(np.tan(th0 / 2) * np.exp(-a * G * B * t / (1 + a * a)))
    ph = G * B * t / (1 + a * a)
    exact = np.array([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
    np.testing.assert_allclose(traj[-1], exact, atol=1e-9)


def _frequency(sig, dt):
    """Mean frequency from upward zero crossings (linear interpolation)."""
    s = sig - sig.mean()
    idx = np.where((s[:-1] < 0) & (s[1:] >= 0))[0]
    tc = (idx + (-s[idx]) / (s[idx + 1] - s[idx])) * dt
    return (len(tc) - 1) / (tc[-1] - tc[0])


def test_anisotropy_shifts_precession():
    B, Ku, Ms = 0.05, 4e4, 8e5
    mod = macrospin(B_bias=(0.0, 0.0, B), Ku=Ku, ku=(0.0, 0.0, 1.0), Ms=Ms, dt=2e-13)
    th = 1e-3
    traj = run(mod, [np.sin(th), 0.0, np.cos(th)], 6000)
    f = _frequency(traj[:, 0], 2e-13)
    expect = G * (B + 2 * Ku / Ms) / (2 * np.pi)
    assert f == pytest.approx(expect, rel=2e-5)


def test_kittel_platelet_macrospin():
    """A single 60x60x5 nm cell: its demag self term is the prism's factor, so
    the small-angle precession about an in-plane bias is Kittel's
    omega = gamma sqrt((B + mu0 Ms (Ny-Nx))(B + mu0 Ms (Nz-Nx)))."""
    dx = dy = 60e-9
    dz = 5e-9
    Ms, B = 8e5, 0.05
    mod = macrospin(dx=dx, dy=dy, dz=dz, Ms=Ms, B_bias=(B, 0.0, 0.0), dt=2e-13)
    Nx = aharoni_factor(dy / 2, dz / 2, dx / 2)
    Ny = aharoni_factor(dz / 2, dx / 2, dy / 2)
    Nz = aharoni_factor(dx / 2, dy / 2, dz / 2)
    w = G * np.sqrt((B + MU0 * Ms * (Ny - Nx)) * (B + MU0 * Ms * (Nz - Nx)))
    th = 1e-4
    traj = run(mod, [np.cos(th), np.sin(th), 0.0], 8000)
    f = _frequency(traj[:, 1], 2e-13)
    assert f == pytest.approx(w / (2 * np.pi), rel=2e-5)


def _film_frequency(n, h, A, B, dt, T, Ms=8e5):
    p = W.Problem(nx=n, ny=n, nz=1, dx=h, dy=h, dz=5e-9, Ms=Ms, A=A, alpha=0.0,
                  B_bias=(B, 0.0, 0.0), dt=dt, nsteps=1, weights=(0.0, 0.0))
    mod = llg.Model(p, np.ones((1, n, n)))
    th = 2e-3
    m = np.zeros((3, 1, n, n))
    m[0], m[1] = np.cos(th), np.sin(th)
    ys = []
    for k in range(int(round(T / dt))):
        m = mod.step(m, k)
        ys.append(m[2].mean())
    return _frequency(np.array(ys), dt)


def _film_kittel(B, Ms=8e5):
    a, b, c = 80e-9, 80e-9, 2.5e-9
    Nx, Ny, Nz = aharoni_factor(b, c, a), aharoni_factor(c, a, b), aharoni_factor(a, b, c)
    return G * np.sqrt((B + MU0 * Ms * (Ny - Nx)) * (B + MU0 * Ms * (Nz - Nx))) / (2 * np.pi)


def test_kittel_film_rigid_limit():
    """A 160x160x5 nm film held nearly uniform by a stiff exchange (A = 100x
    Permalloy) precesses at Kittel's frequency with the film's average
    (Aharoni) factors: the inter-cell demag sum reproduces the prism."""
    f = _film_frequency(4, 40e-9, 1.3e-9, 0.5, 5e-14, 1.6e-10)
    assert f == pytest.approx(_film_kittel(0.5), rel=2e-3)


def test_kittel_film_uniform_mode():
    """With Permalloy's own exchange the quasi-uniform mode of the same film
    stays within a few percent of Kittel (its profile is not uniform)."""
    f = _film_frequency(8, 20e-9, 1.3e-11, 0.5, 1e-13, 1.5e-10)
    assert f == pytest.approx(_film_kittel(0.5), rel=0.05)


def test_exchange_neumann_eigenmode():
    """On a uniform 1D chain with free ends, cos(pi k (i+1/2)/n) is an
    eigenvector of the discrete Laplacian with eigenvalue -(4/h^2) sin^2(pi k/2n)."""
    n, h, A, Ms, k = 12, 3e-9, 1.3e-11, 8e5, 3
    p = W.Problem(nx=n, ny=1, nz=1, dx=h, dy=h, dz=h, Ms=Ms, A=A, weights=(0.0, 0.0))
    mod = llg.Model(p, np.ones((1, 1, n)))
    i = np.arange(n)
    mode = np.cos(np.pi * k * (i + 0.5) / n)
    m = np.zeros((3, 1, 1, n))
    m[1, 0, 0] = mode
    Bex = mod.exchange(m)
    lam = -(4 / h ** 2) * np.sin(np.pi * k / (2 * n)) ** 2
    np.testing.assert_allclose(Bex[1, 0, 0], 2 * A / Ms * lam * mode, atol=1e-12 * abs(2 * A / Ms * lam))
    assert np.abs(Bex[0]).max() == 0.0


def test_fields_are_energy_gradients():
    """B_ex and B_d equal -(1/(Ms psi_i V)) dE/dm_i of the independently
    written energies (edge sum of A_ij |dm|^2 and -1/2 sum M.B_d)."""
    inst = W.random_small(5, 4, 2, seed=3)
    mod = llg.Model(inst.problem, inst.phi)
    p = inst.problem
    m = inst.m0
    Bex, Bd = mod.exchange(m), mod.demag(m)
    rng = np.random.default_rng(0)
    for _ in range(6):
        c, z, y, x = (rng.integers(0, s) for s in m.shape)
        h = 1e-6
        mp, mm = m.copy(), m.copy()
        mp[c, z, y, x] += h
        mm[c, z, y, x] -= h
        Ep, Em = mod.energy_terms(mp), mod.energy_terms(mm)
        scale = -1.0 / (p.Ms * mod.psi[z, y, x] * mod.V * 2 * h)
        assert scale * (Ep[1] - Em[1]) == pytest.approx(Bex[c, z, y, x], rel=1e-6, abs=1e-9)
        assert scale * (Ep[0] - Em[0]) == pytest.approx(Bd[c, z, y, x], rel=1e-6, abs=1e-9)


def test_energy_decays_with_damping():
    inst = W.particle64()
    p = inst.problem.replace(nx=32, ny=32, nsteps=150)
    phi = inst.phi[:, 16:48, 16:48]
    m0 = inst.m0[:, :, 16:48, 16:48]
    mod = llg.Model(p, phi)
    m = m0
    E = [sum(mod.energy_terms(m))]
    for n in range(p.nsteps):
        m = mod.step(m, n)
        E.append(sum(mod.energy_terms(m)))
    E = np.array(E)
    assert E[-1] < E[0]
    assert (np.diff(E) <= 1e-12 * abs(E[0])).all()


def test_norm_invariant_converges():
    """The LL right-hand side is orthogonal to m, so |m| = 1 is exact for the
    flow; RK4 breaks it only at its truncation order."""
    inst = W.film32()
    p0 = inst.problem
    drift = []
    for k in (1, 2):
        p = p0.replace(dt=p0.dt / k, nsteps=200 * k)
        mod = llg.Model(p, inst.phi)
        m = inst.m0
        worst = 0.0
        for n in range(p.nsteps):
            m = mod.step(m, n)
            worst = max(worst, np.abs(np.sqrt((m * m).sum(0)) - 1).max())
        drift.append(worst)
    assert drift[0] < 1e-5
    assert drift[1] < drift[0] / 16


def test_zeeman_rf_on_source_only():
    inst = W.random_small(6, 4, seed=1)
    mod = llg.Model(inst.problem, inst.phi)
    p = inst.problem
    n, ci = 330, 1                                  # t = 330.5 dt
    t = 330.5 * p.dt
    B = mod.zeeman_stage(n, ci)
    x0, x1, y0, y1 = p.src
    np.testing.assert_array_equal(B, mod.zeeman(t))
    s = p.b_rf * np.sin(2 * np.pi * p.f_rf * t)
    assert B[1, 0, y0, x0] == pytest.approx(p.B_bias[1] + s, rel=1e-12)
    assert B[1, 0, 0, x1] == pytest.approx(p.B_bias[1], rel=1e-14)


def test_tabulated_drive_replaces_the_sine_and_matches_a_bias():
    """A drive table that is constant b along z on a source box covering the
    grid gives the same trajectory as a bias b z (no sine, no box edge)."""
    base = W.random_small(6, 4, seed=2, nsteps=12)
    p = base.problem
    b = 0.013
    p_tab = p.replace(b_rf=0.0, rf_dir=(0.0, 0.0, 1.0), src=(0, p.nx, 0, p.ny), drive=(b,) * (3 * p.nsteps + 3))
    p_bias = p.replace(b_rf=0.0, B_bias=(p.B_bias[0], p.B_bias[1], p.B_bias[2] + b))
    _, m_tab, _ = llg.Model(p_tab, base.phi).forward(base.m0, keep=False)
    _, m_bias, _ = llg.Model(p_bias, base.phi).forward(base.m0, keep=False)
    np.testing.assert_allclose(m_tab, m_bias, rtol=0, atol=1e-13)
    # a table read per (step, stage time): a pulse at one stage time only
    # changes the trajectory from that step on
    pulse = [0.0] * (3 * p.nsteps + 3)
    pulse[3 * 7 + 1] = 0.05
    p_pulse = p_tab.replace(drive=tuple(pulse))
    mod = llg.Model(p_pulse, base.phi)
    m = np.array(base.m0, float)
    ref = llg.Model(p_tab.replace(drive=(0.0,) * (3 * p.nsteps + 3)), base.phi)
    mr = m.copy()
    for n in range(p.nsteps):
        m, mr = mod.step(m, n), ref.step(mr, n)
        assert (np.abs(m - mr).max() > 0) == (n >= 7)


def test_port_functional_closed_form():
    """Constant m_y: J = sum_{n>=n_from} sum_b w_b m_y^p."""
    p = W.Problem(nx=6, ny=4, nz=1, alpha=0.0, dt=1e-13, nsteps=7, comp=1, power=2,
                  boxes=((0, 2, 0, 2), (3, 6, 1, 4)), weights=(0.7, -0.2), n_from=3)
    mod = llg.Model(p, np.ones((1, 4, 6)))
    m = np.zeros((3, 1, 4, 6))
    m[1] = 1.0      # m along y, no field: the oracle keeps it (demag is parallel? no: check J only)
    val = mod.port_term(m)
    assert val == pytest.approx(0.7 - 0.2, rel=1e-15)


@pytest.mark.parametrize("power,n_from", [(1, 0), (2, 1), (2, 37)])
def test_port_objective_on_a_precessing_macrospin(power, n_from):
    """Running port sum over a Larmor macrospin (alpha = 0, B along z,
    m0 = x): m_y(t_n) = sin(w n dt), so J = sum_{n >= n_from} (w_0 + w_1)
    sin(w n dt)^p, with both boxes on the one node; the window start and the
    exponent are both exercised."""
    B, dt, N = 0.1, 1e-13, 120
    p = W.Problem(nx=1, ny=1, nz=1, Ms=8e5, A=1.3e-11, alpha=0.0, B_bias=(0.0, 0.0, B), dt=dt, nsteps=N,
                  objective=W.J_PORT, comp=1, power=power, boxes=((0, 1, 0, 1), (0, 1, 0, 1)),
                  weights=(0.8, -0.3), n_from=n_from)
    J, _, _ = llg.Model(p, np.ones((1, 1, 1))).forward(np.array([1.0, 0.0, 0.0]), keep=False)
    n = np.arange(n_from, N + 1)
    expect = 0.5 * (np.sin(G * B * n * dt) ** power).sum()
    assert J == pytest.approx(expect, rel=1e-9)
