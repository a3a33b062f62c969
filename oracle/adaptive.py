"""Adaptive-step time integration of the LLG forward pass and its discrete
adjoint over the accepted steps, FP64 (test infrastructure only: the tests,
smoke() and bench.py's CPU leg use it).

The paper integrates with an adaptive step size (Methods); this restates it
as the embedded Runge-Kutta pair of Dormand and Prince (1980), 5th order
with a 4th-order error estimate and the first-same-as-last property, with
the usual step-size control:

  y5 = m + h sum_j b_j k_j,   y4 = m + h sum_j b*_j k_j,   e = y5 - y4
  sc = atol + rtol max(|psi m|, |psi y5|)   (per node and component)
  err = sqrt(mean((psi e / sc)^2))          accept if err <= 1
  h <- h min(5, max(0.2, 0.9 err^(-1/5)))   (factor 5 if err = 0)

Readings: the error is measured on the magnetisation psi m, not on m (m at
air nodes carries no magnetisation and its motion is ill-conditioned); the
last step is shortened to end exactly at T = nsteps * dt; the initial step is
dt.  The drive is the sine b_rf sin(2 pi f t) at the stage times t + c_s h.

The gradient is the exact derivative of the map over a FIXED schedule of
accepted steps (h_k): the adjoint of each step y5 = m + h sum b_j k_j(m) taken
through its six stages (b_7 = 0), with kappa_s = h (b_s lam + sum_{i>s}
a_is eta_i), eta_s = (df/dY_s)^T kappa_s.  Objective: the terminal energy and
area objective (J_ENERGY_AREA) at t = T.
"""
from __future__ import annotations

import numpy as np

from . import llg

# Dormand-Prince 5(4) tableau
C = (0.0, 1.0 / 5, 3.0 / 10, 4.0 / 5, 8.0 / 9, 1.0, 1.0)
A = ((),
     (1.0 / 5,),
     (3.0 / 40, 9.0 / 40),
     (44.0 / 45, -56.0 / 15, 32.0 / 9),
     (19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729),
     (9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656),
     (35.0 / 384, 0.0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84))
B5 = (35.0 / 384, 0.0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84, 0.0)
B4 = (5179.0 / 57600, 0.0, 7571.0 / 16695, 393.0 / 640, -92097.0 / 339200, 187.0 / 2100, 1.0 / 40)


def stages(model, m, t, h, k1=None):
    """Stage inputs Y_s, fields B_s and slopes k_s (s = 1..7) of one step of
    size h from (t, m); k1 may be passed in (first same as last)."""
    Y, B, K = [], [], []
    for s in range(7):
        if s == 0:
            y = m
        else:
            y = m + h * sum(A[s][j] * K[j] for j in range(s) if A[s][j] != 0.0)
        b = model.field(y, t + C[s] * h)
        Y.append(y)
        B.append(b)
        K.append(k1 if (s == 0 and k1 is not None) else model.rhs(y, b))
    return Y, B, K


def error_norm(model, m, y5, e, rtol, atol):
    psi = model.psi
    sc = atol + rtol * np.maximum(np.abs(psi * m), np.abs(psi * y5))
    return float(np.sqrt(np.mean((psi * e / sc) ** 2)))


def integrate(model, m0, T, h0, rtol, atol, max_attempts=100000):
    """Adaptive forward.  Returns (m_T, schedule [(t_k, h_k)] of the accepted
    steps, attempts [(t, h, accepted, err)])."""
    m = np.array(m0, float).reshape((3,) + model.shape)
    t, h = 0.0, h0
    sched, attempts = [], []
    k1 = None
    while t < T and len(attempts) < max_attempts:
        last = h >= T - t
        if last:
            h = T - t
        Y, _, K = stages(model, m, t, h, k1)
        y5 = m + h * sum(B5[j] * K[j] for j in range(6) if B5[j] != 0.0)
        e = h * sum((B5[j] - B4[j]) * K[j] for j in range(7) if B5[j] != B4[j])
        err = error_norm(model, m, y5, e, rtol, atol)
        ok = err <= 1.0
        attempts.append((t, h, ok, err))
        if ok:
            sched.append((t, h))
            m = y5
            k1 = K[6]
            t = T if last else t + h
        fac = 5.0 if err == 0.0 else min(5.0, max(0.2, 0.9 * err ** -0.2))
        h = h * fac
    return m, sched, attempts


def replay(model, m0, sched):
    """Forward over a fixed schedule; returns the states m_0..m_K."""
    m = np.array(m0, float).reshape((3,) + model.shape)
    traj = [m]
    for t, h in sched:
        _, _, K = stages(model, m, t, h)
        m = m + h * sum(B5[j] * K[j] for j in range(6) if B5[j] != 0.0)
        traj.append(m)
    return traj


def objective(model, mT):
    """Terminal objective at t = T (J_ENERGY_AREA)."""
    if model.p.objective != llg.J_ENERGY_AREA:
        raise ValueError("the adaptive integrator supports the terminal energy/area objective")
    return model.terminal(mT)


def adjoint(model, m0, sched):
    """(J, dJ/dPhi, dJ/dm0) over the fixed schedule."""
    p = model.p
    traj = replay(model, m0, sched)
    J = objective(model, traj[-1])
    lam, gpsi = model.terminal_grads(traj[-1])
    for k in range(len(sched) - 1, -1, -1):
        t, h = sched[k]
        Y, B, _ = stages(model, traj[k], t, h)
        eta = [None] * 6
        total = np.zeros_like(lam)
        for s in range(5, -1, -1):
            kappa = h * B5[s] * lam
            for i in range(s + 1, 6):
                if A[i][s] != 0.0:
                    kappa = kappa + h * A[i][s] * eta[i]
            g, q = model.stage_vjp(kappa, Y[s], B[s])
            eta[s] = g
            total = total + g
            gpsi = gpsi + q
        lam = lam + total
    dphi = p.sigmoid_a * model.psi * (1.0 - model.psi) * gpsi
    return J, dphi, lam
