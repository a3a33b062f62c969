"""Checkpoint schedules for the reverse sweep (test infrastructure only).

The adjoint recursion of Eq. 6 runs backwards in time and needs the forward
states m_n in reverse order.  The paper's motivation (Introduction; adjoint
section) is to avoid storing all of them.  A schedule is an integer action
list; the reverse sweep is exact for every schedule because each recomputed
step repeats the same arithmetic as the original.

Actions (op, a, b):
  SNAP    (0, n, slot)  copy m_n into checkpoint slot `slot`
  ADVANCE (1, n0, n1)   step m from n0 to n1, recording nothing
  RESTORE (2, slot, n)  load m_n from checkpoint slot `slot`
  RECORD  (3, n0, n1)   step m from n0 to n1, recording each step's stage data
  REVERSE (4, n1, n0)   adjoint steps n1-1, ..., n0 over the recorded data

Periodic schedule with segment length K (K = ceil(sqrt(N)) by default):
checkpoints at n = 0, K, 2K, ...; the forward records the last segment
directly; the reverse restores, re-records and reverses each earlier segment.
Memory: ceil(N/K) checkpoints plus K recorded steps, O(sqrt N) at the default.
Store-all is the periodic schedule with K = 1: all N states are kept.

Binomial schedule with s snapshot slots besides the one holding m_0
(Griewank's binomial checkpointing, as used by revolve): reversing l steps
from a snapshotted start with s free slots, where no step may be advanced
more than r times, is possible exactly when l <= beta(s, r) = C(s + r, s).
The reversal takes the smallest such r, advances m steps and snapshots
there, reverses the right part (l - m steps) with s - 1 slots, then the
left part (m steps) with s slots.  The right part gets as many steps as its
budget beta(s - 1, r) allows (m = l - min(beta(s - 1, r), l - 1)), which
keeps m <= beta(s, r - 1) since beta(s, r) = beta(s, r - 1) + beta(s - 1, r).
With no free slot the steps are re-advanced from the start one by one.
Each step is recorded (one step at a time) just before it is reversed.
The first descent of the recursion (advance, snapshot, advance, ..., record
the last step) covers steps 0..N-1 once in order and is the forward pass.
Memory: s + 1 checkpoints plus one recorded step.
"""
from __future__ import annotations

import math

SNAP, ADVANCE, RESTORE, RECORD, REVERSE = 0, 1, 2, 3, 4


def default_segment(nsteps: int) -> int:
    """Smallest K with K*K >= nsteps (integer square root, rounded up)."""
    if nsteps <= 0:
        return 1
    k = math.isqrt(nsteps)
    return k if k * k >= nsteps else k + 1


def periodic(nsteps: int, seg: int = 0):
    """(forward_actions, reverse_actions) for the periodic schedule."""
    N = nsteps
    K = seg if seg > 0 else default_segment(N)
    if N <= 0:
        return [], []
    nseg = (N + K - 1) // K
    fwd, rev = [], []
    for c in range(nseg):
        a, b = c * K, min(N, (c + 1) * K)
        if c < nseg - 1:
            fwd.append((SNAP, a, c))
            fwd.append((ADVANCE, a, b))
        else:
            fwd.append((RECORD, a, b))
    for c in range(nseg - 1, -1, -1):
        a, b = c * K, min(N, (c + 1) * K)
        if c < nseg - 1:
            rev.append((RESTORE, c, a))
            rev.append((RECORD, a, b))
        rev.append((REVERSE, b, a))
    return fwd, rev


def store_all(nsteps: int):
    """Every state m_n is kept (K = 1); each reverse step re-records its own
    stages from m_n."""
    return periodic(nsteps, 1)


def beta(s: int, r: int, cap: int = 1 << 62) -> int:
    """C(s + r, s), saturated at `cap`."""
    v = 1
    for k in range(1, min(s, r) + 1):
        v = v * (s + r - min(s, r) + k) // k
        if v >= cap:
            return cap
    return v


def binomial(nsteps: int, snaps: int = 0):
    """(forward_actions, reverse_actions) for the binomial schedule with
    `snaps` free checkpoint slots (0 = default_segment(nsteps))."""
    N = nsteps
    if N <= 0:
        return [], []
    s0 = snaps if snaps > 0 else default_segment(N)
    out = [(SNAP, 0, 0)]
    state = {"cur": 0}          # step the working state holds with a valid spectrum, or -1

    def goto(a, slot):
        if state["cur"] != a:
            out.append((RESTORE, slot, a))
            state["cur"] = a

    def rec_rev(n):
        out.append((RECORD, n, n + 1))
        out.append((REVERSE, n + 1, n))
        state["cur"] = -1

    # tasks (a, length, free slots, slot holding m_a), processed last in,
    # first out: a split pushes the left part, then the right part
    tasks = [(0, N, s0, 0)]
    while tasks:
        a, length, s, slot = tasks.pop()
        if length == 1:
            goto(a, slot)
            rec_rev(a)
        elif s == 0:
            for k in range(length - 1, -1, -1):
                goto(a, slot)
                if k > 0:
                    out.append((ADVANCE, a, a + k))
                    state["cur"] = a + k
                rec_rev(a + k)
        else:
            r = 1
            while beta(s, r) < length:
                r += 1
            right = min(beta(s - 1, r), length - 1)
            mid = a + length - right
            goto(a, slot)
            out.append((ADVANCE, a, mid))
            state["cur"] = mid
            out.append((SNAP, mid, slot + 1))
            tasks.append((a, length - right, s, slot))
            tasks.append((mid, right, s - 1, slot + 1))
    first = next(i for i, act in enumerate(out) if act[0] == RECORD)
    return out[:first + 1], out[first + 1:]


def peak_states(fwd, rev):
    """(checkpoint slots, recorded steps) a schedule needs at most."""
    slots = 0
    rec = 0
    for op, a, b in list(fwd) + list(rev):
        if op == SNAP:
            slots = max(slots, b + 1)
        elif op == RECORD:
            rec = max(rec, b - a)
    return slots, rec


def run_adjoint(model, m0, fwd, rev):
    """Execute a schedule with an oracle Model; returns (J, dJ/dPhi, dJ/dm0).
    Used to check that every schedule reproduces the store-all gradient."""
    import numpy as np
    from .llg import J_PORT

    p = model.p
    dt = p.dt
    m = np.array(m0, float).reshape((3,) + model.shape)
    J = 0.0
    if p.objective == J_PORT and p.n_from <= 0:
        J += model.port_term(m)
    slots = {}
    recorded = {}
    cur = 0

    def advance(n0, n1, record):
        nonlocal m, J
        assert cur == n0
        for n in range(n0, n1):
            if record:
                recorded[n] = m
            m = model.step(m, n)
            if first_pass[0] and p.objective == J_PORT and n + 1 >= p.n_from:
                J += model.port_term(m)
        return n1

    first_pass = [True]
    for op, a, b in fwd:
        if op == SNAP:
            slots[b] = m
        elif op in (ADVANCE, RECORD):
            if op == RECORD:
                recorded.clear()
            cur = advance(a, b, op == RECORD)
    mN = m
    J += model.terminal(mN)
    first_pass[0] = False
    lam, gpsi = model.terminal_grads(mN)
    if p.objective == J_PORT and p.nsteps >= p.n_from:
        lam = lam + model.port_term_grad(mN)
    for op, a, b in rev:
        if op == SNAP:
            slots[b] = m
        elif op == RESTORE:
            m = slots[a]
            cur = b
        elif op == RECORD:
            recorded.clear()
            cur = advance(a, b, True)
        elif op == ADVANCE:
            cur = advance(a, b, False)
        elif op == REVERSE:
            for n in range(a - 1, b - 1, -1):
                Y, B, _ = model.stages(recorded[n], n)
                u4 = dt / 6.0 * lam
                g4, q4 = model.stage_vjp(u4, Y[3], B[3])
                u3 = dt / 3.0 * lam + dt * g4
                g3, q3 = model.stage_vjp(u3, Y[2], B[2])
                u2 = dt / 3.0 * lam + 0.5 * dt * g3
                g2, q2 = model.stage_vjp(u2, Y[1], B[1])
                u1 = dt / 6.0 * lam + 0.5 * dt * g2
                g1, q1 = model.stage_vjp(u1, Y[0], B[0])
                gpsi = gpsi + q1 + q2 + q3 + q4
                lam = lam + g1 + g2 + g3 + g4
                if p.objective == J_PORT and n >= p.n_from:
                    lam = lam + model.port_term_grad(recorded[n])
    dphi = p.sigmoid_a * model.psi * (1.0 - model.psi) * gpsi
    return J, dphi, lam
