"""Invariants of the oracle's checkpoint schedules (integer artefacts)."""
import pytest

from oracle import schedule as S


@pytest.mark.parametrize("N,seg", [(1, 0), (2, 0), (17, 0), (100, 0), (101, 0), (20000, 0),
                                   (50, 7), (50, 50), (50, 80), (9, 1)])
def test_periodic_invariants(N, seg):
    fwd, rev = S.periodic(N, seg)
    K = seg if seg > 0 else S.default_segment(N)
    # forward advances every step exactly once, in order
    n = 0
    for op, a, b in fwd:
        if op in (S.ADVANCE, S.RECORD):
            assert a == n and b > a
            n = b
        elif op == S.SNAP:
            assert a == n and a == b * K
    assert n == N
    # reverse visits each step exactly once, from N-1 down to 0, over
    # freshly recorded data
    recorded = None
    for op, a, b in fwd:
        if op == S.RECORD:
            recorded = (a, b)
    top = N
    snaps = {b: a for op, a, b in fwd if op == S.SNAP}
    pos = None
    for op, a, b in rev:
        if op == S.RESTORE:
            assert snaps[a] == b
            pos = b
        elif op == S.RECORD:
            assert pos == a
            recorded = (a, b)
            pos = b
        elif op == S.REVERSE:
            assert (b, a) == recorded and a == top
            top = b
    assert top == 0
    slots, rec = S.peak_states(fwd, rev)
    assert slots == (N + K - 1) // K - 1
    assert rec == min(K, N)


def test_sqrt_memory():
    for N in (100, 5000, 20000, 50000):
        fwd, rev = S.periodic(N)
        slots, rec = S.peak_states(fwd, rev)
        assert slots + rec <= 2 * int(N ** 0.5) + 2


def test_default_segment():
    assert [S.default_segment(n) for n in (1, 2, 4, 5, 9, 10, 10000, 10001)] == [1, 2, 2, 3, 3, 4, 100, 101]


def test_store_all():
    fwd, rev = S.store_all(3)
    assert fwd == [(S.SNAP, 0, 0), (S.ADVANCE, 0, 1), (S.SNAP, 1, 1), (S.ADVANCE, 1, 2), (S.RECORD, 2, 3)]
    assert rev == [(S.REVERSE, 3, 2), (S.RESTORE, 1, 1), (S.RECORD, 1, 2), (S.REVERSE, 2, 1),
                   (S.RESTORE, 0, 0), (S.RECORD, 0, 1), (S.REVERSE, 1, 0)]
    assert S.store_all(0) == ([], [])


def test_beta_is_the_binomial_coefficient():
    import math
    for s in range(0, 12):
        for r in range(0, 12):
            assert S.beta(s, r) == math.comb(s + r, s)
    assert S.beta(300, 300) == 1 << 62          # saturates instead of growing without bound


def _replay(fwd, rev, N):
    """Checks a schedule action by action; returns (slots used, evaluations
    per step)."""
    evals = [0] * N
    slot_step = {}
    pos = 0                      # step held by the working state, None if unknown
    n = 0
    for op, a, b in fwd:
        if op == S.SNAP:
            assert a == pos
            slot_step[b] = a
        else:
            assert op in (S.ADVANCE, S.RECORD) and a == pos == n and b > a
            for k in range(a, b):
                evals[k] += 1
            n = pos = b
    assert n == N and fwd[-1][0] == S.RECORD
    recorded = (fwd[-1][1], fwd[-1][2])
    pos = None
    top = N
    for op, a, b in rev:
        if op == S.SNAP:
            assert a == pos
            slot_step[b] = a
        elif op == S.RESTORE:
            assert slot_step[a] == b
            pos = b
        elif op == S.ADVANCE:
            assert a == pos and b > a
            for k in range(a, b):
                evals[k] += 1
            pos = b
        elif op == S.RECORD:
            assert a == pos and b > a
            for k in range(a, b):
                evals[k] += 1
            recorded = (a, b)
            pos = None
        else:
            assert op == S.REVERSE and (b, a) == recorded and a == top
            top = b
            pos = None
    assert top == 0
    return len(slot_step), evals


@pytest.mark.parametrize("N,snaps", [(1, 0), (2, 0), (3, 1), (10, 0), (10, 2), (17, 3), (100, 0), (100, 1),
                                     (1000, 10), (10000, 0), (5000, 64)])
def test_binomial_invariants(N, snaps):
    fwd, rev = S.binomial(N, snaps)
    s = snaps if snaps > 0 else S.default_segment(N)
    used, evals = _replay(fwd, rev, N)
    slots, rec = S.peak_states(fwd, rev)
    assert used <= s + 1 and slots <= s + 1 and rec == 1
    # every step is advanced at most r times plus its one recording, where r
    # is the smallest repetition number with beta(s, r) >= N
    r = 0
    while S.beta(s, r) < N:
        r += 1
    assert max(evals) <= r + 1 and min(evals) >= 1


def test_binomial_small_case_by_hand():
    # N = 3 with one free slot: r = 2 (beta(1, 1) = 2 < 3 <= beta(1, 2) = 3),
    # right part min(beta(0, 2), 2) = 1 step: snapshot at step 2
    fwd, rev = S.binomial(3, 1)
    assert fwd == [(S.SNAP, 0, 0), (S.ADVANCE, 0, 2), (S.SNAP, 2, 1), (S.RECORD, 2, 3)]
    assert rev == [(S.REVERSE, 3, 2),
                   (S.RESTORE, 0, 0), (S.ADVANCE, 0, 1), (S.SNAP, 1, 1), (S.RECORD, 1, 2), (S.REVERSE, 2, 1),
                   (S.RESTORE, 0, 0), (S.RECORD, 0, 1), (S.REVERSE, 1, 0)]
