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
