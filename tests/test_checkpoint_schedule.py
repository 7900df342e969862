"""The binomial checkpoint schedule of the adjoint (Sec. 2.5, Eq. checkpointing).

``binomial_schedule(n, s)`` is run on a stand-in state machine (the position
along the trajectory): every step is recorded exactly once, at its own position,
its adjoint follows immediately, in reverse order n-1 .. 0; at most s states are
stored besides the initial one; and the plain forward steps add up to the least
possible number, computed here by brute force over all split points (and equal to
Griewank's binomial closed form ``binomial_cost``).
"""
from functools import lru_cache

import pytest

from paper_2603_15920_b300.difvm import binomial_cost, binomial_schedule


@lru_cache(None)
def _brute(n, s):
    """Fewest plain steps to reverse n steps from a stored start with s free slots."""
    if n <= 1:
        return 0
    if s == 0:
        return n * (n - 1) // 2         # re-run from the start for every step
    return min(k + _brute(n - k, s - 1) + _brute(k, s) for k in range(1, n))


def _run(acts, n):
    pos, slots, live_max, adv = None, {0: 0}, 1, 0
    reversed_steps, last_record = [], None
    for a in acts:
        if a[0] == "load":
            pos = slots[a[1]]
        elif a[0] == "advance":
            pos += a[1]
            adv += a[1]
        elif a[0] == "save":
            assert a[1] not in slots
            slots[a[1]] = pos
            live_max = max(live_max, len(slots))
        elif a[0] == "free":
            del slots[a[1]]
        elif a[0] == "record":
            assert pos == a[1], (pos, a)
            last_record, pos = a[1], None
        elif a[0] == "bwd":
            assert last_record == a[1]
            reversed_steps.append(a[1])
            last_record = None
    return reversed_steps, live_max, adv


@pytest.mark.parametrize("s", [0, 1, 2, 3, 5])
def test_binomial_schedule_reverses_every_step_with_least_recomputation(s):
    for n in range(1, 46):
        steps, live, adv = _run(binomial_schedule(n, s), n)
        assert steps == list(range(n - 1, -1, -1))
        assert live <= s + 1
        assert adv == _brute(n, s) == binomial_cost(n, s), (n, s, adv, _brute(n, s))


def test_binomial_cost_closed_form_values():
    # c = s + 1 checkpoints reverse beta(c, r) = C(c + r, c) steps with r sweeps;
    # cost r n - beta(c + 1, r - 1)
    assert binomial_cost(28, 5) == 2 * 28 - 8           # n = beta(6, 2): r = 2
    assert binomial_cost(56, 5) == 3 * 56 - 36          # beta(6, 2) < 56 <= beta(6, 3): r = 3
    assert binomial_cost(1000, 9) == 4 * 1000 - 364     # beta(10, 3) = 286 < 1000 <= beta(10, 4) = 1001
    assert binomial_cost(1000, 9) < 4 * 1000            # ten states reverse 1000 steps in < 4 sweeps
