"""Which warp counts a derived pair as new on the worklist path (csrc/cfpq_worklist.cu), as a
host-side model.

A pair (x, a, b) of a derived non-terminal x has two bits: bit b of row a of T_x and bit a of
row b of T_x^T, which the worklist keeps for every derived non-terminal. Three kinds of
update can set the same pair at the same time from different warps:
  wl_set and the left-operand join: atomic OR into T_x (the pair is new where the bit was
  clear), then into T_x^T;
  the right-operand join: a word-wide atomic OR into T_x^T; for the bits that were clear
  there, an atomic OR into T_x, and the pair is new where that bit of T_x was clear.
Every warp that counts a pair as new also pushes it on the stack, so exactly one warp may
count it, whatever the interleaving of the atomics. The model enumerates every interleaving
of up to four such updates (each a sequence of atomic steps on the two bits) and checks
that. A planted mistake (the right-operand join deciding on T_x^T alone, as it once did)
must be caught."""
import itertools

import pytest


def set_first(state):
    """wl_set or the left join: T, then T^T."""
    old = state["T"]
    state["T"] = 1
    new = old == 0
    yield new
    state["TT"] = 1


def right_join(state):
    """The right-operand join: T^T word-wide, then T for the bits that were clear in T^T."""
    old_tt = state["TT"]
    state["TT"] = 1
    if old_tt:
        return  # another update set it first: that one decides
    yield None
    old = state["T"]
    state["T"] = 1
    yield old == 0


def right_join_planted(state):
    """The planted mistake: new where the bit of T^T was clear; T set after."""
    old_tt = state["TT"]
    state["TT"] = 1
    yield old_tt == 0
    state["T"] = 1


def run(kinds, order):
    """Runs the updates' steps in the given order of update indices; returns the number of
    updates that counted the pair as new, and the final bits."""
    state = {"T": 0, "TT": 0}
    gens = [k(state) for k in kinds]
    done = [False] * len(kinds)
    counted = 0
    for i in order:
        if done[i]:
            continue
        try:
            r = next(gens[i])
            if r:
                counted += 1
        except StopIteration:
            done[i] = True
    for i, g in enumerate(gens):  # finish whatever is left, in index order
        while not done[i]:
            try:
                if next(g):
                    counted += 1
            except StopIteration:
                done[i] = True
    return counted, state


def interleavings(n_updates, steps=3):
    """Every order in which n updates take up to `steps` atomic steps each."""
    seq = [i for i in range(n_updates) for _ in range(steps)]
    return set(itertools.permutations(seq))


MIXES = [
    (set_first, right_join),
    (right_join, right_join),
    (set_first, set_first),
    (set_first, right_join, right_join),
    (right_join, set_first, right_join, set_first),
]


@pytest.mark.parametrize("kinds", MIXES, ids=lambda ks: "+".join(k.__name__ for k in ks))
def test_exactly_one_update_counts_the_pair(kinds):
    orders = interleavings(len(kinds), steps=3 if len(kinds) <= 3 else 2)
    for order in orders:
        counted, state = run(kinds, order)
        assert counted == 1, (order, counted)
        assert state == {"T": 1, "TT": 1}


def test_planted_decision_on_the_transpose_is_caught():
    """Deciding on T^T lets a right join and a concurrent wl_set both count the pair."""
    kinds = (set_first, right_join_planted)
    bad = [o for o in interleavings(2) if run(kinds, o)[0] != 1]
    assert bad, "the model should expose the double count"
