"""The mbarrier protocol of the tensor-core product's two rings, as a host-side model.

k_tc_bool_gemm (csrc/cfpq_tensor.cu) moves each K stage s through a packed ring of PST slots
(filled by TMA loads that the producer issues in order and that land in any order) and an
unpacked ring of UST slots (filled by one of two unpack groups, which take alternate stages,
and read by the MMA thread in stage order, whose commits free the slots asynchronously). Every
wait is a parity wait on an mbarrier. This model replays the kernel's per-stage sequence of
waits, arrivals and copies under random interleavings and random landing order, with the
mbarrier semantics of the PTX ISA (a phase completes when its arrivals are in and its
transaction bytes are counted; a parity wait passes once the phase of that parity has
completed), and checks that every stage reaches the MMA intact and that no run deadlocks.

With the odd packed ring of the tile-skipping E2M1 kind (PST = 5) the groups alternate on each
slot. Without the wait on the other group's previous use of the slot, a parity wait can pass on
the phase two earlier: the planted variant shows it, the kernel's protocol must not.

The dense E2M1 kind (B landed by TMA beside the packed A) runs a shorter protocol, modelled by
run_single_commit: both rings have six slots, one MMA commit per stage frees the stage in both,
and the unpack groups wait only for the stage's loads. A shallower tensor-memory ring breaks it
(planted)."""
import random

import pytest


class Barrier:
    def __init__(self, count):
        self.count, self.phase, self.pending, self.tx = count, 0, count, 0

    def _complete_if_done(self):
        if self.pending == 0 and self.tx == 0:
            self.phase += 1
            self.pending = self.count

    def arrive(self):
        self.pending -= 1
        self._complete_if_done()

    def expect_tx(self, nbytes):  # mbarrier.arrive.expect_tx
        self.tx += nbytes
        self.arrive()

    def complete_tx(self, nbytes):
        self.tx -= nbytes
        self._complete_if_done()

    def passed(self, parity):  # mbarrier.try_wait.parity
        return (self.phase & 1) != parity


def run(seed, pst, ust, stages, fixed, groups=2):
    """One random schedule; returns None or the first violation found."""
    rng = random.Random(seed)
    full_p = [Barrier(1) for _ in range(pst)]
    empty_p = [Barrier(1) for _ in range(pst)]  # one arrival per group (its threads as one)
    full_u = [Barrier(1) for _ in range(ust)]
    empty_u = [Barrier(1) for _ in range(ust)]
    packed = [None] * pst
    unpacked = [None] * ust
    in_flight = []   # issued TMA loads: (slot, stage)
    commits = []     # MMA commits not yet arrived: slot
    prod = {"s": 0}
    grp = [{"s": g, "step": 0} for g in range(groups)]
    mma = {"s": 0}

    def producer():
        s = prod["s"]
        if s >= stages:
            return False
        slot = s % pst
        if not empty_p[slot].passed(((s // pst) & 1) ^ 1):
            return False
        full_p[slot].expect_tx(1)
        in_flight.append((slot, s))
        prod["s"] = s + 1
        return True

    def land():
        if not in_flight:
            return False
        slot, s = in_flight.pop(rng.randrange(len(in_flight)))  # any order
        packed[slot] = s
        full_p[slot].complete_tx(1)
        return True

    def group(g):
        st = grp[g]
        s = st["s"]
        if s >= stages:
            return False
        ps, us = s % pst, s % ust
        if st["step"] == 0:  # the wait that the odd ring needs
            if fixed and pst % groups != 0 and s >= pst and not empty_p[ps].passed(((s // pst) - 1) & 1):
                return False
            st["step"] = 1
            return True
        if st["step"] == 1:
            if not full_p[ps].passed((s // pst) & 1):
                return False
            st["step"] = 2
            return True
        if not empty_u[us].passed(((s // ust) & 1) ^ 1):
            return False
        if packed[ps] != s:
            return f"group {g} read stage {packed[ps]} from packed slot {ps} as stage {s}"
        empty_p[ps].arrive()
        unpacked[us] = s
        full_u[us].arrive()
        st["s"] = s + groups
        st["step"] = 0
        return True

    def mma_thread():
        s = mma["s"]
        if s >= stages:
            return False
        us = s % ust
        if not full_u[us].passed((s // ust) & 1):
            return False
        if unpacked[us] != s:
            return f"MMA read stage {unpacked[us]} from unpacked slot {us} as stage {s}"
        commits.append(us)
        mma["s"] = s + 1
        return True

    def commit():
        if not commits:
            return False
        empty_u[commits.pop(0)].arrive()  # tcgen05.commit arrivals come in issue order
        return True

    actors = [producer, land, mma_thread, commit] + [lambda g=g: group(g) for g in range(groups)]
    while mma["s"] < stages:
        order = list(range(len(actors)))
        rng.shuffle(order)
        moved = False
        for k in order:
            r = actors[k]()
            if isinstance(r, str):
                return r
            if r:
                moved = True
                break
        if not moved:
            return f"deadlock at MMA stage {mma['s']}, producer {prod['s']}, groups {[x['s'] for x in grp]}"
    return None


@pytest.mark.parametrize("pst,ust", [(5, 5), (8, 5), (6, 5), (4, 5), (3, 5), (5, 3)],
                         ids=["odd-5", "e4m3", "e2m1", "even-4", "odd-3", "odd-5-ust-3"])
def test_ring_protocol_is_exact(pst, ust):
    for seed in range(400):
        err = run(seed, pst, ust, stages=70, fixed=True)
        assert err is None, (seed, err)


def test_planted_parity_alias_is_caught():
    """Without the wait on the other group's use of the slot, the odd packed ring of the
    E2M1 kind lets a group pass a full barrier on the phase two earlier."""
    bad = [seed for seed in range(400) if run(seed, 5, 5, stages=70, fixed=False) is not None]
    assert bad, "the model should expose the aliasing of the unfixed protocol"
    assert all(run(seed, 8, 5, stages=70, fixed=False) is None for seed in range(200))  # even ring: no alias


def run_single_commit(seed, pst, ust, stages, groups=2):
    """The dense E2M1 kind's protocol (B landed by TMA in the packed slot beside the packed A):
    one MMA commit per stage on empty_p frees the stage's packed slot and, with ust == pst,
    its tensor-memory A slot; the unpack groups wait only for the stage's loads, and the MMA
    thread only for the unpacked stage (which implies the stage's B). Returns None or the first violation
    (a slot overwritten while an earlier stage's MMAs still read it, a wrong stage read)."""
    rng = random.Random(seed)
    full_p = [Barrier(1) for _ in range(pst)]
    empty_p = [Barrier(1) for _ in range(pst)]  # the MMA commit alone
    full_u = [Barrier(1) for _ in range(ust)]
    packed = [None] * pst     # stage whose A (packed) and B sit in the slot
    unpacked = [None] * ust   # stage whose A sits in the tensor-memory slot
    done = set()              # stages whose MMAs completed
    in_flight, commits = [], []
    prod, mma = {"s": 0}, {"s": 0}
    grp = [{"s": g} for g in range(groups)]

    def producer():
        s = prod["s"]
        if s >= stages or not empty_p[s % pst].passed(((s // pst) & 1) ^ 1):
            return False
        full_p[s % pst].expect_tx(1)
        in_flight.append((s % pst, s))
        prod["s"] = s + 1
        return True

    def land():
        if not in_flight:
            return False
        slot, s = in_flight.pop(rng.randrange(len(in_flight)))
        old = packed[slot]
        if old is not None and old not in done:
            return f"load of stage {s} overwrote packed slot {slot} of stage {old} before its MMAs completed"
        packed[slot] = s
        full_p[slot].complete_tx(1)
        return True

    def group(g):
        s = grp[g]["s"]
        if s >= stages or not full_p[s % pst].passed((s // pst) & 1):
            return False
        if packed[s % pst] != s:
            return f"group {g} read stage {packed[s % pst]} as stage {s}"
        us = s % ust
        old = unpacked[us]
        if old is not None and old not in done:
            return f"group {g} overwrote tensor-memory slot {us} of stage {old} before its MMAs completed"
        unpacked[us] = s
        full_u[us].arrive()
        grp[g]["s"] = s + groups
        return True

    def mma_thread():
        s = mma["s"]
        if s >= stages:
            return False
        # only the unpacked stage's barrier: the unpack group waited for the stage's loads
        # (the B tile lands with the packed A) before arriving on it
        if not full_u[s % ust].passed((s // ust) & 1):
            return False
        if unpacked[s % ust] != s or packed[s % pst] != s:
            return f"MMA of stage {s} read A {unpacked[s % ust]} / B {packed[s % pst]}"
        commits.append(s)
        mma["s"] = s + 1
        return True

    def commit():
        if not commits:
            return False
        s = commits.pop(0)
        done.add(s)
        empty_p[s % pst].arrive()
        return True

    actors = [producer, land, mma_thread, commit] + [lambda g=g: group(g) for g in range(groups)]
    while mma["s"] < stages or commits:
        order = list(range(len(actors)))
        rng.shuffle(order)
        moved = False
        for k in order:
            r = actors[k]()
            if isinstance(r, str):
                return r
            if r:
                moved = True
                break
        if not moved:
            return f"deadlock at MMA stage {mma['s']}"
    return None


def test_single_commit_protocol_is_exact():
    for seed in range(400):
        err = run_single_commit(seed, 6, 6, stages=70)
        assert err is None, (seed, err)


def test_single_commit_needs_equal_ring_depths():
    """With a tensor-memory ring shallower than the packed ring, a stage's loads landing no
    longer means its tensor-memory slot is free: the model must catch the overwrite."""
    bad = [seed for seed in range(300) if run_single_commit(seed, 6, 5, stages=70) is not None]
    assert bad
