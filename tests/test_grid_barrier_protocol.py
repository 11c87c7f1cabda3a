"""The grid barrier of the persistent gather loop (k_gather_loop, csrc/cfpq_api.cu; grid_sync
and grid_sync_start, csrc/cfpq_device.cuh), as a host-side model.

Every block of a launch reads the solve's arrival counter once at its start and takes the
next multiple of the grid size as its first target; at each barrier it adds one and waits
until the counter reaches the target, then moves the target on by the grid size. The counter
is never reset, across the barriers of a launch nor across the launches of a solve. The model
replays launches of G blocks, each block a sequence of phases and barriers, under random
interleavings and random block start times (a block may start after others have already
arrived at the first barrier), and checks that no block leaves barrier k before every block
has arrived at it, that every launch finishes, and that the counter ends each launch at a
multiple of G. A planted mistake (the target taken as the counter read plus G, without
rounding down) must be caught."""
import random

import pytest


def run_launches(seed, grid, barriers, launches, round_down=True):
    """Returns None, or the first violation."""
    rng = random.Random(seed)
    counter = 0
    for launch in range(launches):
        started = [False] * grid
        target = [0] * grid
        arrived = [0] * grid      # barriers this block has arrived at
        passed = [0] * grid       # barriers this block has left
        waiting = [False] * grid  # arrived at barrier passed[b] + 1, not yet left
        done = [False] * grid
        steps = 0
        while not all(done):
            steps += 1
            if steps > 100000:
                return f"launch {launch}: no progress (arrived {arrived}, passed {passed})"
            b = rng.randrange(grid)
            if done[b]:
                continue
            if not started[b]:
                c = counter
                target[b] = (c - c % grid + grid) if round_down else (c + grid)
                started[b] = True
                continue
            if waiting[b]:
                if counter >= target[b]:
                    k = passed[b] + 1
                    # every block must have arrived at barrier k
                    if any(arrived[o] < k for o in range(grid)):
                        return f"launch {launch}: block {b} left barrier {k} early (arrived {arrived})"
                    passed[b] = k
                    waiting[b] = False
                    target[b] += grid
                    if passed[b] == barriers:
                        done[b] = True
                continue
            # a phase of work, then the arrival at the next barrier
            if rng.random() < 0.5:
                continue
            arrived[b] += 1
            counter += 1
            waiting[b] = True
        if counter % grid != 0:
            return f"launch {launch}: counter {counter} not a multiple of {grid}"
    return None


@pytest.mark.parametrize("grid", [1, 2, 3, 7, 16])
def test_barrier_protocol_is_exact(grid):
    for seed in range(300):
        err = run_launches(seed, grid, barriers=5, launches=4)
        assert err is None, (grid, seed, err)


def test_planted_target_without_rounding_is_caught():
    """Taking the target as the count read plus the grid size lets a block that starts after
    others have arrived wait for one barrier too many, or one that starts first leave early."""
    bad = [seed for seed in range(300) if run_launches(seed, 4, barriers=3, launches=3, round_down=False)]
    assert bad, "the model should expose the unrounded target"
