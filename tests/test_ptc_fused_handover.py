"""The buffer hand-over of the persistent fused network kernel, modelled on
the host: producers (transports) and consumers (tensor-core GEMMs) of one
block walk the same tiles t = b, b + G, ... and pass two shared-memory
buffers through hardware named barriers: producers arrive on FULL[it & 1]
after filling a buffer, consumers sync on it; consumers arrive on
EMPTY[it & 1] once GEMM1 has read the buffer, only when the block has a tile
two iterations later, and producers sync on EMPTY before refilling a buffer
from their third iteration on.  A barrier completes when both groups have
reached it.  Under random interleavings and for many tile counts and grid
sizes the model never deadlocks, every tile is read once and in order, no
buffer is refilled before it has been read, and no arrival is left pending
when the block exits (which a stray bar.arrive would do)."""
import random

import pytest


def role_ops(role, block, grid, ntiles):
    ops, it, t = [], 0, block
    while t < ntiles:
        buf = it & 1
        if role == "producer":
            if it >= 2:
                ops.append(("sync", "EMPTY", buf))
            ops.append(("write", buf, t))
            ops.append(("arrive", "FULL", buf))
        else:
            ops.append(("sync", "FULL", buf))
            ops.append(("read", buf, t))
            if t + 2 * grid < ntiles:
                ops.append(("arrive", "EMPTY", buf))
        t += grid
        it += 1
    return ops


def run_block(block, grid, ntiles, seed, ops=role_ops):
    rng = random.Random(seed)
    seq = {r: ops(r, block, grid, ntiles) for r in ("producer", "consumer")}
    pc = dict.fromkeys(seq, 0)
    waiting = dict.fromkeys(seq)
    arrived = {}      # (barrier, buffer) -> groups arrived in the current phase
    buffers = {0: None, 1: None}
    reads = []
    for _ in range(100000):
        movable = [r for r in seq if waiting[r] is None and pc[r] < len(seq[r])]
        if not movable:
            break
        role = rng.choice(movable)
        op = seq[role][pc[role]]
        pc[role] += 1
        if op[0] == "write":
            assert buffers[op[1]] is None or buffers[op[1]][1], "buffer refilled before it was read"
            buffers[op[1]] = (op[2], False)
        elif op[0] == "read":
            assert buffers[op[1]] == (op[2], False), "consumer read a stale or wrong tile"
            buffers[op[1]] = (op[2], True)
            reads.append(op[2])
        else:
            key = (op[1], op[2])
            arrived[key] = arrived.get(key, 0) + 1
            if op[0] == "sync":
                waiting[role] = key
            if arrived[key] == 2:   # both groups: the barrier completes and resets
                arrived[key] = 0
                for r in seq:
                    if waiting[r] == key:
                        waiting[r] = None
    assert all(pc[r] == len(seq[r]) and waiting[r] is None for r in seq), "deadlock"
    assert not any(arrived.values()), "an arrival is left pending at exit"
    assert reads == list(range(block, ntiles, grid))


@pytest.mark.parametrize("grid", [1, 2, 3, 7, 152])
def test_handover_never_deadlocks_and_reads_every_tile_once(grid):
    for ntiles in range(1, 3 * grid + 9):
        if ntiles < grid:
            continue
        for block in sorted({0, 1, grid // 2, grid - 1}):
            for seed in range(12):
                run_block(block, grid, ntiles, seed)


def test_the_model_catches_a_missing_wait():
    """Planted mistake: producers that never wait on EMPTY refill a buffer
    the consumers have not read yet."""
    def careless(role, block, grid, ntiles):
        return [op for op in role_ops(role, block, grid, ntiles) if op[:2] != ("sync", "EMPTY")]

    caught = 0
    for seed in range(50):
        try:
            run_block(0, 1, 6, seed, ops=careless)
        except AssertionError:
            caught += 1
    assert caught > 0
