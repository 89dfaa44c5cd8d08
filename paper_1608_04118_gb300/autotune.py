"""Launch-schedule autotuner for the batched form.

Times candidate schedules (tile shape x persistent grid size x nodes per
thread) of a ``Batch`` with CUDA events on its stream and keeps the
fastest.  Candidate grid sizes are multiples of the SM count; 0 means one
block per tile.
"""
from __future__ import annotations

import itertools

# (tile_x, tile_y, nodes per thread): tiles in nodes, tile_x / npt threads across
TILE_SHAPES = ((32, 4, 1), (64, 2, 1), (64, 4, 1), (128, 1, 1), (128, 2, 1), (256, 1, 1),
               (64, 2, 2), (64, 4, 2), (128, 1, 2), (128, 2, 2), (256, 1, 2))
BLOCKS_PER_SM = (2, 4, 8, 16)


def candidates(sm_count):
    for (tx, ty, npt), k in itertools.product(TILE_SHAPES, BLOCKS_PER_SM + (0,)):
        yield tx, ty, (k * sm_count if k else 0), npt


def time_schedule(batch, schedule, steps, warmup=2):
    import torch

    batch.set_schedule(*schedule)
    with torch.cuda.stream(batch.stream):
        batch.step(warmup)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(batch.stream)
        batch.step(steps)
        e1.record(batch.stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / 1e3 / steps


def tune_batch(batch, steps=8, warmup=2):
    """Pick the fastest schedule for ``batch`` (its state is advanced by the
    trial steps; call ``set_fields`` afterwards).  Returns (schedule,
    seconds per step, table of all trials)."""
    import torch

    sm = torch.cuda.get_device_properties(batch.workspace.device).multi_processor_count
    batch.set_fields()
    table = []
    for sch in candidates(sm):
        table.append((sch, time_schedule(batch, sch, steps, warmup)))
    best = min(table, key=lambda r: r[1])
    batch.set_schedule(*best[0])
    return best[0], best[1], table


# Single-lattice step kernel: block shapes (threads per block <= 256) and
# nodes per thread (2 = paired FP32 arithmetic, not for FP64 storage).
CAVITY_SHAPES = ((32, 2), (32, 4), (64, 1), (64, 2), (64, 4), (128, 1), (128, 2), (256, 1))


def cavity_candidates(storage):
    for npt in ((1,) if storage == "f64" else (1, 2)):
        for bx, by in CAVITY_SHAPES:
            if npt == 1 or bx * by <= 128:  # the two-node kernels take <= 128 threads
                yield bx, by, npt


def tune_cavity(cav, steps=20, warmup=4):
    """Pick the fastest step-kernel schedule for ``cav`` (a ``Cavity`` whose
    fields are set; the trial steps advance its state).  Returns (schedule,
    seconds per step, table of all trials)."""
    import torch

    from .ltne import LtneError

    table = []
    for sch in cavity_candidates(cav.storage):
        try:
            cav.set_schedule(*sch)
        except LtneError:  # a form this lattice does not take (e.g. rows without cavity walls)
            continue
        with torch.cuda.stream(cav.stream):
            cav.step(warmup)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(cav.stream)
            cav.step(steps)
            e1.record(cav.stream)
        e1.synchronize()
        table.append((sch, e0.elapsed_time(e1) / 1e3 / steps))
    best = min(table, key=lambda r: r[1])
    cav.set_schedule(*best[0])
    return best[0], best[1], table
