"""Launch autotuner for the fused update kernel.

Times each candidate kernel and launch shape on the caller's own handle with
CUDA events and leaves the fastest one set.  Candidates are the row-staged
kernel with a number of shared-memory stages ("rows", stages) and the
register kernels with a block size ("cell" one cell per thread, "vec2" /
"vec4" that many x cells per thread).  Tuning advances the simulation by the
steps it times (ordinary steps of the same problem), so run it during warm-up.
"""
from __future__ import annotations

from . import lbm

CANDIDATES = {
    lbm.LBM_FP64: [("cell", 64), ("cell", 128), ("vec2", 32), ("vec2", 64), ("vec2", 128)],
    lbm.LBM_FP32: [("rows", 2), ("rows", 3), ("rows", 4), ("cell", 64), ("cell", 128), ("vec2", 64)],
    lbm.LBM_FP16_SHIFTED: [("rows", 2), ("rows", 3), ("rows", 4), ("vec2", 32), ("vec2", 64), ("vec4", 32)],
    lbm.LBM_BF16_SHIFTED: [("rows", 2), ("rows", 3), ("rows", 4), ("vec2", 32), ("vec2", 64), ("vec4", 32)],
}


def name(cand) -> str:
    kind, knob = cand
    return f"rows s{knob}" if kind == "rows" else f"{kind} b{knob}"


def apply(handle, cand) -> bool:
    """Select a candidate; False when it does not apply to this lattice."""
    kind, knob = cand
    if kind == "rows":
        lbm.lbm_set_staging(handle, 1, knob, 0)
        return lbm.lbm_get_staging(handle)[0] == 1
    lbm.lbm_set_staging(handle, 0, 0, 0)
    vec = 1 if kind == "cell" else int(kind[3:])
    lbm.lbm_set_launch(handle, knob, vec)
    return lbm.lbm_get_launch(handle) == (knob, vec)


def describe(handle) -> dict:
    """The kernel and launch shape lbm_step uses now."""
    active, stages, block, rows, grid = lbm.lbm_get_staging(handle)
    if active:
        return {"kernel": "rows", "stages": stages, "block": block, "rows_per_tile": rows, "grid": grid}
    block, vec = lbm.lbm_get_launch(handle)
    return {"kernel": "cell" if vec == 1 else f"vec{vec}", "block": block, "cells_per_thread": vec}


def autotune(handle, precision: int, stream, steps: int = 5, torch=None):
    """Time each applicable candidate for `steps` steps on `stream` (a
    torch.cuda.Stream); set the fastest.  Returns (best candidate name,
    {candidate name: ms per step})."""
    if torch is None:
        import torch
    times, cands = {}, {}
    for cand in CANDIDATES[precision]:
        if not apply(handle, cand):
            continue
        lbm.lbm_step(handle, 1)  # untimed: first launch of this shape
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            lbm.lbm_step(handle, steps)
            e1.record(stream)
        e1.synchronize()
        times[name(cand)] = e0.elapsed_time(e1) / steps
        cands[name(cand)] = cand
    if not times:
        lbm.lbm_set_staging(handle, -1, 0, 0)
        lbm.lbm_set_launch(handle, 0, 0)
        return None, times
    best = min(times, key=times.get)
    apply(handle, cands[best])
    return best, times
