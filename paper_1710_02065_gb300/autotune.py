"""Launch autotuner for the fused update kernel.

Times each candidate kernel, launch shape and streaming pattern on the
caller's own handle with CUDA events and leaves the fastest one set.
Candidates are the row-staged kernel with a number of shared-memory stages
("rows", stages), the register kernels with a block size ("cell" one cell per
thread, "vec2" / "vec4" that many x cells per thread) on the two-lattice pull
pattern, and the same register kernels on the in-place AA pattern ("aa-cell",
"aa-vec2", "aa-vec4"; one lattice, half the memory).  Tuning advances the
simulation by the steps it times (ordinary steps of the same problem), so run
it during warm-up; switching the pattern keeps the state.
"""
from __future__ import annotations

from . import lbm

CANDIDATES = {
    lbm.LBM_FP64: [("cell", 64), ("cell", 128), ("vec2", 32), ("vec2", 64), ("vec2", 128),
                   ("aa-cell", 128), ("aa-vec2", 64)],
    lbm.LBM_FP32: [("rows", 2), ("rows", 3), ("rows", 4), ("cell", 64), ("cell", 128), ("vec2", 64),
                   ("aa-cell", 128), ("aa-vec2", 64)],
    lbm.LBM_FP16_SHIFTED: [("rows", 2), ("rows", 3), ("rows", 4), ("vec2", 32), ("vec2", 64), ("vec4", 32),
                           ("aa-vec2", 32), ("aa-vec2", 64), ("aa-vec4", 32)],
    lbm.LBM_BF16_SHIFTED: [("rows", 2), ("rows", 3), ("rows", 4), ("vec2", 32), ("vec2", 64), ("vec4", 32),
                           ("aa-vec2", 32), ("aa-vec2", 64), ("aa-vec4", 32)],
}


def name(cand) -> str:
    kind, knob = cand
    return f"rows s{knob}" if kind == "rows" else f"{kind} b{knob}"


def apply(handle, cand) -> bool:
    """Select a candidate; False when it does not apply to this lattice."""
    kind, knob = cand
    aa = kind.startswith("aa-")
    try:
        lbm.lbm_set_streaming(handle, lbm.LBM_STREAM_AA if aa else lbm.LBM_STREAM_PULL)
    except lbm.LBMError:
        return False
    if aa:
        kind = kind[3:]
    if kind == "rows":
        lbm.lbm_set_staging(handle, 1, knob, 0)
        return lbm.lbm_get_staging(handle)[0] == 1
    lbm.lbm_set_staging(handle, 0, 0, 0)
    vec = 1 if kind == "cell" else int(kind[3:])
    lbm.lbm_set_launch(handle, knob, vec)
    return lbm.lbm_get_launch(handle) == (knob, vec)


def describe(handle) -> dict:
    """The kernel, launch shape and streaming pattern lbm_step uses now."""
    streaming = "aa" if lbm.lbm_get_streaming(handle) == lbm.LBM_STREAM_AA else "pull"
    active, stages, block, rows, grid = lbm.lbm_get_staging(handle)
    if active:
        return {"kernel": "rows", "streaming": streaming, "stages": stages, "block": block, "rows_per_tile": rows,
                "grid": grid}
    block, vec = lbm.lbm_get_launch(handle)
    return {"kernel": "cell" if vec == 1 else f"vec{vec}", "streaming": streaming, "block": block,
            "cells_per_thread": vec}


def autotune(handle, precision: int, stream, steps: int = 6, torch=None):
    """Time each applicable candidate for `steps` steps (even: the AA pattern
    alternates two step types) on `stream` (a torch.cuda.Stream); set the
    fastest.  Returns (best candidate name, {candidate name: ms per step})."""
    if torch is None:
        import torch
    steps += steps % 2
    times, cands = {}, {}
    for cand in CANDIDATES[precision]:
        if not apply(handle, cand):
            continue
        lbm.lbm_step(handle, 2)  # untimed: first launches of this shape
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
        lbm.lbm_set_streaming(handle, lbm.LBM_STREAM_PULL)
        lbm.lbm_set_staging(handle, -1, 0, 0)
        lbm.lbm_set_launch(handle, 0, 0)
        return None, times
    best = min(times, key=times.get)
    apply(handle, cands[best])
    return best, times
