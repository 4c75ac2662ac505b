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


# ---------------------------------------------------------------------------
# Serving engine: launch shape of each (lattice, precision) group's batched
# update, (cells per lane, warps per block)
# ---------------------------------------------------------------------------
SERVER_CANDIDATES = [(1, 2), (1, 4), (1, 8), (2, 2), (2, 4), (2, 8)]


def tune_server(kinds, sizes, aa: bool = False, round_steps: int = 20, rounds: int = 3,
                budget_bytes: int = 8 << 30):
    """Pick the batched update's launch shape per (lattice, precision) group.

    kinds: (lattice, precision) pairs; sizes: {lattice: [extents, ...]}, one
    request of each extents per group, the batch the group is timed on (at
    rest; the update's cost does not depend on the state).  Each candidate
    runs one warm round and then `rounds` rounds of `round_steps` steps on a
    temporary server; the rate is cell updates over the device time of those
    rounds' graphs.  Returns {(lattice, precision): {"cells_per_lane",
    "warps_per_block", "mlups", "table"}}."""
    out = {}
    for lat, prec in kinds:
        s = lbm.lbm_server_create(budget_bytes, 256, None)
        try:
            if aa:
                lbm.lbm_server_set_streaming(s, lbm.LBM_STREAM_AA)
            cells = 0
            for ext in sizes[lat]:
                lbm.lbm_server_submit(s, lat, prec, ext, 0.6, 1 << 40)
                cells += int(ext[0]) * int(ext[1]) * int(ext[2])
            table = {}
            for v, w in SERVER_CANDIDATES:
                lbm.lbm_server_set_launch(s, lat, prec, v, w)
                lbm.lbm_server_run(s, round_steps)
                t0 = lbm.lbm_server_gpu_time(s)
                for _ in range(rounds):
                    lbm.lbm_server_run(s, round_steps)
                ms = lbm.lbm_server_gpu_time(s) - t0
                table[f"{v}x{w}"] = cells * round_steps * rounds / (ms / 1e3) / 1e6
            best = max(table, key=table.get)
            v, w = (int(t) for t in best.split("x"))
            out[(lat, prec)] = {"cells_per_lane": v, "warps_per_block": w, "mlups": table[best], "table": table}
        finally:
            lbm.lbm_server_destroy(s)
    return out
