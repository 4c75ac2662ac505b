"""Launch-shape autotuner for the fused update kernel.

Times each candidate (threads per block, cells per thread) on the caller's
own handle with CUDA events and leaves the fastest one set.  Tuning advances
the simulation by the steps it times (they are ordinary steps of the same
problem), so run it during warm-up.
"""
from __future__ import annotations

from . import lbm

CANDIDATES = {
    lbm.LBM_FP64: [(64, 1), (128, 1), (32, 2), (64, 2), (128, 2)],
    lbm.LBM_FP32: [(64, 1), (128, 1), (256, 1), (32, 2), (64, 2), (128, 4)],
    lbm.LBM_FP16_SHIFTED: [(128, 1), (32, 2), (64, 2), (128, 2), (32, 4), (128, 4)],
    lbm.LBM_BF16_SHIFTED: [(128, 1), (32, 2), (64, 2), (128, 2), (32, 4), (128, 4)],
}


def autotune(handle, precision: int, stream, steps: int = 5, torch=None):
    """Time each candidate for `steps` steps on `stream` (a torch.cuda.Stream);
    set the fastest.  Returns (best (block, vec), {candidate: ms per step})."""
    if torch is None:
        import torch
    times = {}
    for block, vec in CANDIDATES[precision]:
        lbm.lbm_set_launch(handle, block, vec)
        if lbm.lbm_get_launch(handle) != (block, vec):
            continue  # shape not applicable (mask present or row length)
        lbm.lbm_step(handle, 1)  # untimed: first launch of this shape
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            lbm.lbm_step(handle, steps)
            e1.record(stream)
        e1.synchronize()
        times[(block, vec)] = e0.elapsed_time(e1) / steps
    if not times:
        lbm.lbm_set_launch(handle, 0, 0)
        return lbm.lbm_get_launch(handle), times
    best = min(times, key=times.get)
    lbm.lbm_set_launch(handle, *best)
    return best, times
