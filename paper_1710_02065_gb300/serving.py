"""Continuous-batching driver of the solve server (lbm_server_* in include/lbm.h).

Requests arrive in real time (their `arrival` offsets, seconds); every round
submits what has arrived, lets the server admit by HBM budget and advance all
admitted requests together, and collects what finished.  Reports aggregate
MLUPS and time-to-solution percentiles (arrival to result on the host).

The request payloads (initial rho, u) are the clients' data: a client thread
synthesises each one ahead of its arrival (at most `lookahead_s` early and
`max_ready` payloads held), the way a client holds its data before it
submits, so that payload synthesis on the host does not stall the server
loop.  A payload that is not ready at its arrival time is submitted when it
is, and the wait counts in that request's time to solution.
"""
from __future__ import annotations

import threading
import time

import numpy as np

from . import inputs, lbm


class Server:
    def __init__(self, hbm_budget_bytes: int, max_slots: int = 256, stream: int | None = None, aa: bool = False,
                 launch: dict | None = None):
        """launch: {(lattice, precision): (cells_per_lane, warps_per_block)}"""
        self.s = lbm.lbm_server_create(hbm_budget_bytes, max_slots, stream)
        if aa:
            lbm.lbm_server_set_streaming(self.s, lbm.LBM_STREAM_AA)
        for (lat, prec), (v, w) in (launch or {}).items():
            lbm.lbm_server_set_launch(self.s, lat, prec, v, w)

    def close(self):
        if self.s:
            lbm.lbm_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, req: dict, rho=None, u=None) -> int:
        return lbm.lbm_server_submit(self.s, req["lattice"], req["precision"], req["extents"], req["tau"],
                                     req["steps"], rho, u)

    def run(self, steps: int) -> int:
        return lbm.lbm_server_run(self.s, steps)

    def poll(self, rid: int):
        return lbm.lbm_server_poll(self.s, rid)

    def result(self, rid: int, ncell: int):
        rho = np.zeros(ncell)
        u = np.zeros((ncell, 3))
        rc = lbm.lbm_server_result(self.s, rid, rho, u)
        return rho, u, rc

    def stats(self):
        return lbm.lbm_server_stats(self.s)


class _Client(threading.Thread):
    """Synthesises request payloads in arrival order, ahead of arrival."""

    def __init__(self, pending, t0: float, lookahead_s: float, max_ready: int):
        super().__init__(daemon=True)
        self.pending, self.t0, self.lookahead, self.max_ready = pending, t0, lookahead_s, max_ready
        self.ready = {}  # index -> (rho, u)
        self.cv = threading.Condition()
        self.stop = False

    def run(self):
        for k, req in enumerate(self.pending):
            with self.cv:
                while not self.stop and len(self.ready) >= self.max_ready:
                    self.cv.wait(0.05)
                if self.stop:
                    return
            wait = req["arrival"] - self.lookahead - (time.perf_counter() - self.t0)
            if wait > 0:
                with self.cv:
                    if self.cv.wait_for(lambda: self.stop, timeout=wait):
                        return
            payload = inputs.request_initial_state(req)
            with self.cv:
                self.ready[k] = payload
                self.cv.notify_all()

    def take(self, k: int):
        with self.cv:
            p = self.ready.pop(k, None)
            if p is not None:
                self.cv.notify_all()
            return p


_Q = {lbm.LBM_D2Q9: 9, lbm.LBM_D3Q19: 19, lbm.LBM_D3Q27: 27}
_BYTES = {lbm.LBM_FP64: 8, lbm.LBM_FP32: 4, lbm.LBM_FP16_SHIFTED: 2, lbm.LBM_BF16_SHIFTED: 2}


def algorithmic_bytes(req) -> int:
    """Populations read and written by a request's updates: 2 Q s per cell update."""
    return 2 * _Q[req["lattice"]] * _BYTES[req["precision"]] * int(np.prod(req["extents"])) * int(req["steps"])


_NAMES = {lbm.LBM_D2Q9: "D2Q9", lbm.LBM_D3Q19: "D3Q19", lbm.LBM_D3Q27: "D3Q27"}
_PREC = {lbm.LBM_FP64: "fp64", lbm.LBM_FP32: "fp32", lbm.LBM_FP16_SHIFTED: "fp16", lbm.LBM_BF16_SHIFTED: "bf16"}


def tune_for(requests, aa: bool = False, budget_bytes: int = 8 << 30):
    """Launch shapes for the groups of a request stream (autotune.tune_server
    on one request of each extents the stream holds, per lattice, capped at
    half the budget per group)."""
    from . import autotune
    kinds = sorted({(r["lattice"], r["precision"]) for r in requests})
    sizes = {}
    for r in requests:
        sizes.setdefault(r["lattice"], set()).add(tuple(r["extents"]))
    sizes = {k: sorted(v, key=lambda e: e[0] * e[1] * e[2]) for k, v in sizes.items()}
    picked = {}
    for lat, prec in kinds:
        keep, total = [], 0
        for e in sizes[lat]:
            b = (1 if aa else 2) * _Q[lat] * _BYTES[prec] * e[0] * e[1] * e[2]
            if total + b <= budget_bytes // 2:
                keep.append(e)
                total += b
        picked.update(autotune.tune_server([(lat, prec)], {lat: keep}, aa=aa, budget_bytes=budget_bytes))
    return picked


def serve(requests, hbm_budget_bytes: int = 8 << 30, max_slots: int = 256, steps_per_round: int = 100,
          keep_results: bool = False, lookahead_s: float = 2.0, max_ready: int = 16, aa: bool = False,
          tune: bool = False):
    """Run a request stream to completion; returns a summary dict (and results).
    aa: serve with the in-place AA pattern (one lattice per request).
    tune: pick each group's launch shape first (tune_for; not timed)."""
    tuned = tune_for(requests, aa, hbm_budget_bytes) if tune else {}
    srv = Server(hbm_budget_bytes, max_slots, aa=aa,
                 launch={k: (t["cells_per_lane"], t["warps_per_block"]) for k, t in tuned.items()})
    launch = {}
    for lat, prec in sorted({(r["lattice"], r["precision"]) for r in requests}):
        v, w = lbm.lbm_server_get_launch(srv.s, lat, prec)
        launch[f"{_NAMES[lat]}/{_PREC[prec]}"] = {"cells_per_lane": v, "warps_per_block": w}
        if (lat, prec) in tuned:
            launch[f"{_NAMES[lat]}/{_PREC[prec]}"]["tuned_mlups"] = {
                k: round(x) for k, x in tuned[(lat, prec)]["table"].items()}
    max_running = 0
    pending = sorted(requests, key=lambda r: r["arrival"])
    inflight = {}  # id -> (request, arrival wall time)
    tts, results, failed = [], {}, 0
    t0 = time.perf_counter()
    client = _Client(pending, t0, lookahead_s, max_ready)
    client.start()
    i = 0
    try:
        while i < len(pending) or inflight:
            now = time.perf_counter() - t0
            while i < len(pending) and pending[i]["arrival"] <= now:
                payload = client.take(i)
                if payload is None:
                    break  # not synthesised yet: submitted in a later round
                req = pending[i]
                rid = srv.submit(req, *payload)
                inflight[rid] = (req, t0 + req["arrival"], i)
                i += 1
            if not inflight:
                dt = pending[i]["arrival"] - (time.perf_counter() - t0)
                with client.cv:
                    client.cv.wait(0.05 if dt <= 0 else min(0.05, dt))
                continue
            srv.run(steps_per_round)
            max_running = max(max_running, srv.stats()["running"])
            for rid in list(inflight):
                state, _ = srv.poll(rid)
                if state in (lbm.LBM_REQ_DONE, lbm.LBM_REQ_FAILED):
                    req, t_arr, k = inflight.pop(rid)
                    ncell = int(np.prod(req["extents"]))
                    rho, u, rc = srv.result(rid, ncell)
                    tts.append(time.perf_counter() - t_arr)
                    failed += rc != lbm.LBM_OK
                    if keep_results:
                        results[k] = (rho, u)
    finally:
        with client.cv:
            client.stop = True
            client.cv.notify_all()
        client.join()
    wall = time.perf_counter() - t0
    cells = srv.stats()["cell_updates"]
    gpu_s = lbm.lbm_server_gpu_time(srv.s) / 1e3
    srv.close()
    moved = sum(algorithmic_bytes(r) for r in requests)
    tts = np.array(tts)
    out = {
        "requests": len(requests), "failed": int(failed), "wall_s": wall,
        "aggregate_mlups": cells / wall / 1e6, "cell_updates": int(cells),
        "tts_p50_s": float(np.percentile(tts, 50)), "tts_p99_s": float(np.percentile(tts, 99)),
        "tts_max_s": float(tts.max()), "hbm_budget_bytes": int(hbm_budget_bytes),
        "steps_per_round": steps_per_round, "streaming": "aa" if aa else "pull",
        "max_resident_requests": int(max_running), "gpu_busy_s": gpu_s,
        "algorithmic_bytes": int(moved), "gpu_gbs": moved / gpu_s / 1e9 if gpu_s > 0 else None,
        "launch": launch,
    }
    return (out, results) if keep_results else out
