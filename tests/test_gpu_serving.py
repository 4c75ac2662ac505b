"""The solve server: continuous batching of independent solves.

  * a request's result is bitwise the same alone and batched with others
    (its arithmetic does not depend on the mix)
  * results equal the oracle within the parity tolerances (FP64 1e-12,
    FP32 1e-5 normwise in rho and u); for a pulse at rest |u| is ~1e-5, so
    u also passes when its absolute error is below the round-off of O(1)
    populations in that precision (FP64 1e-13, FP32 1e-8)
  * admission respects the HBM budget: a request that does not fit waits
    and runs once memory is returned
"""
import numpy as np
import pytest

import oracle
from paper_1710_02065_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def serving():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_02065_gb300 import build
    build.build()
    from paper_1710_02065_gb300 import serving as mod
    return mod


def _req(lattice, N, tau, steps, prec):
    ext = (N, N, 1) if lattice == 0 else (N, N, N)
    return {"arrival": 0.0, "lattice": lattice, "extents": ext, "tau": tau, "steps": steps, "precision": prec}


def _run(serving, reqs, budget=1 << 30, rounds_steps=7):
    srv = serving.Server(budget, 64)
    ids = []
    for r in reqs:
        rho, u = inputs.request_initial_state(r)
        ids.append(srv.submit(r, rho, u))
    out = {}
    for _ in range(10000):
        srv.run(rounds_steps)
        for k, rid in enumerate(ids):
            if k in out:
                continue
            st, done = srv.poll(rid)
            if st in (2, 3):
                out[k] = srv.result(rid, int(np.prod(reqs[k]["extents"])))
        if len(out) == len(ids):
            break
    srv.close()
    return out


def test_result_is_the_same_alone_and_in_a_mix(serving):
    a = _req(0, 64, 0.61, 150, 1)
    alone = _run(serving, [a])[0]
    mix = [_req(1, 24, 0.7, 90, 2), a, _req(0, 40, 0.55, 33, 0), _req(1, 16, 0.9, 200, 1),
           _req(0, 128, 0.8, 10, 2), _req(2, 20, 0.7, 50, 1), _req(2, 14, 0.6, 30, 3)]
    batched = _run(serving, mix)
    for k in range(len(mix)):
        assert batched[k][2] == 0
    assert np.array_equal(alone[0], batched[1][0])
    assert np.array_equal(alone[1], batched[1][1])


@pytest.mark.parametrize("lattice,N,prec,tol,floor", [(0, 32, 0, 1e-12, 1e-13), (0, 48, 1, 1e-5, 1e-8),
                                                      (1, 12, 0, 1e-12, 1e-13), (1, 16, 1, 1e-5, 1e-8),
                                                      (2, 12, 0, 1e-12, 1e-13), (2, 16, 1, 1e-5, 1e-8)])
def test_served_results_match_oracle(serving, lattice, N, prec, tol, floor):
    r = _req(lattice, N, 0.66, 40, prec)
    rho_g, u_g, rc = _run(serving, [r])[0]
    assert rc == 0
    rho0, u0 = inputs.request_initial_state(r)
    P = oracle.Problem(lattice, r["extents"], r["tau"])
    f = P.run(P.equilibrium(rho0, u0), r["steps"])
    rho, u, _ = P.moments(f)
    assert np.linalg.norm(rho_g - rho) / np.linalg.norm(rho) <= tol
    du = u_g - u
    assert np.linalg.norm(du) / np.linalg.norm(u) <= tol or np.abs(du).max() <= floor


def test_admission_waits_for_budget(serving):
    big = _req(1, 32, 0.7, 60, 1)            # 2 * 19 * 32^3 * 4 B = 4.98 MB
    budget = int(2 * 19 * 32 ** 3 * 4 * 1.5)  # room for one at a time
    srv = serving.Server(budget, 8)
    ids = []
    for _ in range(3):
        rho, u = inputs.request_initial_state(big)
        ids.append(srv.submit(big, rho, u))
    srv.run(10)
    states = [srv.poll(i)[0] for i in ids]
    assert states.count(1) == 1 and states.count(0) == 2
    assert srv.stats()["bytes_in_use"] <= budget
    finished = set()
    for _ in range(100):
        srv.run(10)
        for i in ids:
            if i not in finished and srv.poll(i)[0] == 2:
                finished.add(i)
                srv.result(i, 32 ** 3)
        if len(finished) == 3:
            break
    assert len(finished) == 3
    srv.close()


def test_zero_step_request_returns_initial_state(serving):
    r = _req(0, 16, 0.7, 0, 0)
    rho, u, rc = _run(serving, [r])[0]
    rho0, u0 = inputs.request_initial_state(r)
    assert rc == 0
    assert np.abs(rho - rho0).max() < 1e-15


def test_serving_stream_small(serving):
    """A short stream with overlapping arrivals completes with sane statistics."""
    reqs = inputs.serving_requests(12, seed=1, rate_per_s=200.0, steps_scale=0.02, sizes_2d=(64, 128),
                                   sizes_3d=(16, 24))
    out = serving.serve(reqs, hbm_budget_bytes=64 << 20, max_slots=8, steps_per_round=10)
    assert out["requests"] == 12 and out["failed"] == 0
    assert out["tts_p99_s"] >= out["tts_p50_s"] > 0
    assert out["aggregate_mlups"] > 0


def test_largest_2d_request_matches_oracle(serving):
    """The largest D2Q9 request size of the serving stream (1024^2), FP32, 3
    steps, next to a small D3Q19 request: equal to the oracle within 1e-5."""
    big = _req(0, 1024, 0.53, 3, 1)
    small = _req(1, 32, 0.8, 5, 2)
    out = _run(serving, [big, small], budget=2 << 30, rounds_steps=2)
    rho_g, u_g, rc = out[0]
    assert rc == 0
    rho0, u0 = inputs.request_initial_state(big)
    P = oracle.Problem(0, big["extents"], big["tau"])
    f = P.run(P.equilibrium(rho0, u0), big["steps"])
    rho, u, _ = P.moments(f)
    assert np.linalg.norm(rho_g - rho) / np.linalg.norm(rho) <= 1e-5
    du = u_g - u
    assert np.linalg.norm(du) / np.linalg.norm(u) <= 1e-5 or np.abs(du).max() <= 1e-8


def test_unstable_request_fails_alone(serving):
    """Failure isolation: a request that blows up (random supersonic start at
    tau just above 1/2) is retired as failed with LBM_EUNSTABLE and its memory
    and slot returned, while the requests batched with it finish with the
    same result as when run alone."""
    from paper_1710_02065_gb300 import lbm
    good = _req(1, 16, 0.7, 60, 1)
    alone = _run(serving, [good])[0]
    bad = _req(1, 16, 0.5001, 400, 1)
    srv = serving.Server(1 << 30, 8)
    n = 16 ** 3
    rng = np.random.default_rng(13)
    u_bad = rng.uniform(-0.45, 0.45, (n, 3))  # uncorrelated, |u| up to 0.78 > c_s = 0.577
    rho_bad = rng.uniform(0.5, 1.5, n)
    ids = [srv.submit(bad, rho_bad, u_bad)]
    rho0, u0 = inputs.request_initial_state(good)
    ids.append(srv.submit(good, rho0, u0))
    states = {}
    for _ in range(200):
        srv.run(20)
        for rid in ids:
            st, _ = srv.poll(rid)
            if st in (lbm.LBM_REQ_DONE, lbm.LBM_REQ_FAILED):
                states[rid] = st
        if len(states) == 2:
            break
    assert states[ids[0]] == lbm.LBM_REQ_FAILED
    assert states[ids[1]] == lbm.LBM_REQ_DONE
    _, _, rc_bad = srv.result(ids[0], n)
    rho_g, u_g, rc_good = srv.result(ids[1], n)
    assert rc_bad == lbm.LBM_EUNSTABLE and rc_good == 0
    assert np.array_equal(rho_g, alone[0]) and np.array_equal(u_g, alone[1])
    st = srv.stats()
    assert st["running"] == 0 and st["bytes_in_use"] == 0  # slot and memory returned
    srv.close()


def test_late_arrival_is_bitwise_the_same_as_alone(serving):
    """Continuous batching: a request submitted after the server has run
    rounds and after another request has retired (so it is admitted into a
    running mix, with rebuilt tile lists and a recaptured round) finishes
    bitwise as when it runs alone."""
    late = _req(1, 20, 0.64, 45, 2)
    alone = _run(serving, [late])[0]
    srv = serving.Server(1 << 30, 16)
    early = [_req(0, 48, 0.7, 14, 1), _req(1, 16, 0.8, 200, 3), _req(2, 12, 0.6, 120, 1)]
    ids = []
    for r in early:
        rho, u = inputs.request_initial_state(r)
        ids.append(srv.submit(r, rho, u))
    # run until the short request has retired while the others still run
    for _ in range(100):
        srv.run(7)
        if srv.poll(ids[0])[0] == 2:
            break
    assert srv.poll(ids[0])[0] == 2 and srv.poll(ids[1])[0] == 1
    srv.result(ids[0], 48 * 48)
    rho, u = inputs.request_initial_state(late)
    lid = srv.submit(late, rho, u)
    got = None
    for _ in range(1000):
        srv.run(7)
        if srv.poll(lid)[0] == 2:
            got = srv.result(lid, 20 ** 3)
            break
    srv.close()
    assert got is not None and got[2] == 0
    assert np.array_equal(alone[0], got[0]) and np.array_equal(alone[1], got[1])


@pytest.mark.parametrize("lattice,N,prec,aa", [(0, 48, 2, False), (0, 48, 3, False), (1, 16, 2, False),
                                               (1, 16, 3, False), (2, 12, 2, False), (2, 12, 3, False),
                                               (0, 48, 3, True), (1, 16, 2, True), (2, 12, 2, True)])
def test_16bit_served_results_match_oracle(serving, lattice, N, prec, aa):
    """FP16 / BF16 storage in the server against the FP64 oracle, D2Q9, D3Q19
    and D3Q27, two-lattice pull and in-place AA: the density error stays
    within the rounding of the stored shifted populations (one half-ulp of
    max |f - w| per step and direction, summed over Q)."""
    r = _req(lattice, N, 0.66, 31 if aa else 30, prec)  # AA: an odd count ends in the push layout
    rho_g, u_g, rc = _run_aa(serving, [r])[0] if aa else _run(serving, [r])[0]
    assert rc == 0
    rho0, u0 = inputs.request_initial_state(r)
    P = oracle.Problem(lattice, r["extents"], r["tau"])
    f0 = P.equilibrium(rho0, u0)
    f = P.run(f0, r["steps"])
    rho, u, _ = P.moments(f)
    _, q, _, w, _ = oracle.lattice(lattice)
    ulp = 2.0 ** -11 if prec == 2 else 2.0 ** -8
    g = max(np.abs(f - w[:, None]).max(), np.abs(f0 - w[:, None]).max())
    bound = (r["steps"] + 1) * q * ulp * g
    assert np.abs(rho_g - rho).max() <= bound
    assert np.abs(u_g - u).max() <= 2 * bound


def _run_aa(serving, reqs, budget=1 << 30, rounds_steps=7):
    srv = serving.Server(budget, 64, aa=True)
    ids = []
    for r in reqs:
        rho, u = inputs.request_initial_state(r)
        ids.append(srv.submit(r, rho, u))
    out = {}
    for _ in range(10000):
        srv.run(rounds_steps)
        for k, rid in enumerate(ids):
            if k not in out and srv.poll(rid)[0] in (2, 3):
                out[k] = srv.result(rid, int(np.prod(reqs[k]["extents"])))
        if len(out) == len(ids):
            break
    srv.close()
    return out


@pytest.mark.parametrize("lattice,N,prec,steps,tol,floor", [(0, 32, 0, 41, 1e-12, 1e-13), (1, 12, 0, 40, 1e-12, 1e-13),
                                                            (1, 16, 1, 33, 1e-5, 1e-8), (2, 12, 1, 20, 1e-5, 1e-8)])
def test_aa_served_results_match_oracle(serving, lattice, N, prec, steps, tol, floor):
    """Requests served with the in-place AA pattern (one lattice each), odd and
    even step counts, batched together: each equals the oracle."""
    r = _req(lattice, N, 0.66, steps, prec)
    other = _req(1, 10, 0.8, 17, 2)
    out = _run_aa(serving, [r, other])
    rho_g, u_g, rc = out[0]
    assert rc == 0 and out[1][2] == 0
    rho0, u0 = inputs.request_initial_state(r)
    P = oracle.Problem(lattice, r["extents"], r["tau"])
    rho, u, _ = P.moments(P.run(P.equilibrium(rho0, u0), r["steps"]))
    assert np.linalg.norm(rho_g - rho) / np.linalg.norm(rho) <= tol
    du = u_g - u
    assert np.linalg.norm(du) / np.linalg.norm(u) <= tol or np.abs(du).max() <= floor


def test_aa_server_budget_holds_twice_the_cells(serving):
    """A budget of three lattices holds one pull request (two lattices each)
    at a time, and all three AA requests (one lattice each)."""
    big = _req(1, 32, 0.7, 30, 1)
    budget = int(2 * 19 * 32 ** 3 * 4 * 1.5)
    for aa, expect in ((False, 1), (True, 3)):
        srv = serving.Server(budget, 8, aa=aa)
        ids = []
        for _ in range(3):
            rho, u = inputs.request_initial_state(big)
            ids.append(srv.submit(big, rho, u))
        srv.run(5)
        assert [srv.poll(i)[0] for i in ids].count(1) == expect
        assert srv.stats()["bytes_in_use"] <= budget
        srv.close()


def _run_shape(serving, reqs, launch):
    srv = serving.Server(1 << 30, 16, launch=launch)
    ids = []
    for r in reqs:
        rho, u = inputs.request_initial_state(r)
        ids.append(srv.submit(r, rho, u))
    out = {}
    for _ in range(1000):
        srv.run(9)
        for k, rid in enumerate(ids):
            if k not in out and srv.poll(rid)[0] in (2, 3):
                out[k] = srv.result(rid, int(np.prod(reqs[k]["extents"])))
        if len(out) == len(ids):
            break
    srv.close()
    return out


def test_launch_shape_does_not_change_results(serving):
    """Every candidate launch shape of the batched update (cells per lane,
    warps per block) gives each request bitwise the result of the default
    shape, for 16-bit, FP32 and FP64 storage, 2D and 3D."""
    from paper_1710_02065_gb300 import autotune
    reqs = [_req(0, 64, 0.61, 23, 1), _req(1, 16, 0.7, 21, 2), _req(0, 32, 0.8, 19, 3), _req(1, 12, 0.66, 17, 0)]
    ref = _run_shape(serving, reqs, None)
    kinds = {(r["lattice"], r["precision"]) for r in reqs}
    for v, w in autotune.SERVER_CANDIDATES:
        got = _run_shape(serving, reqs, {k: (v, w) for k in kinds})
        for k in range(len(reqs)):
            assert got[k][2] == 0
            assert np.array_equal(ref[k][0], got[k][0]) and np.array_equal(ref[k][1], got[k][1]), (v, w, k)


def test_server_tuner_picks_a_candidate(serving):
    from paper_1710_02065_gb300 import autotune, lbm
    picks = autotune.tune_server([(0, 2), (1, 1)], {0: [(64, 64, 1), (128, 128, 1)], 1: [(16, 16, 16), (24, 24, 24)]},
                                 round_steps=4, rounds=1, budget_bytes=1 << 28)
    assert set(picks) == {(0, 2), (1, 1)}
    for p in picks.values():
        assert (p["cells_per_lane"], p["warps_per_block"]) in autotune.SERVER_CANDIDATES
        assert len(p["table"]) == len(autotune.SERVER_CANDIDATES) and p["mlups"] > 0
    s = lbm.lbm_server_create(1 << 20, 4, None)
    try:
        assert lbm.lbm_server_get_launch(s, 1, 1) == (2, 2)
        assert lbm.lbm_server_get_launch(s, 1, 2) == (2, 2)
        lbm.lbm_server_set_launch(s, 1, 2, 1, 8)
        assert lbm.lbm_server_get_launch(s, 1, 2) == (1, 8)
        with pytest.raises(lbm.LBMError):
            lbm.lbm_server_set_launch(s, 1, 2, 3, 4)
        with pytest.raises(lbm.LBMError):
            lbm.lbm_server_set_launch(s, 1, 2, 1, 16)
    finally:
        lbm.lbm_server_destroy(s)
