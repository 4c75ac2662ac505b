"""CPU checks of the seeded serving request stream (input generation only)."""
import numpy as np

from paper_1710_02065_gb300 import inputs


def test_request_stream_is_seeded_and_follows_the_recipe():
    a = inputs.serving_requests(512, seed=5, rate_per_s=8.0)
    b = inputs.serving_requests(512, seed=5, rate_per_s=8.0)
    assert a == b
    arr = np.array([r["arrival"] for r in a])
    assert (np.diff(arr) > 0).all()
    # Poisson arrivals: mean gap 1/rate within a few percent over 512 draws
    assert abs(np.diff(arr).mean() * 8.0 - 1.0) < 0.15
    lat = np.array([r["lattice"] for r in a])
    assert 0.4 < lat.mean() < 0.6
    for r in a:
        N = r["extents"][0]
        if r["lattice"] == 0:
            assert N in (64, 128, 256, 512, 1024) and r["extents"][2] == 1
        else:
            assert N in (32, 48, 64, 96, 128, 192) and r["extents"] == (N, N, N)
        assert 0.52 <= r["tau"] <= 0.9
        assert 500 <= r["steps"] <= 5000
        assert r["precision"] in (1, 2)


def test_request_initial_states():
    r2 = {"lattice": 0, "extents": (64, 64, 1)}
    rho, u = inputs.request_initial_state(r2)
    assert rho.shape == (64 * 64,) and u.shape == (64 * 64, 3)
    assert abs(rho.max() - 1 - 1e-3) < 1e-6
    r3 = {"lattice": 1, "extents": (16, 16, 16)}
    rho, u = inputs.request_initial_state(r3)
    assert rho.shape == (16 ** 3,) and np.abs(u).max() <= 0.02
