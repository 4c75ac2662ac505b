"""The in-place AA streaming pattern (lbm_set_streaming) against the FP64
oracle and against the two-lattice pull update.

The AA pattern keeps one lattice and alternates a gather-push step with a
local step; every boundary rule of the pull update (velocity inflow with a
profile and noise, zero-gradient outflow, sponges, halfway bounce-back at a
solid, periodic axes) must give the same populations, after an odd and after
an even number of steps (the odd-step lattice is in the push layout and is
brought back to the standard layout by the reads).  Tolerances as in
test_gpu_parity: FP64 1e-13 absolute, FP32 1e-5 of max |f|, FP16 / BF16 the
rounding of every stored value per step.
"""
import numpy as np
import pytest

import oracle
from cases import D2Q9, D3Q19, D3Q27, round_jet, to_gpu, to_oracle, acoustic_pulse
from test_gpu_parity import PRECS, _boxed_case, _open_box, _pop_tol

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_02065_gb300 import build
    build.build()


def _aa(c, prec, kernel=None):
    from paper_1710_02065_gb300 import lbm
    s = to_gpu(c, PRECS[prec])
    lbm.lbm_set_streaming(s.h, lbm.LBM_STREAM_AA)
    assert lbm.lbm_get_streaming(s.h) == lbm.LBM_STREAM_AA
    if kernel is not None:
        lbm.lbm_set_launch(s.h, 64, kernel)
    return s


@pytest.mark.parametrize("prec", list(PRECS))
@pytest.mark.parametrize("lattice", [D2Q9, D3Q19, D3Q27])
def test_aa_every_boundary_rule_matches_oracle(lattice, prec):
    c = _boxed_case(lattice)
    P, f = to_oracle(c)
    _, _, _, w, _ = oracle.lattice(lattice)
    done = 0
    s = _aa(c, prec)
    for n in (1, 1, 2, 3):  # step counts 1, 2, 4, 7: odd and even
        f = P.run(f, n, step0=done)
        s.step(n)
        done += n
        err = np.abs(s.populations() - f).max()
        assert err <= _pop_tol(prec, f, w, done), (done, err)
    s.close()


@pytest.mark.parametrize("kernel", [1, 2, 4])
@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("lattice", [D2Q9, D3Q19, D3Q27])
def test_aa_open_box_and_periodic_axes_match_oracle(lattice, prec, kernel):
    """No cell-type mask: open box with inflow profile and noise, outflow,
    sponges; and the same box periodic in y / z.  One, two and four cells
    per thread (the vector kernel updates the x-face nodes in registers; on
    D3Q27, which has the two-cell form only, a request for four runs the
    general in-place kernel)."""
    _, _, _, w, _ = oracle.lattice(lattice)
    n = (40, 12, 1) if lattice == D2Q9 else (24, 10, 8)
    for periodic in (False, True):
        c = _open_box(lattice, n, seed=7, rest=True)
        if periodic:
            for face in range(2, 4 if lattice == D2Q9 else 6):
                c.faces.pop(face, None)
            c.sponges = {1: (5, 0.8)}
        P, f = to_oracle(c)
        ref = P.run(f, 5)
        s = _aa(c, prec, kernel)
        s.step(5)
        err = np.abs(s.populations() - ref).max()
        assert err <= _pop_tol(prec, ref, w, 5), (periodic, err)
        s.close()


@pytest.mark.parametrize("prec", list(PRECS))
@pytest.mark.parametrize("lattice", [D2Q9, D3Q19, D3Q27])
def test_aa_whole_warp_rows_match_oracle(lattice, prec):
    """Two cells per thread on rows of whole warps (nx = 128: two warps per
    row, and the x-moving populations cross from warp to warp; only the row's
    first and last threads push values out of the row): an open x axis
    (inflow with profile and noise, outflow, sponges; values leaving through
    a face are kept at the node) and a periodic one (they wrap around), after
    odd and even step counts."""
    _, _, _, w, _ = oracle.lattice(lattice)
    n = (128, 10, 1) if lattice == D2Q9 else (128, 8, 6)
    for xper in (False, True):
        c = _open_box(lattice, n, seed=31, rest=True)
        if xper:
            c.faces.pop(0)
            c.faces.pop(1)
            c.sponges = {2: (3, 0.6)}
        P, f = to_oracle(c)
        s = _aa(c, prec, 2)
        done = 0
        for k in (3, 2):  # step counts 3 and 5
            f = P.run(f, k, step0=done)
            s.step(k)
            done += k
            err = np.abs(s.populations() - f).max()
            assert err <= _pop_tol(prec, f, w, done), (xper, done, err)
        s.close()


def test_aa_equals_pull_and_survives_switches_and_checkpoints(tmp_path):
    """FP32 jet box: AA and pull agree to round-off after 9 steps; switching the
    pattern in the middle of a run (at an odd step) and a checkpoint written in
    AA at an odd step and resumed in pull continue the same trajectory."""
    from paper_1710_02065_gb300 import lbm
    c = round_jet(48, 32, 32, diameter=6.0, sponge=6, Re=1000.0)
    a = to_gpu(c, PRECS["fp32"])
    b = _aa(c, "fp32")
    a.step(9)
    b.step(9)
    fa, fb = a.populations(), b.populations()
    assert np.abs(fa - fb).max() <= 1e-6 * np.abs(fa).max()
    # pull -> AA at step 9, AA -> pull at step 14
    lbm.lbm_set_streaming(a.h, lbm.LBM_STREAM_AA)
    a.step(5)
    lbm.lbm_set_streaming(a.h, lbm.LBM_STREAM_PULL)
    a.step(4)
    path = str(tmp_path / "aa.bin")
    b.step(5)
    lbm.lbm_save(b.h, path)  # AA, odd step 14
    c2 = to_gpu(c, PRECS["fp32"])
    lbm.lbm_load(c2.h, path)
    assert c2.info()["step"] == 14
    c2.step(4)
    b.step(4)
    fa, fb, fc = a.populations(), b.populations(), c2.populations()
    assert np.abs(fa - fb).max() <= 1e-5 * np.abs(fa).max()
    assert np.array_equal(fb, fc) or np.abs(fb - fc).max() <= 1e-6 * np.abs(fb).max()
    for s in (a, b, c2):
        s.close()


def test_aa_graph_replay_matches_direct_launches():
    """lbm_step on a non-default stream replays captured (gather-push, local)
    step pairs; bitwise the same as direct launches, also across calls that
    start at an odd step."""
    import torch
    from paper_1710_02065_gb300 import lbm
    stream = torch.cuda.Stream()
    c = acoustic_pulse(64)
    a = _aa(c, "fp32")
    b = lbm.Solver(c.lattice, c.n, c.tau, PRECS["fp32"], stream=stream.cuda_stream)
    lbm.lbm_set_streaming(b.h, lbm.LBM_STREAM_AA)
    b.set_state(c.rho0, c.u0)
    a.step(37)
    b.step(5)
    b.step(32)
    torch.cuda.synchronize()
    assert np.array_equal(a.populations(), b.populations())
    a.close()
    b.close()


def test_aa_rejects_refinement_and_reports_memory():
    from paper_1710_02065_gb300 import lbm
    torch = pytest.importorskip("torch")
    c = acoustic_pulse(256)
    s = to_gpu(c, PRECS["fp64"])
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    lbm.lbm_set_streaming(s.h, lbm.LBM_STREAM_AA)
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 - free0 >= 9 * 256 * 256 * 8 - (2 << 20)  # one lattice returned (allocator granularity aside)
    with pytest.raises(lbm.LBMError):
        lbm.lbm_add_refinement_patch(s.h, (8, 8, 0), (17, 17, 1))
    s.close()
