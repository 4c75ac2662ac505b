"""The parity tests against the checked build of the library.

compute-sanitizer is not available where these tests run, so the library has
a checked build instead (build(checked=True), -DLBM_BOUNDS_CHECK): every index
the update kernels read or write is tested before the access, and a cell with
an index outside its lattice is skipped and flagged in the handle's error
word (lbm_sync reports it).  Here the oracle-parity tests of every kernel
path (general and vectorised kernels at every precision and launch shape,
every boundary rule, D3Q27, the row-staged kernel, 2D and 3D refinement)
run in a child process that loads the checked build (LBM_CHECKED=1): a
skipped cell would break parity.  A second child runs every kernel path on
open and walled boxes and checks the error word itself through lbm_sync.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_parity_suite_passes_on_the_checked_build():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_02065_gb300 import build
    build.build(checked=True)
    env = dict(os.environ, LBM_CHECKED="1")
    sel = ("all_boundary_rules or launch_shapes or d3q27_all or staged_kernel_matches or radial_sponge "
           "or free_slip or two_level_3d_parity or two_level_cylinder_parity or three_level")
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "-m", "gpu",
           os.path.join(ROOT, "tests", "test_gpu_parity.py"), os.path.join(ROOT, "tests", "test_gpu_refinement.py"),
           "-k", sel]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
    assert " passed" in r.stdout


def test_checked_build_is_the_library_loaded_under_lbm_checked():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_02065_gb300 import build
    path = build.build(checked=True)
    code = ("import paper_1710_02065_gb300.lbm as m, sys; "
            "sys.exit(0 if m.LIB_PATH.endswith('liblbm_checked.so') else 1)")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=dict(os.environ, LBM_CHECKED="1"))
    assert r.returncode == 0 and os.path.exists(path)


SYNC_SCRIPT = r"""
import sys, numpy as np
sys.path.insert(0, "tests")
from paper_1710_02065_gb300 import lbm
from cases import Case, to_gpu, with_random_state, VELOCITY, OUTFLOW
for lattice, n in ((0, (37, 23, 1)), (1, (19, 13, 11)), (2, (16, 12, 10))):
    for prec in (0, 1, 2, 3):
        for cand in ((128, 1), (64, 2), (32, 4)) if prec != 0 else ((128, 1), (64, 2)):
            for walled in (False, True):
                c = with_random_state(Case("chk", lattice, n, 0.6), seed=3, spread=0.02)
                c.faces = {0: (VELOCITY, (0.03, 0, 0), None), 1: (OUTFLOW, (0, 0, 0), None)}
                c.sponges = {1: (4, 0.4)}
                if walled:
                    m = np.zeros(c.ncell, np.uint8)
                    m[c.ncell // 2] = 1
                    c.solid = m
                s = to_gpu(c, prec)
                lbm.lbm_set_launch(s.h, *cand)
                s.step(3)
                lbm.lbm_sync(s.h)  # raises if the error word has the index-check bit
                s.close()
print("checked build: every kernel path ran without an index fault")
"""


def test_every_kernel_path_reports_no_index_fault():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_02065_gb300 import build
    build.build(checked=True)
    r = subprocess.run([sys.executable, "-c", SYNC_SCRIPT], cwd=ROOT, env=dict(os.environ, LBM_CHECKED="1"),
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "without an index fault" in r.stdout
