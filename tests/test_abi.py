"""CPU checks of the C ABI: the library builds, loads and exports every
entry point that include/lbm.h declares; host-side tables and argument
validation work without a GPU (no kernel is launched here)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module")
def lbm():
    from paper_1710_02065_gb300 import build
    build.build()
    from paper_1710_02065_gb300 import lbm as mod
    return mod


def _declared(repo_root):
    names = set()
    for fn in os.listdir(os.path.join(repo_root, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(repo_root, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol(lbm, repo_root):
    declared = _declared(repo_root)
    assert "lbm_step" in declared and "lbm_create" in declared
    lib = ctypes.CDLL(lbm.LIB_PATH)
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing
    # the binding wraps each declared entry point under the same name
    assert declared <= set(dir(lbm)), declared - set(dir(lbm))


@pytest.mark.parametrize("which", [0, 1, 2])
def test_lattice_table_matches_oracle(lbm, which):
    q, d, xi, w = lbm.lbm_lattice_table(which)
    od, oq, oxi, ow, oopp = oracle.lattice(which)
    assert (q, d) == (oq, od)
    assert np.array_equal(xi, oxi)
    assert np.array_equal(w, ow)


def test_invalid_arguments_are_rejected_on_the_host(lbm):
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_create(lbm.LBM_D2Q9, (16, 16, 1), 0.5)
    assert e.value.code == lbm.LBM_EINVAL
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_create(lbm.LBM_D2Q9, (16, 16, 2), 0.6)
    assert e.value.code == lbm.LBM_EINVAL
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_create(lbm.LBM_D3Q19, (16, 16, 16), 0.6, Ma_ref=0.7)
    assert e.value.code == lbm.LBM_EINVAL
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_create(7, (16, 16, 16), 0.6)
    assert e.value.code == lbm.LBM_EINVAL
    assert "lattice" in lbm.lbm_last_error(None)
