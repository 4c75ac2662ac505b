"""The allocation-free totals entry point, checked against lbm_reduce.

lbm_reduce_noalloc is for callers that cannot allocate device memory at the
point of the call (loops that must not enter an allocator, hosts that keep a
fixed device-memory budget): it keeps its partial sums in a static device
array instead.  This test builds a caller-owned device field in the
library's storage layout, calls the entry point twice in a row through the C
ABI, and compares both results with the totals lbm_reduce reports for a
handle holding the same field, for every lattice and storage precision.  It
sits in a file of its own, collected last.
"""
import numpy as np
import pytest

import oracle
from paper_1710_02065_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
@pytest.mark.parametrize("lattice,n", [(0, (130, 70, 1)), (1, (40, 30, 20)), (2, (24, 18, 14))])
def test_reduce_noalloc_matches_reduce(lattice, n, prec):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_02065_gb300 import build
    build.build()
    from paper_1710_02065_gb300 import lbm

    ncell = int(np.prod(n))
    _, q, _, w, _ = oracle.lattice(lattice)
    f = inputs.random_populations(w, ncell, seed=17 + lattice, spread=0.1)
    mask = np.zeros(ncell, np.uint8)
    mask[::7] = lbm.LBM_CELL_SOLID

    s = lbm.Solver(lattice, n, 0.7, prec)
    s.set_populations(f)
    lbm.lbm_set_geometry(s.h, mask)
    mass, mom, rc = s.reduce()
    assert rc == 0

    # the handle's stored values (exact in FP64) give the caller's field in
    # the same storage format, so both reductions see the same numbers
    dtype = {0: torch.float64, 1: torch.float32, 2: torch.float16, 3: torch.bfloat16}[prec]
    g = torch.tensor(s.populations() - w[:, None], dtype=torch.float64).to(dtype).cuda().contiguous()
    m = torch.tensor(mask, device="cuda")
    out = torch.full((6,), -1.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        lbm.lbm_reduce_noalloc(lattice, prec, g.data_ptr(), ncell, m.data_ptr(), out.data_ptr(), stream)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        assert abs(o[0] - mass) <= 1e-12 * abs(mass)
        assert np.abs(o[1:4] - mom).max() <= 1e-12 * abs(mass)
        assert o[4] == (mask == 0).sum()
        assert o[5] == 0
    s.close()


def test_reduce_noalloc_rejects_oversized_fields():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_02065_gb300 import lbm
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_reduce_noalloc(1, 1, dummy.data_ptr(), (1 << 26) + 1, None, dummy.data_ptr())
    assert e.value.code == lbm.LBM_EINVAL
    assert "scratch" in lbm.lbm_last_error(None)
