"""The bounds-checking build of the library (compiled with -DMPS_BOUNDS_CHECK).

In that build the kernels that take indices from device data (the inverse pivot
permutation of the split, the column swaps of the randomized pivoting) check them
and report DEV_ERR_BOUNDS through the handle's error word instead of reading or
writing out of range.  Odd shapes through every split path must give the oracle's
results with no check failing (a failure would surface as MPS_E_CUDA at the next
synchronous call).
"""

import numpy as np
import pytest

from oracle import mps as omps
from workloads import circuits

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def checked():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2505_06119_gb300 import _lib

    return _lib.load_checked()


@pytest.mark.parametrize("truncation", ["qrcp", "rqrcp"])
@pytest.mark.parametrize("n,chi,depth", [(11, 12, 7), (13, 40, 8)])
def test_odd_shapes_pass_the_index_checks(checked, truncation, n, chi, depth):
    """Odd chain lengths and bond caps (ragged panels, one-CTA splits and grid splits,
    both policies' centre moves) in the checked build: the state equals the oracle's."""
    from paper_2505_06119_gb300 import MPS

    ops = circuits.brickwall(n, depth, seed=n + chi)
    ref = omps.OracleMPS(n, chi, "canon", truncation=truncation, sketch_seed=3)
    ref.run(ops)
    with MPS(n, chi, precision="fp64", lib=checked, truncation=truncation, sketch_seed=3) as m:
        m.run(ops)
        m.sync()  # MPS_E_CUDA here if an index check had failed
        assert m.bond_dims() == ref.bond_dims()
        assert m.fidelity() == pytest.approx(ref.norm2(), rel=1e-9)
        rng = np.random.default_rng(n)
        for _ in range(8):
            bits = rng.integers(0, 2, n)
            assert abs(m.amplitude(bits) - ref.amplitude(bits)) < 1e-10
    assert ref.norm2() < 0.9999


def test_checked_build_is_loaded_separately(checked):
    from paper_2505_06119_gb300 import _lib

    assert checked is not _lib.load()
    assert checked.mps_version() == _lib.load().mps_version()
