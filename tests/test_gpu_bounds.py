"""The index checks of the FSC_BOUNDS_CHECK build (libfsc_checked.so, FSC_LIBRARY=checked).

A column index that leaves the iterate's rows after the graph was validated (the graph borrows the
caller's CSR, so the caller can overwrite it) must be recorded with its site, value and range, and
the access skipped.  The iterate buffers are allocated with spare rows past n, so even the index
tried here stays inside them.  Skipped unless the checked library is the one loaded.
"""
import os

import numpy as np
import pytest

import workloads as W
from _helpers import require_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_cuda()


def test_library_reports_whether_it_checks(torch):
    import paper_2310_10939_gb300 as fsc
    rep = fsc.bounds_report()
    if os.environ.get("FSC_LIBRARY") == "checked":
        assert rep is None
    else:
        assert rep == -1


@pytest.mark.skipif(os.environ.get("FSC_LIBRARY") != "checked", reason="needs the library built with index checks")
def test_out_of_range_column_is_recorded_and_skipped(torch):
    import paper_2310_10939_gb300 as fsc
    g = W.sbm([200] * 3, 0.1, 0.01, 1)
    col = torch.as_tensor(g.col, device="cuda")
    G = fsc.Graph(torch.as_tensor(g.row_ptr, device="cuda"), col)
    spare = 16
    z_in = torch.zeros((g.n + spare, 4), dtype=torch.float32, device="cuda")
    z_out = torch.zeros_like(z_in)
    assert fsc.bounds_report(clear=True) is None
    col[5] = g.n + 3                                  # inside z_in's spare rows, outside the graph
    torch.cuda.synchronize()
    fsc.power_step(G, 4, z_in, z_out)
    torch.cuda.synchronize()
    site, idx, lo, hi = fsc.bounds_report(clear=True)
    assert (site, idx, lo, hi) == (1, g.n + 3, 0, g.n)
    assert fsc.bounds_report() is None
    col[5] = int(g.col[5])
    G.close()
