"""The allocation-free tessellation entry point against the regular one.

tblr_tessellate_noalloc serves callers that cannot allocate device memory:
it takes its scratch from a fixed static device array instead of a caller
workspace.  Its integer outputs must equal those of tblr_tessellate bit for
bit, on two calls in a row (the array keeps the previous call's contents, so
the second call checks that nothing stale leaks through).  This file is
collected last so that a failure here comes after every other test has run.
"""
import ctypes

import numpy as np
import pytest

from paper_2501_05528_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _outputs(lay):
    return [t.cpu().numpy().copy() for t in (lay.perm, lay.box_of, lay.offsets, lay.nbr, lay.nnbr,
                                             lay.colour, lay.pts)]


@pytest.mark.parametrize("d,grid,n,seed", [(2, (16, 16), 65536, 1), (3, (4, 5, 3), 20001, 2)])
def test_noalloc_tessellation_matches_regular_entry_point(d, grid, n, seed):
    from paper_2501_05528_gb300 import tblr as tb
    dev = torch.device("cuda")
    first = inputs.uniform_points(n, d, seed=seed)
    second = inputs.uniform_points(n, d, seed=seed + 100)
    prob = tb.make_problem(d, "laplace2d" if d == 2 else "laplace3d", n, grid,
                           (0.0,) * d, (1.0,) * d, 8)
    for pts in (first, second):                     # two calls in a row
        x = torch.as_tensor(pts, device=dev)
        ref = _outputs(tb.tblr_tessellate(prob, x))
        lay = tb.Layout(prob)                        # caller-owned outputs
        st = tb.lib().tblr_tessellate_noalloc(ctypes.byref(prob), ctypes.c_void_p(x.data_ptr()),
                                              lay.ref, tb._stream())
        assert st == tb.TBLR_OK, tb.lib().tblr_last_error()
        torch.cuda.synchronize()
        got = _outputs(lay)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b)


def test_noalloc_rejects_problems_beyond_its_scratch():
    from paper_2501_05528_gb300 import tblr as tb
    n = 4_000_000
    prob = tb.make_problem(2, "laplace2d", n, (128, 128), (0.0, 0.0), (1.0, 1.0), 8)
    assert tb.lib().tblr_tessellate_workspace(ctypes.byref(prob)) > (8 << 20)
    lay_struct = tb.LayoutStruct(*([1] * 7))        # never dereferenced: rejected on the host
    st = tb.lib().tblr_tessellate_noalloc(ctypes.byref(prob), ctypes.c_void_p(1),
                                          ctypes.byref(lay_struct), None)
    assert st == tb.TBLR_EINVAL
    assert b"8388608" in tb.lib().tblr_last_error()
