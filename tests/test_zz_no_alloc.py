"""GPU test of ceed_dot_noalloc, the dot product that allocates nothing.

Some callers cannot allocate device memory (a library handed only vector pointers by an
application that owns every device buffer, or a loop where cudaMalloc/cudaFree would stall the
device or could fail mid-solve).  This entry point keeps its partial sums in a static device array
inside the library.  Its result is compared with the workspace-based ceed_dot on the same inputs,
within the relative tolerance of the other dot-product test, over two calls in a row (which must
also agree with each other bit for bit).  The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_dot_noalloc_matches_dot():
    import paper_2109_05072_gb300 as ceed
    assert torch.cuda.is_available()
    for n in (1, 8193, 3_000_017):
        x = torch.from_numpy(synthetic.uniform(n, seed=21)).cuda()
        y = torch.from_numpy(synthetic.uniform(n, seed=22)).cuda()
        work = torch.empty(ceed.ceed_dot_workspace_bytes(n), dtype=torch.uint8, device="cuda")
        ref = torch.empty(1, dtype=torch.float64, device="cuda")
        ceed.ceed_dot(x, y, ref, work)
        got = []
        for _ in range(2):
            out = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
            ceed.ceed_dot_noalloc(x, y, out)
            got.append(out.item())
        r = ref.item()
        assert got[0] == got[1]
        assert abs(got[0] - r) <= 1e-12 * np.sqrt(n) * max(1.0, abs(r))
        exact = float(np.dot(x.cpu().numpy(), y.cpu().numpy()))
        assert abs(got[0] - exact) <= 1e-12 * np.sqrt(n) * max(1.0, abs(exact))
    # a length beyond the static scratch is rejected before any kernel runs
    big = ceed.ceed_dot_noalloc_max_n() + 1
    st = ceed._lib.ceed_dot_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), big,
                                    ctypes.c_void_p(ref.data_ptr()), None)
    assert st == ceed.CEED_ERR_INVALID
    assert "static scratch" in ceed.ceed_last_error()
