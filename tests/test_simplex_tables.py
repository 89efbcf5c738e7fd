"""The library's host helper for the degree-p tetrahedron (ceed_simplex_basis: Silvester basis, conical
Gauss-Jacobi rule, written in C++) against the oracle's independent numpy construction.  Host code
only: no GPU is touched."""
import numpy as np
import pytest

from oracle import simplex as sx


@pytest.mark.parametrize("p", range(1, 8))
def test_simplex_tables_match_oracle(p):
    ceed = pytest.importorskip("paper_2109_05072_gb300")
    for q in (p, p + 1, min(p + 2, 10)):
        interp, grad, qw, qref = ceed.ceed_simplex_basis(p, q)
        s = sx.SimplexSpace(p, q)
        assert ceed.ceed_simplex_sizes(p, q) == (s.nd, s.nq)
        np.testing.assert_allclose(qref, s.XI, atol=1e-15)
        np.testing.assert_allclose(qw, s.W, rtol=1e-13, atol=1e-18)
        np.testing.assert_allclose(interp, s.Phi, atol=1e-13 * p)
        np.testing.assert_allclose(grad, s.dPhi, atol=5e-14 * p ** 3)


def test_simplex_sizes_reject_out_of_range():
    ceed = pytest.importorskip("paper_2109_05072_gb300")
    with pytest.raises(ceed.CeedError):
        ceed.ceed_simplex_sizes(8, 3)
    with pytest.raises(ceed.CeedError):
        ceed.ceed_simplex_sizes(3, 11)
