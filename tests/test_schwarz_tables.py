"""The library's host-side fast-diagonalization tables (its own Jacobi eigensolver in C++) against the
oracle's definition of the 1D extended operators (scipy's generalized eigensolver): no GPU needed."""
import numpy as np
import pytest

from oracle import schwarz as sw


@pytest.mark.parametrize("p", range(1, 9))
def test_fdm_tables_diagonalize_the_oracle_operators(p):
    import paper_2109_05072_gb300 as ceed
    S, lam = ceed.ceed_schwarz_fdm_1d(p)
    A, B = sw.reference_1d(p)
    np.testing.assert_allclose(S.T @ B @ S, np.eye(p + 1), atol=1e-12)
    np.testing.assert_allclose(S.T @ A @ S, np.diag(lam), atol=1e-11 * max(1.0, np.abs(lam).max()))
    _, lam_ref = sw.fdm_1d(p)
    np.testing.assert_allclose(np.sort(lam), np.sort(lam_ref), rtol=1e-12, atol=1e-13)


def test_fdm_tables_reject_out_of_range_orders():
    import paper_2109_05072_gb300 as ceed
    for p in (0, 9):
        with pytest.raises(ceed.CeedError):
            ceed.ceed_schwarz_fdm_1d(p)
