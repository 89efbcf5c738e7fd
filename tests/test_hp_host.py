"""The library's host-built conforming hp prolongation P (C++) against the oracle's (numpy), with no
GPU: the same true-dof numbering, the same rows (order groups ascending, elements ascending, nodes a
fastest), the same weights, and the same Dirichlet true dofs."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import hp as hpo


def _group_rows(h):
    rows = []
    for p in np.unique(h.orders):
        for e in np.nonzero(h.orders == p)[0]:
            rows.append(np.arange(h.row0[e], h.row0[e + 1]))
    return np.concatenate(rows)


@pytest.mark.parametrize("dims,choices,seed", [((3, 3, 2), [1, 2, 3, 4, 5], 0), ((2, 3, 2), [2, 5, 8], 1),
                                               ((4, 1, 1), [3, 7], 2), ((2, 2, 2), [4], 3)])
def test_host_prolongation_matches_oracle(dims, choices, seed):
    import paper_2109_05072_gb300 as ceed
    nx, ny, nz = dims
    orders = np.random.default_rng(seed).choice(choices, size=nx * ny * nz)
    h = hpo.HpSpace(nx, ny, nz, orders)
    n_true, rp, col, val, d = ceed.ceed_hp_prolongation(nx, ny, nz, orders)
    assert n_true == h.n_true
    P = sp.csr_matrix((val, col, rp), shape=(len(rp) - 1, n_true))
    ref = h.P[_group_rows(h)]
    assert P.shape == ref.shape
    diff = abs(P - ref)
    assert (diff.max() if diff.nnz else 0.0) <= 1e-13
    np.testing.assert_array_equal(d.astype(bool), h.boundary_mask())
    # every row is a partition of unity (constants are in every element space)
    np.testing.assert_allclose(np.asarray(P.sum(axis=1)).ravel(), 1.0, atol=1e-13)


def test_host_prolongation_rejects_bad_orders():
    import paper_2109_05072_gb300 as ceed
    with pytest.raises(ceed.CeedError):
        ceed.ceed_hp_prolongation(2, 1, 1, [3, 9])
    with pytest.raises(ceed.CeedError):
        ceed.ceed_hp_prolongation(2, 1, 1, [0, 2])
    with pytest.raises(ValueError):
        ceed.ceed_hp_prolongation(2, 2, 1, [1, 2])
