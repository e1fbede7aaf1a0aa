"""The largest-magnitude split rule (keep="largest", the other rule of
section 4) through the C ABI against the oracle.

Each irregular column keeps its diagonal and the p-1 entries of largest
magnitude (equal magnitudes to the smaller row; p largest without a stored
diagonal). Checked: A~, U and J bit for bit against the oracle on the 2D,
3D and Zipf-count workloads and on a matrix with many equal magnitudes
(values on a half-integer grid, explicit zeros included); then Procedure *
with this rule: per-system BiCGStab iterations within +-1 of the oracle's
solves with its own split and M, rr < eps, and x against a dense solve.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
import workloads as W
from gpu_helpers import lib, need_gpu, to_dev, to_scipy, torch

pytestmark = pytest.mark.gpu

SPAI = dict(delta=0.4, mn=5, max_aug=10)


def _ties():
    A = sp.csc_matrix(W.random_sparse_dominant(600, 5, 4, 120, 7).A)
    A.data = np.round(A.data * 2.0) / 2.0  # many equal magnitudes, some stored zeros
    return A


CASES = {
    "2d": (lambda: W.convdiff2d_irregular().A, {}),
    "3d": (lambda: W.convdiff3d_irregular(m=16, s=3, density=0.2).A, {}),
    "zipf": (lambda: W.zipf_columns(n=2000).A, dict(abs_tau=200.0)),
    "ties": (_ties, {}),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_split_largest_matches_oracle(case):
    need_gpu()
    sai = lib()
    make, kw = CASES[case]
    A = sp.csc_matrix(make())
    A.sort_indices()
    J, p, _ = O.detect(A, **kw)
    At, U = O.split(A, J, p, rule=1)
    At, U = sp.csc_matrix(At), sp.csc_matrix(U)
    sp_ = sai.split(to_dev(A), keep="largest", **kw)
    assert sp_.s == len(J) and sp_.p == p
    Atg, Ug, Jg = sp_.arrays()
    G = to_scipy(Atg)
    assert np.array_equal(G.indptr, At.indptr) and np.array_equal(G.indices, At.indices)
    assert np.array_equal(G.data, At.data)
    ucp, uri, uv = (t.cpu().numpy() for t in Ug)
    assert np.array_equal(ucp, U.indptr) and np.array_equal(uri, U.indices) and np.array_equal(uv, U.data)
    assert np.array_equal(Jg.cpu().numpy(), np.asarray(J))
    # the nearest rule differs on these matrices
    At0, _ = O.split(A, J, p, rule=0)
    assert len(J) == 0 or (sp.csc_matrix(At0) != At).nnz > 0


def test_procedure_with_largest_rule():
    need_gpu()
    sai = lib()
    P = W.convdiff2d_irregular()
    A = sp.csc_matrix(P.A)
    x, iters, rep = sai.solve(to_dev(A), torch.as_tensor(P.b, device="cuda"), krylov="bicgstab", eps=1e-8,
                              keep="largest", **SPAI)
    assert rep["status"] == sai.SAI_OK and rep["rr"] < 1e-8
    J, p, _ = O.detect(A)
    At, U = O.split(A, J, p, rule=1)
    At, U = sp.csc_matrix(At), sp.csc_matrix(U)
    Mo = O.spai(At, **SPAI)[0]
    bn = np.linalg.norm(P.b)
    rhs = [P.b] + [U[:, t].toarray().ravel() for t in range(len(J))]
    thr = [0.5e-8 * bn] + [1e-8 * bn / (2 * np.sqrt(len(J)))] * len(J)
    for q, (r, th) in enumerate(zip(rhs, thr)):
        _, it, st = O.bicgstab(At, Mo, r, th)
        assert st == O.OK and abs(iters[q] - it) <= 1, (q, iters[q], it)
    xd = np.linalg.solve(A.toarray(), P.b)
    np.testing.assert_allclose(x.cpu().numpy(), xd, rtol=0, atol=1e-6)
