"""Zero-diagonal repair (section 5 preprocessing): sai_dmperm, sai_permute_rows
and sai_solve with zero_diag = 1, through the C ABI, against the oracle.

A maximum transversal is not unique: the tests compare its size (the
structural rank, unique) with the oracle's and check that the GPU's
transversal is valid (each matched column has a stored nonzero at its row,
no row used twice) and reproducible. The row permutation B = A(p,:) has one
answer for a given p: it is compared bit for bit with the oracle's, on
permutations drawn by the seeded generator. The repaired solve returns A's
unique solution: x is compared with the oracle's repaired solve (each with
its own transversal) and with the exact solution, rr < eps.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
import workloads as W
from gpu_helpers import lib, need_gpu, to_dev, torch

pytestmark = pytest.mark.gpu


def _dev(v):
    return torch.as_tensor(np.ascontiguousarray(v, dtype=np.float64), device="cuda")


def _check_transversal(A, p, rank):
    A = sp.csc_matrix(A)
    matched = p >= 0
    assert matched.sum() == rank
    assert len(np.unique(p[matched])) == rank
    rows = p[matched]
    cols = np.nonzero(matched)[0]
    assert np.all(np.asarray(A[rows, cols]).ravel() != 0)


def _random_pattern(n, density, seed, zero_vals=0):
    rng = np.random.default_rng(seed)
    M = sp.random(n, n, density=density, random_state=rng, format="csc")
    M.data = rng.standard_normal(M.data.size)
    M = W.canonical(M)
    if zero_vals and M.nnz:
        M.data[rng.choice(M.nnz, size=min(zero_vals, M.nnz), replace=False)] = 0.0
    return M


CASES = {
    "displaced_2d": lambda: W.rows_displaced(W.convdiff2d_irregular()).A,
    "displaced_3d_long": lambda: W.rows_displaced(W.convdiff3d_irregular(m=24, s=4, density=0.1)).A,
    "displaced_zipf": lambda: W.rows_displaced(W.zipf_columns(n=2000), frac=0.2).A,
    "random_singular": lambda: _random_pattern(3000, 0.0004, 11, zero_vals=50),
    "random_dense": lambda: _random_pattern(800, 0.02, 12, zero_vals=200),
    "zero_free_diagonal": lambda: W.convdiff2d_irregular().A,
    "one_by_one": lambda: W.canonical(sp.csc_matrix(np.array([[2.0]]))),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_dmperm_rank_matches_oracle_and_is_valid(case):
    need_gpu()
    sai = lib()
    A = CASES[case]()
    n = A.shape[0]
    p_o, rank_o = O.dmperm(A)
    p, rank, moved = sai.dmperm(to_dev(A))
    p = p.cpu().numpy()
    assert rank == rank_o, (rank, rank_o)
    _check_transversal(A, p, rank)
    assert moved == int((p != np.arange(n)).sum())
    if case == "zero_free_diagonal":
        assert moved == 0 and np.array_equal(p, np.arange(n))
    if case.startswith("displaced"):
        assert rank == n and moved > 0
    p2, _, _ = sai.dmperm(to_dev(A))
    assert np.array_equal(p2.cpu().numpy(), p)  # ties go to the smaller index: reproducible


def test_dmperm_empty_matrix():
    need_gpu()
    sai = lib()
    A = W.canonical(sp.csc_matrix((0, 0)))
    p, rank, moved = sai.dmperm(to_dev(A))
    assert rank == 0 and moved == 0 and p.numel() == 0


@pytest.mark.parametrize("case", ["displaced_2d", "displaced_3d_long", "displaced_zipf", "zipf20000"])
def test_permute_rows_bit_exact(case):
    need_gpu()
    sai = lib()
    A = W.zipf_columns(n=20000).A if case == "zipf20000" else CASES[case]()
    n = A.shape[0]
    rng = np.random.default_rng(13)
    for p in (rng.permutation(n).astype(np.int32), np.arange(n, dtype=np.int32)[::-1].copy()):
        B_o = O.permute_rows(A, p)
        B = sai.permute_rows(to_dev(A), torch.as_tensor(p, device="cuda"))
        assert np.array_equal(B.col_ptr.cpu().numpy(), B_o.indptr)
        assert np.array_equal(B.row_idx.cpu().numpy(), B_o.indices)
        assert np.array_equal(B.val.cpu().numpy(), B_o.data)


def test_permute_rows_rejects_non_permutations():
    need_gpu()
    sai = lib()
    A = CASES["displaced_2d"]()
    n = A.shape[0]
    for bad in (np.zeros(n, np.int32), np.full(n, n, np.int32), np.r_[np.arange(n - 1), -1].astype(np.int32)):
        with pytest.raises(sai.SaiError) as e:
            sai.permute_rows(to_dev(A), torch.as_tensor(bad, device="cuda"))
        assert e.value.status == sai.SAI_INVALID_ARG


@pytest.mark.parametrize("case,kw", [
    ("2d_spai", dict(sai="spai", delta=0.4, mn=5, max_aug=10, krylov="bicgstab", eps=1e-8)),
    ("3d_psai_gmres", dict(sai="psai", delta=0.3, tol=1e-3, tol_mode=1, lmax=10, krylov="gmres", restart=50,
                           eps=1e-10)),
])
def test_repaired_solve_against_oracle(case, kw):
    need_gpu()
    sai = lib()
    P = W.rows_displaced(W.convdiff2d_irregular() if case == "2d_spai" else
                         W.convdiff3d_irregular(m=16, s=3, density=0.2))
    assert (P.A.diagonal() == 0).sum() > 0
    x_o, it_o, rep_o, p_o = O.solve_repaired(P.A, P.b, **kw)
    x, iters, rep = sai.solve(to_dev(P.A), _dev(P.b), zero_diag=True, **kw)
    assert rep["status"] == sai.SAI_OK and rep["moved"] > 0
    assert rep["s"] == rep_o["s"] and rep["p"] == rep_o["p"]  # the split's counts ignore row order
    eps = kw["eps"]
    assert rep["rr"] < eps and rep_o["rr"] < eps
    x = x.cpu().numpy()
    # both solve A x = b to rr < eps; A's solution is the ones vector
    np.testing.assert_allclose(x, x_o, rtol=0, atol=1e3 * eps)
    np.testing.assert_allclose(x, np.ones(P.n), rtol=0, atol=1e3 * eps)


def test_repair_is_a_no_op_on_a_zero_free_diagonal():
    need_gpu()
    sai = lib()
    P = W.convdiff2d_irregular()
    kw = dict(delta=0.4, mn=5, max_aug=10, eps=1e-8)
    x0, it0, r0 = sai.solve(to_dev(P.A), _dev(P.b), **kw)
    x1, it1, r1 = sai.solve(to_dev(P.A), _dev(P.b), zero_diag=True, **kw)
    assert r1["moved"] == 0 and it0 == it1
    assert torch.equal(x0, x1)


def test_repair_reports_structural_singularity():
    need_gpu()
    sai = lib()
    P = W.rows_displaced(W.convdiff2d_irregular(m=20, s=1, density=0.3))
    A = P.A.copy()
    A.data[A.indptr[7]:A.indptr[8]] = 0.0  # column 7 keeps its pattern, but no entry counts
    assert O.dmperm(A)[1] == P.n - 1
    with pytest.raises(sai.SaiError) as e:
        sai.solve(to_dev(A), _dev(P.b), zero_diag=True)
    assert e.value.status == sai.SAI_SINGULAR


def test_split_create_rejects_the_flag():
    need_gpu()
    sai = lib()
    P = W.convdiff2d_irregular(m=12, s=1, density=0.3)
    L = sai.load()
    v = to_dev(P.A).view()
    prm = sai._SplitParams(10.0, -1.0, 0, 0, 0, 1)
    h = sai.C.c_void_p()
    assert L.sai_split_create(sai.C.byref(v), sai.C.byref(prm), None, sai.C.byref(h)) == sai.SAI_INVALID_ARG


def test_repaired_solve_full_size_64cubed():
    """The 64^3 system (n = 262144, ten 5 % columns) with 5 % of its rows
    cycled: rank n as the oracle finds it, valid transversal, and the
    repaired GMRES(50) solve meets eps = 1e-10 with A's solution."""
    need_gpu()
    sai = lib()
    P = W.rows_displaced(W.convdiff3d_irregular())
    p_o, rank_o = O.dmperm(P.A)
    p, rank, moved = sai.dmperm(to_dev(P.A))
    assert rank == rank_o == P.n and moved > 0
    _check_transversal(P.A, p.cpu().numpy(), rank)
    x, iters, rep = sai.solve(to_dev(P.A), _dev(P.b), sai="spai", delta=0.3, mn=5, max_aug=10, krylov="gmres",
                              restart=50, eps=1e-10, zero_diag=True)
    assert rep["status"] == sai.SAI_OK and rep["moved"] == moved and rep["s"] == 10
    assert rep["rr"] < 1e-10
    np.testing.assert_allclose(x.cpu().numpy(), np.ones(P.n), rtol=0, atol=1e-6)
