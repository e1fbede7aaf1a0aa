"""CUDA path vs the oracle, element by element, on seeded inputs.

Bars: the split is bit-exact; M has the oracle's exact sparsity pattern with
values within 1e-10 relative (FP64 configs); Krylov iteration counts within
+-1; the recovered x meets ||b - A x||/||b|| < eps as the oracle's does.
Every call goes through the C ABI (ctypes binding of libsaismw.so).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
import workloads as W
from gpu_helpers import assert_same_pattern_and_values, lib, need_gpu, to_dev, to_scipy, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _split_both(A, **kw):
    sai = lib()
    h = sai.split(to_dev(A), **kw)
    At_d, U_d, J_d = h.arrays()
    J, p, tau = O.detect(A, mult=kw.get("thresh_mult", 10.0), abs_tau=kw.get("abs_tau", -1.0))
    At, U = O.split(A, J, p)
    return h, At_d, U_d, J_d, At, U, J, p


SPLIT_CASES = {
    "convdiff2d_45": lambda: W.convdiff2d_irregular().A,
    "convdiff3d_12": lambda: W.convdiff3d_irregular(m=12, s=4, density=0.3).A,
    "random_400": lambda: W.random_sparse_dominant(400, 4, 5, 120, seed=7).A,
    "no_dense": lambda: W.convdiff2d_irregular(m=10, s=0).A,
}


@pytest.mark.parametrize("case", sorted(SPLIT_CASES))
def test_split_bit_exact(case):
    A = SPLIT_CASES[case]()
    h, At_d, U_d, J_d, At, U, J, p = _split_both(A)
    assert (h.s, h.p) == (len(J), p)
    assert np.array_equal(J_d.cpu().numpy(), J)
    Atg = to_scipy(At_d)
    assert np.array_equal(Atg.indptr, At.indptr) and np.array_equal(Atg.indices, At.indices)
    assert np.array_equal(Atg.data, At.data)
    ucp, uri, uv = (t.cpu().numpy() for t in U_d)
    assert np.array_equal(ucp, U.indptr) and np.array_equal(uri, U.indices) and np.array_equal(uv, U.data)
    assert h.norm1_At == pytest.approx(abs(At).sum(axis=0).max(), rel=1e-14)


def test_split_missing_diagonal_and_user_tau():
    n = 300
    rng = np.random.default_rng(5)
    A = sp.lil_matrix((n, n))
    for j in range(n):
        A[j, j] = 4.0
        A[(j + 1) % n, j] = -1.0
    for j in (17, 150):
        rows = rng.choice(n, 80, replace=False)
        for i in rows:
            A[i, j] = rng.standard_normal()
    A[150, 150] = 0.0  # removes the stored diagonal of column 150
    A = sp.csc_matrix(A)
    A.eliminate_zeros()
    for kw in ({}, {"abs_tau": 30.0}):
        h, At_d, U_d, J_d, At, U, J, p = _split_both(A, **kw)
        assert np.array_equal(J_d.cpu().numpy(), J)
        Atg = to_scipy(At_d)
        assert np.array_equal(Atg.indices, At.indices) and np.array_equal(Atg.data, At.data)


def test_split_rejects_unsorted_rows():
    sai = lib()
    A = W.convdiff2d_irregular(m=8, s=0).A
    d = to_dev(A)
    ri = d.row_idx.clone()
    ri[0], ri[1] = ri[1].item(), ri[0].item()   # column 0 now unsorted
    bad = sai.CscMatrix(d.n, d.col_ptr, ri, d.val)
    with pytest.raises(sai.SaiError) as e:
        sai.split(bad)
    assert e.value.status == sai.SAI_INVALID_ARG


# ------------------------------------------------------------------ SPAI

SPAI_CASES = {
    # name: (matrix maker, delta, mn, max_aug)
    "convdiff2d_45_paper": (lambda: W.convdiff2d_irregular().A, 0.4, 5, 10),
    "convdiff3d_14": (lambda: W.convdiff3d_irregular(m=14, s=3, density=0.2).A, 0.3, 5, 10),
    "random_600_deep": (lambda: W.random_sparse_dominant(600, 4, 3, 150, seed=11).A, 0.1, 3, 6),
    "tier1_forced": (lambda: W.convdiff2d_irregular(m=20, s=2, density=0.2).A, 0.0, 5, 5),
    "tier2_forced": (lambda: W.convdiff2d_irregular(m=14, s=1, density=0.2).A, 0.0, 8, 9),
}


@pytest.mark.parametrize("case", sorted(SPAI_CASES))
def test_spai_matches_oracle(case):
    mk, delta, mn, max_aug = SPAI_CASES[case]
    A = mk()
    sai = lib()
    h = sai.split(to_dev(A))
    P = sai.build_spai(h, delta=delta, mn=mn, max_aug=max_aug)
    Md, loops_d, res_d, _ = P.arrays()
    J, p, _ = O.detect(A)
    At, _ = O.split(A, J, p)
    Mo, loops_o, res_o = O.spai(At, delta, mn, max_aug)
    assert_same_pattern_and_values(to_scipy(Md), Mo)
    assert np.array_equal(loops_d.cpu().numpy(), loops_o)
    np.testing.assert_allclose(res_d.cpu().numpy(), res_o, rtol=1e-9, atol=1e-13)
    assert P.n_c == int((res_o > delta).sum()) and P.l_m == int(loops_o.max())
    if case == "tier1_forced":
        assert P.n_tier[1] > 0
    if case == "tier2_forced":
        assert P.n_tier[2] > 0


def test_spai_diagonal_and_tiny():
    sai = lib()
    d = np.linspace(1.0, 2.0, 33)
    A = sp.diags(d).tocsc()
    P = sai.build_spai(sai.split(to_dev(A)), delta=0.4)
    Md, loops, res, _ = P.arrays()
    np.testing.assert_allclose(to_scipy(Md).toarray(), np.diag(1.0 / d), rtol=1e-15)
    assert int(loops.max()) == 0
    A1 = sp.csc_matrix(np.array([[3.0]]))
    P1 = sai.build_spai(sai.split(to_dev(A1)), delta=0.4)
    M1 = to_scipy(P1.arrays()[0]).toarray()
    assert M1[0, 0] == pytest.approx(1.0 / 3.0, rel=1e-15)


# ------------------------------------------------------------------ PSAI(tol)

PSAI_CASES = {
    # name: (maker, delta, tol, tol_mode, lmax)
    "convdiff2d_45_paper_tolk": (lambda: W.convdiff2d_irregular().A, 0.4, 0.0, 0, 10),
    "convdiff3d_14_fixed": (lambda: W.convdiff3d_irregular(m=14, s=3, density=0.2).A, 0.3, 1e-3, 1, 10),
    "random_500_tolk": (lambda: W.random_sparse_dominant(500, 3, 3, 120, seed=13).A, 0.2, 0.0, 0, 4),
    "growth_tiers": (lambda: W.convdiff2d_irregular(m=18, s=1, density=0.2).A, 0.0, 0.02, 1, 4),
}


@pytest.mark.parametrize("case", sorted(PSAI_CASES))
def test_psai_matches_oracle(case):
    mk, delta, tol, mode, lmax = PSAI_CASES[case]
    A = mk()
    sai = lib()
    h = sai.split(to_dev(A))
    P = sai.build_psai(h, delta=delta, tol=tol, tol_mode=mode, lmax=lmax)
    Md, loops_d, pre_d, post_d = P.arrays()
    J, p, _ = O.detect(A)
    At, _ = O.split(A, J, p)
    Mo, loops_o, pre_o, post_o = O.psai(At, delta, tol, mode, lmax)
    assert_same_pattern_and_values(to_scipy(Md), Mo)
    assert np.array_equal(loops_d.cpu().numpy(), loops_o)
    np.testing.assert_allclose(pre_d.cpu().numpy(), pre_o, rtol=1e-9, atol=1e-13)
    np.testing.assert_allclose(post_d.cpu().numpy(), post_o, rtol=1e-9, atol=1e-13)


# ------------------------------------------------------------------ Krylov + SMW

@pytest.mark.parametrize("method,restart", [("bicgstab", 30), ("gmres", 30), ("gmres", 20), ("cgs", 30),
                                            ("bicg", 30)])
def test_krylov_multi_rhs_matches_oracle(method, restart):
    """The s+1 systems in one call against the oracle's solves one by one;
    GMRES(20) is the restart length of the paper's remark on other solvers (section 5)."""
    sai = lib()
    P = W.convdiff2d_irregular()
    A = P.A
    h = sai.split(to_dev(A))
    Pc = sai.build_spai(h, delta=0.4, mn=5, max_aug=10)
    J, p, _ = O.detect(A)
    At, U = O.split(A, J, p)
    Mo, _, _ = O.spai(At, 0.4, 5, 10)
    s = len(J)
    B = np.zeros((A.shape[0], s + 1))
    B[:, 0] = P.b
    B[:, 1:] = U.toarray()
    bn = np.linalg.norm(P.b)
    thr = [0.5e-8 * bn] + [1e-8 * bn / (2 * np.sqrt(s))] * s
    meth = {"bicgstab": sai.BICGSTAB, "gmres": sai.GMRES, "cgs": sai.CGS, "bicg": sai.BICG}[method]
    X, iters, stat, st = sai.krylov_solve(h, Pc, torch.as_tensor(B, device="cuda"), thr, method=meth,
                                          restart=restart)
    X = X.cpu().numpy()
    assert st == sai.SAI_OK and all(v == 0 for v in stat)
    for q in range(s + 1):
        if method == "bicgstab":
            y, it, sto = O.bicgstab(At, Mo, B[:, q], thr[q])
        elif method == "cgs":
            y, it, sto = O.cgs(At, Mo, B[:, q], thr[q])
        elif method == "bicg":
            y, it, sto = O.bicg(At, Mo, B[:, q], thr[q])
        else:
            y, it, sto = O.gmres(At, Mo, B[:, q], thr[q], restart=restart)
        assert sto == O.OK
        assert abs(iters[q] - it) <= 1, (q, iters[q], it)
        assert np.linalg.norm(B[:, q] - At @ X[:, q]) < 1.01 * thr[q]
        np.testing.assert_allclose(X[:, q], y, rtol=0, atol=1e-7 * max(1.0, np.abs(y).max()))


def test_krylov_maxit_and_zero_rhs():
    sai = lib()
    A = W.convdiff2d_irregular(m=30, s=0).A
    h = sai.split(to_dev(A))
    Pc = sai.build_spai(h, delta=0.4, mn=1, max_aug=0)
    n = A.shape[0]
    B = np.zeros((n, 2))
    B[:, 0] = A @ np.ones(n)
    X, iters, stat, st = sai.krylov_solve(h, Pc, torch.as_tensor(B, device="cuda"), [1e-14, 1.0], maxit=3)
    assert st == sai.SAI_MAXITER and stat[0] == sai.SAI_MAXITER and iters[0] == 3
    assert stat[1] == sai.SAI_OK and iters[1] == 0  # zero right-hand side converges at once
    assert np.all(X[:, 1].cpu().numpy() == 0.0)


def test_smw_matches_oracle():
    sai = lib()
    A = W.random_sparse_dominant(300, 3, 4, 100, seed=3).A
    h = sai.split(to_dev(A))
    J, p, _ = O.detect(A)
    At, U = O.split(A, J, p)
    rng = np.random.default_rng(9)
    Y = rng.standard_normal((A.shape[0], len(J) + 1)) * 0.1
    x_d, c_d = sai.smw_recover(h, torch.as_tensor(Y, device="cuda"))
    x_o, z_o, c_o = O.smw(Y[:, 0], Y[:, 1:], J)
    np.testing.assert_allclose(x_d.cpu().numpy(), x_o, rtol=1e-12, atol=1e-14)
    assert c_d == pytest.approx(c_o, rel=1e-12)


@pytest.mark.parametrize("sai_kind,krylov", [("spai", "bicgstab"), ("psai", "bicgstab"), ("spai", "gmres")])
def test_procedure_star_matches_oracle(sai_kind, krylov):
    sai = lib()
    P = W.convdiff2d_irregular()
    kw = dict(sai=sai_kind, krylov=krylov, eps=1e-8, delta=0.4, mn=5, max_aug=10, tol_mode=0, lmax=10, restart=50)
    x_d, it_d, rep_d = sai.solve(to_dev(P.A), torch.as_tensor(P.b, device="cuda"), **kw)
    x_o, it_o, rep_o = O.solve(P.A, P.b, **kw)
    assert rep_d["s"] == rep_o["s"] and rep_d["nnz_M"] == rep_o["nnz_M"] and rep_d["l_m"] == rep_o["l_m"]
    assert all(abs(a - b) <= 1 for a, b in zip(it_d, it_o)), (it_d, list(it_o))
    assert rep_d["rr"] < 1e-8 and rep_o["rr"] < 1e-8
    assert rep_d["rr"] == pytest.approx(O.rel_resid(P.A, P.b, x_d.cpu().numpy()), rel=1e-6)
    np.testing.assert_allclose(x_d.cpu().numpy(), x_o, rtol=0, atol=1e-6)
    assert rep_d["c"] == pytest.approx(rep_o["c"], rel=1e-6)
