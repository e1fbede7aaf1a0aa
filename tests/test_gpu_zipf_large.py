"""The heavy-tailed Zipf-count workload at n = 1e5: forward and backward at scale.

n = 100000, column counts min(Zipf(1.5), 5000) at random rows, N(0,1) values,
a_jj = 1.2 sum |a_ij|; irregular columns are those above tau = 200, which
gives s = 5343 and p = 107, so every solve carries 5344 systems and the SMW
system is 5343 x 5343. SPAI(0.4, 5, 10), BiCGStab, FP64. Checked:
 - the split (s, p, J) and every column of M against the oracle's;
 - the 5344-system solve: sampled systems meet their Theorem 2 thresholds on
   the true residual (scipy), five systems give the same bits when solved on
   their own (a system's arithmetic does not depend on how many run with it),
   and four systems agree with the oracle's BiCGStab with its own M
   (iterations within +-1);
 - the SMW recovery (blocked LU for s > 256) against LAPACK on the same
   Y = [yhat, What], and Procedure * meeting the Theorem 2 bound on
   ||b - A x|| / ||b||;
 - the backward pass: ||g - A^T lambda|| within the Theorem 2 bound, dL/dA on
   A's pattern equal to -lambda_i x_j bit for bit, the adjoint SMW (U^T What
   for s > 256 and the blocked LU) against LAPACK on the transposed solves'
   Y, and central finite differences at h = 1e-6 of L = g^T x along b and on
   two stored entries of A, one in A~ and one in U.
The oracle's Procedure * on all 5344 systems takes about 15 minutes on one
core, so the whole-run comparisons are on sampled systems and on properties
that hold at any size.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
import workloads as W
from gpu_helpers import assert_same_pattern_and_values, lib, need_gpu, to_dev, to_scipy, torch

pytestmark = pytest.mark.gpu

SPAI = dict(delta=0.4, mn=5, max_aug=10)
TAU = 200.0
EPS = 1e-10


@pytest.fixture(scope="module")
def zipf():
    P = W.zipf_columns(n=100000)
    J, p, _ = O.detect(P.A, abs_tau=TAU)
    At, U = O.split(P.A, J, p)
    Mo = O.spai(At, **SPAI)[0]
    return P, np.asarray(J), p, sp.csc_matrix(At), sp.csc_matrix(U), sp.csc_matrix(Mo)


@pytest.fixture(scope="module")
def dev(zipf):
    """Device copies: A, its split and M (built once for the module)."""
    need_gpu()
    sai = lib()
    P = zipf[0]
    dA = to_dev(P.A)
    sp_ = sai.split(dA, abs_tau=TAU)
    Pc = sai.build_spai(sp_, **SPAI)
    return dA, sp_, Pc


def _rhs_block(P, U, s):
    """B = [b, u_1 .. u_s] (n x (s+1), row-major) assembled on the device."""
    n = P.n
    B = torch.zeros((n, s + 1), dtype=torch.float64, device="cuda")
    B[:, 0] = torch.as_tensor(P.b, device="cuda")
    coo = U.tocoo()
    B[torch.as_tensor(coo.row, device="cuda").long(), 1 + torch.as_tensor(coo.col, device="cuda").long()] = \
        torch.as_tensor(coo.data, device="cuda")
    return B


def _thresholds(bnorm, s):
    return [0.5 * EPS * bnorm] + [EPS * bnorm / (2.0 * np.sqrt(s))] * s


def test_zipf_1e5_split_and_build_match_oracle(zipf, dev):
    sai = lib()
    P, J, p, At, U, Mo = zipf
    dA, sp_, Pc = dev
    assert sp_.s == J.size == 5343 and sp_.p == p == 107
    Atg, Ug, Jg = sp_.arrays()
    assert np.array_equal(Jg.cpu().numpy(), J)
    Ag = to_scipy(Atg)
    assert np.array_equal(Ag.indptr, At.indptr) and np.array_equal(Ag.indices, At.indices)
    assert np.array_equal(Ag.data, At.data)
    assert_same_pattern_and_values(to_scipy(Pc.arrays()[0]), Mo)


def test_zipf_1e5_forward_5344_systems(zipf, dev):
    sai = lib()
    P, J, p, At, U, Mo = zipf
    dA, sp_, Pc = dev
    s = sp_.s
    B = _rhs_block(P, U, s)
    thr = _thresholds(np.linalg.norm(P.b), s)
    X, iters, status, st = sai.krylov_solve(sp_, Pc, B, thr, method=sai.BICGSTAB, maxit=500)
    assert st == sai.SAI_OK and all(v == sai.SAI_OK for v in status)
    rng = np.random.default_rng(5)
    sel = np.concatenate([[0], np.sort(rng.choice(np.arange(1, s + 1), 300, replace=False))])
    Xs = X[:, torch.as_tensor(sel, device="cuda")].cpu().numpy()
    Bs = B[:, torch.as_tensor(sel, device="cuda")].cpu().numpy()
    R = Bs - At @ Xs
    for q, c in enumerate(sel):
        # the recursive residual met thr; the true residual may differ by rounding
        assert np.linalg.norm(R[:, q]) < 1.5 * thr[c], (c, np.linalg.norm(R[:, q]), thr[c])
    # a system's arithmetic is the same whether it runs alone or with 5343 others
    few = [0, 1, 77, 2500, s]
    idx = torch.as_tensor(few, device="cuda")
    X2, it2, st2, _ = sai.krylov_solve(sp_, Pc, B[:, idx].contiguous(), [thr[c] for c in few],
                                       method=sai.BICGSTAB, maxit=500)
    assert it2 == [iters[c] for c in few]
    assert torch.equal(X2, X[:, idx])
    # four systems against the oracle's BiCGStab with its own M
    for c in (0, 1, 2500, s):
        rhs = B[:, c].cpu().numpy()
        yo, it_o, st_o = O.bicgstab(At, Mo, rhs, thr[c])
        assert st_o == O.OK and abs(iters[c] - it_o) <= 1, (c, iters[c], it_o)
        xc = X[:, c].cpu().numpy()
        assert np.abs(xc - yo).max() <= 1e-6 * np.abs(yo).max()


def test_zipf_1e5_smw_and_procedure(zipf, dev):
    sai = lib()
    P, J, p, At, U, Mo = zipf
    dA, sp_, Pc = dev
    s = sp_.s
    B = _rhs_block(P, U, s)
    Y, _, _, st = sai.krylov_solve(sp_, Pc, B, _thresholds(np.linalg.norm(P.b), s), method=sai.BICGSTAB)
    assert st == sai.SAI_OK
    del B
    x, c = sai.smw_recover(sp_, Y)
    # the same recovery from library routines: LAPACK for the s x s solve,
    # cuBLAS (through torch) for What z
    Jt = torch.as_tensor(J, device="cuda").long()
    Cm = np.eye(s) + Y[Jt, 1:].cpu().numpy()
    z = np.linalg.solve(Cm, Y[Jt, 0].cpu().numpy())
    xr = (Y[:, 0] - Y[:, 1:] @ torch.as_tensor(z, device="cuda")).cpu().numpy()
    del Y
    xg = x.cpu().numpy()
    assert np.abs(xg - xr).max() <= 1e-9 * np.abs(xr).max()
    assert abs(c - np.linalg.norm(z)) <= 1e-9 * np.linalg.norm(z)
    xs, iters, rep = sai.solve(dA, torch.as_tensor(P.b, device="cuda"), krylov="bicgstab", eps=EPS,
                               abs_tau=TAU, **SPAI)
    assert rep["status"] == sai.SAI_OK and rep["s"] == s
    rr = np.linalg.norm(P.b - P.A @ xs.cpu().numpy()) / np.linalg.norm(P.b)
    assert rr <= EPS * (1.0 + rep["c"]) / 2.0, (rr, rep["c"])
    assert abs(rr - rep["rr"]) <= 1e-3 * rr + 1e-15


def test_zipf_1e5_backward(zipf, dev):
    sai = lib()
    P, J, p, At, U, Mo = zipf
    dA, sp_, Pc = dev
    n, s = P.n, sp_.s
    A = sp.csc_matrix(P.A)
    b_d = torch.as_tensor(P.b, device="cuda")
    x, _, rep_f = sai.solve_with(dA, sp_, Pc, b_d, eps=EPS)
    assert rep_f["status"] == sai.SAI_OK
    g = np.random.default_rng(11).standard_normal(n)
    g_d = torch.as_tensor(g, device="cuda")
    lam, gv, iters_b, rep = sai.backward(dA, sp_, Pc, x, g_d, eps=EPS)
    assert rep["status"] == sai.SAI_OK
    lam_h, x_h, gv_h = lam.cpu().numpy(), x.cpu().numpy(), gv.cpu().numpy()
    # Theorem 2 on A^T: ||g - A^T lambda|| <= eps ||g|| (1 + c) / 2
    ra = np.linalg.norm(g - A.T @ lam_h) / np.linalg.norm(g)
    assert ra <= EPS * (1.0 + rep["c"]) / 2.0, (ra, rep["c"])
    # dL/dA_ij = -lambda_i x_j on A's stored pattern, the same product
    cols = np.repeat(np.arange(n), np.diff(A.indptr))
    assert np.array_equal(gv_h, -lam_h[A.indices] * x_h[cols])
    # the adjoint SMW against LAPACK on the transposed solves' Y = [yhat, What]
    Bt = torch.zeros((n, s + 1), dtype=torch.float64, device="cuda")
    Bt[:, 0] = g_d
    Bt[torch.as_tensor(J, device="cuda").long(), 1 + torch.arange(s, device="cuda")] = 1.0
    Yt, _, _, st = sai.krylov_solve(sp_, Pc, Bt, _thresholds(np.linalg.norm(g), s), method=sai.BICGSTAB,
                                    transpose=True)
    assert st == sai.SAI_OK
    del Bt
    # U^T Y by cuSPARSE (through torch; U's CSC arrays are the CSR of U^T),
    # the s x s solve by LAPACK, What z by cuBLAS
    Ut = torch.sparse_csr_tensor(torch.as_tensor(U.indptr, dtype=torch.int64),
                                 torch.as_tensor(U.indices, dtype=torch.int64),
                                 torch.as_tensor(U.data, dtype=torch.float64), size=(s, n)).to("cuda")
    UY = (Ut @ Yt).cpu().numpy()
    Cm = np.eye(s) + UY[:, 1:]
    z = np.linalg.solve(Cm, UY[:, 0])
    lr = (Yt[:, 0] - Yt[:, 1:] @ torch.as_tensor(z, device="cuda")).cpu().numpy()
    del Yt, Ut
    assert np.abs(lam_h - lr).max() <= 1e-8 * np.abs(lr).max()
    # central differences at h = 1e-6 of L = g^T x. For an approximate x with
    # residual r = b - A x, g^T x = g^T A^{-1} b - lambda^T r exactly, so the
    # raw difference quotient carries the solves' error term
    # -lambda^T (r+ - r-) / (2h). The test checks that the raw quotient
    # differs from the gradient by about that term, and that the quotient with
    # the term put back agrees with the gradient: to 1e-6 along b (an inner
    # product over all of lambda), to 1e-5 on single entries -lambda_i x_j,
    # taken from a forward and a backward pass at eps = 1e-12 (one component
    # of lambda or x carries more of its solve's error than their norms do).
    h = 1e-6
    x12, _, r12 = sai.solve_with(dA, sp_, Pc, b_d, eps=1e-12)
    assert r12["status"] == sai.SAI_OK
    lam12, gv12, _, rb12 = sai.backward(dA, sp_, Pc, x12, g_d, eps=1e-12)
    assert rb12["status"] == sai.SAI_OK
    lam_h, gv_h = lam12.cpu().numpy(), gv12.cpu().numpy()

    def L_and_r(Ad, As, bv):
        xx, _, r = sai.solve(Ad, torch.as_tensor(bv, device="cuda"), krylov="bicgstab", eps=1e-11, abs_tau=TAU,
                             **SPAI)
        assert r["status"] == sai.SAI_OK
        xv = xx.cpu().numpy()
        return float(g @ xv), bv - As @ xv

    def check_fd(Ad_p, As_p, b_p, Ad_m, As_m, b_m, an, tol):
        Lp, rp = L_and_r(Ad_p, As_p, b_p)
        Lm, rm = L_and_r(Ad_m, As_m, b_m)
        fd = (Lp - Lm) / (2 * h)
        term = float(lam_h @ (rp - rm)) / (2 * h)
        assert abs(fd + term - an) <= tol * abs(an), (fd, term, an)
        assert abs(fd - an) <= 1.5 * abs(term) + tol * abs(an), (fd, term, an)

    db = np.random.default_rng(12).standard_normal(n)
    check_fd(dA, A, P.b + h * db, dA, A, P.b - h * db, float(lam_h @ db), 1e-6)
    # one entry in a regular column (part of A~) and one dropped entry of an
    # irregular column (part of U), each where |lambda_i x_j| is largest
    Jset = set(J.tolist())
    reg = np.array([j for j in np.argsort(-np.abs(x_h))[:200] if j not in Jset][:20])
    cand = [(abs(lam_h[A.indices[q]] * x_h[j]), q) for j in reg for q in range(A.indptr[j], A.indptr[j + 1])]
    q_reg = max(cand)[1]
    jd = int(J[np.argmax(np.abs(x_h[J]))])
    t = int(np.searchsorted(J, jd))
    urows = set(U.indices[U.indptr[t]:U.indptr[t + 1]].tolist())
    cand = [(abs(lam_h[A.indices[q]]), q) for q in range(A.indptr[jd], A.indptr[jd + 1]) if A.indices[q] in urows]
    q_u = max(cand)[1]
    for q in (q_reg, q_u):
        Ap, Am = A.copy(), A.copy()
        Ap.data[q] += h
        Am.data[q] -= h
        check_fd(to_dev(Ap), Ap, P.b, to_dev(Am), Am, P.b, float(gv_h[q]), 1e-5)
