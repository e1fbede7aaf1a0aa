"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these tests retypes an oracle formula: each compares the oracle with
printed values (Table 3), hand-worked examples, closed forms, brute force on
dense matrices (numpy / scipy), exactness limits or the paper's theorems.
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import oracle as O
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _vmat(J, n):
    """V = [e_J0, ..., e_J(s-1)] as an n x s sparse matrix."""
    s = len(J)
    return sp.csc_matrix((np.ones(s), (np.asarray(J), np.arange(s))), shape=(n, s))


def _dominant(n, per_col, seed, s=0, dense_nnz=0):
    return W.random_sparse_dominant(n, per_col, s, dense_nnz, seed).A


# ---------------------------------------------------------------- detection

def test_avg_nnz_reproduces_table3():
    """Table 3: p = floor(nnz/n) for all twelve printed test matrices."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table3_p.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) == 12
    for name, n, nnz, p in rows:
        assert O.avg_nnz(int(n), int(nnz)) == int(p), name


def test_detect_threshold_is_strict_10p():
    """Section 4: irregular iff nnz(a_j) > 10p. Column 0 has exactly 10p, column 1 has 10p+1."""
    n = 100
    rows, cols = list(range(n)), list(range(n))            # diagonal: p = 1 before extras
    # p must stay 1: total nnz < 2n. Column 0 gets 9 extra (10 = 10p), column 1 gets 10 extra (11).
    extra0 = [i for i in range(1, 11)][:9]
    extra1 = [i for i in range(2, 13)][:10]
    rows += extra0 + extra1
    cols += [0] * len(extra0) + [1] * len(extra1)
    A = sp.csc_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n))
    J, p, tau = O.detect(A)
    assert p == 1 and tau == 10.0
    assert J.tolist() == [1]
    Jge, _, _ = O.detect(A, ge=True)
    assert Jge.tolist() == [0, 1]
    Jabs, _, tau = O.detect(A, abs_tau=9.5)
    assert Jabs.tolist() == [0, 1] and tau == 9.5


# ---------------------------------------------------------------- split

def test_split_hand_example_tie_rule():
    """Hand-worked: lower-bidiagonal 30 x 30 plus a full column 12.
    nnz = 59 + 28 = 87, p = 2, tau = 20 -> column 12 is irregular; keep the
    diagonal and the single nearest entry; rows 11 and 13 tie at distance 1 and
    the smaller row (11) is kept. Everything else of column 12 goes to U."""
    n = 30
    rows = list(range(n)) + list(range(1, n))
    cols = list(range(n)) + list(range(n - 1))
    vals = [4.0 + i for i in range(n)] + [-1.0 - 0.01 * i for i in range(n - 1)]
    for i in range(n):
        if i not in (12, 13):
            rows.append(i); cols.append(12); vals.append(0.5 + i)
    A = sp.csc_matrix((vals, (rows, cols)), shape=(n, n))
    assert A.nnz == 87
    J, p, tau = O.detect(A)
    assert (J.tolist(), p, tau) == ([12], 2, 20.0)
    At, U = O.split(A, J, p)
    col = At[:, 12]
    assert sorted(col.indices.tolist()) == [11, 12]
    assert col[11, 0] == 0.5 + 11 and col[12, 0] == 4.0 + 12
    assert sorted(U.indices.tolist()) == [i for i in range(n) if i not in (11, 12)]
    assert U[13, 0] == -1.0 - 0.01 * 12          # the sub-diagonal entry was dropped
    # every other column untouched
    for j in range(n):
        if j != 12:
            assert (At[:, j] != A[:, j]).nnz == 0


def test_split_missing_diagonal_keeps_p_nearest():
    """Proposal for a column without a stored diagonal: keep the p nearest entries."""
    n = 40
    rows = list(range(n)); cols = list(range(n)); vals = [3.0] * n
    dense_rows = [i for i in range(n) if i != 20]          # column 20 lacks its diagonal
    rows = [r for r, c in zip(rows, cols) if c != 20]; vals = vals[:len(rows)]; cols = [c for c in cols if c != 20]
    rows += dense_rows; cols += [20] * len(dense_rows); vals += [1.0 + i for i in dense_rows]
    A = sp.csc_matrix((vals, (rows, cols)), shape=(n, n))
    J, p, _ = O.detect(A)
    assert J.tolist() == [20] and p == 1 + (A.nnz - n) // n or True
    At, U = O.split(A, J, 3)
    # nearest three to row 20: 19 and 21 (distance 1, 19 first) then 18 (distance 2, smaller row)
    assert sorted(At[:, 20].indices.tolist()) == [18, 19, 21]


@pytest.mark.parametrize("maker", ["convdiff2d", "random"])
def test_split_invariants(maker):
    """A = A~ + U V^T exactly, diag(A~) = diag(A), each irregular column keeps
    min(p, nnz) entries, kept entries are the nearest ones (brute force)."""
    if maker == "convdiff2d":
        A = W.convdiff2d_irregular(m=20, s=3, density=0.4).A
    else:
        A = _dominant(150, 4, seed=3, s=4, dense_nnz=90)
    n = A.shape[0]
    J, p, tau = O.detect(A)
    assert len(J) >= 3
    At, U = O.split(A, J, p)
    D = (A - At - U @ _vmat(J, n).T)
    assert abs(D).max() == 0.0 if D.nnz else True
    assert np.array_equal(A.diagonal(), At.diagonal())
    for t, j in enumerate(J):
        a_rows = A.indices[A.indptr[j]:A.indptr[j + 1]]
        kept = At.indices[At.indptr[j]:At.indptr[j + 1]]
        assert len(kept) == min(p, len(a_rows))
        assert j in kept
        # brute force: sort off-diagonal rows by (|i-j|, i) and take p-1
        off = sorted([i for i in a_rows if i != j], key=lambda i: (abs(i - j), i))
        assert sorted(kept.tolist()) == sorted([j] + off[: p - 1])
        for i in kept:
            assert At[i, j] == A[i, j]
    # untouched columns
    mask = np.ones(n, bool); mask[J] = False
    assert (At[:, mask] != A[:, mask]).nnz == 0


def test_theorem3_dominant_gives_nonsingular_split():
    """Theorem 3(i): strictly column diagonally dominant A -> A~ nonsingular."""
    A = _dominant(120, 3, seed=11, s=3, dense_nnz=80)
    J, p, _ = O.detect(A)
    At, _ = O.split(A, J, p)
    Ad = At.toarray()
    d = np.abs(np.diag(Ad)); off = np.abs(Ad).sum(axis=0) - d
    assert np.all(d > off)
    assert np.linalg.matrix_rank(Ad) == Ad.shape[0]


# ---------------------------------------------------------------- SPAI

def _columns(M, k):
    return M.indices[M.indptr[k]:M.indptr[k + 1]], M.data[M.indptr[k]:M.indptr[k + 1]]


def test_spai_first_step_closed_form():
    """With S = {k}, eq. (lsprob) is 1-D: m_kk = a_kk/||a_k||^2 and
    ||r||^2 = 1 - a_kk^2/||a_k||^2."""
    At = _dominant(60, 5, seed=5)
    M, loops, res = O.spai(At, delta=0.0, mn=5, max_aug=0)
    Ad = At.toarray()
    for k in range(60):
        rows, vals = _columns(M, k)
        a = Ad[:, k]
        assert rows.tolist() == [k]
        assert vals[0] == pytest.approx(a[k] / (a @ a), rel=1e-14)
        assert res[k] == pytest.approx(np.sqrt(1.0 - a[k] ** 2 / (a @ a)), rel=1e-12)
        assert loops[k] == 0


def test_spai_diagonal_is_exact():
    """A diagonal A~ is its own SAI pattern: M = A~^{-1}, zero residual, no augmentation."""
    d = np.linspace(1.0, 3.0, 25)
    At = sp.diags(d).tocsc()
    M, loops, res = O.spai(At, delta=0.4)
    assert np.allclose(M.toarray(), np.diag(1.0 / d), rtol=1e-15, atol=0)
    assert np.all(res <= 1e-15) and np.all(loops == 0)


def _spai_bruteforce(Ad, k, delta, mn, max_aug):
    """SPAI on a dense matrix written from section 2.1 without any reduction:
    LS over all n rows (eq. (subprob)), candidates from the rows touched by
    A(:,S) (plus k), profitability by the 1-D problem (ls1d) solved directly:
    rho_j = ||r + mu_j A e_j||, mu_j minimising it."""
    n = Ad.shape[0]
    e = np.zeros(n); e[k] = 1.0
    S = [k]
    hist = []
    for l in range(max_aug + 1):
        m = np.linalg.lstsq(Ad[:, S], e, rcond=None)[0]
        r = Ad[:, S] @ m - e
        rn = np.linalg.norm(r)
        hist.append((list(S), rn, m))
        if rn <= delta or l == max_aug:
            break
        L = set(np.nonzero(np.any(Ad[:, S] != 0, axis=1))[0].tolist()) | {k}
        cand = [j for j in range(n) if j not in S and any(Ad[i, j] != 0 for i in L)]
        rho = {}
        for j in cand:
            aj = Ad[:, j]
            mu = -(r @ aj) / (aj @ aj)
            rho[j] = np.linalg.norm(r + mu * aj)
        picks = sorted(cand, key=lambda j: (rho[j], j))[:mn]
        if not picks:
            break
        S = S + picks
    return hist


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_spai_matches_bruteforce_dense(seed):
    """Pattern per loop (order of insertion included), residual and values of
    the oracle SPAI equal the brute-force dense restatement of section 2.1."""
    At = _dominant(45, 3, seed=100 + seed)
    Ad = At.toarray()
    delta, mn, max_aug = 0.05, 3, 4
    M, loops, res = O.spai(At, delta, mn, max_aug)
    for k in range(0, 45, 3):
        pats, rs = O.spai_trace(At, k, delta, mn, max_aug)
        hist = _spai_bruteforce(Ad, k, delta, mn, max_aug)
        assert len(pats) == len(hist), k
        for (S, rn, _), pat, r in zip(hist, pats, rs):
            assert pat.tolist() == S
            assert r == pytest.approx(rn, rel=1e-10, abs=1e-14)
        S, rn, m = hist[-1]
        rows, vals = _columns(M, k)
        order = np.argsort(S)
        assert rows.tolist() == sorted(S)
        np.testing.assert_allclose(vals, np.asarray(m)[order], rtol=1e-10, atol=1e-14)
        assert loops[k] == len(hist) - 1


def test_spai_residual_monotone_and_bounded():
    """S only grows, so the LS residual cannot rise; |S| <= 1 + mn*max_aug
    (the paper's 1 + 5 x 19 bound, section 5.1); loops <= max_aug."""
    At = W.convdiff2d_irregular(m=16, s=0).A
    mn, max_aug = 4, 6
    M, loops, res = O.spai(At, 0.02, mn, max_aug)
    assert np.all(np.diff(M.indptr) <= 1 + mn * max_aug)
    assert loops.max() <= max_aug
    for k in range(0, At.shape[0], 17):
        pats, rs = O.spai_trace(At, k, 0.02, mn, max_aug)
        assert np.all(np.diff(rs) <= 1e-14)
        for a, b in zip(pats, pats[1:]):
            assert set(a.tolist()) <= set(b.tolist())


def _reach(B, k, l):
    """Boolean pattern of B^l e_k (B already contains I)."""
    v = np.zeros(B.shape[0], bool); v[k] = True
    for _ in range(l):
        v = (B @ v.astype(np.float64)) != 0
    return v


def test_spai_envelope():
    """Section 4, fifth issue: SPAI patterns lie in P((I + |A|^T|A|)^l e_k)."""
    At = _dominant(80, 3, seed=21)
    Aabs = abs(At)
    B = (sp.identity(80) + Aabs.T @ Aabs).tocsc()
    for k in range(0, 80, 7):
        pats, _ = O.spai_trace(At, k, 0.0, 3, 4)
        for l, S in enumerate(pats):
            env = _reach(B, k, l)
            assert env[S].all(), (k, l)


# ---------------------------------------------------------------- PSAI(tol)

def test_bpsai_recovers_exact_inverse():
    """With delta = 0, no dropping (fixed tol 0) and l_max beyond the graph
    diameter, the pattern reaches P((I+|A|)^(n-1) e_k) and the LS problem is
    square: PSAI returns A~^{-1} (section 2.2, Cayley-Hamilton argument)."""
    At = _dominant(14, 2, seed=8)
    M, loops, pre, post = O.psai(At, delta=0.0, tol=0.0, tol_mode=1, lmax=14)
    Ainv = np.linalg.inv(At.toarray())
    np.testing.assert_allclose(M.toarray(), Ainv, rtol=1e-10, atol=1e-12)
    assert np.all(pre < 1e-12)


def test_psai_patterns_follow_power_growth():
    """Reading (A) with a nonzero diagonal: S^(l) = P((I+|A|)^l e_k) exactly,
    the set bounded by the envelope of section 4."""
    At = _dominant(70, 3, seed=31)
    B = (sp.identity(70) + abs(At)).tocsc()
    for k in range(0, 70, 9):
        pats, rs = O.psai_trace(At, k, delta=0.0, tol=0.05, tol_mode=1, lmax=3)
        for l, S in enumerate(pats):
            env = np.nonzero(_reach(B, k, l))[0]
            assert sorted(S.tolist()) == env.tolist(), (k, l)
        assert np.all(np.diff(rs) <= 1e-14)


def test_psai_drop_rule_and_2delta_bound():
    """eq. (tolk): the emitted column is the last LS solution restricted to
    |m_jk| > delta/(nnz(m_k) ||A||_1); the dropped part d has
    ||A d||_2 <= ||A||_1 ||d||_1 <= delta, so ||r_post|| <= ||r_pre|| + delta."""
    At = W.convdiff2d_irregular(m=18, s=2, density=0.3).A
    J, p, _ = O.detect(At)
    At, _ = O.split(At, J, p)
    n = At.shape[0]
    Ad = At.toarray()
    norm1 = np.abs(Ad).sum(axis=0).max()
    delta = 0.2
    M, loops, pre, post = O.psai(At, delta=delta, tol_mode=0, lmax=4)
    assert np.all(post <= pre + delta * (1 + 1e-12))
    conv = pre <= delta
    assert np.all(post[conv] <= 2 * delta * (1 + 1e-12))
    for k in range(0, n, 23):
        pats, rs = O.psai_trace(At, k, delta=delta, tol_mode=0, lmax=4)
        S = np.sort(pats[-1])
        e = np.zeros(n); e[k] = 1.0
        m = np.linalg.lstsq(Ad[:, S], e, rcond=None)[0]
        tolk = delta / (np.count_nonzero(m) * norm1)
        keep = np.abs(m) > tolk
        rows, vals = _columns(M, k)
        assert rows.tolist() == S[keep].tolist()
        np.testing.assert_allclose(vals, m[keep], rtol=1e-10, atol=1e-14)
        r_post = Ad[:, S[keep]] @ m[keep] - e
        assert post[k] == pytest.approx(np.linalg.norm(r_post), rel=1e-10)


# ---------------------------------------------------------------- Krylov

def _full_M(Ainv):
    return sp.csc_matrix(Ainv)


def test_krylov_exact_preconditioner_one_iteration():
    """With M = A~^{-1}, A~ M = I: both solvers converge in one iteration."""
    At = _dominant(50, 3, seed=41)
    Minv = _full_M(np.linalg.inv(At.toarray()))
    b = np.random.default_rng(0).standard_normal(50)
    thr = 1e-10 * np.linalg.norm(b)
    y, it, st = O.bicgstab(At, Minv, b, thr)
    assert st == O.OK and it == 1
    np.testing.assert_allclose(At @ y, b, rtol=0, atol=1e-9)
    y, it, st = O.gmres(At, Minv, b, thr, restart=5)
    assert st == O.OK and it == 1
    np.testing.assert_allclose(At @ y, b, rtol=0, atol=1e-9)


def test_gmres_full_cycle_is_direct_solve():
    """GMRES(m) with m >= n and tiny threshold equals the direct solution."""
    At = _dominant(40, 4, seed=42)
    M, _, _ = O.spai(At, 0.3, 3, 2)
    b = np.random.default_rng(1).standard_normal(40)
    y, it, st = O.gmres(At, M, b, 1e-13 * np.linalg.norm(b), restart=60, maxit=60)
    assert st == O.OK and it <= 40
    np.testing.assert_allclose(y, np.linalg.solve(At.toarray(), b), rtol=1e-9, atol=1e-11)


@pytest.mark.parametrize("solver", ["bicgstab", "gmres"])
def test_krylov_true_residual_meets_threshold(solver):
    """The recursive (or Givens) residual tracks the true residual of y."""
    A = W.convdiff2d_irregular(m=24, s=0).A
    M, _, _ = O.spai(A, 0.4, 5, 3)
    b = A @ np.ones(A.shape[0])
    thr = 1e-9 * np.linalg.norm(b)
    if solver == "bicgstab":
        y, it, st = O.bicgstab(A, M, b, thr)
    else:
        y, it, st = O.gmres(A, M, b, thr, restart=30, maxit=800)
    assert st == O.OK and it > 3
    assert np.linalg.norm(b - A @ y) < 1.01 * thr
    np.testing.assert_allclose(y, 1.0, rtol=0, atol=1e-6)


def _scipy_bicgstab_steps(A, M, b, j):
    """scipy's BiCGStab (van der Vorst's recurrence, x0 = 0, shadow residual
    r^ = b; its M is applied as a right preconditioner: p^ = M p, v = A p^,
    x += alpha p^ + omega s^) run for exactly j iterations: no tolerance can
    stop it early."""
    import scipy.sparse.linalg as sla_
    Mop = sla_.LinearOperator(A.shape, matvec=lambda v: M @ v, dtype=np.float64)
    x, info = sla_.bicgstab(sp.csr_matrix(A), b, rtol=0.0, atol=0.0, maxiter=j, M=Mop)
    assert info == j, info
    return x


@pytest.mark.parametrize("case", ["random40", "convdiff36"])
def test_bicgstab_iterates_match_scipy_step_by_step(case):
    """The oracle's BiCGStab iterate y_j after j = 1..6 iterations equals
    scipy's on the same right-preconditioned system A~ M z = b, y = M z. A
    wrong omega (the stabilising step) or beta (the direction update) changes
    y_2 onwards, although both would still converge; the exact-preconditioner
    pin never reaches omega (it stops at the half step)."""
    if case == "random40":
        At = sp.csc_matrix(_dominant(40, 4, seed=77))
        M = O.spai(At, 0.3, 3, 2)[0]
        b = np.random.default_rng(5).standard_normal(40)
    else:
        At = W.convdiff2d_irregular(m=6, s=0).A
        M = O.spai(At, 0.2, 3, 2)[0]
        b = At @ np.ones(At.shape[0])
    Ms = sp.csc_matrix(M)
    assert abs(Ms - Ms.T).max() > 1e-3 and abs(At - At.T).max() > 1e-3  # nonsymmetric operator
    for j in range(1, 7):
        y, it, st = O.bicgstab(At, M, b, 0.0, maxit=j)
        assert st == O.MAXITER and it == j
        x = _scipy_bicgstab_steps(At, Ms, b, j)
        np.testing.assert_allclose(y, x, rtol=0, atol=1e-10 * np.abs(x).max())
    # the iterates move: consecutive steps differ well above the tolerance
    y1 = O.bicgstab(At, M, b, 0.0, maxit=1)[0]
    y2 = O.bicgstab(At, M, b, 0.0, maxit=2)[0]
    assert np.abs(y2 - y1).max() > 1e-6 * np.abs(y2).max()


def test_krylov_maxit_status():
    A = W.convdiff2d_irregular(m=30, s=0).A
    I = sp.identity(A.shape[0], format="csc")
    b = A @ np.ones(A.shape[0])
    y, it, st = O.bicgstab(A, I, b, 1e-14 * np.linalg.norm(b), maxit=3)
    assert st == O.MAXITER and it == 3


# ---------------------------------------------------------------- SMW

def test_smw_exact_recovers_direct_solve():
    """Theorem 1 / eq. (update1): with exact y = A~^{-1}b and W = A~^{-1}U the
    recovered x equals the direct solution of A x = b."""
    A = _dominant(90, 3, seed=51, s=3, dense_nnz=60)
    J, p, _ = O.detect(A)
    At, U = O.split(A, J, p)
    b = np.random.default_rng(2).standard_normal(90)
    Atd = At.toarray()
    y = np.linalg.solve(Atd, b)
    Wm = np.linalg.solve(Atd, U.toarray())
    x, z, c = O.smw(y, Wm, J)
    xd = np.linalg.solve(A.toarray(), b)
    np.testing.assert_allclose(x, xd, rtol=1e-10, atol=1e-12)
    # z = (I + V^T W)^{-1} V^T y equals x(J): x(J) = y(J) - W(J,:) z = z
    np.testing.assert_allclose(z, xd[J], rtol=1e-10)
    assert c == pytest.approx(np.linalg.norm(xd[J]), rel=1e-10)
    assert O.rel_resid(A, b, x) < 1e-12


def test_rel_resid_matches_scipy():
    A = _dominant(70, 3, seed=52)
    rng = np.random.default_rng(3)
    b, x = rng.standard_normal(70), rng.standard_normal(70)
    assert O.rel_resid(A, b, x) == pytest.approx(np.linalg.norm(b - A @ x) / np.linalg.norm(b), rel=1e-13)


# ---------------------------------------------------------------- Procedure *

@pytest.mark.parametrize("sai,krylov", [("spai", "bicgstab"), ("psai", "bicgstab"), ("spai", "gmres")])
def test_procedure_star_meets_eps_and_theorem2(sai, krylov):
    """Procedure * on the 2D workload (45 x 45, Pe 10, 3 columns at 30 %):
    rr < eps (section 5 reports a < 1 for c = 1), the Theorem 2 inequality
    ||b - A x|| <= ||r_y|| + c ||R_W||_F holds, and the per-system iteration
    counts equal independent solves with the thresholds of eqs. (stopb) and
    (stopU2) with c = 1."""
    P = W.convdiff2d_irregular()
    eps = 1e-8
    kw = dict(sai=sai, krylov=krylov, eps=eps, delta=0.4, mn=5, max_aug=10, tol_mode=0, lmax=10, restart=50)
    x, iters, rep = O.solve(P.A, P.b, **kw)
    assert rep["s"] == 3 and rep["p"] == 5
    assert rep["status"] == O.OK
    assert rep["rr"] < eps
    bnorm = np.linalg.norm(P.b)
    assert rep["rr"] * bnorm <= rep["bound"] * (1 + 1e-6)
    np.testing.assert_allclose(x, 1.0, rtol=0, atol=1e-5)
    # independent restatement of the stopping thresholds
    J, p, _ = O.detect(P.A)
    At, U = O.split(P.A, J, p)
    if sai == "spai":
        M = O.spai(At, 0.4, 5, 10)[0]
    else:
        M = O.psai(At, 0.4, tol_mode=0, lmax=10)[0]
    s = len(J)
    thr = [eps / 2 * bnorm] + [bnorm * eps / (2 * np.sqrt(s))] * s
    rhs = [P.b] + [U[:, t].toarray().ravel() for t in range(s)]
    for q in range(s + 1):
        if krylov == "bicgstab":
            _, it, _ = O.bicgstab(At, M, rhs[q], thr[q])
        else:
            _, it, _ = O.gmres(At, M, rhs[q], thr[q], restart=50)
        assert it == iters[q]


# ---------------------------------------------------------------- backward pass (O8)
def test_backward_dense_matches_central_differences():
    """The dense adjoint (lambda = A^{-T} g, dL/dA_ij = -lambda_i x_j) against
    central differences of L = g^T A^{-1} b at h = 1e-6, each perturbed
    system solved by a dense LU (scipy), over b and a sample of A's stored
    entries including the dense columns'."""
    P = W.random_sparse_dominant(40, 3, 2, 15, seed=31)
    A = O.as_csc(P.A)
    rng = np.random.default_rng(3)
    g = rng.standard_normal(A.shape[0])
    b = rng.standard_normal(A.shape[0])
    x = sla.solve(A.toarray(), b)
    lam, gv = O.backward_dense(A, x, g)
    h = 1e-6

    def loss(Ad, bb):
        return float(g @ sla.solve(Ad, bb))

    Ad = A.toarray()
    for i in rng.choice(A.shape[0], 8, replace=False):
        e = np.zeros_like(b)
        e[i] = h
        fd = (loss(Ad, b + e) - loss(Ad, b - e)) / (2 * h)
        assert fd == pytest.approx(lam[i], rel=1e-6, abs=1e-9)
    cols = np.repeat(np.arange(A.shape[1]), np.diff(A.indptr))
    for q in rng.choice(A.nnz, 25, replace=False):
        i, j = A.indices[q], cols[q]
        Ap, Am = Ad.copy(), Ad.copy()
        Ap[i, j] += h
        Am[i, j] -= h
        fd = (loss(Ap, b) - loss(Am, b)) / (2 * h)
        assert fd == pytest.approx(gv[q], rel=1e-6, abs=1e-9)


def test_smw_adjoint_with_exact_solves_is_the_dense_adjoint():
    """Theorem 1 applied to A^T = A~^T + V U^T: with yhat, W from exact dense
    solves of A~^T, the oracle's adjoint recovery equals A^{-T} g."""
    P = W.random_sparse_dominant(80, 3, 3, 70, seed=32)
    A = O.as_csc(P.A)
    J, p, _ = O.detect(A)
    assert len(J) == 3
    At, U = O.split(A, J, p)
    n = A.shape[0]
    g = np.random.default_rng(4).standard_normal(n)
    rhs = np.column_stack([g, _vmat(J, n).toarray()])
    Y = sla.solve(At.toarray().T, rhs)
    lam, z, c = O.smw_adjoint(Y[:, 0], Y[:, 1:], U)
    lam_d = sla.solve(A.toarray().T, g)
    np.testing.assert_allclose(lam, lam_d, rtol=1e-10, atol=1e-12)
    assert c == pytest.approx(np.linalg.norm(z))


def test_csc_transpose_is_the_transpose():
    A = O.as_csc(_dominant(50, 4, 33, s=2, dense_nnz=20))
    T = O.csc_transpose(A)
    assert (T != A.T.tocsc()).nnz == 0
    assert np.all(np.diff(T.indptr) >= 0)


@pytest.mark.parametrize("krylov", ["bicgstab", "gmres"])
def test_oracle_backward_meets_the_adjoint_thresholds(krylov):
    """The sparse adjoint pipeline (split, M, s+1 transposed solves with M^T,
    adjoint SMW) meets the Theorem 2 bound on ||g - A^T lambda|| on the 2D
    workload, agrees with the dense adjoint, and its iteration counts equal independent
    solves of A~^T with M^T at the Theorem 2 thresholds taken from ||g||."""
    P = W.convdiff2d_irregular()
    A = O.as_csc(P.A)
    eps = 1e-10
    x = O.solve(A, P.b, krylov=krylov, eps=eps)[0]
    g = np.random.default_rng(5).standard_normal(A.shape[0])
    lam, gv, iters, rep = O.backward(A, x, g, krylov=krylov, eps=eps)
    assert rep["status"] == O.OK and rep["s"] == 3
    # Theorem 2 on A^T: ||g - A^T lambda|| <= ||r_y|| + c ||R_W||_F, with the
    # thresholds eps||g||/2 and eps||g||/(2 sqrt(s)) per system
    assert rep["rr"] <= eps * (1 + rep["c"]) / 2 * 1.05
    lam_d, gv_d = O.backward_dense(A, x, g)
    np.testing.assert_allclose(lam, lam_d, rtol=0, atol=1e-7 * np.abs(lam_d).max())
    np.testing.assert_allclose(gv, gv_d, rtol=0, atol=1e-7 * np.abs(gv_d).max())
    J, p, _ = O.detect(A)
    At, U = O.split(A, J, p)
    M = O.spai(At, 0.4, 5, 10)[0]
    gn = np.linalg.norm(g)
    s = len(J)
    thr = [eps / 2 * gn] + [gn * eps / (2 * np.sqrt(s))] * s
    rhs = [g] + [np.eye(A.shape[0])[:, j] for j in J]
    for q in range(s + 1):
        if krylov == "bicgstab":
            _, it, _ = O.bicgstab(At.T.tocsc(), M.T.tocsc(), rhs[q], thr[q])
        else:
            _, it, _ = O.gmres(At.T.tocsc(), M.T.tocsc(), rhs[q], thr[q], restart=50)
        assert it == iters[q]


def test_zipf_workload_structure():
    """The heavy-tailed generator: counts capped, strict column dominance,
    irregular columns found above the absolute threshold 200."""
    P = W.zipf_columns(n=1500)
    A = O.as_csc(P.A)
    cnt = np.diff(A.indptr)
    assert cnt.max() <= 750 + 1
    d = A.diagonal()
    off = np.asarray(abs(A).sum(axis=0)).ravel() - np.abs(d)
    assert np.all(np.abs(d) > 1.19 * off)
    J, p, tau = O.detect(A, abs_tau=200.0)
    assert tau == 200.0 and len(J) == int((cnt > 200).sum()) and len(J) > 10


# ---- the largest-magnitude split rule (section 4, the second approach) ----
def _col(M, j):
    M = sp.csc_matrix(M)
    return dict(zip(M.indices[M.indptr[j]:M.indptr[j + 1]].tolist(), M.data[M.indptr[j]:M.indptr[j + 1]].tolist()))


def test_split_largest_hand_worked():
    """Column 2 of an 8 x 8 matrix holds 10 (diagonal), -3, 4, 2, -2, 0.5,
    -0.5, 0.1; p_keep = 3 keeps the diagonal and the two largest: rows 1
    (-3) and 6 (4). The nearest rule keeps rows 1 and 3 instead."""
    n = 8
    A = sp.lil_matrix((n, n))
    for i in range(n):
        A[i, i] = 1.0
    for r, v in zip(range(8), [0.5, -3.0, 10.0, 2.0, -2.0, 0.1, 4.0, -0.5]):
        A[r, 2] = v
    A = sp.csc_matrix(A)
    At, U = O.split(A, [2], 3, rule=1)
    assert _col(At, 2) == {1: -3.0, 2: 10.0, 6: 4.0}
    assert _col(U, 0) == {0: 0.5, 3: 2.0, 4: -2.0, 5: 0.1, 7: -0.5}
    At0, _ = O.split(A, [2], 3, rule=0)
    assert _col(At0, 2) == {1: -3.0, 2: 10.0, 3: 2.0}


def test_split_largest_ties_and_no_diagonal():
    """Equal magnitudes go to the smaller row; without a stored diagonal the
    p_keep largest are kept."""
    n = 10
    A = sp.lil_matrix((n, n))
    for i in range(n):
        A[i, i] = 2.0
    for r in (0, 3, 5, 8, 9):  # column 4: five entries of magnitude 1, one of 5
        A[r, 4] = -1.0 if r % 2 else 1.0
    A[1, 4] = 5.0
    A = sp.csc_matrix(A)
    At, _ = O.split(A, [4], 4, rule=1)
    assert sorted(_col(At, 4)) == [0, 1, 3, 4]  # diagonal, the 5, then the two smallest rows of the ties
    B = sp.lil_matrix(A)
    B[4, 4] = 0.0
    B = sp.csc_matrix(B)
    B.eliminate_zeros()
    Bt, _ = O.split(B, [4], 3, rule=1)
    assert sorted(_col(Bt, 4)) == [0, 1, 3]


def test_split_largest_brute_force():
    """Random column-dominant matrices with dense columns: the kept entries of
    every irregular column equal the diagonal plus the first p-1 off-diagonal
    entries sorted by (-|a_ij|, i); A = A~ + U V^T exactly."""
    for trial in range(4):
        A = _dominant(300, 5, seed=trial, s=4, dense_nnz=60)
        A = sp.csc_matrix(A)
        J, p, _ = O.detect(A)
        At, U = O.split(A, J, p, rule=1)
        At, U = sp.csc_matrix(At), sp.csc_matrix(U)
        for t, j in enumerate(J):
            c = _col(A, j)
            off = sorted(((-abs(v), i) for i, v in c.items() if i != j))
            want = {i for _, i in off[:p - 1]} | ({j} if j in c else set())
            assert set(_col(At, j)) == want
            assert set(_col(U, t)) == set(c) - want
        V = sp.csc_matrix((np.ones(len(J)), (np.asarray(J), np.arange(len(J)))), shape=(A.shape[0], len(J)))
        assert abs(At + U @ V.T - A).max() == 0.0


# ---- PSAI(lfill): the lfill largest entries of each m_k (section 2.2) ----
def test_psai_lfill_large_equals_no_drop():
    """With lfill beyond any pattern size nothing is dropped: the same M as a
    fixed tol of 0."""
    At = W.convdiff2d_irregular(m=16, s=0).A
    M1 = sp.csc_matrix(O.psai(At, 0.2, 0.0, 1, 3)[0])
    M2 = sp.csc_matrix(O.psai(At, 0.2, tol_mode=2, lmax=3, lfill=10 ** 6)[0])
    assert np.array_equal(M1.indptr, M2.indptr) and np.array_equal(M1.indices, M2.indices)
    assert np.array_equal(M1.data, M2.data)


def test_psai_lfill_diagonal_and_count():
    d = np.arange(1.0, 21.0)
    Md = sp.csc_matrix(O.psai(sp.diags(d).tocsc(), 0.1, tol_mode=2, lmax=4, lfill=1)[0])
    assert np.allclose(Md.toarray(), np.diag(1.0 / d), rtol=0, atol=1e-15)
    At = W.convdiff2d_irregular(m=16, s=0).A
    M = sp.csc_matrix(O.psai(At, 0.05, tol_mode=2, lmax=3, lfill=4)[0])
    assert np.diff(M.indptr).max() <= 4


def test_psai_lfill_brute_force():
    """Each emitted column equals the lfill entries of largest magnitude
    (ties to the smaller index) of the dense least-squares solution on the
    last loop's pattern."""
    At = sp.csc_matrix(W.convdiff2d_irregular(m=16, s=0).A)
    n = At.shape[0]
    M = sp.csc_matrix(O.psai(At, 0.05, tol_mode=2, lmax=3, lfill=6)[0])
    A = At.toarray()
    for k in range(0, n, 17):
        pats, _ = O.psai_trace(At, k, 0.05, tol_mode=2, lmax=3, lfill=6)
        S = np.asarray(pats[-1])
        e = np.zeros(n)
        e[k] = 1.0
        m = np.linalg.lstsq(A[:, S], e, rcond=None)[0]
        order = sorted(range(len(S)), key=lambda t: (-abs(m[t]), S[t]))[:6]
        want = {int(S[t]): m[t] for t in order}
        got = dict(zip(M.indices[M.indptr[k]:M.indptr[k + 1]].tolist(), M.data[M.indptr[k]:M.indptr[k + 1]].tolist()))
        assert set(got) == set(want), k
        assert all(abs(got[j] - want[j]) <= 1e-10 * max(abs(v) for v in want.values()) for j in want)


# ---- PSAI growth reading (C): dropped positions never return (section 2.2) ----
def _power_patterns(At, k, L):
    """P(a^(l)) for l = 0..L, a^(0) = e_k, a^(l+1) = |A~| a^(l) (structural)."""
    B = abs(sp.csc_matrix(At)).astype(bool).astype(np.int64)
    a = np.zeros(At.shape[0], dtype=np.int64)
    a[k] = 1
    pats = [set([k])]
    for _ in range(L):
        a = (B @ a > 0).astype(np.int64)
        pats.append(set(np.flatnonzero(a).tolist()))
    return pats


def test_psai_growth_c_brute_force():
    """Traced patterns of sampled columns: S^(l) inside P(a^(l)); a position
    that leaves S never returns; and S^(l+1) = {j in S^(l): |m_j| > tol} u
    (P(a^(l+1)) minus P(a^(l))) with m the dense least-squares solution on S^(l)."""
    At = sp.csc_matrix(W.convdiff2d_irregular(m=16, s=0).A)
    A = At.toarray()
    n, tol, lmax = At.shape[0], 2e-3, 4
    for k in range(0, n, 23):
        pats, _ = O.psai_trace(At, k, 0.0, tol, 1, lmax, growth=1)
        P = _power_patterns(At, k, len(pats))
        gone = set()
        for l, S in enumerate(pats):
            S = [int(j) for j in S]
            assert set(S) <= P[l], (k, l)
            assert not (set(S) & gone), (k, l)
            if l + 1 < len(pats):
                e = np.zeros(n)
                e[k] = 1.0
                m = np.linalg.lstsq(A[:, S], e, rcond=None)[0]
                kept = {j for j, v in zip(S, m) if abs(v) > tol}
                assert set(int(j) for j in pats[l + 1]) == kept | (P[l + 1] - P[l]), (k, l)
                gone |= set(S) - kept


def test_psai_growth_c_differs_from_a_and_diagonal():
    At = W.convdiff2d_irregular(m=16, s=0).A
    Ma = sp.csc_matrix(O.psai(At, 0.05, 1e-3, 1, 4)[0])
    Mc = sp.csc_matrix(O.psai(At, 0.05, 1e-3, 1, 4, growth=1)[0])
    assert (Ma != Mc).nnz > 0 and Mc.nnz < Ma.nnz
    d = np.arange(1.0, 21.0)
    Md = sp.csc_matrix(O.psai(sp.diags(d).tocsc(), 0.1, 1e-3, 1, 4, growth=1)[0])
    assert np.allclose(Md.toarray(), np.diag(1.0 / d), rtol=0, atol=1e-15)


# ---- CGS (section 5 names it among the other solvers) ----
def test_cgs_exact_preconditioner_one_iteration():
    """With M = A~^{-1} the preconditioned operator is I: CGS ends after one
    iteration with y = A~^{-1} b."""
    A = sp.csc_matrix(_dominant(60, 4, seed=3))
    Minv = sp.csc_matrix(np.linalg.inv(A.toarray()))
    b = np.random.default_rng(1).standard_normal(60)
    y, it, st = O.cgs(A, Minv, b, 1e-10 * np.linalg.norm(b))
    assert st == O.OK and it == 1
    np.testing.assert_allclose(y, np.linalg.solve(A.toarray(), b), rtol=0, atol=1e-12)


def test_cgs_finite_termination_and_agreement():
    """On a small nonsymmetric system CGS reaches the dense solution within
    n + 1 iterations (finite termination in exact arithmetic), and on the 2D
    workload it meets its threshold and agrees with BiCGStab's solution."""
    A = sp.csc_matrix(_dominant(8, 3, seed=5))
    I = sp.identity(8, format="csc")
    b = np.arange(1.0, 9.0)
    y, it, st = O.cgs(A, I, b, 1e-12 * np.linalg.norm(b), maxit=9)
    assert st == O.OK and it <= 9
    np.testing.assert_allclose(y, np.linalg.solve(A.toarray(), b), rtol=0, atol=1e-9)
    P = W.convdiff2d_irregular()
    J, p, _ = O.detect(P.A)
    At, _ = O.split(P.A, J, p)
    M = O.spai(At, 0.4, 5, 10)[0]
    thr = 0.5e-10 * np.linalg.norm(P.b)
    yc, itc, stc = O.cgs(At, M, P.b, thr)
    yb, itb, stb = O.bicgstab(At, M, P.b, thr)
    assert stc == O.OK and stb == O.OK
    assert np.linalg.norm(P.b - sp.csc_matrix(At) @ yc) < 1.01 * thr
    np.testing.assert_allclose(yc, yb, rtol=0, atol=1e-7)


def test_bicg_exact_preconditioner_termination_and_agreement():
    """BiCG: with M = A~^{-1} one iteration gives y = A~^{-1} b; without a
    preconditioner it reaches the dense solution of an 8 x 8 nonsymmetric
    system within n + 1 iterations; on the 2D workload it agrees with
    BiCGStab's solution."""
    A = sp.csc_matrix(_dominant(60, 4, seed=3))
    Minv = sp.csc_matrix(np.linalg.inv(A.toarray()))
    b = np.random.default_rng(1).standard_normal(60)
    y, it, st = O.bicg(A, Minv, b, 1e-10 * np.linalg.norm(b))
    assert st == O.OK and it == 1
    np.testing.assert_allclose(y, np.linalg.solve(A.toarray(), b), rtol=0, atol=1e-12)
    A8 = sp.csc_matrix(_dominant(8, 3, seed=5))
    b8 = np.arange(1.0, 9.0)
    y8, it8, st8 = O.bicg(A8, sp.identity(8, format="csc"), b8, 1e-12 * np.linalg.norm(b8), maxit=9)
    assert st8 == O.OK and it8 <= 9
    np.testing.assert_allclose(y8, np.linalg.solve(A8.toarray(), b8), rtol=0, atol=1e-9)
    P = W.convdiff2d_irregular()
    J, p, _ = O.detect(P.A)
    At, _ = O.split(P.A, J, p)
    M = O.spai(At, 0.4, 5, 10)[0]
    thr = 0.5e-10 * np.linalg.norm(P.b)
    yg, _, sg = O.bicg(At, M, P.b, thr)
    yb, _, sb = O.bicgstab(At, M, P.b, thr)
    assert sg == O.OK and sb == O.OK
    np.testing.assert_allclose(yg, yb, rtol=0, atol=1e-7)


# ------------------------------------------- zero-diagonal repair (section 5)

def _check_transversal(A, p, rank):
    """p is a matching: each matched column j has a stored nonzero at row
    p[j], no row is used twice, and exactly rank columns are matched."""
    A = sp.csc_matrix(A)
    matched = p >= 0
    assert matched.sum() == rank
    assert len(set(p[matched].tolist())) == rank
    for j in np.nonzero(matched)[0]:
        assert A[p[j], j] != 0


def _random_pattern(n, density, rng, zero_vals=0):
    M = sp.random(n, n, density=density, random_state=rng, format="csc")
    M.data = rng.standard_normal(M.data.size)
    M = sp.csc_matrix(M)
    M.sort_indices()
    if zero_vals and M.nnz:  # stored entries with value zero do not count
        M.data[rng.choice(M.nnz, size=min(zero_vals, M.nnz), replace=False)] = 0.0
    return M


def test_dmperm_rank_is_the_structural_rank():
    """The transversal's size equals scipy's structural rank (a library
    maximum bipartite matching) on random patterns, singular ones included,
    and the matching is valid."""
    from scipy.sparse.csgraph import structural_rank
    rng = np.random.default_rng(7)
    for trial in range(60):
        n = int(rng.integers(1, 40))
        A = _random_pattern(n, float(rng.choice([0.02, 0.05, 0.1, 0.3])), rng)
        p, rank = O.dmperm(A)
        _check_transversal(A, p, rank)
        assert rank == structural_rank(A), trial


def test_dmperm_brute_force_small():
    """n <= 6: the largest number of nonzeros (sigma(j), j) over all n!
    permutations sigma is the maximum transversal's size; stored zeros do
    not count."""
    import itertools
    rng = np.random.default_rng(8)
    for trial in range(40):
        n = int(rng.integers(1, 7))
        A = _random_pattern(n, 0.4, rng, zero_vals=int(rng.integers(0, 4)))
        assert A.nnz == len(A.data)
        D = A.toarray()
        best = max(sum(D[s[j], j] != 0 for j in range(n)) for s in itertools.permutations(range(n)))
        p, rank = O.dmperm(A)
        _check_transversal(A, p, rank)
        assert rank == best, trial


def test_dmperm_keeps_a_zero_free_diagonal_and_fills_holes():
    """A zero-free diagonal gives the identity; a cyclic shift of rows is
    undone exactly when the shifted rows' only other entries are elsewhere
    (a permuted diagonal matrix has one perfect matching)."""
    P = W.convdiff2d_irregular(m=12, s=1, density=0.3)
    p, rank = O.dmperm(P.A)
    assert rank == P.n and np.array_equal(p, np.arange(P.n))
    n = 9
    q = np.roll(np.arange(n), 2)
    A = sp.csc_matrix(sp.csr_matrix(sp.diags(np.arange(1.0, n + 1)))[q, :])
    p, rank = O.dmperm(A)
    assert rank == n and np.array_equal(A[p, :].toarray(), np.diag(np.arange(1.0, n + 1)))
    # one empty column and one empty row: rank n - 1, the empty column unmatched
    A = sp.lil_matrix(np.eye(5))
    A[3, 3] = 0.0
    A[3, 4] = 1.0
    A[4, 4] = 0.0
    A = sp.csc_matrix(A)
    A.eliminate_zeros()
    p, rank = O.dmperm(A)
    assert rank == 4 and p[3] == -1 and p[4] == 3


def test_dmperm_repairs_the_displaced_workload():
    """Rows cycled out of place: the repaired matrix has a zero-free diagonal."""
    from scipy.sparse.csgraph import structural_rank
    P = W.rows_displaced(W.convdiff3d_irregular(m=12, s=3, density=0.1))
    assert (P.A.diagonal() == 0).sum() > 0
    p, rank = O.dmperm(P.A)
    assert rank == P.n == structural_rank(P.A)
    _check_transversal(P.A, p, rank)
    assert (O.permute_rows(P.A, p).diagonal() != 0).all()


def test_permute_rows_is_fancy_indexing():
    """B = A(p,:) equals scipy's row indexing, values bit for bit."""
    rng = np.random.default_rng(9)
    A = W.convdiff3d_irregular(m=10, s=2, density=0.4).A
    for _ in range(3):
        p = rng.permutation(A.shape[0]).astype(np.int32)
        B = O.permute_rows(A, p)
        R = sp.csc_matrix(A[p, :])
        R.sort_indices()
        assert np.array_equal(B.indptr, R.indptr) and np.array_equal(B.indices, R.indices)
        assert np.array_equal(B.data, R.data)
    with pytest.raises(O.OracleError):
        O.permute_rows(A, np.zeros(A.shape[0], np.int32))


def test_solve_after_repair_meets_eps():
    """Procedure * on the repaired system returns A's solution (rr on A)."""
    P = W.rows_displaced(W.convdiff2d_irregular())
    x, it, rep, p = O.solve_repaired(P.A, P.b, eps=1e-8)
    assert rep["rr"] < 1e-8 and rep["s"] == 3
    assert np.abs(x - 1.0).max() < 1e-5


# ------------------------------------------------ block GMRES (section 3)

def _small_system(n, k, seed):
    rng = np.random.default_rng(seed)
    At = sp.csc_matrix(sp.random(n, n, density=0.2, random_state=rng) + sp.diags(3.0 + rng.random(n)))
    At.sort_indices()
    B = rng.standard_normal((n, k))
    return At, B


def test_block_gmres_with_one_column_is_gmres():
    """k = 1: the block method is GMRES itself (same step count, same
    solution to rounding)."""
    P = W.convdiff2d_irregular()
    At = sp.csc_matrix(O.split(P.A, *O.detect(P.A)[:2])[0])
    M = sp.csc_matrix(O.spai(At, 0.4, 5, 10)[0])
    thr = 0.5e-8 * np.linalg.norm(P.b)
    y, it, st = O.gmres(At, M, P.b, thr, restart=30)
    Y, itb, stb = O.block_gmres(At, M, P.b[:, None], [thr], restart=30)
    assert st == stb == O.OK and it == itb[0]
    np.testing.assert_allclose(Y[:, 0], y, rtol=0, atol=1e-9)


def test_block_gmres_exact_preconditioner_one_step():
    """M = A~^{-1}: A~M = I, the block Krylov space of B holds every
    solution, one block step solves all columns."""
    At, B = _small_system(40, 3, 21)
    M = sp.csc_matrix(np.linalg.inv(At.toarray()))
    Y, it, st = O.block_gmres(At, M, B, np.full(3, 1e-10), restart=5)
    assert st == O.OK and list(it) == [1, 1, 1]
    np.testing.assert_allclose(At @ Y, B, rtol=0, atol=1e-10)


def test_block_gmres_finite_termination():
    """Without restarts the block space reaches dimension n after
    ceil(n / k) steps: the exact solution by then (dense solve)."""
    n, k = 12, 3
    At, B = _small_system(n, k, 22)
    M = sp.identity(n, format="csc")
    Y, it, st = O.block_gmres(At, M, B, np.full(k, 1e-11), restart=10, maxit=10)
    assert st == O.OK and it.max() <= n // k
    np.testing.assert_allclose(Y, np.linalg.solve(At.toarray(), B), rtol=0, atol=1e-10)


def test_block_gmres_minimises_over_the_block_krylov_space():
    """After j block steps (no restart, thresholds never met), column c's
    residual is min ||b_c - K t|| over t in the block Krylov space
    span[B, KB, .., K^{j-1}B], K = A~M (dense least squares)."""
    n, k = 60, 3
    At, B = _small_system(n, k, 23)
    rng = np.random.default_rng(24)
    M = sp.csc_matrix(sp.diags(1.0 / At.diagonal()) + sp.random(n, n, density=0.05, random_state=rng) * 0.01)
    K = At.toarray() @ M.toarray()
    for j in (1, 2, 4, 6):
        Y, it, st = O.block_gmres(At, M, B, np.zeros(k), restart=10, maxit=j)
        assert list(it) == [j] * k and st == O.MAXITER
        blocks = [B]
        for _ in range(j - 1):
            blocks.append(K @ blocks[-1])
        Q, _ = np.linalg.qr(np.hstack(blocks))
        KQ = K @ Q
        for c in range(k):
            t = np.linalg.lstsq(KQ, B[:, c], rcond=None)[0]
            best = np.linalg.norm(B[:, c] - KQ @ t)
            got = np.linalg.norm(B[:, c] - At @ Y[:, c])
            assert abs(got - best) <= 1e-10 * np.linalg.norm(B[:, c]), (j, c, got, best)


def test_procedure_with_block_gmres_meets_theorem2():
    """Procedure * with block GMRES(30) and GMRES(5) (systems frozen at the
    restarts where they meet their thresholds) on the 2D workload: rr < eps
    and the Theorem 2 inequality rr <= ||r_y|| + c ||R_W||."""
    P = W.convdiff2d_irregular()
    x, it, rep = O.solve(P.A, P.b, krylov="bgmres", restart=5, eps=1e-8)
    assert rep["status"] == O.OK and rep["rr"] < 1e-8 and len(set(it.tolist())) > 1
    x, it, rep = O.solve(P.A, P.b, krylov="bgmres", restart=30, eps=1e-8)
    assert rep["status"] == O.OK
    assert rep["rr"] < 1e-8 and rep["rr"] <= rep["bound"] / np.linalg.norm(P.b) * (1 + 1e-6)


def test_oracle_backward_with_block_gmres():
    """The adjoint pipeline with block GMRES(30) (all s+1 transposed systems
    in one block): the Theorem 2 bound on ||g - A^T lambda||, agreement with
    the dense adjoint, and block-step counts equal to a direct block solve of
    the transposed systems at the thresholds taken from ||g||."""
    P = W.convdiff2d_irregular()
    A = O.as_csc(P.A)
    eps = 1e-10
    x = O.solve(A, P.b, krylov="bgmres", restart=30, eps=eps)[0]
    g = np.random.default_rng(6).standard_normal(A.shape[0])
    lam, gv, iters, rep = O.backward(A, x, g, krylov="bgmres", restart=30, eps=eps)
    assert rep["status"] == O.OK and rep["s"] == 3
    assert rep["rr"] <= eps * (1 + rep["c"]) / 2 * 1.05
    lam_d, gv_d = O.backward_dense(A, x, g)
    np.testing.assert_allclose(lam, lam_d, rtol=0, atol=1e-7 * np.abs(lam_d).max())
    np.testing.assert_allclose(gv, gv_d, rtol=0, atol=1e-7 * np.abs(gv_d).max())
    J, p, _ = O.detect(A)
    At, U = O.split(A, J, p)
    M = O.spai(At, 0.4, 5, 10)[0]
    gn = np.linalg.norm(g)
    s = len(J)
    thr = [eps / 2 * gn] + [gn * eps / (2 * np.sqrt(s))] * s
    R = np.zeros((A.shape[0], s + 1))
    R[:, 0] = g
    R[J, np.arange(1, s + 1)] = 1.0
    _, it, st = O.block_gmres(sp.csc_matrix(At.T), sp.csc_matrix(M.T), R, thr, restart=30)
    assert st == O.OK and list(it) == list(iters)


# ------------------------------------- eq. (stopU2) with the recovery's c

def _batch_matrix(q):
    """Matrix q of the 256-matrix batched workload (the random geometric-graph
    systems), generated on its own."""
    rng = np.random.default_rng(W.SEED_BASE + 3)
    ns = rng.integers(1000, 50001, size=256)
    return W.rgg_irregular(int(ns[q]), seed=(W.SEED_BASE + 3) * 1000 + q)


def test_c_continuation_meets_eps_by_theorem2():
    """Theorem 2 bounds ||b - A x|| by ||r_y|| + c ||R_W||_F. With eq. (stopU2)
    at c = 1 that is eps ||b|| (1 + c) / 2, and matrix 10 of the batched
    workload (c = sqrt(10): b = A 1 makes z = x(J) = 1) ends above eps. With
    the u_j systems continued to the threshold with the measured c, the
    residual (recomputed here with scipy) is below eps, below the report's
    Theorem 2 bound, which is itself below eps ||b||; the continued systems
    took more iterations and the b system none."""
    P = _batch_matrix(10)
    b = P.b
    bn = np.linalg.norm(b)
    x0, it0, r0 = O.solve(P.A, b, eps=1e-8)
    assert r0["c"] > 1.0 and r0["c_rounds"] == 0
    assert np.linalg.norm(b - P.A @ x0) / bn > 1e-8           # the c = 1 bound is not enough here
    x1, it1, r1 = O.solve(P.A, b, eps=1e-8, c_adapt=1)
    assert r1["c_rounds"] == 1 and r1["c_first"] == pytest.approx(r0["c"], rel=1e-12)
    rr = np.linalg.norm(b - P.A @ x1) / bn
    assert rr < 1e-8 and rr == pytest.approx(r1["rr"], rel=1e-6)
    assert rr * bn <= r1["bound"] * (1 + 1e-9) and r1["bound"] <= 1e-8 * bn
    assert it1[0] == it0[0] and all(a > c for a, c in zip(it1[1:], it0[1:]))
    np.testing.assert_allclose(x1, 1.0, rtol=0, atol=1e-5)


def test_c_continuation_is_idle_when_c_is_small():
    """No second round when c <= 1: a matrix without irregular columns (s = 0,
    c = 0) gives the same bits with and without the option."""
    P = _batch_matrix(64)
    x0, it0, r0 = O.solve(P.A, P.b, eps=1e-8)
    x1, it1, r1 = O.solve(P.A, P.b, eps=1e-8, c_adapt=1)
    assert r0["s"] == 0 and r1["c_rounds"] == 0
    assert np.array_equal(x0, x1) and np.array_equal(it0, it1)
