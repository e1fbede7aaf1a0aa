"""ctypes front end of the plain FP64 C oracle (``oracle/*.c``).

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package. The
product path (``paper_1211_6866_gb300``) never does, and shares no code with
it. Sparse matrices go in and come out as ``scipy.sparse.csc_matrix`` with
int64 column pointers, int32 row indices sorted inside each column.
"""
import ctypes as C
import os

import numpy as np
import scipy.sparse as sp

from .build import build_oracle

OK, BAD_INPUT, SINGULAR, MAXITER, BREAKDOWN, NOMEM = range(6)
STATUS_NAMES = {0: "OK", 1: "BAD_INPUT", 2: "SINGULAR", 3: "MAXITER", 4: "BREAKDOWN", 5: "NOMEM"}

_i32p = C.POINTER(C.c_int32)
_i64p = C.POINTER(C.c_int64)
_f64p = C.POINTER(C.c_double)


class _Csc(C.Structure):
    _fields_ = [("nrows", C.c_int32), ("ncols", C.c_int32), ("col_ptr", _i64p),
                ("row_idx", _i32p), ("val", _f64p)]


class _SpaiParams(C.Structure):
    _fields_ = [("delta", C.c_double), ("mn", C.c_int32), ("max_aug", C.c_int32), ("key_bits", C.c_int32)]


class _PsaiParams(C.Structure):
    _fields_ = [("delta", C.c_double), ("tol", C.c_double), ("tol_mode", C.c_int32), ("lmax", C.c_int32),
                ("lfill", C.c_int32), ("growth", C.c_int32)]


class _SolveParams(C.Structure):
    _fields_ = [("thresh_mult", C.c_double), ("abs_tau", C.c_double), ("sai", C.c_int32),
                ("spai", _SpaiParams), ("psai", _PsaiParams), ("krylov", C.c_int32),
                ("restart", C.c_int32), ("maxit", C.c_int32), ("eps", C.c_double), ("c_adapt", C.c_int32),
                ("reserved", C.c_int32)]


class _SolveReport(C.Structure):
    _fields_ = [("s", C.c_int32), ("p", C.c_int32), ("tau", C.c_double), ("nnz_At", C.c_int64),
                ("nnz_M", C.c_int64), ("n_c", C.c_int32), ("l_m", C.c_int32), ("iter_max", C.c_int32),
                ("status", C.c_int32), ("c", C.c_double), ("rr", C.c_double), ("bound", C.c_double),
                ("c_first", C.c_double), ("c_rounds", C.c_int32), ("reserved", C.c_int32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build_oracle()
        L = C.CDLL(path)
        L.orc_avg_nnz.restype = C.c_int32
        L.orc_avg_nnz.argtypes = [C.c_int32, C.c_int64]
        L.orc_rel_resid.restype = C.c_double
        L.orc_csc_free.restype = None
        _lib = L
    return _lib


def _ptr(a, t):
    return a.ctypes.data_as(t)


def as_csc(A):
    """Canonical CSC copy: sorted rows, int64 pointers, int32 rows, float64 values."""
    A = sp.csc_matrix(A)
    A.sort_indices()
    A.sum_duplicates()
    return A


class _In:
    """Keeps the numpy buffers alive for the lifetime of the ctypes struct."""

    def __init__(self, A):
        A = as_csc(A)
        self.indptr = np.ascontiguousarray(A.indptr, dtype=np.int64)
        self.indices = np.ascontiguousarray(A.indices, dtype=np.int32)
        self.data = np.ascontiguousarray(A.data, dtype=np.float64)
        self.s = _Csc(A.shape[0], A.shape[1], _ptr(self.indptr, _i64p), _ptr(self.indices, _i32p),
                      _ptr(self.data, _f64p))
        self.shape = A.shape
        self.nnz = int(A.nnz)


def _take(c):
    """Copy an oracle-allocated orc_csc into scipy and free the C arrays."""
    nnz = int(c.col_ptr[c.ncols]) if c.col_ptr else 0
    indptr = np.ctypeslib.as_array(c.col_ptr, shape=(c.ncols + 1,)).copy()
    if nnz:
        rows = np.ctypeslib.as_array(c.row_idx, shape=(nnz,)).copy()
        vals = np.ctypeslib.as_array(c.val, shape=(nnz,)).copy()
    else:
        rows = np.zeros(0, np.int32)
        vals = np.zeros(0, np.float64)
    lib().orc_csc_free(C.byref(c))
    return sp.csc_matrix((vals, rows, indptr), shape=(c.nrows, c.ncols))


class OracleError(RuntimeError):
    def __init__(self, what, status):
        super().__init__("%s: oracle status %s" % (what, STATUS_NAMES.get(status, status)))
        self.status = status


def _check(what, st):
    if st != OK:
        raise OracleError(what, st)


def avg_nnz(n, nnz):
    return int(lib().orc_avg_nnz(int(n), int(nnz)))


def detect(A, mult=10.0, abs_tau=-1.0, ge=False):
    a = _In(A)
    n = a.shape[1]
    J = np.zeros(max(n, 1), np.int32)
    s, p, tau = C.c_int32(), C.c_int32(), C.c_double()
    _check("detect", lib().orc_detect(C.byref(a.s), C.c_double(mult), C.c_double(abs_tau), int(ge),
                                      _ptr(J, _i32p), C.byref(s), C.byref(p), C.byref(tau)))
    return J[: s.value].copy(), p.value, tau.value


def split(A, J, p_keep, rule=0):
    """A = A~ + U V^T; rule 0 keeps the p_keep entries nearest to the diagonal,
    rule 1 the diagonal and the p_keep-1 largest in magnitude (section 4)."""
    a = _In(A)
    J = np.ascontiguousarray(J, dtype=np.int32)
    At, U = _Csc(), _Csc()
    _check("split", lib().orc_split_rule(C.byref(a.s), _ptr(J, _i32p), len(J), int(p_keep), int(rule), C.byref(At),
                                         C.byref(U)))
    return _take(At), _take(U)


def _cols(n, cols):
    if cols is None:
        return 0, n
    return int(cols[0]), int(cols[1])


def spai(At, delta, mn=5, max_aug=10, key_bits=20, cols=None):
    """Returns (M csc, loops[n], res[n]); entries outside ``cols`` are 0 / empty."""
    a = _In(At)
    n = a.shape[1]
    c0, c1 = _cols(n, cols)
    prm = _SpaiParams(delta, mn, max_aug, key_bits)
    loops = np.zeros(max(n, 1), np.int32)
    res = np.zeros(max(n, 1), np.float64)
    M = _Csc()
    _check("spai", lib().orc_spai(C.byref(a.s), C.byref(prm), c0, c1, C.byref(M), _ptr(loops, _i32p),
                                  _ptr(res, _f64p)))
    return _take(M), loops[:n], res[:n]


def _trace(fn, At, prm, k, cap):
    a = _In(At)
    S_hist = np.zeros(cap, np.int32)
    S_off = np.zeros(256, np.int32)
    res = np.zeros(256, np.float64)
    nl = fn(C.byref(a.s), C.byref(prm), int(k), _ptr(S_hist, _i32p), cap, _ptr(S_off, _i32p), _ptr(res, _f64p))
    if nl < 0:
        raise OracleError("trace", -nl)
    pats = [S_hist[S_off[l]: S_off[l + 1]].copy() for l in range(nl)]
    return pats, res[:nl].copy()


def spai_trace(At, k, delta, mn=5, max_aug=10, key_bits=20, cap=1 << 20):
    """Pattern S^(l) (in insertion order) and LS residual for every loop of column k."""
    return _trace(lib().orc_spai_trace, At, _SpaiParams(delta, mn, max_aug, key_bits), k, cap)


def psai(At, delta, tol=0.0, tol_mode=0, lmax=10, cols=None, lfill=0, growth=0):
    """Returns (M csc, loops[n], res_pre[n], res_post[n]). tol_mode 2: PSAI(lfill);
    growth 1: pattern growth reading (C)."""
    a = _In(At)
    n = a.shape[1]
    c0, c1 = _cols(n, cols)
    prm = _PsaiParams(delta, tol, tol_mode, lmax, lfill, growth)
    loops = np.zeros(max(n, 1), np.int32)
    pre = np.zeros(max(n, 1), np.float64)
    post = np.zeros(max(n, 1), np.float64)
    M = _Csc()
    _check("psai", lib().orc_psai(C.byref(a.s), C.byref(prm), c0, c1, C.byref(M), _ptr(loops, _i32p),
                                  _ptr(pre, _f64p), _ptr(post, _f64p)))
    return _take(M), loops[:n], pre[:n], post[:n]


def psai_trace(At, k, delta, tol=0.0, tol_mode=0, lmax=10, cap=1 << 22, lfill=0, growth=0):
    return _trace(lib().orc_psai_trace, At, _PsaiParams(delta, tol, tol_mode, lmax, lfill, growth), k, cap)


def bicgstab(At, M, rhs, thr, maxit=500):
    a, m = _In(At), _In(M)
    rhs = np.ascontiguousarray(rhs, dtype=np.float64)
    y = np.zeros_like(rhs)
    it = C.c_int32()
    st = lib().orc_bicgstab(C.byref(a.s), C.byref(m.s), _ptr(rhs, _f64p), C.c_double(thr), int(maxit),
                            _ptr(y, _f64p), C.byref(it))
    return y, it.value, st


def bicg(At, M, rhs, thr, maxit=500):
    a, m = _In(At), _In(M)
    rhs = np.ascontiguousarray(rhs, dtype=np.float64)
    y = np.zeros_like(rhs)
    it = C.c_int32()
    st = lib().orc_bicg(C.byref(a.s), C.byref(m.s), _ptr(rhs, _f64p), C.c_double(thr), int(maxit), _ptr(y, _f64p),
                        C.byref(it))
    return y, it.value, st


def cgs(At, M, rhs, thr, maxit=500):
    a, m = _In(At), _In(M)
    rhs = np.ascontiguousarray(rhs, dtype=np.float64)
    y = np.zeros_like(rhs)
    it = C.c_int32()
    st = lib().orc_cgs(C.byref(a.s), C.byref(m.s), _ptr(rhs, _f64p), C.c_double(thr), int(maxit), _ptr(y, _f64p),
                       C.byref(it))
    return y, it.value, st


def gmres(At, M, rhs, thr, restart=50, maxit=500):
    a, m = _In(At), _In(M)
    rhs = np.ascontiguousarray(rhs, dtype=np.float64)
    y = np.zeros_like(rhs)
    it = C.c_int32()
    st = lib().orc_gmres(C.byref(a.s), C.byref(m.s), _ptr(rhs, _f64p), C.c_double(thr), int(restart),
                         int(maxit), _ptr(y, _f64p), C.byref(it))
    return y, it.value, st


def block_gmres(At, M, B, thr, restart=50, maxit=500):
    """Block GMRES(restart) on A~ M Z = B (n x k), Y = M Z; thr: k thresholds.
    Returns (Y (n x k), block steps per column, status)."""
    a, m = _In(At), _In(M)
    B = np.asfortranarray(B, dtype=np.float64)
    n, k = B.shape
    thr = np.ascontiguousarray(thr, dtype=np.float64)
    Y = np.zeros((n, k), order="F")
    it = np.zeros(k, np.int32)
    st = lib().orc_block_gmres(C.byref(a.s), C.byref(m.s), int(k), _ptr(B, _f64p), _ptr(thr, _f64p), int(restart),
                               int(maxit), _ptr(Y, _f64p), _ptr(it, _i32p))
    if st == BAD_INPUT:
        raise OracleError("block_gmres", st)
    return Y, it, st


def smw(yhat, W, J):
    """W: (n, s) array. Returns (xhat, z, c)."""
    yhat = np.ascontiguousarray(yhat, dtype=np.float64)
    n = yhat.shape[0]
    J = np.ascontiguousarray(J, dtype=np.int32)
    s = len(J)
    Wc = np.asfortranarray(np.asarray(W, dtype=np.float64).reshape(n, s))
    x = np.zeros(n)
    z = np.zeros(max(s, 1))
    c = C.c_double()
    _check("smw", lib().orc_smw(n, s, _ptr(yhat, _f64p), Wc.ctypes.data_as(_f64p), _ptr(J, _i32p),
                                _ptr(x, _f64p), _ptr(z, _f64p), C.byref(c)))
    return x, z[:s], c.value


def rel_resid(A, b, x):
    a = _In(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    return float(lib().orc_rel_resid(C.byref(a.s), _ptr(b, _f64p), _ptr(x, _f64p)))


def solve(A, b, sai="spai", krylov="bicgstab", eps=1e-8, maxit=500, restart=50, thresh_mult=10.0,
          abs_tau=-1.0, delta=0.4, mn=5, max_aug=10, key_bits=20, tol=0.0, tol_mode=0, lmax=10, c_adapt=0):
    """Procedure * end to end. Returns (x, iters[s+1], report dict). c_adapt=1:
    when the recovery's c exceeds 1, the u_j systems are continued to
    eq. (stopU2) with that c and x is recovered again."""
    a = _In(A)
    n = a.shape[1]
    b = np.ascontiguousarray(b, dtype=np.float64)
    prm = _SolveParams(thresh_mult, abs_tau, 0 if sai == "spai" else 1,
                       _SpaiParams(delta, mn, max_aug, key_bits), _PsaiParams(delta, tol, tol_mode, lmax),
                       {"bicgstab": 0, "gmres": 1, "cgs": 2, "bicg": 3, "bgmres": 4}[krylov], restart, maxit, eps,
                       int(c_adapt), 0)
    x = np.zeros(n)
    iters = np.zeros(n + 1, np.int32)
    rep = _SolveReport()
    _check("solve", lib().orc_solve(C.byref(a.s), _ptr(b, _f64p), C.byref(prm), _ptr(x, _f64p),
                                    _ptr(iters, _i32p), C.byref(rep)))
    report = {f: getattr(rep, f) for f, _ in _SolveReport._fields_}
    return x, iters[: rep.s + 1].copy(), report


def dmperm(A):
    """Zero-diagonal repair of section 5: a maximum transversal of A.
    Returns (p, rank): p[j] = row matched to column j (-1 if unmatched)."""
    a = _In(A)
    n = a.shape[1]
    p = np.zeros(max(n, 1), np.int32)
    r = C.c_int32()
    _check("dmperm", lib().orc_dmperm(C.byref(a.s), _ptr(p, _i32p), C.byref(r)))
    return p[:n].copy(), r.value


def permute_rows(A, p):
    """B = A(p,:): row j of B is row p[j] of A."""
    a = _In(A)
    p = np.ascontiguousarray(p, dtype=np.int32)
    out = _Csc()
    _check("permute_rows", lib().orc_permute_rows(C.byref(a.s), _ptr(p, _i32p), C.byref(out)))
    return _take(out)


def solve_repaired(A, b, **kw):
    """Procedure * after the section 5 preprocessing: when A has a zero
    diagonal, solve A(p,:) x = b(p) with p = dmperm(A) (the solution x is
    A's). Returns (x, iters, report, p); report["rr"] is taken on A itself."""
    p, rank = dmperm(A)
    n = A.shape[0]
    if rank < n:
        raise OracleError("solve_repaired: structurally singular", SINGULAR)
    b = np.ascontiguousarray(b, dtype=np.float64)
    if np.array_equal(p, np.arange(n)):
        x, it, rep = solve(A, b, **kw)
    else:
        x, it, rep = solve(permute_rows(A, p), b[p], **kw)
    rep["rr"] = rel_resid(A, b, x)
    return x, it, rep, p


def csc_transpose(A):
    """A^T as a canonical CSC (the oracle's own transpose)."""
    a = _In(A)
    out = _Csc()
    _check("csc_transpose", lib().orc_csc_transpose(C.byref(a.s), C.byref(out)))
    return _take(out)


def smw_adjoint(yhat, W, U):
    """Theorem 1 on A^T = A~^T + V U^T. W: (n, s) array, U: n x s CSC.
    Returns (lambda, z, c)."""
    yhat = np.ascontiguousarray(yhat, dtype=np.float64)
    n = yhat.shape[0]
    u = _In(U)
    s = u.shape[1]
    Wc = np.asfortranarray(np.asarray(W, dtype=np.float64).reshape(n, s))
    lam = np.zeros(n)
    z = np.zeros(max(s, 1))
    c = C.c_double()
    _check("smw_adjoint", lib().orc_smw_adjoint(n, s, _ptr(yhat, _f64p), Wc.ctypes.data_as(_f64p), C.byref(u.s),
                                                _ptr(lam, _f64p), _ptr(z, _f64p), C.byref(c)))
    return lam, z[:s], c.value


def backward(A, x, g, sai="spai", krylov="bicgstab", eps=1e-8, maxit=500, restart=50, thresh_mult=10.0,
             abs_tau=-1.0, delta=0.4, mn=5, max_aug=10, key_bits=20, tol=0.0, tol_mode=0, lmax=10):
    """Backward pass of x = A^{-1} b (adjoint of Procedure *).
    Returns (lambda = dL/db, grad_vals aligned with A's CSC values, iters[s+1], report)."""
    a = _In(A)
    n = a.shape[1]
    x = np.ascontiguousarray(x, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    prm = _SolveParams(thresh_mult, abs_tau, 0 if sai == "spai" else 1,
                       _SpaiParams(delta, mn, max_aug, key_bits), _PsaiParams(delta, tol, tol_mode, lmax),
                       {"bicgstab": 0, "gmres": 1, "cgs": 2, "bicg": 3, "bgmres": 4}[krylov], restart, maxit, eps,
                       0, 0)
    lam = np.zeros(n)
    gv = np.zeros(a.nnz)
    iters = np.zeros(n + 1, np.int32)
    rep = _SolveReport()
    _check("backward", lib().orc_backward(C.byref(a.s), _ptr(x, _f64p), _ptr(g, _f64p), C.byref(prm),
                                          _ptr(lam, _f64p), _ptr(gv, _f64p), _ptr(iters, _i32p), C.byref(rep)))
    report = {f: getattr(rep, f) for f, _ in _SolveReport._fields_}
    return lam, gv, iters[: rep.s + 1].copy(), report


def backward_dense(A, x, g):
    """The plain definition, small n only: lambda = A^{-T} g by dense LU
    (numpy.linalg.solve), dL/dA_ij = -lambda_i x_j on A's stored pattern.
    Returns (lambda, grad_vals aligned with A's canonical CSC values)."""
    Ac = as_csc(A)
    lam = np.linalg.solve(Ac.toarray().T, np.asarray(g, dtype=np.float64))
    cols = np.repeat(np.arange(Ac.shape[1]), np.diff(Ac.indptr))
    return lam, -lam[Ac.indices] * np.asarray(x, dtype=np.float64)[cols]
