"""Seeded synthetic irregular sparse systems A x = b.

Input generation only: this module builds matrices and right-hand sides and
holds none of the method's arithmetic (no detection, splitting, SAI, Krylov or
SMW step). Both the CUDA path's tests/benchmark and the oracle read the same
generated arrays.

The paper evaluates on SuiteSparse circuit / device / CFD matrices that have a
few (nearly) dense columns on top of a 2-50 nonzeros-per-column body, with
b = A * ones and x0 = 0 (section 5, Tables 2 and 3). Those matrices are not
available here; these generators reproduce their structural traits on PDE
stencils and random graphs instead:

* ``convdiff2d`` / ``convdiff3d``: -Lap(u) + beta . grad(u) on the unit square /
  cube, first-order upwind, interior grid m^d, h = 1/(m+1), scaled by h^2 so
  the diagonal is 2d + h*sum(beta).
* ``add_dense_columns``: s columns at seeded positions receive extra nonzeros
  in Bernoulli(density) rows outside their stencil pattern, N(0,1) values,
  optionally rescaled so that sum|added| = scale * |a_jj| (keeps A column
  diagonally dominant, the class of Theorem 3(i)).

All matrices are returned as canonical scipy CSC (sorted rows, no
duplicates, int64 column pointers, int32 row indices, float64 values).
"""
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

SEED_BASE = 12116866  # arXiv 1211.6866


@dataclass
class Problem:
    name: str
    A: sp.csc_matrix
    b: np.ndarray
    params: dict = field(default_factory=dict)

    @property
    def n(self):
        return self.A.shape[0]


def canonical(A):
    A = sp.csc_matrix(A)
    A.sum_duplicates()
    A.sort_indices()
    A.indptr = A.indptr.astype(np.int64)
    A.indices = A.indices.astype(np.int32)
    A.data = A.data.astype(np.float64)
    return A


def _stencil(m, dim, beta):
    """Upwind convection-diffusion stencil on an m^dim interior grid (h^2-scaled)."""
    h = 1.0 / (m + 1)
    n = m ** dim
    idx = np.arange(n, dtype=np.int64)
    coords = [(idx // (m ** d)) % m for d in range(dim)]
    rows, cols, vals = [idx], [idx], [np.full(n, 2.0 * dim + h * float(np.sum(beta)))]
    for d in range(dim):
        stride = m ** d
        c = coords[d]
        lo = c > 0          # neighbour at -stride (upwind side for beta_d > 0)
        rows.append(idx[lo]); cols.append(idx[lo] - stride); vals.append(np.full(lo.sum(), -1.0 - h * beta[d]))
        hi = c < m - 1      # neighbour at +stride
        rows.append(idx[hi]); cols.append(idx[hi] + stride); vals.append(np.full(hi.sum(), -1.0))
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    return canonical(A)


def convdiff2d(m, pe=10.0):
    return _stencil(m, 2, (pe, pe))


def convdiff3d(m, pe=10.0):
    return _stencil(m, 3, (pe, pe, pe))


def add_dense_columns(A, s, density, rng, scale_to_diag=None, cols=None):
    """Make s columns of A dense: Bernoulli(density) new rows with N(0,1) values."""
    n = A.shape[0]
    if cols is None:
        cols = np.sort(rng.choice(n, size=s, replace=False))
    add_r, add_c, add_v = [], [], []
    Acsc = canonical(A)
    if len(cols) == 0:
        return Acsc, np.asarray(cols, dtype=np.int64)
    for j in cols:
        present = np.zeros(n, bool)
        present[Acsc.indices[Acsc.indptr[j]:Acsc.indptr[j + 1]]] = True
        pick = (rng.random(n) < density) & ~present
        rows = np.nonzero(pick)[0]
        v = rng.standard_normal(rows.size)
        if scale_to_diag is not None and rows.size:
            v *= scale_to_diag * abs(Acsc[j, j]) / np.abs(v).sum()
        add_r.append(rows); add_c.append(np.full(rows.size, j)); add_v.append(v)
    add = sp.coo_matrix((np.concatenate(add_v), (np.concatenate(add_r), np.concatenate(add_c))), shape=(n, n))
    return canonical(Acsc + add), np.asarray(cols, dtype=np.int64)


def _finish(name, A, params):
    A = canonical(A)
    b = A @ np.ones(A.shape[0])
    return Problem(name, A, np.ascontiguousarray(b), params)


def convdiff2d_irregular(m=45, pe=10.0, s=3, density=0.3, seed=SEED_BASE + 1):
    """2D 5-point convection-diffusion on m x m (n = m^2) plus s dense N(0,1) columns.

    Default sizes: the 45 x 45 grid (n = 2025), Peclet 10, 3 columns at 30 %."""
    rng = np.random.default_rng(seed)
    A, cols = add_dense_columns(convdiff2d(m, pe), s, density, rng)
    return _finish("convdiff2d_m%d_s%d" % (m, s), A, dict(m=m, pe=pe, s=s, density=density, seed=seed,
                                                        dense_cols=cols.tolist()))


def convdiff3d_irregular(m=64, pe=10.0, s=10, density=0.05, scale=0.5, seed=SEED_BASE + 2):
    """3D 7-point convection-diffusion on m^3 plus s dense columns scaled to the diagonal.

    Default sizes: the 64^3 grid (n = 262144), Peclet 10, 10 columns at 5 %,
    sum|added| = 0.5 |a_jj|."""
    rng = np.random.default_rng(seed)
    A, cols = add_dense_columns(convdiff3d(m, pe), s, density, rng, scale_to_diag=scale)
    return _finish("convdiff3d_m%d_s%d" % (m, s), A, dict(m=m, pe=pe, s=s, density=density, scale=scale,
                                                        seed=seed, dense_cols=cols.tolist()))


def rows_displaced(P, frac=0.05, seed=SEED_BASE + 6):
    """The system of P with a seeded cycle over round(frac*n) of its rows
    (A' = A(q,:), b' = b(q), same solution x): most of the moved rows put a
    zero on the diagonal, like the circuit matrices that section 5 permutes
    before the method."""
    rng = np.random.default_rng(seed)
    n = P.A.shape[0]
    m = max(2, int(round(frac * n)))
    R = rng.choice(n, size=m, replace=False)
    q = np.arange(n)
    q[R] = np.roll(R, -1)  # row R[t] of A' is row R[t+1] of A
    A = canonical(P.A[q, :])
    params = dict(P.params, displaced=m, frac=frac, seed_rows=seed)
    return Problem(P.name + "_zd%d" % m, A, np.ascontiguousarray(P.b[q]), params)


def random_sparse_dominant(n, nnz_per_col, s, dense_nnz, seed, dominance=1.2):
    """Small irregular test matrix: random sparse body, s dense columns, column dominance.

    Used by tests for generic (non-stencil, nonsymmetric) patterns."""
    rng = np.random.default_rng(seed)
    rows, cols, vals = [], [], []
    dense = np.sort(rng.choice(n, size=s, replace=False)) if s else np.zeros(0, np.int64)
    for j in range(n):
        k = dense_nnz if j in set(dense.tolist()) else nnz_per_col
        k = min(k, n - 1)
        r = rng.choice(np.delete(np.arange(n), j), size=k, replace=False)
        v = rng.standard_normal(k)
        rows += [r, [j]]
        cols += [np.full(k, j), [j]]
        vals += [v, [dominance * np.abs(v).sum() + 1.0]]
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    return _finish("random_n%d" % n, A, dict(n=n, s=s, dense_cols=dense.tolist(), seed=seed))


def zipf_columns(n=2000, alpha=1.5, cap=None, dominance=1.2, seed=SEED_BASE + 5):
    """Heavy-tailed irregular matrix (the Zipf-count workload): column j holds
    min(Zipf(alpha), cap) off-diagonal entries at distinct random rows with
    N(0,1) values, and a diagonal a_jj = dominance * sum_{i != j} |a_ij|
    (strict column dominance, so A~ stays nonsingular by Theorem 3(i)).
    Irregular columns are those above the absolute threshold tau = 200.
    The recipe is that of a 1e5-column system scaled to n; cap defaults to
    min(5000, n // 2)."""
    rng = np.random.default_rng(seed)
    cap = min(5000, n // 2) if cap is None else cap
    counts = np.minimum(rng.zipf(alpha, size=n), cap)
    rows, cols, vals = [], [], []
    for j in range(n):
        k = int(counts[j])
        r = rng.choice(n - 1, size=k, replace=False)
        r = r + (r >= j)  # skip the diagonal
        v = rng.standard_normal(k)
        rows += [r, [j]]
        cols += [np.full(k, j), [j]]
        vals += [v, [dominance * np.abs(v).sum() + 1e-3]]
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    return _finish("zipf_n%d" % n, A, dict(n=n, alpha=alpha, cap=cap, abs_tau=200.0, seed=seed))


def aniso9(m, eps=1e-3, theta_deg=30.0):
    """-div(K grad u) on an m x m interior grid, K = R diag(1, eps) R^T rotated by
    theta, the 9-point stencil (central second differences, the four-point
    cross difference for u_xy), Dirichlet boundary, h^2-scaled."""
    th = np.deg2rad(theta_deg)
    c, s = np.cos(th), np.sin(th)
    k11, k22, k12 = c * c + eps * s * s, s * s + eps * c * c, (1.0 - eps) * c * s
    n = m * m
    idx = np.arange(n, dtype=np.int64)
    x, y = idx % m, idx // m
    rows, cols, vals = [idx], [idx], [np.full(n, 2.0 * (k11 + k22))]
    for dx, dy, v in ((-1, 0, -k11), (1, 0, -k11), (0, -1, -k22), (0, 1, -k22),
                      (1, 1, -0.5 * k12), (-1, -1, -0.5 * k12), (1, -1, 0.5 * k12), (-1, 1, 0.5 * k12)):
        ok = (x + dx >= 0) & (x + dx < m) & (y + dy >= 0) & (y + dy < m)
        rows.append(idx[ok]); cols.append(idx[ok] + dx + dy * m); vals.append(np.full(ok.sum(), v))
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    return canonical(A)


def aniso9_irregular(m=1024, eps=1e-3, theta_deg=30.0, s=50, density=0.02, seed=SEED_BASE + 4):
    """The rotated anisotropic diffusion operator on m x m plus s dense N(0,1)
    columns. Default sizes: the 1024 x 1024 grid (n = 1048576), anisotropy
    1e-3 at 30 degrees, 50 columns at 2 %."""
    rng = np.random.default_rng(seed)
    A, cols = add_dense_columns(aniso9(m, eps, theta_deg), s, density, rng)
    return _finish("aniso9_m%d_s%d" % (m, s), A, dict(m=m, eps=eps, theta_deg=theta_deg, s=s, density=density,
                                                    seed=seed, dense_cols=cols.tolist()))


def rgg_irregular(n, seed, smax=20):
    """One matrix of the batched workload: the Laplacian D - Adj of a random
    geometric graph on n uniform points in the unit square with radius
    sqrt(8/(pi n)) (average degree 8); each stored off-diagonal perturbed by
    xi |a_ii|, xi ~ U(-0.1, 0.1) (nonsymmetric); then
    a_jj = max(a_jj, 1.05 sum_{i != j} |a_ij|, 1) (strict column dominance, so
    A~ stays nonsingular by Theorem 3(i); the 1 covers isolated points); plus
    s ~ U{1..smax} dense N(0,1) columns of density ~U[1%, 10%]."""
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(seed)
    pts = rng.random((n, 2))
    pairs = cKDTree(pts).query_pairs(np.sqrt(8.0 / (np.pi * n)), output_type="ndarray")
    i, j = pairs[:, 0], pairs[:, 1]
    deg = np.bincount(np.concatenate([i, j]), minlength=n).astype(np.float64)
    r = np.concatenate([i, j])
    c = np.concatenate([j, i])
    v = -1.0 + rng.uniform(-0.1, 0.1, size=r.size) * deg[r]
    A = sp.coo_matrix((np.concatenate([v, deg]), (np.concatenate([r, np.arange(n)]), np.concatenate([c, np.arange(n)]))),
                      shape=(n, n)).tocsc()
    A.sum_duplicates()

    def dominate(A, floor):
        d = A.diagonal()
        off = np.asarray(abs(A).sum(axis=0)).ravel() - np.abs(d)
        return sp.csc_matrix(A + sp.diags(np.maximum(np.maximum(np.abs(d), 1.05 * off), floor) - d))

    A = dominate(A, 1.0)
    s = int(rng.integers(1, smax + 1))
    A, cols = add_dense_columns(A, s, float(rng.uniform(0.01, 0.10)), rng)
    A = dominate(sp.csc_matrix(A, dtype=np.float64), 0.0)  # dominance again over the enlarged columns
    return _finish("rgg_n%d" % n, A, dict(n=n, s_generated=s, dense_cols=cols.tolist(), seed=seed))


def rgg_batch(count=256, nmin=1000, nmax=50000, seed=SEED_BASE + 3):
    """The batched workload: count matrices of rgg_irregular with n ~ U[nmin, nmax]."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(nmin, nmax + 1, size=count)
    return [rgg_irregular(int(n), seed=seed * 1000 + q) for q, n in enumerate(ns)]
