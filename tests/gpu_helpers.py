"""Helpers shared by the GPU parity tests (device <-> scipy conversion)."""
import numpy as np
import pytest
import scipy.sparse as sp

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def lib():
    import paper_1211_6866_gb300 as sai
    sai.load()
    return sai


def to_dev(A):
    sai = lib()
    A = sp.csc_matrix(A)
    A.sort_indices()
    return sai.CscMatrix.from_arrays(A.indptr, A.indices, A.data, A.shape[0])


def to_scipy(M, nrows=None):
    cp = M.col_ptr.cpu().numpy()
    ri = M.row_idx.cpu().numpy()
    v = M.val.cpu().numpy()
    ncols = cp.size - 1
    return sp.csc_matrix((v, ri, cp), shape=(nrows or M.n, ncols))


def assert_same_pattern_and_values(Mg, Mo, rtol=1e-10, cols=None):
    """Bit-exact sparsity pattern, values within rtol (relative to each column's max)."""
    Mg = sp.csc_matrix(Mg)
    Mo = sp.csc_matrix(Mo)
    if cols is None:
        cols = range(Mo.shape[1])
    bad = []
    for k in cols:
        gi = Mg.indices[Mg.indptr[k]:Mg.indptr[k + 1]]
        oi = Mo.indices[Mo.indptr[k]:Mo.indptr[k + 1]]
        if not np.array_equal(gi, oi):
            bad.append(k)
            continue
        gv = Mg.data[Mg.indptr[k]:Mg.indptr[k + 1]]
        ov = Mo.data[Mo.indptr[k]:Mo.indptr[k + 1]]
        scale = np.abs(ov).max() if ov.size else 1.0
        if ov.size and np.abs(gv - ov).max() > rtol * scale:
            bad.append(k)
    assert not bad, "columns differing from the oracle: %s (of %d)" % (bad[:10], len(bad))
