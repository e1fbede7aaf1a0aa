"""Saving M and loading it again for later right-hand sides (sai_precond_create).

M built once, written to a file, read back as a new handle: the loaded M is
the same CSC bit for bit, and Procedure * steps 3-5 with it give the same x
and iteration counts as with the built handle (rr to its atomic-sum noise). Malformed CSC input is
refused with SAI_INVALID_ARG.
"""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import lib, need_gpu, to_dev, to_scipy, torch

pytestmark = pytest.mark.gpu


def _dev(v):
    return torch.as_tensor(np.ascontiguousarray(v, dtype=np.float64), device="cuda")


@pytest.mark.parametrize("kind", ["spai", "psai"])
def test_saved_m_solves_like_the_built_one(kind, tmp_path):
    need_gpu()
    sai = lib()
    P = W.convdiff2d_irregular()
    dA = to_dev(P.A)
    sp_ = sai.split(dA)
    Pc = (sai.build_spai(sp_, delta=0.4, mn=5, max_aug=10) if kind == "spai"
          else sai.build_psai(sp_, delta=0.4, tol=1e-3, tol_mode=1, lmax=10))
    path = str(tmp_path / "m.npz")
    sai.save_precond(Pc, path)
    Pl = sai.load_precond(path)
    assert Pl.n == Pc.n and Pl.nnz == Pc.nnz
    a, b = to_scipy(Pc.arrays()[0]), to_scipy(Pl.arrays()[0])
    assert np.array_equal(a.indptr, b.indptr) and np.array_equal(a.indices, b.indices)
    assert np.array_equal(a.data, b.data)
    rng = np.random.default_rng(3)
    for rhs in (P.b, rng.standard_normal(P.n)):
        x1, it1, r1 = sai.solve_with(dA, sp_, Pc, _dev(rhs), eps=1e-8)
        x2, it2, r2 = sai.solve_with(dA, sp_, Pl, _dev(rhs), eps=1e-8)
        # rr sums A x with atomics (its last bits vary between runs); x is the same bits
        assert it1 == it2 and torch.equal(x1, x2) and r1["rr"] < 1e-8
        assert r2["rr"] == pytest.approx(r1["rr"], rel=1e-9)


def test_malformed_m_is_refused():
    need_gpu()
    sai = lib()
    n = 4
    cp = np.array([0, 2, 3, 4, 5])
    bad_rows = np.array([1, 0, 2, 3, 0])  # column 0's rows are not ascending
    M = sai.CscMatrix.from_arrays(cp, bad_rows, np.ones(5), n)
    with pytest.raises(sai.SaiError) as e:
        sai.precond_from_csc(M)
    assert e.value.status == sai.SAI_INVALID_ARG
    out_of_range = np.array([0, 1, 2, 3, 7])
    M = sai.CscMatrix.from_arrays(cp, out_of_range, np.ones(5), n)
    with pytest.raises(sai.SaiError) as e:
        sai.precond_from_csc(M)
    assert e.value.status == sai.SAI_INVALID_ARG
