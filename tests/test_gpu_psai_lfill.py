"""PSAI(lfill) (tol_mode 2): the lfill entries of largest magnitude of each
newly computed m_k are kept (equal magnitudes to the smaller column index),
with the power growth and stop test of PSAI(tol). Against the oracle: M's
pattern bit-exact and values 1e-10 (FP64) or 1e-4 (FP32 QR + FP64
refinement) on the 2D and 3D workloads; Procedure * with it meeting eps with
per-system iterations within +-1 of the oracle's; lfill < 1 refused.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
import workloads as W
from gpu_helpers import assert_same_pattern_and_values, lib, need_gpu, to_dev, to_scipy, torch

pytestmark = pytest.mark.gpu

CASES = {
    "2d": (lambda: W.convdiff2d_irregular().A, dict(delta=0.3, lmax=4, lfill=10)),
    "3d": (lambda: W.convdiff3d_irregular(m=16, s=3, density=0.2).A, dict(delta=0.3, lmax=3, lfill=12)),
}


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("case", sorted(CASES))
def test_psai_lfill_matches_oracle(case, precision):
    need_gpu()
    sai = lib()
    make, kw = CASES[case]
    A = sp.csc_matrix(make())
    J, p, _ = O.detect(A)
    At, _ = O.split(A, J, p)
    Mo = O.psai(At, kw["delta"], tol_mode=2, lmax=kw["lmax"], lfill=kw["lfill"])[0]
    sp_ = sai.split(to_dev(A))
    Pc = sai.build_psai(sp_, delta=kw["delta"], tol_mode=2, lmax=kw["lmax"], lfill=kw["lfill"], precision=precision)
    Mg = to_scipy(Pc.arrays()[0])
    assert np.diff(Mg.indptr).max() <= kw["lfill"]
    assert_same_pattern_and_values(Mg, Mo, rtol=1e-10 if precision == 0 else 1e-4)


def test_procedure_with_psai_lfill():
    need_gpu()
    sai = lib()
    P = W.convdiff2d_irregular()
    A = sp.csc_matrix(P.A)
    kw = dict(delta=0.3, lmax=4, lfill=10)
    x, iters, rep = sai.solve(to_dev(A), torch.as_tensor(P.b, device="cuda"), sai="psai", tol_mode=2,
                              krylov="bicgstab", eps=1e-8, **kw)
    assert rep["status"] == sai.SAI_OK and rep["rr"] < 1e-8
    J, p, _ = O.detect(A)
    At, U = O.split(A, J, p)
    At, U = sp.csc_matrix(At), sp.csc_matrix(U)
    Mo = O.psai(At, kw["delta"], tol_mode=2, lmax=kw["lmax"], lfill=kw["lfill"])[0]
    bn = np.linalg.norm(P.b)
    rhs = [P.b] + [U[:, t].toarray().ravel() for t in range(len(J))]
    thr = [0.5e-8 * bn] + [1e-8 * bn / (2 * np.sqrt(len(J)))] * len(J)
    for q, (r, th) in enumerate(zip(rhs, thr)):
        _, it, st = O.bicgstab(At, Mo, r, th)
        assert st == O.OK and abs(iters[q] - it) <= 1, (q, iters[q], it)


def test_psai_lfill_needs_a_positive_lfill():
    need_gpu()
    sai = lib()
    sp_ = sai.split(to_dev(W.convdiff2d_irregular(m=10, s=0).A))
    with pytest.raises(sai.SaiError) as e:
        sai.build_psai(sp_, delta=0.3, tol_mode=2, lmax=2, lfill=0)
    assert e.value.status == sai.SAI_INVALID_ARG
