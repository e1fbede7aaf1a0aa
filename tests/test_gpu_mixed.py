"""Reduced-precision forms against the FP64 oracle.

The refined GMRES runs its inner solves in FP32 and keeps the residual, the
correction and every stop test in FP64; the bar is the same final accuracy as
the FP64 form: ||b - A x|| / ||b|| < eps for the recovered x, and x close to
the oracle's solution.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import lib, need_gpu, to_dev, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("sai_kind", ["spai", "psai"])
def test_refined_gmres_2d_meets_eps(sai_kind):
    sai = lib()
    P = W.convdiff2d_irregular()
    kw = dict(sai=sai_kind, krylov="gmres", eps=1e-8, delta=0.4, mn=5, max_aug=10, tol_mode=0, lmax=10, restart=50)
    x, iters, rep = sai.solve(to_dev(P.A), torch.as_tensor(P.b, device="cuda"), krylov_precision=1, **kw)
    assert rep["status"] == sai.SAI_OK
    assert rep["rr"] < 1e-8
    assert O.rel_resid(P.A, P.b, x.cpu().numpy()) < 1e-8
    x_o, it_o, rep_o = O.solve(P.A, P.b, **kw)
    np.testing.assert_allclose(x.cpu().numpy(), x_o, rtol=0, atol=1e-6)
    assert rep["c"] == pytest.approx(rep_o["c"], rel=1e-6)


def test_refined_krylov_multi_rhs_thresholds():
    """Every system meets its own FP64 threshold on its true residual."""
    sai = lib()
    P = W.convdiff2d_irregular(m=30, s=3, density=0.3)
    A = P.A
    h = sai.split(to_dev(A))
    Pc = sai.build_spai(h, delta=0.4, mn=5, max_aug=10)
    J, p, _ = O.detect(A)
    At, U = O.split(A, J, p)
    s = len(J)
    B = np.zeros((A.shape[0], s + 1))
    B[:, 0] = P.b
    B[:, 1:] = U.toarray()
    bn = np.linalg.norm(P.b)
    thr = [0.5e-10 * bn] + [1e-10 * bn / (2 * np.sqrt(s))] * s
    X, iters, stat, st = sai.krylov_solve(h, Pc, torch.as_tensor(B, device="cuda"), thr, method=sai.GMRES,
                                          restart=30, precision=1)
    assert st == sai.SAI_OK and all(v == 0 for v in stat)
    X = X.cpu().numpy()
    for q in range(s + 1):
        assert np.linalg.norm(B[:, q] - At @ X[:, q]) < thr[q]


@pytest.mark.parametrize("sai_kind", ["spai", "psai"])
def test_refined_gmres_fullsize_meets_eps(sai_kind):
    sai = lib()
    P = W.convdiff3d_irregular()
    kw = dict(sai=sai_kind, krylov="gmres", eps=1e-10, restart=50, maxit=500, delta=0.3, mn=5, max_aug=10,
              tol=1e-3, tol_mode=1, lmax=10)
    x, iters, rep = sai.solve(to_dev(P.A), torch.as_tensor(P.b, device="cuda"), krylov_precision=1, **kw)
    assert rep["status"] == sai.SAI_OK
    assert rep["rr"] < 1e-10
    assert O.rel_resid(P.A, P.b, x.cpu().numpy()) < 1e-10
    np.testing.assert_allclose(x.cpu().numpy(), 1.0, rtol=0, atol=1e-7)
