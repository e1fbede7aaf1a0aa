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


# ------------------------------------------------------------------ FP32 QR + FP64 refinement build
from gpu_helpers import assert_same_pattern_and_values, to_scipy  # noqa: E402

BUILD_CASES = {
    # name: (maker, kind, params)
    "spai_2d_paper": (lambda: W.convdiff2d_irregular().A, "spai", dict(delta=0.4, mn=5, max_aug=10)),
    "spai_3d": (lambda: W.convdiff3d_irregular(m=14, s=3, density=0.2).A, "spai", dict(delta=0.3, mn=5, max_aug=10)),
    "spai_random_deep": (lambda: W.random_sparse_dominant(600, 4, 3, 150, seed=11).A, "spai",
                         dict(delta=0.1, mn=3, max_aug=6)),
    "spai_tier2": (lambda: W.convdiff2d_irregular(m=14, s=1, density=0.2).A, "spai", dict(delta=0.0, mn=8, max_aug=9)),
    "psai_3d_fixed": (lambda: W.convdiff3d_irregular(m=14, s=3, density=0.2).A, "psai",
                      dict(delta=0.3, tol=1e-3, tol_mode=1, lmax=10)),
    "psai_growth": (lambda: W.convdiff2d_irregular(m=18, s=1, density=0.2).A, "psai",
                    dict(delta=0.0, tol=0.02, tol_mode=1, lmax=4)),
}


@pytest.mark.parametrize("case", sorted(BUILD_CASES))
def test_refined_build_matches_fp64_oracle(case):
    """M within 1e-4 relative of the FP64 oracle (the refinement step brings the
    LS solutions back to FP64 accuracy, so the patterns agree as well)."""
    mk, kind, kw = BUILD_CASES[case]
    A = mk()
    sai = lib()
    h = sai.split(to_dev(A))
    J, p, _ = O.detect(A)
    At, _ = O.split(A, J, p)
    if kind == "spai":
        P = sai.build_spai(h, precision=1, **kw)
        Mo = O.spai(At, kw["delta"], kw["mn"], kw["max_aug"])[0]
    else:
        P = sai.build_psai(h, precision=1, **kw)
        Mo = O.psai(At, kw["delta"], kw["tol"], kw["tol_mode"], kw["lmax"])[0]
    assert_same_pattern_and_values(to_scipy(P.arrays()[0]), Mo, rtol=1e-4)


@pytest.mark.parametrize("sai_kind", ["spai", "psai"])
def test_fully_reduced_precision_pipeline_meets_eps(sai_kind):
    """FP32 QR + FP64 refinement build, FP32-inner refined GMRES: same final
    accuracy as the FP64 form on the 64^3 workload."""
    sai = lib()
    P = W.convdiff3d_irregular()
    kw = dict(sai=sai_kind, krylov="gmres", eps=1e-10, restart=50, maxit=500, delta=0.3, mn=5, max_aug=10,
              tol=1e-3, tol_mode=1, lmax=10)
    x, iters, rep = sai.solve(to_dev(P.A), torch.as_tensor(P.b, device="cuda"), krylov_precision=1,
                              sai_precision=1, **kw)
    assert rep["status"] == sai.SAI_OK and rep["rr"] < 1e-10
    assert O.rel_resid(P.A, P.b, x.cpu().numpy()) < 1e-10
