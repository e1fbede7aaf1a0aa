"""The rotated anisotropic 9-point workload (mixed precision at scale).

-div(K grad u) on a grid, K = R diag(1, 1e-3) R^T at 30 degrees, plus dense
N(0,1) columns; SPAI(0.4, 5, 10) and BiCGStab to tol 1e-8.
 - 96 x 96 (n = 9216, s = 5): the FP64 build column by column against the
   oracle (pattern bit-exact, values 1e-10), the solve meeting tol and agreeing
   with the oracle's x (BiCGStab's iteration counts on this operator depend on
   the rounding order, so they are compared within 20%); the FP32-QR +
   FP64-refined build against the FP64 oracle (pattern bit-exact, values 1e-4)
   and the solve with it meeting tol.
 - 1024 x 1024 (n = 1048576, s = 50): the refined build on three column
   ranges against the oracle (pattern, 1e-4) and the FP64 build on the same
   ranges (pattern, 1e-10).
 - 256 x 256 (n = 65536, s = 8): the refined-build solve with FP64 BiCGStab,
   FP64 SMW and FP64 stopping tests meeting ||b - A x||/||b|| < 1e-8 and
   agreeing with the oracle's x.
 - 512 x 512 with all 50 dense columns (n = 262144, s = 50), the largest grid
   on which the method reaches 1e-8 in reasonable time: SPAI(0.2, 5, 10)
   refined, FP64 BiCGStab with the u_j systems continued with the measured c
   (c = sqrt(50)), rr < 1e-8 on the device and recomputed on the host, x
   within 1e-2 of the exact solution (all ones). At 1024 x 1024 the b system
   takes 26165 iterations and some u_j systems do not reach their thresholds
   within 60000 (the operator's condition grows like h^-2 / 1e-3).
 - 1024 x 1024: the SPAI(0.2, 5, 10) refined build (the 512 x 512 solve's
   setting; its columns reach the global-memory tiers) on three column
   ranges against the oracle.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import assert_same_pattern_and_values, lib, need_gpu, to_dev, to_scipy, torch

pytestmark = pytest.mark.gpu

SPAI = dict(delta=0.4, mn=5, max_aug=10)


def _dev(v):
    return torch.as_tensor(np.ascontiguousarray(v, dtype=np.float64), device="cuda")


@pytest.fixture(scope="module")
def small():
    P = W.aniso9_irregular(m=96, s=5)
    J, p, _ = O.detect(P.A)
    At, _ = O.split(P.A, J, p)
    Mo = O.spai(At, **SPAI)[0]
    return P, At, Mo


def test_aniso_small_fp64_build_and_solve(small):
    need_gpu()
    sai = lib()
    P, At, Mo = small
    sp_ = sai.split(to_dev(P.A))
    assert sp_.s == 5 and sp_.p == 8
    Pc = sai.build_spai(sp_, **SPAI)
    assert_same_pattern_and_values(to_scipy(Pc.arrays()[0]), Mo)
    x, iters, rep = sai.solve(to_dev(P.A), _dev(P.b), krylov="bicgstab", eps=1e-8, **SPAI)
    xo, it_o, rep_o = O.solve(P.A, P.b, krylov="bicgstab", eps=1e-8, **SPAI)
    # BiCGStab's residual history on this operator is erratic and the iteration
    # counts depend on the rounding order (both sides take ~280 +- 40); the bar
    # here is the FP64 true residual and agreement with the oracle's solution.
    assert rep["status"] == sai.SAI_OK and rep_o["status"] == O.OK
    assert all(abs(a - b) <= 0.2 * b for a, b in zip(iters, it_o)), (iters, list(it_o))
    assert rep["rr"] < 1e-8 and rep_o["rr"] < 1e-8
    np.testing.assert_allclose(x.cpu().numpy(), xo, rtol=0, atol=1e-5)


def test_aniso_small_refined_build(small):
    need_gpu()
    sai = lib()
    P, At, Mo = small
    sp_ = sai.split(to_dev(P.A))
    Pc = sai.build_spai(sp_, precision=1, **SPAI)
    assert_same_pattern_and_values(to_scipy(Pc.arrays()[0]), Mo, rtol=1e-4)
    x, iters, rep = sai.solve(to_dev(P.A), _dev(P.b), krylov="bicgstab", eps=1e-8, sai_precision=1, **SPAI)
    assert rep["status"] == sai.SAI_OK and rep["rr"] < 1e-8


def test_aniso_fullsize_builds_match_oracle():
    """1024 x 1024, 50 dense columns: the FP64 and the refined builds on three
    column ranges against the oracle."""
    need_gpu()
    sai = lib()
    P = W.aniso9_irregular()
    J, p, _ = O.detect(P.A)
    At, _ = O.split(P.A, J, p)
    sp_ = sai.split(to_dev(P.A))
    assert sp_.s == len(J) == 50 and sp_.p == p
    Mr = to_scipy(sai.build_spai(sp_, precision=1, **SPAI).arrays()[0])
    Md = to_scipy(sai.build_spai(sp_, **SPAI).arrays()[0])
    n = P.n
    for c0, c1 in ((0, 1500), (n // 2, n // 2 + 1500), (n - 1500, n)):
        Mo = O.spai(At, cols=(c0, c1), **SPAI)[0]
        assert_same_pattern_and_values(Md, Mo, cols=range(c0, c1))
        assert_same_pattern_and_values(Mr, Mo, rtol=1e-4, cols=range(c0, c1))


def test_aniso_256_refined_solve_meets_tol():
    """256 x 256, 8 dense columns: the refined build with FP64 BiCGStab, SMW and
    stopping tests meets ||b - A x||/||b|| < 1e-8 and agrees with the oracle's x
    (the FP64 oracle takes ~1000 iterations per system here)."""
    need_gpu()
    sai = lib()
    P = W.aniso9_irregular(m=256, s=8)
    x, iters, rep = sai.solve(to_dev(P.A), _dev(P.b), krylov="bicgstab", eps=1e-8, maxit=5000, sai_precision=1,
                              **SPAI)
    assert rep["status"] == sai.SAI_OK, (rep["status"], iters)
    assert rep["rr"] < 1e-8
    assert O.rel_resid(P.A, P.b, x.cpu().numpy()) < 1e-8
    xo, it_o, rep_o = O.solve(P.A, P.b, krylov="bicgstab", eps=1e-8, maxit=5000, **SPAI)
    assert rep_o["status"] == O.OK
    # both meet rr < 1e-8; with cond(A) ~ 1e5 on this grid two such solutions
    # (and the exact one, all ones) agree to about 1e-3
    np.testing.assert_allclose(x.cpu().numpy(), xo, rtol=0, atol=1e-3)
    np.testing.assert_allclose(x.cpu().numpy(), 1.0, rtol=0, atol=1e-3)


def test_aniso_512_all_columns_refined_solve_meets_tol():
    need_gpu()
    sai = lib()
    P = W.aniso9_irregular(m=512)
    x, iters, rep = sai.solve(to_dev(P.A), _dev(P.b), krylov="bicgstab", eps=1e-8, maxit=30000, delta=0.2, mn=5,
                              max_aug=10, sai_precision=1, c_adapt=1)
    assert rep["s"] == 50 and rep["status"] == sai.SAI_OK, (rep["status"], max(iters))
    assert rep["c_rounds"] == 1 and rep["c"] == pytest.approx(np.sqrt(50.0), rel=1e-6)
    assert rep["rr"] < 1e-8
    assert O.rel_resid(P.A, P.b, x.cpu().numpy()) < 1e-8
    np.testing.assert_allclose(x.cpu().numpy(), 1.0, rtol=0, atol=1e-2)


def test_aniso_fullsize_delta02_refined_build_matches_oracle():
    need_gpu()
    sai = lib()
    P = W.aniso9_irregular()
    J, p, _ = O.detect(P.A)
    At, _ = O.split(P.A, J, p)
    sp_ = sai.split(to_dev(P.A))
    kw = dict(delta=0.2, mn=5, max_aug=10)
    Pc = sai.build_spai(sp_, precision=1, **kw)
    assert Pc.n_tier[1] > 0.9 * P.n  # |S| past 16: the global-memory tier 1
    Mr = to_scipy(Pc.arrays()[0])
    n = P.n
    for c0, c1 in ((0, 1000), (n // 2, n // 2 + 1000), (n - 1000, n)):
        Mo = O.spai(At, cols=(c0, c1), **kw)[0]
        assert_same_pattern_and_values(Mr, Mo, rtol=1e-4, cols=range(c0, c1))
