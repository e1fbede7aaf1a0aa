"""Block GMRES(m) (krylov="bgmres", the block Krylov alternative named after
Theorem 2) through the C ABI against the oracle's block GMRES.

The GPU orthogonalises by two passes of block classical Gram-Schmidt and a
shifted Cholesky QR; the oracle by block modified Gram-Schmidt and
Householder QR. In exact arithmetic both give the same iterates, so each
system's block-step count agrees to +-1 (systems are frozen at the restart
where their true residual meets the threshold) and the solutions to
rounding.
 - 2D workload (k = s+1 = 4), SPAI(0.4, 5, 10): the s+1 solves by
   sai_krylov_solve at restart 30 (one cycle) and restart 5 (many cycles),
   forward and transposed; Procedure * and the backward pass with bgmres;
 - a 3D workload with 11 systems at restart 20 (the size class of the 64^3
   benchmark, k = 11);
 - the 64^3 benchmark system itself: GMRES(50) in block form to 1e-10
   meets eps and returns A's solution (the oracle's block GMRES is too slow
   there, so the check is the residual and the known solution);
 - the refined form (FP32 inner block solves, FP64 outside) against the
   oracle's FP64 answer, and at 64^3;
 - limits: more than 32 systems and restart 0 are refused.
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
import workloads as W
from gpu_helpers import lib, need_gpu, to_dev, to_scipy, torch

pytestmark = pytest.mark.gpu

SPAI = dict(delta=0.4, mn=5, max_aug=10)


def _system(P, spai=SPAI, **split_kw):
    sai = lib()
    sp_ = sai.split(to_dev(P.A), **split_kw)
    Pc = sai.build_spai(sp_, **spai)
    At_d, (ucp, uri, uv), _ = sp_.arrays()
    At = to_scipy(At_d)
    U = sp.csc_matrix((uv.cpu().numpy(), uri.cpu().numpy(), ucp.cpu().numpy()), shape=(P.n, sp_.s))
    M = to_scipy(Pc.arrays()[0])
    s = sp_.s
    B = np.zeros((P.n, s + 1))
    B[:, 0] = P.b
    B[:, 1:] = U.toarray()
    bn = np.linalg.norm(P.b)
    thr = [0.5e-8 * bn] + [1e-8 * bn / (2 * np.sqrt(max(s, 1)))] * s
    return sp_, Pc, sp.csc_matrix(At), sp.csc_matrix(M), B, thr


@pytest.mark.parametrize("restart", [30, 5])
@pytest.mark.parametrize("transpose", [False, True])
def test_block_solves_match_oracle(restart, transpose):
    need_gpu()
    sai = lib()
    P = W.convdiff2d_irregular()
    sp_, Pc, At, M, B, thr = _system(P)
    if transpose:
        At, M = sp.csc_matrix(At.T), sp.csc_matrix(M.T)
    X, iters, status, st = sai.krylov_solve(sp_, Pc, torch.as_tensor(B, device="cuda"), thr, method=sai.BGMRES,
                                            restart=restart, transpose=transpose)
    Yo, it_o, st_o = O.block_gmres(At, M, B, thr, restart=restart)
    assert st == sai.SAI_OK and st_o == O.OK
    assert all(abs(a - b) <= 1 for a, b in zip(iters, it_o)), (iters, list(it_o))
    X = X.cpu().numpy()
    for c in range(B.shape[1]):
        assert np.linalg.norm(B[:, c] - At @ X[:, c]) < thr[c] * 1.000001
    np.testing.assert_allclose(X, Yo, rtol=0, atol=1e-6 * np.abs(Yo).max())


def test_eleven_systems_match_oracle():
    need_gpu()
    sai = lib()
    P = W.convdiff3d_irregular(m=16, s=10, density=0.1)
    sp_, Pc, At, M, B, thr = _system(P, dict(delta=0.3, mn=5, max_aug=10))
    assert B.shape[1] == 11
    X, iters, status, st = sai.krylov_solve(sp_, Pc, torch.as_tensor(B, device="cuda"), thr, method=sai.BGMRES,
                                            restart=20)
    Yo, it_o, st_o = O.block_gmres(At, M, B, thr, restart=20)
    assert st == sai.SAI_OK and st_o == O.OK
    assert all(abs(a - b) <= 1 for a, b in zip(iters, it_o)), (iters, list(it_o))
    np.testing.assert_allclose(X.cpu().numpy(), Yo, rtol=0, atol=1e-6 * np.abs(Yo).max())


def test_procedure_and_backward_with_block_gmres():
    need_gpu()
    sai = lib()
    P = W.convdiff2d_irregular()
    kw = dict(krylov="bgmres", restart=30, eps=1e-8, **SPAI)
    x, iters, rep = sai.solve(to_dev(P.A), torch.as_tensor(P.b, device="cuda"), **kw)
    xo, it_o, rep_o = O.solve(P.A, P.b, **kw)
    assert rep["status"] == sai.SAI_OK and rep_o["status"] == O.OK
    assert all(abs(a - b) <= 1 for a, b in zip(iters, it_o)) and rep["rr"] < 1e-8
    np.testing.assert_allclose(x.cpu().numpy(), xo, rtol=0, atol=1e-6)
    # backward: lambda = A^{-T} g with the transposed block solves
    g = np.random.default_rng(5).standard_normal(P.n)
    dA = to_dev(P.A)
    sp_ = sai.split(dA)
    Pc = sai.build_spai(sp_, **SPAI)
    lam, gv, it_b, rep_b = sai.backward(dA, sp_, Pc, x, torch.as_tensor(g, device="cuda"), krylov="bgmres",
                                        restart=30, eps=1e-8)
    lam_o, gv_o, it_bo, rep_bo = O.backward(P.A, xo, g, **kw)
    assert rep_b["status"] == sai.SAI_OK and rep_b["rr"] < 1e-8
    assert all(abs(a - b) <= 1 for a, b in zip(it_b, it_bo)), (it_b, list(it_bo))
    np.testing.assert_allclose(lam.cpu().numpy(), lam_o, rtol=0, atol=1e-6 * np.abs(lam_o).max())


def test_refined_block_gmres_matches_oracle():
    """FP32 inner block GMRES refined in FP64 (every stop test in FP64)
    reaches the FP64 answer: x against the oracle's FP64 block GMRES."""
    need_gpu()
    sai = lib()
    P = W.convdiff2d_irregular()
    kw = dict(krylov="bgmres", restart=30, eps=1e-8, **SPAI)
    x, iters, rep = sai.solve(to_dev(P.A), torch.as_tensor(P.b, device="cuda"), krylov_precision=1, **kw)
    xo, it_o, rep_o = O.solve(P.A, P.b, **kw)
    assert rep["status"] == sai.SAI_OK and rep["rr"] < 1e-8
    np.testing.assert_allclose(x.cpu().numpy(), xo, rtol=0, atol=1e-6)


GOLDEN_BG = os.path.join(os.path.dirname(__file__), "golden", "oracle_bgmres_m64_s10.json")


@pytest.mark.parametrize("precision", [0, 1])
def test_block_gmres_full_size_64cubed(precision):
    """The 64^3 benchmark system (n = 262144, 11 systems), SPAI(0.3, 5, 10),
    block GMRES(50) in FP64 and in the refined form to eps = 1e-10. The FP64
    form's block steps per system against the oracle's complete block solve
    (stored by the oracle-only tests/golden/make_oracle_bgmres64.py), +-1."""
    need_gpu()
    sai = lib()
    P = W.convdiff3d_irregular()
    x, iters, rep = sai.solve(to_dev(P.A), torch.as_tensor(P.b, device="cuda"), sai="spai", delta=0.3, mn=5,
                              max_aug=10, krylov="bgmres", restart=50, eps=1e-10, krylov_precision=precision)
    assert rep["status"] == sai.SAI_OK and rep["s"] == 10
    assert rep["rr"] < 1e-10
    np.testing.assert_allclose(x.cpu().numpy(), np.ones(P.n), rtol=0, atol=1e-6)
    if precision == 0:
        with open(GOLDEN_BG) as f:
            gold = json.load(f)
        assert gold["status"] == O.OK and gold["report"]["rr"] < 1e-10
        assert all(abs(a - b) <= 1 for a, b in zip(iters, gold["block_steps"])), (iters, gold["block_steps"])


def test_block_gmres_limits():
    need_gpu()
    sai = lib()
    P = W.convdiff2d_irregular()
    sp_, Pc, At, M, B, thr = _system(P)
    B33 = torch.as_tensor(np.random.default_rng(6).standard_normal((P.n, 33)), device="cuda")
    with pytest.raises(sai.SaiError) as e:
        sai.krylov_solve(sp_, Pc, B33, [1e-8] * 33, method=sai.BGMRES)
    assert e.value.status == sai.SAI_INVALID_ARG
    with pytest.raises(sai.SaiError) as e:
        sai.krylov_solve(sp_, Pc, torch.as_tensor(B, device="cuda"), thr, method=sai.BGMRES, restart=0)
    assert e.value.status == sai.SAI_INVALID_ARG


def test_identical_right_hand_sides_keep_x_sound():
    """Two identical right-hand sides make the first block numerically rank
    deficient, so the shifted Cholesky QR may break down. Whatever happens,
    each system ends with OK (and meets its threshold) or BREAKDOWN, and a
    broken block step never enters X: every returned column's residual is at
    most the starting one (x0 = 0) and the two columns agree."""
    need_gpu()
    sai = lib()
    P = W.convdiff2d_irregular()
    sp_, Pc, At, M, B, thr = _system(P)
    B2 = np.stack([P.b, P.b], axis=1)
    thr2 = [thr[0], thr[0]]
    for fp in (0, 1):
        X, iters, status, st = sai.krylov_solve(sp_, Pc, torch.as_tensor(B2, device="cuda"), thr2,
                                                method=sai.BGMRES, restart=30, precision=fp)
        X = X.cpu().numpy()
        assert st in (sai.SAI_OK, sai.SAI_BREAKDOWN), st
        for c in range(2):
            r = np.linalg.norm(P.b - At @ X[:, c])
            assert status[c] in (sai.SAI_OK, sai.SAI_BREAKDOWN), status
            assert np.all(np.isfinite(X[:, c]))
            assert r <= np.linalg.norm(P.b) * (1 + 1e-12)
            if status[c] == sai.SAI_OK:
                assert r < thr2[c] * 1.000001
        np.testing.assert_allclose(X[:, 0], X[:, 1], rtol=0, atol=1e-6 * max(np.abs(X).max(), 1.0))
