"""Batches of independent irregular systems through sai_solve_batched.

Matrices: random geometric-graph Laplacians with a nonsymmetric perturbation
and 1-20 dense columns (workloads.rgg_irregular), n uniform in a range.
Per matrix against the oracle's Procedure * on that matrix alone: the split
(s, p), the iteration counts (the largest of its s+1 systems within +-1),
rr < eps and x. The batch builds every column in one SAI launch (its M
compared block by block with the oracle's M of each matrix) and runs all
systems in one batched BiCGStab; with c_adapt the u_j systems of a matrix
whose c exceeds 1 are continued with that c, as the oracle does, so that all
256 matrices of the batched workload meet eps.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import lib, need_gpu, to_dev, torch

pytestmark = pytest.mark.gpu

SPAI = dict(delta=0.4, mn=5, max_aug=10)


def _dev(v):
    return torch.as_tensor(np.ascontiguousarray(v, dtype=np.float64), device="cuda")


def _run(Ps, **kw):
    sai = lib()
    return sai.solve_batched([to_dev(P.A) for P in Ps], [_dev(P.b) for P in Ps], **kw)


@pytest.mark.parametrize("sai_precision", [0, 1])
def test_batch_matches_oracle_per_matrix(sai_precision):
    need_gpu()
    sai = lib()
    Ps = W.rgg_batch(count=10, nmin=1000, nmax=4000)
    xs, per, rep = _run(Ps, eps=1e-8, sai_precision=sai_precision, **SPAI)
    assert rep["status"] == sai.SAI_OK
    assert rep["columns"] == sum(P.n for P in Ps)
    assert rep["systems"] == sum(r["s"] + 1 for r in per)
    for P, x, r in zip(Ps, xs, per):
        xo, it_o, rep_o = O.solve(P.A, P.b, krylov="bicgstab", eps=1e-8, **SPAI)
        assert r["s"] == rep_o["s"] and r["p"] == rep_o["p"]
        assert r["status"] == sai.SAI_OK
        assert abs(r["iter_max"] - int(np.max(it_o))) <= 1, (r["iter_max"], list(it_o))
        assert r["rr"] < 1e-8
        np.testing.assert_allclose(x.cpu().numpy(), xo, rtol=0, atol=1e-6)


def test_batch_equals_single_solves():
    """Each matrix of the batch gives the x of its own sai_solve (same split, M,
    thresholds; only the summation order of the inner products differs)."""
    need_gpu()
    sai = lib()
    Ps = W.rgg_batch(count=6, nmin=2000, nmax=6000, seed=W.SEED_BASE + 31)
    xs, per, rep = _run(Ps, eps=1e-10, **SPAI)
    for P, x, r in zip(Ps, xs, per):
        x1, it1, rep1 = sai.solve(to_dev(P.A), _dev(P.b), krylov="bicgstab", eps=1e-10, **SPAI)
        assert r["s"] == rep1["s"] and abs(r["iter_max"] - rep1["iter_max"]) <= 1
        np.testing.assert_allclose(x.cpu().numpy(), x1.cpu().numpy(), rtol=0, atol=1e-8)


def test_batch_psai_fixed_tol():
    need_gpu()
    sai = lib()
    Ps = W.rgg_batch(count=6, nmin=1000, nmax=3000, seed=W.SEED_BASE + 32)
    kw = dict(sai="psai", delta=0.4, tol=1e-3, tol_mode=1, lmax=10)
    xs, per, rep = _run(Ps, eps=1e-8, **kw)
    for P, x, r in zip(Ps, xs, per):
        xo, it_o, rep_o = O.solve(P.A, P.b, krylov="bicgstab", eps=1e-8, **kw)
        assert abs(r["iter_max"] - int(np.max(it_o))) <= 1 and r["rr"] < 1e-8
        np.testing.assert_allclose(x.cpu().numpy(), xo, rtol=0, atol=1e-6)


def test_batch_uneven_sizes_large():
    """48 matrices with n uniform in [1k, 50k] (the batched workload's range):
    every matrix meets eps; three sampled matrices against the oracle."""
    need_gpu()
    sai = lib()
    Ps = W.rgg_batch(count=48, nmin=1000, nmax=50000, seed=W.SEED_BASE + 33)
    xs, per, rep = _run(Ps, eps=1e-8, sai_precision=1, **SPAI)
    assert rep["status"] == sai.SAI_OK
    assert all(r["rr"] < 1e-8 for r in per)
    for q in (0, 17, 41):
        xo, it_o, rep_o = O.solve(Ps[q].A, Ps[q].b, krylov="bicgstab", eps=1e-8, **SPAI)
        assert per[q]["s"] == rep_o["s"] and abs(per[q]["iter_max"] - int(np.max(it_o))) <= 1
        np.testing.assert_allclose(xs[q].cpu().numpy(), xo, rtol=0, atol=1e-6)


def test_batch_rejects_unsupported_forms():
    need_gpu()
    sai = lib()
    Ps = W.rgg_batch(count=2, nmin=1000, nmax=1500)
    with pytest.raises(sai.SaiError) as e:
        _run(Ps, sai="psai", delta=0.4, tol_mode=0)
    assert e.value.status == sai.SAI_NOT_IMPLEMENTED


def _batch_matrix(q):
    """Matrix q of the 256-matrix batched workload, generated on its own."""
    rng = np.random.default_rng(W.SEED_BASE + 3)
    ns = rng.integers(1000, 50001, size=256)
    return W.rgg_irregular(int(ns[q]), seed=(W.SEED_BASE + 3) * 1000 + q)


@pytest.mark.parametrize("sai_precision", [0, 1])
def test_batched_build_matches_oracle_per_matrix(sai_precision):
    """sai_build_batched: the M of the stacked A~ is block diagonal and each
    diagonal block is the oracle's M of that matrix alone (pattern bit for
    bit, values within 1e-10 / 1e-4)."""
    need_gpu()
    sai = lib()
    from gpu_helpers import assert_same_pattern_and_values, to_scipy
    Ps = W.rgg_batch(count=8, nmin=1000, nmax=5000, seed=W.SEED_BASE + 34)
    Pc = sai.build_batched([to_dev(P.A) for P in Ps], sai_precision=sai_precision, **SPAI)
    M = to_scipy(Pc.arrays()[0])
    r0 = np.cumsum([0] + [P.n for P in Ps])
    assert M.shape == (r0[-1], r0[-1])
    for m, P in enumerate(Ps):
        J, p, _ = O.detect(P.A)
        At, _ = O.split(P.A, J, p)
        Mo = O.spai(At, **SPAI)[0]
        blk = M[:, r0[m]:r0[m + 1]].tocsc()
        rows = blk.indices
        assert rows.size == 0 or (rows.min() >= r0[m] and rows.max() < r0[m + 1])  # block diagonal
        assert_same_pattern_and_values(blk[r0[m]:r0[m + 1], :], Mo, rtol=1e-10 if sai_precision == 0 else 1e-4)


def test_batch_c_continuation_matches_oracle():
    """c_adapt: matrix 10 of the batched workload (rr 1.07e-8 > eps with c = 1
    in the oracle) and two others; per matrix the oracle's Procedure * with
    the same option: c_rounds equal, largest iteration count +-1, rr < eps
    (the first one only reaches it through the continuation), x within 1e-6."""
    need_gpu()
    sai = lib()
    Ps = [_batch_matrix(q) for q in (10, 32, 64)]
    xs, per, rep = _run(Ps, eps=1e-8, c_adapt=1, **SPAI)
    assert rep["status"] == sai.SAI_OK
    for P, x, r in zip(Ps, xs, per):
        xo, it_o, rep_o = O.solve(P.A, P.b, krylov="bicgstab", eps=1e-8, c_adapt=1, **SPAI)
        assert r["s"] == rep_o["s"] and r["c_rounds"] == rep_o["c_rounds"]
        assert abs(r["iter_max"] - int(np.max(it_o))) <= 1, (r["iter_max"], list(it_o))
        assert r["rr"] < 1e-8 and O.rel_resid(P.A, P.b, x.cpu().numpy()) < 1e-8
        np.testing.assert_allclose(x.cpu().numpy(), xo, rtol=0, atol=1e-6)
    assert per[0]["c_rounds"] == 1 and per[2]["c_rounds"] == 0


def test_single_solve_c_continuation_matches_oracle():
    """sai_solve with c_adapt on matrix 10 of the batched workload: every
    system's iteration count (both rounds) within +-1 of the oracle's, rr < eps."""
    need_gpu()
    sai = lib()
    P = _batch_matrix(10)
    x, iters, rep = sai.solve(to_dev(P.A), _dev(P.b), krylov="bicgstab", eps=1e-8, c_adapt=1, **SPAI)
    xo, it_o, rep_o = O.solve(P.A, P.b, krylov="bicgstab", eps=1e-8, c_adapt=1, **SPAI)
    assert rep["c_rounds"] == 1 == rep_o["c_rounds"]
    assert all(abs(a - b) <= 1 for a, b in zip(iters, it_o)), (iters, list(it_o))
    assert rep["rr"] < 1e-8
    np.testing.assert_allclose(x.cpu().numpy(), xo, rtol=0, atol=1e-6)


def test_batch256_every_matrix_meets_eps():
    """The 256-matrix batched workload (n uniform in [1k, 50k]) as the
    benchmark runs it (autotuned build schedule, FP32 QR + FP64 refinement,
    c_adapt): every matrix ends with rr < eps and status OK, on the device
    and recomputed on the host for a sample; sampled matrices against the
    oracle (iterations +-1, x within 1e-6), the two that c = 1 leaves above
    eps among them."""
    need_gpu()
    sai = lib()
    Ps = W.rgg_batch(count=256)
    As = [to_dev(P.A) for P in Ps]
    try:
        sai.build_autotune_batched(As, sai_precision=1, **SPAI)
        xs, per, rep = sai.solve_batched(As, [_dev(P.b) for P in Ps], eps=1e-8, sai_precision=1, c_adapt=1, **SPAI)
    finally:
        sai.build_set_config()
    assert rep["status"] == sai.SAI_OK and len(per) == 256
    assert all(r["status"] == sai.SAI_OK and r["rr"] < 1e-8 for r in per), \
        [(q, r["rr"]) for q, r in enumerate(per) if not r["rr"] < 1e-8]
    for q in (0, 10, 79, 200):
        P = Ps[q]
        assert O.rel_resid(P.A, P.b, xs[q].cpu().numpy()) < 1e-8
        xo, it_o, rep_o = O.solve(P.A, P.b, krylov="bicgstab", eps=1e-8, c_adapt=1, **SPAI)
        assert per[q]["s"] == rep_o["s"] and abs(per[q]["iter_max"] - int(np.max(it_o))) <= 1
        np.testing.assert_allclose(xs[q].cpu().numpy(), xo, rtol=0, atol=1e-6)
