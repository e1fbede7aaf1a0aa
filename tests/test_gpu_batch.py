"""Batches of independent irregular systems through sai_solve_batched.

Matrices: random geometric-graph Laplacians with a nonsymmetric perturbation
and 1-20 dense columns (workloads.rgg_irregular), n uniform in a range.
Per matrix against the oracle's Procedure * on that matrix alone: the split
(s, p), the iteration counts (the largest of its s+1 systems within +-1),
rr < eps and x. The batch builds every column in one SAI launch and runs all
systems in one batched BiCGStab.
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
