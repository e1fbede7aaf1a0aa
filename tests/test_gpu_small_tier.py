"""The small shared-memory tier of the SAI build (first_tier 1: four columns
per warp in 8-lane groups; 2: two columns per warp in 16-lane groups; 3: one
column per lane, 32 per warp) against the oracle, through the C ABI.

The tier holds |L| <= 32 rows and |S| <= 8 columns; a column that outgrows it
restarts in tier 0. Bars as for the other tiers: the oracle's sparsity
pattern bit for bit, values within 1e-10 (FP64) or 1e-4 (FP32 QR + FP64
refinement) of each column's largest entry, loop counts exact, LS residuals
within 1e-9; the same first_tier gives the same bits under every other
schedule setting.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import assert_same_pattern_and_values, lib, need_gpu, to_dev, to_scipy

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu_and_config():
    need_gpu()
    yield
    lib().build_set_config()


def _oracle_split(A, **kw):
    J, p, _ = O.detect(A, **kw)
    return O.split(A, J, p)[0]


CASES = {
    # name: (matrix maker, builder, parameters, which tiers finish the columns: "small" all in the
    # small tier, "restart" some restarted in tier 0 or later, None not checked)
    "spai_3d_24": (lambda: W.convdiff3d_irregular(m=24, s=4, density=0.1).A, "spai",
                   dict(delta=0.3, mn=5, max_aug=10), "small"),
    "spai_2d_paper": (lambda: W.convdiff2d_irregular().A, "spai", dict(delta=0.4, mn=5, max_aug=10), None),
    "spai_2d_deep": (lambda: W.convdiff2d_irregular(m=30, s=2, density=0.2).A, "spai",
                     dict(delta=0.05, mn=5, max_aug=3), "restart"),
    "psai_3d_fixed": (lambda: W.convdiff3d_irregular(m=20, s=3, density=0.1).A, "psai",
                      dict(delta=0.3, tol=1e-3, tol_mode=1, lmax=10), "small"),
    "psai_2d_tolk": (lambda: W.convdiff2d_irregular().A, "psai", dict(delta=0.4, tol_mode=0, lmax=10), None),
    "psai_2d_deep": (lambda: W.convdiff2d_irregular(m=30, s=2, density=0.2).A, "psai",
                     dict(delta=0.05, tol=1e-4, tol_mode=1, lmax=3), "restart"),
    "psai_3d_growth_c": (lambda: W.convdiff3d_irregular(m=16, s=3, density=0.1).A, "psai",
                         dict(delta=0.3, tol=0.05, tol_mode=1, lmax=4, growth="C"), None),
    "spai_random": (lambda: W.random_sparse_dominant(500, 3, 3, 120, seed=13).A, "spai",
                    dict(delta=0.2, mn=3, max_aug=4), None),
}


def _oracle_build(At, kind, kw):
    if kind == "spai":
        M, loops, res = O.spai(At, kw["delta"], kw["mn"], kw["max_aug"])
        return M, loops, res
    M, loops, pre, _ = O.psai(At, kw["delta"], kw.get("tol", 0.0), kw["tol_mode"], kw["lmax"],
                              growth=1 if kw.get("growth", "A") == "C" else 0)
    return M, loops, pre


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("first_tier", [1, 2, 3])
@pytest.mark.parametrize("case", sorted(CASES))
def test_small_tier_matches_oracle(case, first_tier, precision):
    sai = lib()
    mk, kind, kw, tiers = CASES[case]
    A = mk()
    h = sai.split(to_dev(A))
    sai.build_set_config(8, 2, 0, first_tier)
    P = sai.build_spai(h, precision=precision, **kw) if kind == "spai" else \
        sai.build_psai(h, precision=precision, **kw)
    Md, loops_d, res_d, _ = P.arrays()
    Mo, loops_o, res_o = _oracle_build(_oracle_split(A), kind, kw)
    assert_same_pattern_and_values(to_scipy(Md), Mo, rtol=1e-10 if precision == 0 else 1e-4)
    assert np.array_equal(loops_d.cpu().numpy(), loops_o)
    np.testing.assert_allclose(res_d.cpu().numpy(), res_o, rtol=1e-9 if precision == 0 else 1e-5,
                               atol=1e-13 if precision == 0 else 1e-9)
    assert sum(P.n_tier) == A.shape[0]
    if tiers == "small":
        assert P.n_tier[4] == A.shape[0], P.n_tier
    elif tiers == "restart":
        assert sum(P.n_tier[:4]) > 0, P.n_tier  # columns that outgrew the tier restarted in tier 0 or later


@pytest.mark.parametrize("first_tier", [1, 2, 3])
def test_small_tier_bits_do_not_depend_on_the_rest_of_the_schedule(first_tier):
    sai = lib()
    A = W.convdiff2d_irregular().A
    h = sai.split(to_dev(A))
    kw = dict(delta=0.4, mn=5, max_aug=10, precision=1)
    sai.build_set_config(8, 2, 0, first_tier)
    ref = to_scipy(sai.build_spai(h, **kw).arrays()[0])
    for w, b, hf in ((4, 1, 1), (4, 4, 0), (8, 4, 1)):
        sai.build_set_config(w, b, hf, first_tier)
        got = to_scipy(sai.build_spai(h, **kw).arrays()[0])
        assert np.array_equal(got.indptr, ref.indptr) and np.array_equal(got.indices, ref.indices)
        assert np.array_equal(got.data, ref.data)


@pytest.mark.parametrize("first_tier", [1, 3])
def test_procedure_star_with_the_small_tier(first_tier):
    """Procedure * on the 2D workload with the small tier: every system's
    BiCGStab iteration count within +-1 of the oracle's, rr < eps, x within
    1e-6 of the oracle's."""
    sai = lib()
    import torch
    P = W.convdiff2d_irregular()
    sai.build_set_config(8, 2, 0, first_tier)
    dA = to_dev(P.A)
    b = torch.as_tensor(P.b, device="cuda")
    x, iters, rep = sai.solve(dA, b, sai="spai", krylov="bicgstab", eps=1e-8, delta=0.4, mn=5, max_aug=10)
    xo, it_o, rep_o = O.solve(P.A, P.b, sai="spai", krylov="bicgstab", eps=1e-8, delta=0.4, mn=5, max_aug=10)
    assert all(abs(a - c) <= 1 for a, c in zip(iters, it_o)), (iters, it_o)
    assert rep["rr"] < 1e-8
    np.testing.assert_allclose(x.cpu().numpy(), xo, rtol=0, atol=1e-6)
    assert rep["n_tier"][4] > 0
