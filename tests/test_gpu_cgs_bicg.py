"""CGS and BiCG (krylov="cgs" / "bicg", the other solvers section 5 names):
Procedure * with them against the oracle's, the transposed solves, and the
solvers over a thousand systems (the panel SpMV path).

 - 2D workload, SPAI(0.4, 5, 10), eps = 1e-8: per-system iterations within
   +-1 of the oracle's Procedure * with the same solver, rr < eps, x within
   1e-6; transposed solves (A~^T with M^T, BiCG's shadow then runs with A~ M)
   against the oracle's solver on the transposes.
 - Zipf-count matrix at n = 20000 (s = 1066, so 1067 systems): every sampled
   system meets its threshold on the true residual, and four systems give
   the same bits when solved on their own.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
import workloads as W
from gpu_helpers import lib, need_gpu, to_dev, to_scipy, torch

pytestmark = pytest.mark.gpu

SPAI = dict(delta=0.4, mn=5, max_aug=10)


@pytest.mark.parametrize("krylov", ["cgs", "bicg"])
def test_procedure_with_cgs_matches_oracle(krylov):
    need_gpu()
    sai = lib()
    P = W.convdiff2d_irregular()
    x, iters, rep = sai.solve(to_dev(P.A), torch.as_tensor(P.b, device="cuda"), krylov=krylov, eps=1e-8, **SPAI)
    xo, it_o, rep_o = O.solve(P.A, P.b, krylov=krylov, eps=1e-8, **SPAI)
    assert rep["status"] == sai.SAI_OK and rep_o["status"] == O.OK
    assert all(abs(a - b) <= 1 for a, b in zip(iters, it_o)), (iters, list(it_o))
    assert rep["rr"] < 1e-8
    np.testing.assert_allclose(x.cpu().numpy(), xo, rtol=0, atol=1e-6)


@pytest.mark.parametrize("krylov", ["cgs", "bicg"])
def test_transposed_solves_match_oracle(krylov):
    need_gpu()
    sai = lib()
    P = W.convdiff2d_irregular()
    sp_ = sai.split(to_dev(P.A))
    Pc = sai.build_spai(sp_, **SPAI)
    At, M = to_scipy(sp_.arrays()[0]), to_scipy(Pc.arrays()[0])
    AtT, MT = sp.csc_matrix(At.T), sp.csc_matrix(M.T)
    B = np.random.default_rng(4).standard_normal((P.n, 3))
    thr = [1e-9 * np.linalg.norm(B[:, q]) for q in range(3)]
    meth = sai.CGS if krylov == "cgs" else sai.BICG
    X, iters, status, st = sai.krylov_solve(sp_, Pc, torch.as_tensor(B, device="cuda"), thr, method=meth,
                                            transpose=True)
    assert st == sai.SAI_OK
    fn = O.cgs if krylov == "cgs" else O.bicg
    for q in range(3):
        yo, it, sto = fn(AtT, MT, B[:, q], thr[q])
        assert sto == O.OK and abs(iters[q] - it) <= 1, (q, iters[q], it)
        np.testing.assert_allclose(X[:, q].cpu().numpy(), yo, rtol=0, atol=1e-6 * np.abs(yo).max())


@pytest.mark.parametrize("krylov", ["cgs", "bicg"])
def test_cgs_over_a_thousand_systems(krylov):
    need_gpu()
    sai = lib()
    P = W.zipf_columns(n=20000)
    A = sp.csc_matrix(P.A)
    sp_ = sai.split(to_dev(A), abs_tau=200.0)
    Pc = sai.build_spai(sp_, **SPAI)
    J, p, _ = O.detect(A, abs_tau=200.0)
    At, U = O.split(A, J, p)
    At, U = sp.csc_matrix(At), sp.csc_matrix(U)
    s = sp_.s
    assert s == len(J) > 256
    B = np.zeros((P.n, s + 1))
    B[:, 0] = P.b
    B[:, 1:] = U.toarray()
    bn = np.linalg.norm(P.b)
    thr = [0.5e-10 * bn] + [1e-10 * bn / (2 * np.sqrt(s))] * s
    Bd = torch.as_tensor(B, device="cuda")
    meth = sai.CGS if krylov == "cgs" else sai.BICG
    X, iters, status, st = sai.krylov_solve(sp_, Pc, Bd, thr, method=meth)
    assert st == sai.SAI_OK
    Xh = X.cpu().numpy()
    sel = np.concatenate([[0], np.random.default_rng(2).choice(np.arange(1, s + 1), 100, replace=False)])
    for c in sel:
        assert np.linalg.norm(B[:, c] - At @ Xh[:, c]) < 1.5 * thr[c], c
    few = [0, 1, 300, s]
    idx = torch.as_tensor(few, device="cuda")
    X2, it2, _, _ = sai.krylov_solve(sp_, Pc, Bd[:, idx].contiguous(), [thr[c] for c in few], method=meth)
    assert it2 == [iters[c] for c in few]
    assert torch.equal(X2, X[:, idx])
