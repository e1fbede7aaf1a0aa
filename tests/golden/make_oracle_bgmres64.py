"""Writes tests/golden/oracle_bgmres_m64_s10.json by running ONLY the oracle.

Workload: the 64^3 system of workloads.convdiff3d_irregular (n = 262144, ten
5 % columns); Procedure * with SPAI(delta=0.3, mn=5, max_aug=10) and block
GMRES(50) over the s+1 = 11 systems, eps = 1e-10, maxit 500.
Stored: the per-system block-step counts, the solve report, the oracle's
seconds for the complete block solve, and for its first 10 block steps alone
(the sample the benchmark times on its own host to scale the former).
Run: python tests/golden/make_oracle_bgmres64.py   (tens of minutes on one core)
"""
import json
import os
import sys
import time

import numpy as np
import scipy.sparse as sp

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402

SPAI = dict(delta=0.3, mn=5, max_aug=10)
EPS = 1e-10
SAMPLE_STEPS = 10


def main():
    P = W.convdiff3d_irregular()
    J, p, _ = O.detect(P.A)
    At, U = O.split(P.A, J, p)
    At = sp.csc_matrix(At)
    M = sp.csc_matrix(O.spai(At, SPAI["delta"], SPAI["mn"], SPAI["max_aug"])[0])
    s = len(J)
    B = np.hstack([P.b[:, None], sp.csc_matrix(U).toarray()])
    bn = np.linalg.norm(P.b)
    thr = np.array([0.5 * EPS * bn] + [EPS * bn / (2.0 * np.sqrt(s))] * s)
    t = time.time()
    O.block_gmres(At, M, B, thr, restart=50, maxit=SAMPLE_STEPS)
    t_sample = time.time() - t
    t = time.time()
    Y, it, st = O.block_gmres(At, M, B, thr, restart=50, maxit=500)
    t_full = time.time() - t
    x, iters, rep = O.solve(P.A, P.b, krylov="bgmres", restart=50, eps=EPS, maxit=500, **SPAI)
    rep = {k: (float(v) if isinstance(v, float) else int(v)) for k, v in rep.items()}
    out = {"workload": P.name, "n": P.n, "nnz": int(P.A.nnz), "params": P.params,
           "krylov": {"method": "block gmres", "restart": 50, "eps": EPS, "maxit": 500}, "sai_params": SPAI,
           "block_steps": [int(i) for i in it], "status": int(st), "report": rep,
           "krylov_seconds": round(t_full, 2), "sample_steps": SAMPLE_STEPS, "sample_seconds": round(t_sample, 3)}
    print(list(it), rep["rr"], t_full, t_sample, file=sys.stderr)
    with open(os.path.join(HERE, "oracle_bgmres_m64_s10.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
