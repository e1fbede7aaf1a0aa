"""Writes tests/golden/oracle_zerodiag_m64_s10.json by running ONLY the oracle.

Workload: the 64^3 system of workloads.convdiff3d_irregular (n = 262144, ten
5 % columns) with a seeded cycle over 5 % of its rows (workloads.rows_displaced
defaults), which puts zeros on the diagonal. Procedure * after the oracle's
zero-diagonal repair (section 5): maximum transversal, A(p,:), SPAI(delta=0.3,
mn=5, max_aug=10), GMRES(50), eps = 1e-10, maxit 500.
Stored: the transversal's size and moved columns, the s+1 iteration counts,
the solve report and the oracle's time.
Run: python tests/golden/make_oracle_zerodiag64.py   (under a minute on one core)
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402

SPAI = dict(sai="spai", delta=0.3, mn=5, max_aug=10)


def main():
    P = W.rows_displaced(W.convdiff3d_irregular())
    t = time.time()
    x, iters, rep, p = O.solve_repaired(P.A, P.b, krylov="gmres", restart=50, eps=1e-10, maxit=500, **SPAI)
    secs = time.time() - t
    rep = {k: (float(v) if isinstance(v, float) else int(v)) for k, v in rep.items()}
    out = {"workload": P.name, "n": P.n, "nnz": int(P.A.nnz), "params": P.params,
           "krylov": {"method": "gmres", "restart": 50, "eps": 1e-10, "maxit": 500}, "sai_params": SPAI,
           "moved": int((p != np.arange(P.n)).sum()), "rank": int((p >= 0).sum()),
           "iters": [int(i) for i in iters], "report": rep, "oracle_seconds": round(secs, 2)}
    print(iters, rep["rr"], file=sys.stderr)
    with open(os.path.join(HERE, "oracle_zerodiag_m64_s10.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
