"""Writes tests/golden/oracle_convdiff3d_m64_s10.json by running ONLY the oracle.

Workload: 3D 7-point convection-diffusion, 64^3 grid (n = 262144), Peclet 10,
10 dense columns at 5 % scaled to sum|.| = 0.5|a_jj| (workloads.convdiff3d_irregular
defaults); Procedure * with SPAI(delta=0.3, mn=5, max_aug=10) and with
PSAI(delta=0.3, fixed tol 1e-3, lmax=10), GMRES(50), eps = 1e-10, maxit 500.
Stored: split sizes, nnz(M), n_c, l_m, the s+1 iteration counts and rr.
Run: python tests/golden/make_oracle_convdiff3d.py   (about 2 minutes on one core)
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402

CASES = {
    "spai": dict(sai="spai", delta=0.3, mn=5, max_aug=10),
    "psai": dict(sai="psai", delta=0.3, tol=1e-3, tol_mode=1, lmax=10),
}


def main():
    P = W.convdiff3d_irregular()
    out = {"workload": P.name, "n": P.n, "nnz": int(P.A.nnz), "params": P.params,
           "krylov": {"method": "gmres", "restart": 50, "eps": 1e-10, "maxit": 500}, "cases": {}}
    for name, kw in CASES.items():
        t = time.time()
        x, iters, rep = O.solve(P.A, P.b, krylov="gmres", restart=50, eps=1e-10, maxit=500, **kw)
        rep = {k: (float(v) if isinstance(v, float) else int(v)) for k, v in rep.items()}
        out["cases"][name] = {"sai_params": kw, "iters": [int(i) for i in iters], "report": rep,
                              "oracle_seconds": round(time.time() - t, 2)}
        print(name, iters, rep["rr"], file=sys.stderr)
    with open(os.path.join(HERE, "oracle_convdiff3d_m64_s10.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
