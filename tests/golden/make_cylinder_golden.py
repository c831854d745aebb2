"""Write tests/golden/cylinder_oracle.json: FP64 oracle results on the full-size
hollow cylinder (1,073,280 vertices, 16^3 boxes), at sampled vertices.

    python tests/golden/make_cylinder_golden.py

Calls only the oracle (oracle/cgs_oracle.py) and the seeded mesh generator;
nothing here comes from the CUDA path.  The oracle's set-up of this mesh takes
about two minutes and its solve about a quarter of an hour on one core, which
is why the results are stored instead of recomputed by each test.

Stored (vertex indices drawn by default_rng(11) among the free vertices):
  apply_A      (A b)_v                         Sec. 3, A = Q^T A_L Q
  local_w      (W_ov sum_p R_p^T A_p^{-1} R_p b)_v     Eq. (4)
  m_hybrid     (M b)_v, hybrid ASM_1 + ASM_2   Eqs. (4), (5)
  m_additive   (M b)_v, additive               Eq. (3)
  solve        flexible PCG on A x = b, hybrid, rtol 1e-8: iterations, true
               relative residual, x_v
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import cgs_oracle as O  # noqa: E402
from paper_2606_20496_b300 import meshes  # noqa: E402

NSAMPLE = 256


def main():
    m, b = meshes.workload_cylinder()
    t0 = time.time()
    P = O.Problem(m.xyz, m.conn, m.part, m.boxes)
    t_setup = time.time() - t0
    b = np.where(P.dir, 0.0, b)
    idx = np.sort(np.random.default_rng(11).choice(P.free, NSAMPLE, replace=False))
    out = {"citation": "Sec. 3 (A = Q^T A_L Q, Eq. (4)), Sec. 4 (box coarse space, Eq. (5)), flexible PCG; "
                       "written by tests/golden/make_cylinder_golden.py from the FP64 oracle",
           "mesh": "hollow cylinder 64 x 128 x 128 hexes (workload_cylinder(), RHS seed 6), 16^3 boxes, "
                   "2^3-element subdomains grown by one layer",
           "nv": m.nv, "n_r": int(P.nr), "idx": idx.tolist()}
    out["apply_A"] = P.apply_A(b)[idx].tolist()
    out["local_w"] = P.local_solves(b, weighted=True)[idx].tolist()
    out["m_hybrid"] = P.apply_M(b, "hybrid")[idx].tolist()
    out["m_additive"] = P.apply_M(b, "additive")[idx].tolist()
    t0 = time.time()
    x, its, rel, ok = P.solve(b, rtol=1e-8, maxit=1000)
    out["solve"] = {"rtol": 1e-8, "form": "hybrid", "iters": int(its), "relres": float(rel),
                    "converged": bool(ok), "x": x[idx].tolist(), "x_norm": float(np.linalg.norm(x))}
    out["oracle_seconds"] = {"setup": round(t_setup, 1), "solve": round(time.time() - t0, 1)}
    with open(os.path.join(HERE, "cylinder_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: out[k] for k in ("nv", "n_r", "oracle_seconds")}), out["solve"]["iters"])


if __name__ == "__main__":
    main()
