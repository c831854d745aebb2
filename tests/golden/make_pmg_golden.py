"""Write tests/golden/pmg_oracle.json: FP64 oracle results of the p-multigrid
wrap on its full-size workload (the 32^3 deformed cube, spectral elements of
order 7, schedule 7 -> 3 -> 1, 11,390,625 nodes), at sampled element-local
nodes.

    python tests/golden/make_pmg_golden.py

Calls only the oracle (oracle/sem_oracle.py, oracle/cgs_oracle.py) and the
seeded input generators; nothing here comes from the CUDA path.  The two
sides number the nodes differently, so every stored value is addressed by
(element, k, j, i) of the element-local layout.

Stored (positions drawn by default_rng(12)):
  apply_A   (A_7 b) at the positions          Sec. 1, A = Q^T A_L Q
  m_pmg     (M b), Eq. (13) with Eq. (14) smoothers and one two-level
            Schwarz sweep at order 1
  solve     flexible GMRES(30) on A_7 x = b, rtol 1e-8: products A z, true
            relative residual, x at the positions, ||x||
b is meshes.sem_rhs at the node coordinates, zero on Dirichlet nodes.
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

from oracle import sem_oracle as S  # noqa: E402
from paper_2606_20496_b300 import meshes  # noqa: E402

NSAMPLE = 256


def main():
    m, orders = meshes.workload_sem()
    t0 = time.time()
    P = S.PMG(m.xyz, m.conn, m.part, m.boxes, orders=orders)
    t_setup = time.time() - t0
    f = P.fine
    b = np.where(f.dir, 0.0, meshes.sem_rhs(f.node_coords()))
    rng = np.random.default_rng(12)
    p = f.p
    pos = np.stack([rng.integers(0, m.ne, NSAMPLE), rng.integers(0, p, NSAMPLE), rng.integers(0, p, NSAMPLE),
                    rng.integers(0, p, NSAMPLE)], axis=1)
    g = f.l2g[pos[:, 0], pos[:, 1], pos[:, 2], pos[:, 3]]
    out = {"citation": "Sec. 1 (SEM operator), Sec. 5 (Eq. (13), Eq. (14), GMRES on the pressure); "
                       "written by tests/golden/make_pmg_golden.py from the FP64 oracle",
           "mesh": "32^3 smoothly deformed cube, elements permuted (workload_cube32), 8^3 boxes, "
                   "spectral elements of order 7, schedule 7 -> 3 -> 1, b = sem_rhs (seed 9)",
           "orders": list(orders), "n_nodes": int(f.ng), "n_free": int((~f.dir).sum()),
           "positions": pos.tolist()}
    out["apply_A"] = P.apply_A(b)[g].tolist()
    out["m_pmg"] = P.apply_M(b)[g].tolist()
    t0 = time.time()
    x, its, rel, ok = P.solve(b, rtol=1e-8, maxit=300, restart=30)
    true_rel = float(np.linalg.norm(b - P.apply_A(x)) / np.linalg.norm(b))
    out["solve"] = {"rtol": 1e-8, "restart": 30, "iters": int(its), "relres": true_rel, "converged": bool(ok),
                    "x": x[g].tolist(), "x_norm": float(np.linalg.norm(x))}
    out["oracle_seconds"] = {"setup": round(t_setup, 1), "solve": round(time.time() - t0, 1)}
    with open(os.path.join(HERE, "pmg_oracle.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps({k: out[k] for k in ("n_nodes", "n_free", "oracle_seconds")}), its, true_rel)


if __name__ == "__main__":
    main()
