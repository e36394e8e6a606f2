"""Writes mixed_nt42_map.json: the oracle's MAP point for one observation vector of the
mixed-precision workload truncated to its first 42 time steps (K 25,200^2).

The full mixed workload's K (252,000^2, 508 GB) cannot be formed, so the forward error of
its matrix-free solve is measured at this truncation, where the oracle's dense Cholesky
solve applies.  The file keeps what bench.py needs to report that error without running
the oracle: x = K^{-1} d, m_map = G^* x and q_map = F_q m_map for d = vectors_d(1)[0] (white
N(0,1) data), as 1,024 seeded sampled entries of x and of m_map with their full norms, and
q_map whole.

Calls only the oracle (and the seeded input generator).  Run from the repository root:
    python tests/golden/mixed_nt42_map.py
A CPU test (tests/test_golden_mixed.py) recomputes it and compares.
"""

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2501_14911_gb300 import synthetic  # noqa: E402

PATH = os.path.join(HERE, "mixed_nt42_map.json")
SAMPLES = 1024


def compute():
    p = synthetic.MIXED_NT42
    F, Fq = p.blocks_F(), p.blocks_Fq()
    d = p.vectors_d(1)
    G = oracle.prior_blocks_separable(F, p.gx, p.gy, p.ell, p.sigma_p)
    K = oracle.assemble_K(F, G, p.sigma2)
    L = oracle.cholesky_lower(K)
    del K
    x = oracle.solve_K(L, d.reshape(1, -1)).reshape(d.shape)
    m = oracle.p2o_apply_adjoint(G, x)
    q = oracle.qoi_map(Fq, m)
    rng = np.random.default_rng(2501)
    xi = np.sort(rng.choice(x.size, SAMPLES, replace=False))
    mi = np.sort(rng.choice(m.size, SAMPLES, replace=False))
    xf, mf = x.reshape(-1), m.reshape(-1)
    out = {
        "_source": "oracle/ (dense Cholesky solve of Sec. 4, Phase 2 and Eq. (4.13) with the SE prior of "
                   "reading R4) on the mixed workload truncated to N_t = 42; written by mixed_nt42_map.py",
        "workload": p.name, "Nm": p.Nm, "Nd": p.Nd, "Nt": p.Nt, "Nq": p.Nq, "sigma2": p.sigma2,
        "data": "vectors_d(1)[0], white N(0,1)",
        "x_norm": float(np.linalg.norm(xf)), "x_idx": xi.tolist(), "x_val": xf[xi].tolist(),
        "m_norm": float(np.linalg.norm(mf)), "m_idx": mi.tolist(), "m_val": mf[mi].tolist(),
        "q": q.reshape(-1).tolist(),
    }
    return out


if __name__ == "__main__":
    rec = compute()
    with open(PATH, "w") as f:
        json.dump(rec, f, indent=0)
    print("wrote", PATH)
