"""The stored oracle solution of the truncated mixed workload (tests/golden/mixed_nt42_map.json,
which bench.py's mixed block compares its matrix-free solve with) equals a fresh run of the
script that wrote it.  CPU only: about a minute of host time (a 25,200^2 Gram product and its
Cholesky factor).  Two FP64 runs on different BLAS builds sum in different orders; through
the solve with kappa(K) of about 1e4 they agree to about 10 kappa(K) 2^-53 = 1e-11, so 1e-10
is required."""

import importlib.util
import json
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
pytestmark = pytest.mark.slow


def test_stored_truncated_mixed_solution_is_the_oracle_s():
    spec = importlib.util.spec_from_file_location("mixed_nt42_map", os.path.join(HERE, "golden", "mixed_nt42_map.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    with open(mod.PATH) as f:
        stored = json.load(f)
    fresh = mod.compute()
    for key in ("x_idx", "m_idx", "workload", "Nm", "Nd", "Nt", "Nq"):
        assert stored[key] == fresh[key], key
    for key in ("x", "m"):
        a, b = np.array(stored[key + "_val"]), np.array(fresh[key + "_val"])
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-10, key
        assert abs(stored[key + "_norm"] - fresh[key + "_norm"]) < 1e-10 * fresh[key + "_norm"], key
    a, b = np.array(stored["q"]), np.array(fresh["q"])
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-10
