"""Parity bookkeeping for the GPU tests: the error metric, tolerances derived from the
conditioning of K and the unit roundoff of the arithmetic, and a record of every measured
error, which the test session prints at its end (tightest margins last).

Error metric (reading R11): normwise ||x - x_ref|| / ||x_ref|| per right-hand side, the
maximum over the batch, in FP64.

Tolerances (reading R20).  Products of the FP64-accurate tiers are held to 1e-12.  A result
that passes through a solve with K (m_map, q_map, x = K^{-1} d, the Cholesky factor) is held
to

    tol = max(1e-12, C kappa(K) u)                                     (solves)
    tol = max(1e-12, C kappa(K) rho u),  rho = ||K^{-1}|| ||d|| / ||K^{-1} d||   (explicit inverse)

with C = 10, kappa(K) = lambda_max / lambda_min measured from the oracle's K at the test's own
size, and u the unit roundoff of the arithmetic that bounds the result: 2^-53 for FP64, 2^-48
for the double-FP32 (float-pair) arithmetic, 2^-47 for the digit planes.  The first form is
the forward-error bound of a backward-stable solve ((K + dK) x = d with ||dK|| ~ u ||K||), and
of iterative refinement whose residual is computed in precision u (the limiting accuracy is of
order kappa(K) u_residual).  The second is that of x = X d with a computed inverse X whose
error is of order kappa(K) u ||K^{-1}||: the error ||dX|| ||d|| relative to ||x|| picks up the
factor rho in [1, kappa(K)], which the test computes from the oracle's solution.  A conjugate-
gradient solve stopped at ||d - K x|| <= eta ||d|| has ||x - x*|| <= ||K^{-1}|| eta ||d||
= rho eta ||x*||, so it is held to max(1e-12, rho eta + C kappa(K) u) with u its operator's.
m_map = G^* x and q_map = F_q m_map are held to the bound of x: the errors a solve amplifies
lie along the eigenvectors v of K's small eigenvalues lambda, and there ||G^* v||^2 <=
||Gamma_prior|| (lambda - sigma^2) is small, so G^* damps rather than amplifies them.  A result
formed by a subtraction that cancels (Gamma_post(q) = X_qq - Q X^T, Gamma_post(m) v = w -
G^* K^{-1} F w) carries the bound of the subtracted term times gamma = ||subtracted term|| /
||result||, from the oracle.
"""

from __future__ import annotations

import inspect
import os

import numpy as np

U_F64 = 2.0 ** -53
U_DF64 = 2.0 ** -48   # float pairs (about 48 significant bits)
U_DIGITS = 2.0 ** -47  # six FP16 digit planes: a 47-bit fixed-point image of each row
FLOOR = 1e-12
C_BOUND = 10.0

RECORDS: list[tuple[str, str, float, float]] = []


def rel(a, b):
    """||a - b|| / ||b|| over the whole array."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def relb(a, b):
    """max over the leading batch axis of ||a_b - b_b|| / ||b_b||."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    a = a.reshape(a.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    num = np.linalg.norm(a - b, axis=1)
    den = np.maximum(np.linalg.norm(b, axis=1), 1e-300)
    return float(np.max(num / den))


def _where():
    test = os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]
    frame = inspect.currentframe().f_back.f_back
    return f"{test}:{frame.f_lineno}"


def check(err, tol, what=""):
    """Assert err < tol and record both for the end-of-session parity table."""
    err = float(err)
    where = _where()
    RECORDS.append((where, what, err, float(tol)))
    assert err < tol, f"{where} {what}: measured error {err:.3e} is not below the tolerance {tol:.3e}"


def spd_extremes(K, L=None):
    """(lambda_min, lambda_max) of the SPD matrix whose lower triangle K holds.

    Up to n = 6000 from the eigenvalues; above that, the largest by Lanczos on K and the
    smallest by Lanczos on K^{-1} applied with the Cholesky factor L (computed if not given),
    to three digits."""
    import scipy.linalg as sla
    import scipy.sparse.linalg as spla

    K = np.asarray(K, dtype=np.float64)
    n = K.shape[0]
    Ks = np.tril(K) + np.tril(K, -1).T
    if n <= 6000:
        ev = np.linalg.eigvalsh(Ks)
        return float(ev[0]), float(ev[-1])
    if L is None:
        L = np.linalg.cholesky(Ks)
    opK = spla.LinearOperator((n, n), matvec=lambda v: Ks @ v, dtype=np.float64)

    def kinv(v):
        w = sla.solve_triangular(L, v, lower=True, check_finite=False)
        return sla.solve_triangular(L, w, lower=True, trans="T", check_finite=False)

    opKi = spla.LinearOperator((n, n), matvec=kinv, dtype=np.float64)
    lmax = float(spla.eigsh(opK, k=1, which="LA", tol=1e-3, return_eigenvectors=False)[0])
    mu = float(spla.eigsh(opKi, k=1, which="LA", tol=1e-3, return_eigenvectors=False)[0])
    return 1.0 / mu, lmax


def kappa_spd(K, L=None):
    """2-norm condition number lambda_max / lambda_min (spd_extremes)."""
    lmin, lmax = spd_extremes(K, L)
    return lmax / lmin


def tol_solve(kappa, u):
    """Forward-error tolerance of a backward-stable solve (or of refinement with residuals in u)."""
    return max(FLOOR, C_BOUND * kappa * u)


def rho_inverse(lmin, d, x):
    """max over the batch of ||K^{-1}|| ||d_b|| / ||x_b||, x = K^{-1} d (the oracle's solution)."""
    d = np.asarray(d, dtype=np.float64).reshape(np.shape(d)[0], -1)
    x = np.asarray(x, dtype=np.float64).reshape(np.shape(x)[0], -1)
    return float(np.max(np.linalg.norm(d, axis=1) / (lmin * np.linalg.norm(x, axis=1))))


def tol_inverse(kappa, u, rho):
    """Forward-error tolerance of x = X d with a computed explicit inverse X."""
    return max(FLOOR, C_BOUND * kappa * rho * u)


def tol_cg(kappa, u, rho, eta):
    """Forward-error tolerance of a conjugate-gradient solve stopped at relative residual eta."""
    return max(FLOOR, rho * eta + C_BOUND * kappa * u)


def summary_lines():
    """The recorded errors as text lines, smallest margin (err / tol largest) last."""
    if not RECORDS:
        return []
    rows = sorted(RECORDS, key=lambda r: r[2] / r[3])
    out = [f"parity: {len(rows)} checks; measured error / tolerance (tightest last)"]
    for where, what, err, tol in rows:
        name = where.split("::", 1)[-1]
        out.append(f"  {err:9.2e} / {tol:8.1e}  ({err / tol:5.3f})  {name} {what}".rstrip())
    return out
