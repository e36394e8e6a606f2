"""Prior covariances for the oracle (FP64).

Test infrastructure only; see the package docstring.

The prior is time-invariant, so Gamma_prior = I_t (x) C_s is block diagonal
(Sec. 5, footnote on the shift invariance of the prior) and
G^* = Gamma_prior F^T is block Toeplitz with blocks G_k = F_k C_s
(Sec. 4, Phase 2, the definition of G^* before Eq. (4.7)).
"""

import numpy as np
import scipy.sparse as sp


def se_covariance_1d(n, ell, sigma):
    """sigma * exp(-(a - b)^2 / (2 ell^2)) on n integer nodes (one grid axis)."""
    a = np.arange(n, dtype=np.float64)
    return sigma * np.exp(-((a[:, None] - a[None, :]) ** 2) / (2.0 * ell * ell))


def se_covariance(gx, gy, ell, sigma):
    """Dense squared-exponential spatial covariance C_s on a gx x gy grid.

    C_s[a, b] = sigma^2 exp(-|x_a - x_b|^2 / (2 ell^2)), nodes at integer
    coordinates (distances in cell units), node index a = ix * gy + iy.
    Written from the coordinates directly (no separable shortcut).
    """
    ix, iy = np.meshgrid(np.arange(gx), np.arange(gy), indexing="ij")
    x = ix.reshape(-1).astype(np.float64)
    y = iy.reshape(-1).astype(np.float64)
    r2 = (x[:, None] - x[None, :]) ** 2 + (y[:, None] - y[None, :]) ** 2
    return (sigma * sigma) * np.exp(-r2 / (2.0 * ell * ell))


def prior_blocks(blocks, Cs):
    """G_k = F_k C_s for every block k, so that G^* = Gamma_prior F^T."""
    blocks = np.asarray(blocks, dtype=np.float64)
    return blocks @ np.asarray(Cs, dtype=np.float64)


def prior_blocks_separable(blocks, gx, gy, ell, sigma):
    """G_k = F_k C_s for the squared-exponential C_s of se_covariance, applied through its
    Kronecker structure: with node index a = ix * gy + iy, C_s = C_x (x) C_y where C_x and C_y
    are the 1-D kernels of se_covariance_1d(., ell, sigma) (sigma^2 = sigma * sigma splits one
    sigma onto each axis, since exp(-(dx^2 + dy^2) / (2 ell^2)) factors).  Row r of F_k viewed
    as a gx x gy array X_r maps to C_x X_r C_y (both factors symmetric).  Equal to
    prior_blocks(blocks, se_covariance(gx, gy, ell, sigma)) at O(N_m (gx + gy)) per row instead
    of O(N_m^2)."""
    blocks = np.asarray(blocks, dtype=np.float64)
    Cx = se_covariance_1d(gx, ell, sigma)
    Cy = se_covariance_1d(gy, ell, sigma)
    X = blocks.reshape(blocks.shape[:-1] + (gx, gy))
    return (Cx @ X @ Cy).reshape(blocks.shape)


def _sym_sqrt(C):
    w, V = np.linalg.eigh(C)
    w = np.clip(w, 0.0, None)
    return (V * np.sqrt(w)) @ V.T


def prior_sample(z, gx, gy, ell, sigma):
    """m = C_s^{1/2} z for each time block (prior draw with zero mean).

    C_s on a regular grid is the Kronecker product of two 1-D SE matrices
    (ix-major ordering), so its symmetric root is the Kronecker product of the
    1-D roots; negative rounding eigenvalues are clipped to zero.  z has shape
    [..., N_t, gx*gy].
    """
    z = np.asarray(z, dtype=np.float64)
    Rx = _sym_sqrt(se_covariance_1d(gx, ell, sigma))
    Ry = _sym_sqrt(se_covariance_1d(gy, ell, sigma))
    Z = z.reshape(z.shape[:-1] + (gx, gy))
    M = Rx @ Z @ Ry  # (Rx (x) Ry) vec(Z) with ix-major vec
    return M.reshape(z.shape)


def elliptic_operator(gx, gy, alpha1, alpha2):
    """A_s = alpha1 I - alpha2 Delta_h on the gx x gy grid, as a sparse matrix.

    Eq. (5.1) defines the prior covariance as (alpha1 I - alpha2 Delta_h)^{-2}.
    Delta_h is the 5-point Laplacian with unit spacing and homogeneous Neumann
    boundaries in its natural (graph) form: (Delta_h u)_p = sum over grid
    neighbours q of (u_q - u_p).  The paper's Robin coefficient is not given,
    so Neumann stands in for it.  Node index a = ix * gy + iy.
    """
    n = gx * gy
    rows, cols, vals = [], [], []
    deg = np.zeros(n)
    for ix in range(gx):
        for iy in range(gy):
            a = ix * gy + iy
            for jx, jy in ((ix - 1, iy), (ix + 1, iy), (ix, iy - 1), (ix, iy + 1)):
                if 0 <= jx < gx and 0 <= jy < gy:
                    rows.append(a)
                    cols.append(jx * gy + jy)
                    vals.append(-alpha2)
                    deg[a] += 1.0
    rows.extend(range(n))
    cols.extend(range(n))
    vals.extend(alpha1 + alpha2 * deg)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
