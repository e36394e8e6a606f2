"""Data-space inversion for the oracle (FP64): K, its Cholesky factor, m_map, q_map.

Test infrastructure only; see the package docstring.

Notation: F (p2o map) with blocks F_k, G^* = Gamma_prior F^T with blocks
G_k = F_k C_s, F_q (p2q map) with blocks (F_q)_k, Gamma_noise diagonal.
"""

import numpy as np
import scipy.linalg as sla

from .toeplitz import p2o_apply, p2o_apply_adjoint


def _noise_diag(noise, Nt, R):
    """Gamma_noise as a [N_t * R] vector of variances (a scalar means sigma^2 I)."""
    v = np.asarray(noise, dtype=np.float64)
    if v.ndim == 0:
        return np.full(Nt * R, float(v))
    return v.reshape(Nt * R).copy()


def assemble_K(F_blocks, G_blocks, noise):
    """K = Gamma_noise + F G^* (Sec. 4, Phase 2, the K of Eq. (4.7)).

    Block (t, t') of F G^* is sum_{s=0}^{min(t,t')} F_{t-s} G_{t'-s}^T, because
    F has block (t, s) = F_{t-s} (s <= t) and G^* has block (s, t') =
    G_{t'-s}^T (s <= t').  With W(k, k') := F_k G_{k'}^T this is
    sum_{u=0}^{min(t,t')} W(t-u, t'-u): the terms of block (t, t') are those
    of block (t-1, t'-1) plus W(t, t').  The oracle therefore forms every
    W(k, k') with one matmul and accumulates along block diagonals:
        K(t, 0) = W(t, 0), K(0, t') = W(0, t'),
        K(t, t') = K(t-1, t'-1) + W(t, t')   (t, t' >= 1),
    then adds the diagonal Gamma_noise.  Returns the full (N_t R)^2 matrix;
    data index (t, i) -> t * R + i.
    """
    F_blocks = np.asarray(F_blocks, dtype=np.float64)
    G_blocks = np.asarray(G_blocks, dtype=np.float64)
    Nt, R, Nm = F_blocks.shape
    n = Nt * R
    W = F_blocks.reshape(n, Nm) @ G_blocks.reshape(n, Nm).T
    K = W.copy()
    for t in range(1, Nt):
        rows = slice(t * R, (t + 1) * R)
        prev = slice((t - 1) * R, t * R)
        # block row t, block columns 1..N_t-1 gain block row t-1, columns 0..N_t-2
        K[rows, R:] += K[prev, : n - R]
    K[np.diag_indices(n)] += _noise_diag(noise, Nt, R)
    return K


def assemble_K_columns(F_blocks, G_blocks, noise):
    """K column by column as Sec. 4, Phase 2 describes: K e_j = Gamma_noise e_j + F (G^* e_j).

    One adjoint (G^*) and one forward (F) Toeplitz matvec per data unit vector;
    only for small sizes (used to pin assemble_K).
    """
    F_blocks = np.asarray(F_blocks, dtype=np.float64)
    Nt, R, Nm = F_blocks.shape
    n = Nt * R
    E = np.eye(n).reshape(n, Nt, R)  # all unit vectors as a batch
    K = p2o_apply(F_blocks, p2o_apply_adjoint(G_blocks, E)).reshape(n, n).T
    K = K + np.diag(_noise_diag(noise, Nt, R))
    return K


def cholesky_lower(K):
    """Lower Cholesky factor L with K = L L^T, from the lower triangle of K.

    K is symmetric positive definite (Gamma_noise SPD plus a Gram matrix).  The
    lower triangle is mirrored and LAPACK's factorisation is the step; a matrix
    that is not SPD raises numpy.linalg.LinAlgError.
    """
    K = np.asarray(K, dtype=np.float64)
    Kl = np.tril(K)
    Ksym = Kl + np.tril(K, -1).T
    return np.linalg.cholesky(Ksym)


def solve_K(L, d):
    """x = K^{-1} d = L^{-T} L^{-1} d; d is [n] or [B, n] (one row per RHS)."""
    d = np.asarray(d, dtype=np.float64)
    rhs = d.T if d.ndim == 2 else d
    y = sla.solve_triangular(L, rhs, lower=True)
    x = sla.solve_triangular(L, y, lower=True, trans="T")
    return x.T if d.ndim == 2 else x


def map_point(F_blocks, G_blocks, noise, d_obs, L=None):
    """m_map = G^* K^{-1} d_obs (zero prior mean).

    Eq. (4.13) with m_prior = 0 reads m_map = (I - G^* K^{-1} F) G^* Gamma_n^{-1} d.
    Since K - F G^* = Gamma_n, (I - G^* K^{-1} F) G^* = G^* K^{-1} (K - F G^*)
    = G^* K^{-1} Gamma_n, so m_map = G^* K^{-1} d_obs exactly; the longer form
    is map_point_woodbury_form.  d_obs: [..., N_t, R].  Returns [..., N_t, N_m].
    """
    F_blocks = np.asarray(F_blocks, dtype=np.float64)
    Nt, R, Nm = F_blocks.shape
    if L is None:
        L = cholesky_lower(assemble_K(F_blocks, G_blocks, noise))
    d = np.asarray(d_obs, dtype=np.float64)
    flat = d.reshape(-1, Nt * R)
    x = solve_K(L, flat).reshape(d.shape)
    return p2o_apply_adjoint(G_blocks, x)


def map_point_woodbury_form(F_blocks, G_blocks, noise, d_obs, L=None):
    """Eq. (4.13) term by term: m_map = (I - G^* K^{-1} F) G^* Gamma_n^{-1} d_obs."""
    F_blocks = np.asarray(F_blocks, dtype=np.float64)
    Nt, R, Nm = F_blocks.shape
    if L is None:
        L = cholesky_lower(assemble_K(F_blocks, G_blocks, noise))
    d = np.asarray(d_obs, dtype=np.float64)
    var = _noise_diag(noise, Nt, R).reshape(Nt, R)
    y = p2o_apply_adjoint(G_blocks, d / var)
    Fy = p2o_apply(F_blocks, y)
    z = solve_K(L, Fy.reshape(-1, Nt * R)).reshape(Fy.shape)
    return y - p2o_apply_adjoint(G_blocks, z)


def qoi_map(Fq_blocks, m_map):
    """q_map = F_q m_map, the push-forward of Eq. (4.2)."""
    return p2o_apply(Fq_blocks, m_map)


def loss(F_blocks, m, d, noise, A_s=None):
    """0.5 ||F m - d||^2_{Gamma_n^{-1}} + 0.5 sum_t ||A_s m_t||^2.

    The data misfit is the negative log-likelihood of Sec. 2 (Eq. (2.9)); the
    prior term uses the elliptic operator A_s of Eq. (5.1), whose square is the
    inverse prior covariance of each time block.  A_s=None drops the prior term.
    """
    F_blocks = np.asarray(F_blocks, dtype=np.float64)
    Nt, R, Nm = F_blocks.shape
    var = _noise_diag(noise, Nt, R).reshape(Nt, R)
    r = p2o_apply(F_blocks, m) - d
    val = 0.5 * np.sum(r * r / var)
    if A_s is not None:
        Am = (A_s @ np.asarray(m, dtype=np.float64).reshape(-1, Nm).T).T
        val += 0.5 * np.sum(Am * Am)
    return float(val)


def loss_gradient(F_blocks, m, d, noise, A_s=None):
    """Gradient of loss(): F^T Gamma_n^{-1} (F m - d) + (I_t (x) A_s^T A_s) m."""
    F_blocks = np.asarray(F_blocks, dtype=np.float64)
    Nt, R, Nm = F_blocks.shape
    var = _noise_diag(noise, Nt, R).reshape(Nt, R)
    m = np.asarray(m, dtype=np.float64)
    g = p2o_apply_adjoint(F_blocks, (p2o_apply(F_blocks, m) - d) / var)
    if A_s is not None:
        flat = m.reshape(-1, Nm).T
        g = g + (A_s.T @ (A_s @ flat)).T.reshape(m.shape)
    return g


def qoi_data_gram(Fq_blocks, G_blocks):
    """X = F_q G^* as a dense (N_q N_t) x (N_d N_t) matrix.

    Block (t, t') is sum_{s=0}^{min(t,t')} (F_q)_{t-s} G_{t'-s}^T (both maps are block
    lower-triangular Toeplitz in time); with W(k, k') = (F_q)_k G_{k'}^T the blocks
    accumulate along block diagonals exactly as in assemble_K, on both sides of the
    diagonal since X is not symmetric.
    """
    Fq_blocks = np.asarray(Fq_blocks, dtype=np.float64)
    G_blocks = np.asarray(G_blocks, dtype=np.float64)
    Nt, Rq, Nm = Fq_blocks.shape
    R = G_blocks.shape[1]
    W = Fq_blocks.reshape(Nt * Rq, Nm) @ G_blocks.reshape(Nt * R, Nm).T
    X = W.copy()
    for t in range(1, Nt):
        rows = slice(t * Rq, (t + 1) * Rq)
        prev = slice((t - 1) * Rq, t * Rq)
        X[rows, R:] += X[prev, : (Nt - 1) * R]
    return X


def d2q_map(Fq_blocks, F_blocks, G_blocks, noise, L=None):
    """The data-to-QoI map Q of Eq. (4.11) with zero prior mean, (N_q N_t) x (N_d N_t).

    Eq. (4.11): Q = F_q (I - G^* K^{-1} F) G^* Gamma_n^{-1}.  Since F G^* = K - Gamma_n,
    K^{-1} F G^* Gamma_n^{-1} = Gamma_n^{-1} - K^{-1}, hence Q = F_q G^* K^{-1}; the rows
    of Q are the rows of F_q G^* times K^{-1} (K symmetric).  The long form is pinned
    against this in the tests.
    """
    F_blocks = np.asarray(F_blocks, dtype=np.float64)
    Nt, R, Nm = F_blocks.shape
    if L is None:
        L = cholesky_lower(assemble_K(F_blocks, G_blocks, noise))
    X = qoi_data_gram(Fq_blocks, G_blocks)
    return solve_K(L, X)


def qoi_posterior_covariance(Fq_blocks, Gq_blocks, F_blocks, G_blocks, noise, L=None):
    """Gamma_post(q) of Eq. (4.10): F_q (I - G^* K^{-1} F) G_q^*, with G_q^* = Gamma_prior F_q^T.

    Expanded: F_q G_q^* - (F_q G^*) K^{-1} (F G_q^*), and F G_q^* = (F_q G^*)^T because
    Gamma_prior is symmetric; so Gamma_post(q) = X_qq - Q X^T with X = F_q G^* and
    X_qq = F_q Gamma_prior F_q^T (the same Gram accumulation with G_q blocks).
    """
    X_qq = qoi_data_gram(Fq_blocks, Gq_blocks)
    X = qoi_data_gram(Fq_blocks, G_blocks)
    Q = d2q_map(Fq_blocks, F_blocks, G_blocks, noise, L)
    return X_qq - Q @ X.T


def prior_apply(Cs, v):
    """Gamma_prior v = (I_t (x) C_s) v: the spatial covariance applied to each time block."""
    v = np.asarray(v, dtype=np.float64)
    return v @ np.asarray(Cs, dtype=np.float64).T


def posterior_cov_apply(F_blocks, G_blocks, Cs, noise, v, L=None):
    """Gamma_post(m) v by Eq. (4.7): (I - G^* K^{-1} F) Gamma_prior v, v: [..., N_t, N_m]."""
    F_blocks = np.asarray(F_blocks, dtype=np.float64)
    Nt, R, Nm = F_blocks.shape
    if L is None:
        L = cholesky_lower(assemble_K(F_blocks, G_blocks, noise))
    w = prior_apply(Cs, v)
    y = p2o_apply(F_blocks, w)
    x = solve_K(L, y.reshape(-1, Nt * R)).reshape(y.shape)
    return w - p2o_apply_adjoint(G_blocks, x)


def posterior_variance_probe(F_blocks, G_blocks, Cs, noise, V, L=None):
    """Probe estimate of the pointwise posterior variances diag(Gamma_post(m)) (Sec. 4, Phase 2
    names them among the quantities that follow from Gamma_post(m) actions): elementwise
    sum_s v_s * (Gamma_post(m) v_s) / sum_s v_s * v_s over caller-drawn probes V [S, N_t, N_m],
    0 where no probe touches an entry.  Exact for the unit vectors, and for sign vectors whose
    products cancel off the diagonal (the rows of a Hadamard matrix)."""
    V = np.asarray(V, dtype=np.float64)
    U = posterior_cov_apply(F_blocks, G_blocks, Cs, noise, V, L=L)
    num = (V * U).sum(axis=0)
    den = (V * V).sum(axis=0)
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), 0.0)


def map_point_with_prior_mean(F_blocks, G_blocks, noise, d_obs, m_prior, L=None):
    """m_map of Eq. (4.13) with the prior-mean term of Eq. (4.8).

    Eq. (4.13): m_map = (I - G^* K^{-1} F) G^* Gamma_n^{-1} d + m_map^prior with
    Eq. (4.8): m_map^prior = (I - G^* K^{-1} F) m_prior.  Using the identity of
    map_point for the first term: m_map = G^* K^{-1} d + m_prior - G^* K^{-1} F m_prior.
    """
    F_blocks = np.asarray(F_blocks, dtype=np.float64)
    Nt, R, Nm = F_blocks.shape
    if L is None:
        L = cholesky_lower(assemble_K(F_blocks, G_blocks, noise))
    m_prior = np.asarray(m_prior, dtype=np.float64)
    r = np.asarray(d_obs, dtype=np.float64) - p2o_apply(F_blocks, m_prior)
    x = solve_K(L, r.reshape(-1, Nt * R)).reshape(r.shape)
    return m_prior + p2o_apply_adjoint(G_blocks, x)


def qoi_time_steps(Nt, stride):
    """0-based fine time steps that carry the QoIs on a grid of N_t^q = N_t / stride points.

    The Remark after Eq. (2.15) lets the QoI time grid be coarser than the time-stepping
    grid, and the example of Sec. 5 takes parameters and data at 10 Hz on (0, 50) s
    (N_t = 500) with QoIs at 1 Hz (N_t^q = 50).  QoI k is read at the end of its
    interval, time (k + 1) * stride * dt, i.e. fine step stride (k + 1) - 1, so the
    last QoI falls on the final time T.
    """
    if stride < 1 or Nt % stride:
        raise ValueError(f"stride {stride} must divide N_t = {Nt}")
    return np.arange(stride - 1, Nt, stride)


def qoi_rows(Nt, Nq, stride):
    """Indices of the coarse-grid QoI entries within a fine-grid QoI vector [N_t][N_q]
    (flattened): the rows of Q, and the rows and columns of Gamma_post(q), that remain
    on the QoI grid of qoi_time_steps."""
    steps = qoi_time_steps(Nt, stride)
    return (steps[:, None] * Nq + np.arange(Nq)[None, :]).reshape(-1)
