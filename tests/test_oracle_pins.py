"""Pins for the CPU oracle: each check ties an oracle routine to something other
than itself (the LTI recursion, the dense matrix of Eq. (2.5), library routines,
closed forms, exact identities, finite differences).  CPU only."""

import json
import os

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from paper_2501_14911_gb300 import synthetic

HERE = os.path.dirname(os.path.abspath(__file__))


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def micro(seed=7, Nt=6, R=3, Nm=5):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((Nt, R, Nm)) * np.exp(-np.arange(Nt) / 3.0)[:, None, None], rng


# ---------------------------------------------------------------- Toeplitz maps

def test_p2o_matches_lti_time_stepping():
    """F_k = B A^k C applied by convolution equals running Eq. (2.2) from w_0 = 0."""
    rng = np.random.default_rng(1)
    Ns, Nm, Nd, Nt = 9, 4, 3, 12
    A = rng.standard_normal((Ns, Ns))
    A *= 0.9 / np.max(np.abs(np.linalg.eigvals(A)))
    B = rng.standard_normal((Nd, Ns))
    C = rng.standard_normal((Ns, Nm))
    m = rng.standard_normal((Nt, Nm))
    blocks = oracle.lti_blocks(A, B, C, Nt)
    np.testing.assert_allclose(blocks[0], B @ C, rtol=1e-15, atol=0)
    np.testing.assert_allclose(blocks[2], B @ A @ A @ C, rtol=1e-13, atol=1e-15)
    d_conv = oracle.p2o_apply(blocks, m)
    d_sim = oracle.lti_simulate(A, B, C, m)
    assert rel(d_conv, d_sim) < 1e-13


def test_p2o_matches_dense_matrix():
    blocks, rng = micro()
    Nt, R, Nm = blocks.shape
    P = oracle.p2o_dense(blocks)
    m = rng.standard_normal((2, Nt, Nm))
    d = oracle.p2o_apply(blocks, m)
    for b in range(2):
        assert rel(d[b].reshape(-1), P @ m[b].reshape(-1)) < 1e-14
    d2 = rng.standard_normal((Nt, R))
    assert rel(oracle.p2o_apply_adjoint(blocks, d2).reshape(-1), P.T @ d2.reshape(-1)) < 1e-14


def test_dense_matrix_is_scipy_toeplitz_in_scalar_case():
    """R = N_m = 1: Eq. (2.5) is the lower-triangular Toeplitz matrix of the block sequence."""
    f = np.random.default_rng(3).standard_normal(7)
    P = oracle.p2o_dense(f.reshape(7, 1, 1))
    T = sla.toeplitz(f, np.r_[f[0], np.zeros(6)])
    np.testing.assert_array_equal(P, T)


def test_scalar_case_is_truncated_convolution():
    rng = np.random.default_rng(4)
    f = rng.standard_normal(11)
    m = rng.standard_normal(11)
    d = oracle.p2o_apply(f.reshape(11, 1, 1), m.reshape(11, 1)).reshape(-1)
    np.testing.assert_allclose(d, np.convolve(f, m)[:11], rtol=1e-13, atol=1e-14)


def test_single_time_step_is_gemv():
    rng = np.random.default_rng(5)
    F0 = rng.standard_normal((1, 4, 9))
    m = rng.standard_normal((1, 9))
    np.testing.assert_allclose(oracle.p2o_apply(F0, m)[0], F0[0] @ m[0], rtol=1e-15)


def test_impulse_response_is_bit_exact():
    """m = e_(s, j) gives d[t] = F_{t-s}[:, j] for t >= s and 0 before (causality)."""
    blocks, _ = micro(Nt=8, R=2, Nm=4)
    Nt, R, Nm = blocks.shape
    for s, j in ((0, 0), (3, 2), (7, 3)):
        m = np.zeros((Nt, Nm))
        m[s, j] = 1.0
        d = oracle.p2o_apply(blocks, m)
        expect = np.zeros((Nt, R))
        for t in range(s, Nt):
            expect[t] = blocks[t - s][:, j]
        np.testing.assert_array_equal(d, expect)
        # adjoint impulse: d = e_(t, i) gives m[s'] = F_{t-s'}[i, :] for s' <= t
        dd = np.zeros((Nt, R))
        dd[s, j % R] = 1.0
        mm = oracle.p2o_apply_adjoint(blocks, dd)
        exp_m = np.zeros((Nt, Nm))
        for sp in range(0, s + 1):
            exp_m[sp] = blocks[s - sp][j % R]
        np.testing.assert_array_equal(mm, exp_m)


def test_shift_invariance():
    blocks, rng = micro(Nt=10)
    Nt, R, Nm = blocks.shape
    m = rng.standard_normal((Nt, Nm))
    m_shift = np.zeros_like(m)
    m_shift[1:] = m[:-1]
    d = oracle.p2o_apply(blocks, m)
    d_shift = oracle.p2o_apply(blocks, m_shift)
    np.testing.assert_array_equal(d_shift[0], 0.0)
    assert rel(d_shift[1:], d[:-1]) < 1e-15


def test_adjoint_identity():
    blocks, rng = micro(Nt=9, R=4, Nm=13)
    Nt, R, Nm = blocks.shape
    m = rng.standard_normal((Nt, Nm))
    d = rng.standard_normal((Nt, R))
    lhs = np.vdot(oracle.p2o_apply(blocks, m), d)
    rhs = np.vdot(m, oracle.p2o_apply_adjoint(blocks, d))
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), 1.0)


def test_paper_storage_figures():
    """Storage of N_t blocks in FP64 reproduces the sizes printed in Sec. 5 (golden)."""
    with open(os.path.join(HERE, "golden", "paper_storage.json")) as f:
        g = json.load(f)
    Nm, Nd, Nq, Nt, Ntq = g["Nm"], g["Nd"], g["Nq"], g["Nt"], g["Ntq"]
    gb = 1e9
    assert abs(Nt * Nd * Nm * 8 / gb - g["p2o_GB"]) / g["p2o_GB"] < 0.01
    assert abs(Nt * Nq * Nm * 8 / gb - g["p2q_GB"]) / g["p2q_GB"] < 0.02
    assert abs(Nm * Nt * 8 / gb - g["column_GB"]) / g["column_GB"] < 0.01
    assert abs((Nd * Nt) ** 2 * 8 / gb - g["K_GB"]) / g["K_GB"] < 0.01
    assert abs((Nq * Ntq) ** 2 * 8 / 1e6 - g["qoi_cov_MB"]) / g["qoi_cov_MB"] < 0.02
    assert abs(Nq * Ntq * Nd * Nt * 8 / 1e6 - g["d2q_MB"]) / g["d2q_MB"] < 0.01
    assert Nm * Nt == g["param_dim"] and Nd * Nt == g["data_dim"] and Nq * Ntq == g["qoi_dim"]
    # the oracle's block array holds exactly N_t blocks: same storage count
    blocks = np.zeros((3, 2, 5))
    assert oracle.p2o_dense(blocks).size == (3 * 2) * (3 * 5)


# ---------------------------------------------------------------- prior

def test_se_covariance_is_kronecker_of_axes():
    gx, gy, ell, sig = 4, 6, 1.7, 1.3
    C = oracle.se_covariance(gx, gy, ell, sig)
    Cx = oracle.se_covariance_1d(gx, ell, sig)
    Cy = oracle.se_covariance_1d(gy, ell, sig)
    np.testing.assert_allclose(C, np.kron(Cx, Cy), rtol=1e-14, atol=1e-300)
    np.testing.assert_allclose(np.diag(C), sig * sig, rtol=1e-15)
    # neighbours along y (index +1) and along x (index +gy) are one cell apart
    np.testing.assert_allclose(C[0, 1], sig * sig * np.exp(-1 / (2 * ell * ell)), rtol=1e-15)
    np.testing.assert_allclose(C[0, gy], sig * sig * np.exp(-1 / (2 * ell * ell)), rtol=1e-15)
    np.testing.assert_allclose(C[0, gy + 1], sig * sig * np.exp(-2 / (2 * ell * ell)), rtol=1e-15)


def test_separable_prior_blocks_equal_the_dense_product():
    """prior_blocks_separable against prior_blocks with the dense SE covariance, on a
    non-square grid (the axes cannot be swapped unnoticed) and with several blocks and rows."""
    gx, gy, ell, sig = 5, 7, 1.6, 1.4
    rng = np.random.default_rng(11)
    blocks = rng.standard_normal((3, 4, gx * gy))
    dense = oracle.prior_blocks(blocks, oracle.se_covariance(gx, gy, ell, sig))
    np.testing.assert_allclose(oracle.prior_blocks_separable(blocks, gx, gy, ell, sig), dense, rtol=1e-13,
                               atol=1e-13 * np.abs(dense).max())


def test_prior_sample_root():
    gx, gy, ell, sig = 5, 3, 2.0, 0.8
    n = gx * gy
    R = oracle.prior_sample(np.eye(n).reshape(n, n), gx, gy, ell, sig)  # rows are R e_a
    C = oracle.se_covariance(gx, gy, ell, sig)
    np.testing.assert_allclose(R @ R.T, C, atol=1e-12)
    np.testing.assert_allclose(R, R.T, atol=1e-13)


def test_elliptic_operator():
    gx, gy, a1, a2 = 5, 7, 0.3, 1.1
    A = oracle.elliptic_operator(gx, gy, a1, a2).toarray()
    np.testing.assert_allclose(A, A.T, rtol=0, atol=0)
    np.testing.assert_allclose(A @ np.ones(gx * gy), a1 * np.ones(gx * gy), rtol=1e-14)
    # interior: Laplacian of a linear field vanishes
    ix, iy = np.meshgrid(np.arange(gx), np.arange(gy), indexing="ij")
    u = (2.0 * ix + 3.0 * iy).reshape(-1).astype(float)
    Au = (A @ u).reshape(gx, gy)
    np.testing.assert_allclose(Au[1:-1, 1:-1], a1 * u.reshape(gx, gy)[1:-1, 1:-1], rtol=1e-13)
    # 1-D special case: Neumann tridiagonal [1 -1; -1 2 -1; ...; -1 1]
    A1 = oracle.elliptic_operator(6, 1, 0.0, 1.0).toarray()
    T = np.diag([1, 2, 2, 2, 2, 1.0]) - np.diag(np.ones(5), 1) - np.diag(np.ones(5), -1)
    np.testing.assert_array_equal(A1, T)


# ---------------------------------------------------------------- K, Cholesky, solves

def _tiny_problem(seed=11, gx=4, gy=3, Nd=3, Nt=7, sigma2=0.05):
    rng = np.random.default_rng(seed)
    Nm = gx * gy
    F = rng.standard_normal((Nt, Nd, Nm)) * np.exp(-np.arange(Nt) / 3.0)[:, None, None]
    Cs = oracle.se_covariance(gx, gy, 1.5, 1.0)
    G = oracle.prior_blocks(F, Cs)
    return F, G, Cs, sigma2, rng


def test_K_matches_dense_definition():
    F, G, Cs, s2, _ = _tiny_problem()
    Nt, Nd, Nm = F.shape
    P = oracle.p2o_dense(F)
    Gamma_p = np.kron(np.eye(Nt), Cs)
    K_dense = s2 * np.eye(Nt * Nd) + P @ Gamma_p @ P.T
    K = oracle.assemble_K(F, G, s2)
    assert rel(K, K_dense) < 1e-14
    assert rel(oracle.assemble_K_columns(F, G, s2), K_dense) < 1e-14
    # G blocks really are the blocks of Gamma_prior F^T (transposed Toeplitz)
    np.testing.assert_allclose(oracle.p2o_dense(G).T, Gamma_p @ P.T, rtol=1e-13, atol=1e-13)


def test_K_symmetric_positive_definite_and_noise_floor():
    F, G, Cs, s2, _ = _tiny_problem(Nt=9)
    K = oracle.assemble_K(F, G, s2)
    np.testing.assert_allclose(K, K.T, rtol=1e-13, atol=1e-13)
    lam = np.linalg.eigvalsh(0.5 * (K + K.T))
    assert lam.min() >= s2 * (1 - 1e-8)


def test_K_with_diagonal_noise():
    F, G, Cs, s2, rng = _tiny_problem()
    Nt, Nd, _ = F.shape
    var = rng.uniform(0.01, 0.1, size=(Nt, Nd))
    K = oracle.assemble_K(F, G, var)
    K0 = oracle.assemble_K(F, G, 0.0)
    np.testing.assert_allclose(np.diag(K - K0), var.reshape(-1), rtol=1e-12)
    np.testing.assert_array_equal(np.tril(K - K0, -1), 0.0)


def _textbook_cholesky(A):
    n = A.shape[0]
    L = np.zeros_like(A)
    for i in range(n):
        for j in range(i + 1):
            s = sum(L[i, k] * L[j, k] for k in range(j))
            if i == j:
                L[i, i] = np.sqrt(A[i, i] - s)
            else:
                L[i, j] = (A[i, j] - s) / L[j, j]
    return L


def test_cholesky_against_textbook_and_reconstruction():
    F, G, Cs, s2, _ = _tiny_problem(Nt=5, Nd=3)
    K = oracle.assemble_K(F, G, s2)
    L = oracle.cholesky_lower(K)
    np.testing.assert_array_equal(np.triu(L, 1), 0.0)
    assert np.all(np.diag(L) > 0)
    assert rel(L @ L.T, np.tril(K) + np.tril(K, -1).T) < 1e-14
    assert rel(L, _textbook_cholesky(np.tril(K) + np.tril(K, -1).T)) < 1e-13
    # only the lower triangle is read
    K_garbage_upper = np.tril(K) + np.triu(np.full_like(K, 7.0), 1)
    np.testing.assert_array_equal(oracle.cholesky_lower(K_garbage_upper), L)


def test_cholesky_rejects_indefinite():
    A = np.array([[1.0, 2.0], [2.0, 1.0]])
    with pytest.raises(np.linalg.LinAlgError):
        oracle.cholesky_lower(A)


def test_solve_K_residual():
    F, G, Cs, s2, rng = _tiny_problem()
    K = oracle.assemble_K(F, G, s2)
    L = oracle.cholesky_lower(K)
    d = rng.standard_normal((3, K.shape[0]))
    x = oracle.solve_K(L, d)
    for b in range(3):
        assert rel(K @ x[b], d[b]) < 1e-12
    assert rel(oracle.solve_K(L, d[0]), x[0]) < 1e-15


# ---------------------------------------------------------------- m_map, q_map

def test_map_point_equals_closed_form_posterior_mean():
    """With an invertible prior, m_map = G^* K^{-1} d solves Eq. (2.12) (Woodbury, Eq. (4.6))."""
    rng = np.random.default_rng(21)
    gx, gy, Nd, Nt, s2 = 4, 4, 3, 6, 0.02
    Nm = gx * gy
    F = rng.standard_normal((Nt, Nd, Nm)) * np.exp(-np.arange(Nt) / 2.5)[:, None, None]
    A_s = oracle.elliptic_operator(gx, gy, 1.0, 1.0).toarray()
    Cs = np.linalg.inv(A_s @ A_s)  # Eq. (5.1): (alpha1 I - alpha2 Delta)^{-2}
    Cs = 0.5 * (Cs + Cs.T)
    G = oracle.prior_blocks(F, Cs)
    d = rng.standard_normal((Nt, Nd))
    P = oracle.p2o_dense(F)
    H = P.T @ P / s2 + np.kron(np.eye(Nt), A_s @ A_s)
    m_closed = np.linalg.solve(H, P.T @ d.reshape(-1) / s2)
    m_map = oracle.map_point(F, G, s2, d)
    assert rel(m_map.reshape(-1), m_closed) < 1e-10
    m_413 = oracle.map_point_woodbury_form(F, G, s2, d)
    assert rel(m_413, m_map) < 1e-10


def test_map_point_fixed_point_with_singular_se_prior():
    """m_map = Gamma_p F^T Gamma_n^{-1} (d - F m_map) holds for the numerically singular SE prior."""
    F, G, Cs, s2, rng = _tiny_problem(gx=5, gy=5, Nd=2, Nt=8, sigma2=1e-3)
    d = rng.standard_normal((2, 8, 2))
    m = oracle.map_point(F, G, s2, d)
    rhs = oracle.p2o_apply_adjoint(G, (d - oracle.p2o_apply(F, m)) / s2)
    assert rel(m, rhs) < 1e-9
    assert rel(oracle.map_point_woodbury_form(F, G, s2, d), m) < 1e-9


def test_map_point_large_noise_limit():
    F, G, Cs, s2, rng = _tiny_problem()
    d = rng.standard_normal((F.shape[0], F.shape[1]))
    big = 1e8
    m = oracle.map_point(F, G, big, d)
    approx = oracle.p2o_apply_adjoint(G, d) / big
    assert rel(m, approx) < 1e-6


def test_qoi_map_is_push_forward():
    F, G, Cs, s2, rng = _tiny_problem()
    Nt, Nd, Nm = F.shape
    Fq = rng.standard_normal((Nt, 2, Nm))
    d = rng.standard_normal((Nt, Nd))
    m = oracle.map_point(F, G, s2, d)
    q = oracle.qoi_map(Fq, m)
    assert rel(q.reshape(-1), oracle.p2o_dense(Fq) @ m.reshape(-1)) < 1e-14


# ---------------------------------------------------------------- loss / gradient

def test_gradient_matches_central_differences_and_dense():
    rng = np.random.default_rng(31)
    gx, gy, Nd, Nt, s2 = 3, 4, 2, 5, 0.1
    Nm = gx * gy
    F = rng.standard_normal((Nt, Nd, Nm))
    A_s = oracle.elliptic_operator(gx, gy, 1.0, 1.0)
    m = rng.standard_normal((Nt, Nm))
    d = rng.standard_normal((Nt, Nd))
    g = oracle.loss_gradient(F, m, d, s2, A_s)
    v = rng.standard_normal((Nt, Nm))
    h = 1e-6
    fd = (oracle.loss(F, m + h * v, d, s2, A_s) - oracle.loss(F, m - h * v, d, s2, A_s)) / (2 * h)
    L0 = oracle.loss(F, m, d, s2, A_s)
    assert abs(fd - np.vdot(g, v)) <= 1e-8 * max(abs(L0), 1.0)
    P = oracle.p2o_dense(F)
    Ad = A_s.toarray()
    g_dense = P.T @ (P @ m.reshape(-1) - d.reshape(-1)) / s2 + np.kron(np.eye(Nt), Ad.T @ Ad) @ m.reshape(-1)
    assert rel(g.reshape(-1), g_dense) < 1e-13


# ---------------------------------------------------------------- synthetic inputs

def test_synthetic_blocks_recipe():
    p = synthetic.small("t", 4, 4, 3, 8, tau=2.0)
    a = p.blocks_F()
    b = p.blocks_F()
    np.testing.assert_array_equal(a, b)  # deterministic
    assert a.shape == (8, 3, 16)
    # decay: block k has std ~ exp(-k / tau)
    big = synthetic.toeplitz_blocks(5, 4, 64, 512, 2.0)
    std = big.reshape(4, -1).std(axis=1)
    np.testing.assert_allclose(std, np.exp(-np.arange(4) / 2.0), rtol=0.02)


def test_single_block_outputs_match_full_products():
    blocks, rng = micro(Nt=9, R=3, Nm=7)
    m = rng.standard_normal((9, 7))
    d = rng.standard_normal((9, 3))
    full = oracle.p2o_apply(blocks, m)
    fullT = oracle.p2o_apply_adjoint(blocks, d)
    P = oracle.p2o_dense(blocks)
    for t in (0, 4, 8):
        assert rel(oracle.p2o_apply_block(blocks, m, t), full[t]) < 1e-15
        assert rel(oracle.p2o_apply_block(blocks, m, t), (P @ m.reshape(-1)).reshape(9, 3)[t]) < 1e-14
        assert rel(oracle.p2o_apply_adjoint_block(blocks, d, t), fullT[t]) < 1e-15


# ---------------------------------------------------------------- d2q map and QoI covariance

def test_d2q_map_equals_eq_4_11_long_form_and_reproduces_q_map():
    F, G, Cs, s2, rng = _tiny_problem(gx=4, gy=3, Nd=3, Nt=6, sigma2=0.02)
    Nt, Nd, Nm = F.shape
    Fq = rng.standard_normal((Nt, 2, Nm)) * np.exp(-np.arange(Nt) / 3.0)[:, None, None]
    Q = oracle.d2q_map(Fq, F, G, s2)
    # Eq. (4.11) term by term with dense matrices
    P, Pq = oracle.p2o_dense(F), oracle.p2o_dense(Fq)
    Gstar = np.kron(np.eye(Nt), Cs) @ P.T
    K = s2 * np.eye(Nt * Nd) + P @ Gstar
    long = Pq @ (np.eye(Nt * Nm) - Gstar @ np.linalg.solve(K, P)) @ Gstar / s2
    assert rel(Q, long) < 1e-10
    # q_map = Q d_obs equals the push-forward of m_map (Eq. (4.14) vs Eq. (4.2))
    d = rng.standard_normal((Nt, Nd))
    q_push = oracle.qoi_map(Fq, oracle.map_point(F, G, s2, d))
    assert rel(Q @ d.reshape(-1), q_push.reshape(-1)) < 1e-12
    # the Gram accumulation equals the dense F_q G^*
    assert rel(oracle.qoi_data_gram(Fq, G), Pq @ Gstar) < 1e-14


def test_qoi_posterior_covariance_equals_eq_4_10_and_push_forward():
    F, G, Cs, s2, rng = _tiny_problem(gx=3, gy=3, Nd=2, Nt=5, sigma2=0.05)
    Nt, Nd, Nm = F.shape
    Fq = rng.standard_normal((Nt, 2, Nm))
    Gq = oracle.prior_blocks(Fq, Cs)
    C = oracle.qoi_posterior_covariance(Fq, Gq, F, G, s2)
    P, Pq = oracle.p2o_dense(F), oracle.p2o_dense(Fq)
    Gp = np.kron(np.eye(Nt), Cs)
    K = s2 * np.eye(Nt * Nd) + P @ Gp @ P.T
    # Eq. (4.10): F_q (I - G* K^-1 F) G_q*
    ref = Pq @ (np.eye(Nt * Nm) - Gp @ P.T @ np.linalg.solve(K, P)) @ Gp @ Pq.T
    assert rel(C, ref) < 1e-11
    np.testing.assert_allclose(C, C.T, rtol=0, atol=1e-10 * np.abs(C).max())
    # Gamma_post(q) = F_q Gamma_post(m) F_q^T with the Woodbury Gamma_post(m) of Eq. (4.6)
    Gpost = Gp @ (np.eye(Nt * Nm) - P.T @ np.linalg.solve(K, P @ Gp))
    assert rel(C, Pq @ Gpost @ Pq.T) < 1e-10


# ---------------------------------------------------------------- posterior covariance actions, prior mean

def _elliptic_problem(seed=41, gx=3, gy=4, Nd=2, Nt=5, s2=0.03):
    rng = np.random.default_rng(seed)
    Nm = gx * gy
    F = rng.standard_normal((Nt, Nd, Nm)) * np.exp(-np.arange(Nt) / 2.0)[:, None, None]
    A = oracle.elliptic_operator(gx, gy, 1.0, 1.0).toarray()
    Cs = np.linalg.inv(A @ A)
    Cs = 0.5 * (Cs + Cs.T)
    return F, oracle.prior_blocks(F, Cs), Cs, A, s2, rng


def test_posterior_covariance_action_is_inverse_hessian():
    """Gamma_post(m) of Eq. (4.7) equals H^{-1} of Eq. (2.13) with an invertible prior."""
    F, G, Cs, A, s2, rng = _elliptic_problem()
    Nt, Nd, Nm = F.shape
    P = oracle.p2o_dense(F)
    H = P.T @ P / s2 + np.kron(np.eye(Nt), A @ A)
    V = rng.standard_normal((3, Nt, Nm))
    got = oracle.posterior_cov_apply(F, G, Cs, s2, V)
    for b in range(3):
        assert rel(got[b].reshape(-1), np.linalg.solve(H, V[b].reshape(-1))) < 1e-10
    np.testing.assert_allclose(oracle.prior_apply(Cs, V[0]), (np.kron(np.eye(Nt), Cs) @ V[0].reshape(-1)).reshape(Nt, Nm),
                               rtol=1e-13, atol=1e-14)


def test_posterior_variance_probe_is_exact_for_unit_and_hadamard_probes():
    """The probe estimate of diag(Gamma_post(m)) equals the diagonal of H^{-1} (Eq. (2.13),
    invertible elliptic prior) for the unit vectors and for the rows of a Hadamard matrix
    (sign vectors whose products cancel off the diagonal); a few random sign probes do not
    give it exactly (the estimator is not the diagonal by construction)."""
    import scipy.linalg as sla

    F, G, Cs, A, s2, rng = _elliptic_problem(gx=2, gy=4, Nt=4)  # N = 4 * 8 = 32 parameters
    Nt, Nd, Nm = F.shape
    P = oracle.p2o_dense(F)
    H = P.T @ P / s2 + np.kron(np.eye(Nt), A @ A)
    diag = np.diag(np.linalg.inv(H)).reshape(Nt, Nm)
    unit = np.eye(Nt * Nm).reshape(-1, Nt, Nm)
    assert rel(oracle.posterior_variance_probe(F, G, Cs, s2, unit), diag) < 1e-10
    had = sla.hadamard(Nt * Nm).astype(np.float64).reshape(-1, Nt, Nm)
    assert rel(oracle.posterior_variance_probe(F, G, Cs, s2, had), diag) < 1e-10
    few = np.sign(rng.standard_normal((3, Nt, Nm)))
    assert rel(oracle.posterior_variance_probe(F, G, Cs, s2, few), diag) > 1e-3
    # entries no probe touches read 0
    part = unit[:5]
    est = oracle.posterior_variance_probe(F, G, Cs, s2, part).reshape(-1)
    assert np.all(est[5:] == 0.0) and rel(est[:5], diag.reshape(-1)[:5]) < 1e-10


def test_map_point_with_prior_mean_is_closed_form():
    """Eq. (4.13) + Eq. (4.8) against the normal equations of Eq. (2.12) with m_prior != 0."""
    F, G, Cs, A, s2, rng = _elliptic_problem(seed=43)
    Nt, Nd, Nm = F.shape
    P = oracle.p2o_dense(F)
    Gpi = np.kron(np.eye(Nt), A @ A)
    d = rng.standard_normal((Nt, Nd))
    m0 = rng.standard_normal((Nt, Nm))
    H = P.T @ P / s2 + Gpi
    closed = np.linalg.solve(H, P.T @ d.reshape(-1) / s2 + Gpi @ m0.reshape(-1))
    got = oracle.map_point_with_prior_mean(F, G, s2, d, m0)
    assert rel(got.reshape(-1), closed) < 1e-10
    # zero prior mean reduces to map_point
    assert rel(oracle.map_point_with_prior_mean(F, G, s2, d, np.zeros_like(m0)), oracle.map_point(F, G, s2, d)) < 1e-14


# ---------------------------------------------------------------- QoI time grid

def test_qoi_time_steps_match_the_example_grid():
    """Sec. 5: N_t = 500 steps at 10 Hz on (0, 50) s, QoIs at 1 Hz, N_t^q = 50, and the
    QoI dimension N_q N_t^q = 800 (golden): one QoI per second, the last at T = 50 s."""
    with open(os.path.join(HERE, "golden", "paper_storage.json")) as f:
        g = json.load(f)
    Nt, Ntq, Nq = g["Nt"], g["Ntq"], g["Nq"]
    stride = Nt // Ntq
    steps = oracle.qoi_time_steps(Nt, stride)
    assert stride == 10 and len(steps) == Ntq
    dt = 50.0 / Nt
    times = (steps + 1) * dt  # step t ends at time (t + 1) dt
    np.testing.assert_allclose(times, np.arange(1, 51), rtol=0, atol=1e-12)
    assert len(oracle.qoi_rows(Nt, Nq, stride)) == g["qoi_dim"]
    np.testing.assert_array_equal(oracle.qoi_time_steps(7, 1), np.arange(7))
    with pytest.raises(ValueError):
        oracle.qoi_time_steps(10, 3)


def _coarse_p2q_dense(Fq, stride):
    """The p2q matrix on the coarse QoI grid, block by block: block (k, s) is
    (F_q)_{t_k - s} for s <= t_k with t_k = stride (k + 1) - 1, else zero."""
    Nt, Rq, Nm = Fq.shape
    Ntq = Nt // stride
    P = np.zeros((Ntq * Rq, Nt * Nm))
    for k in range(Ntq):
        tk = stride * (k + 1) - 1
        for s in range(tk + 1):
            P[k * Rq:(k + 1) * Rq, s * Nm:(s + 1) * Nm] = Fq[tk - s]
    return P


def test_coarse_qoi_grid_selects_from_the_fine_d2q_map_and_covariance():
    """Q and Gamma_post(q) on a QoI grid of every third step: the selected rows (and
    columns) of the fine-grid results equal Eqs. (4.10)-(4.11) written with the coarse
    p2q matrix assembled from its block definition."""
    F, G, Cs, s2, rng = _tiny_problem(seed=17, gx=3, gy=3, Nd=2, Nt=6, sigma2=0.04)
    Nt, Nd, Nm = F.shape
    Fq = rng.standard_normal((Nt, 2, Nm)) * np.exp(-np.arange(Nt) / 4.0)[:, None, None]
    Gq = oracle.prior_blocks(Fq, Cs)
    stride = 3
    rows = oracle.qoi_rows(Nt, 2, stride)
    Q = oracle.d2q_map(Fq, F, G, s2)[rows]
    C = oracle.qoi_posterior_covariance(Fq, Gq, F, G, s2)[np.ix_(rows, rows)]
    P = oracle.p2o_dense(F)
    Pc = _coarse_p2q_dense(Fq, stride)
    Gp = np.kron(np.eye(Nt), Cs)
    K = s2 * np.eye(Nt * Nd) + P @ Gp @ P.T
    post = np.eye(Nt * Nm) - Gp @ P.T @ np.linalg.solve(K, P)
    assert rel(Q, Pc @ post @ Gp @ P.T / s2) < 1e-10
    assert rel(C, Pc @ post @ Gp @ Pc.T) < 1e-10
    # the coarse q_map is the fine q_map read at the QoI steps
    d = rng.standard_normal((Nt, Nd))
    q_fine = oracle.qoi_map(Fq, oracle.map_point(F, G, s2, d))
    steps = oracle.qoi_time_steps(Nt, stride)
    assert rel((Q @ d.reshape(-1)).reshape(-1, 2), q_fine[steps]) < 1e-12
