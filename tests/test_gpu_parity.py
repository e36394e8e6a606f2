"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances are normwise relative errors per right-hand side, the maximum over
the batch (reading R11): 1e-12 for products of the FP64-accurate tiers, 1e-5 for
the FP32 tier, 1e-3 for the FP16 tier.  Results that pass through a solve with K
follow reading R20 (tests/parity.py): a bound from kappa(K), which the oracle
measures for each test problem, and the unit roundoff of the arithmetic, never
below 1e-12.
"""

from types import SimpleNamespace

import numpy as np
import pytest

import oracle
import parity
from paper_2501_14911_gb300 import synthetic
from parity import check, rel, relb

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2501_14911_gb300 as bti  # noqa: E402

TOL = {bti.F64: 1e-12, bti.F32: 1e-5, bti.DF64: 1e-12, bti.F16: 1e-3}


_ORACLE_K = {}


def oracle_K(key, F, G, noise, Fq=None):
    """The oracle's K = Gamma_n + F G^* of one test problem and what the tolerances of
    reading R20 need from it, cached by key: K, its factor L, lambda_min and kappa(K)."""
    if key not in _ORACLE_K:
        K = oracle.assemble_K(F, G, noise)
        L = oracle.cholesky_lower(K)
        lmin, lmax = parity.spd_extremes(K, L)
        _ORACLE_K[key] = SimpleNamespace(K=K, L=L, lmin=lmin, kappa=lmax / lmin, F=F, G=G, Fq=Fq)
    return _ORACLE_K[key]


def solve_bounds(c, d, u, kind="solve", eta=None):
    """Tolerances (reading R20) for x = K^{-1} d and for m_map = G^* x and q_map = F_q m_map,
    which the rule holds to the same bound: kind "solve" (a backward-stable solve, or
    refinement with residuals in u), "inverse" (an explicit inverse formed in u) or "cg"
    (stopped at relative residual eta, operator in u).  Returns the oracle's x, m, q too."""
    d = np.asarray(d, dtype=np.float64)
    B = d.shape[0]
    x = oracle.solve_K(c.L, d.reshape(B, -1)).reshape(d.shape)
    m = oracle.p2o_apply_adjoint(c.G, x)
    rho = parity.rho_inverse(c.lmin, d, x)
    if kind == "solve":
        tol = parity.tol_solve(c.kappa, u)
    elif kind == "inverse":
        tol = parity.tol_inverse(c.kappa, u, rho)
    else:
        tol = parity.tol_cg(c.kappa, u, rho, eta)
    q = oracle.qoi_map(c.Fq, m) if c.Fq is not None else None
    return SimpleNamespace(x=x, m=m, q=q, rho=rho, tol_x=tol, tol_m=tol, tol_q=tol,
                           info=f"kappa(K) = {c.kappa:.0f}, rho = {rho:.1f}")


def d2q_bounds(c, Fq, G, Q_or, C_or, d, u, kind="solve", rows=None):
    """Tolerances (reading R20) for the d2q map Q = X K^{-1} (X = F_q G^*, each row a solve
    with K, or a product with an explicit inverse when kind is "inverse"), for Gamma_post(q) =
    X_qq - Q X^T (the bound of Q times gamma = ||Q|| ||X|| / ||Gamma_post(q)||, the cancellation)
    and for q = Q d (times ||Q|| ||d|| / ||q||).  rows: the rows of the coarse QoI grid."""
    X = oracle.qoi_data_gram(Fq, G)
    if rows is not None:
        X = X[rows]
    if kind == "inverse":
        tQ = parity.tol_inverse(c.kappa, u, parity.rho_inverse(c.lmin, X, Q_or))
    else:
        tQ = parity.tol_solve(c.kappa, u)
    nQ = np.linalg.norm(Q_or, 2)
    gamma = np.linalg.norm(Q_or) * np.linalg.norm(X, 2) / np.linalg.norm(C_or)
    tol_C = max(parity.FLOOR, tQ * gamma + parity.C_BOUND * u)
    out = SimpleNamespace(tol_Q=tQ, tol_C=tol_C, gamma=gamma)
    if d is not None:
        d = np.asarray(d).reshape(np.shape(d)[0], -1)
        qv = d @ Q_or.T
        alpha = float(np.max(nQ * np.linalg.norm(d, axis=1) / np.linalg.norm(qv, axis=1)))
        out.tol_q = max(parity.FLOOR, tQ * alpha + parity.C_BOUND * u)
        out.alpha = alpha
    out.info = f"kappa(K) = {c.kappa:.0f}, gamma = {gamma:.1f}" + (f", alpha_Qd = {out.alpha:.1f}" if d is not None else "")
    return out


def postcov_bound(c, Cs, V, u, probe=False):
    """Tolerance (reading R20) of Gamma_post(m) v = w - G^* K^{-1} F w (Eq. (4.7), w = Gamma_prior v)
    for the vectors V: the bound of the subtracted term G^* K^{-1} F w (a solve, then G^*) times the
    cancellation gamma = ||G^* K^{-1} F w|| / ||Gamma_post(m) v||.  probe: the same for the probe
    estimate sum_s v_s o Gamma_post(m) v_s / sum_s v_s o v_s over the vectors."""
    V = np.asarray(V, dtype=np.float64)
    W = oracle.prior_apply(Cs, V)
    b = solve_bounds(c, oracle.p2o_apply(c.F, W), u)
    if probe:
        den = (V * V).sum(axis=0)
        den = np.where(den > 0, den, 1.0)
        sub = (V * b.m).sum(axis=0) / den
        full = (V * (W - b.m)).sum(axis=0) / den
        gamma = float(np.linalg.norm(sub) / np.linalg.norm(full))
    else:
        B = V.shape[0]
        gamma = float(np.max(np.linalg.norm(b.m.reshape(B, -1), axis=1)
                             / np.linalg.norm((W - b.m).reshape(B, -1), axis=1)))
    tol = max(parity.FLOOR, gamma * b.tol_m + parity.C_BOUND * u)
    return tol, b.info + f", gamma = {gamma:.1f}"


def cuda(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


def host(x):
    torch.cuda.synchronize()
    return x.detach().cpu().numpy().astype(np.float64)


def make_handle(F, Fq=None, store=bti.F64):
    Nt, Nd, Nm = F.shape
    Nq = 0 if Fq is None else Fq.shape[1]
    h = bti.Handle(Nm, Nd, Nq, Nt)
    h.set_blocks(bti.OP_F, cuda(F), store)
    if Fq is not None:
        h.set_blocks(bti.OP_FQ, cuda(Fq), store)
    return h


CASES = [
    # (name, Nm, Nd, Nq, Nt, B): ragged chunks / warps / column pairs, several radices
    ("L90_ragged", 3000, 13, 5, 45, 3),
    ("L128_b6", 1024, 8, 4, 64, 6),
    ("L420", 700, 6, 3, 210, 2),
    ("L400_batched_shape", 4096, 100, 32, 200, 1),
    ("L512_sweep_shape_ragged", 2051, 9, 3, 256, 2),  # the headline sweep's length, ragged column pairs
    ("L840_odd", 333, 7, 2, 420, 1),
    ("Nt1_gemv", 257, 5, 3, 1, 2),
    ("scalar", 1, 1, 1, 16, 2),
    ("R1100_row_tiles", 600, 1100, 3, 20, 5),  # adjoint stages d-hat in 512-row tiles
    # FP16 tier with B >= 8: tensor-core forward product (row tiles of 128, groups of 16/32)
    ("tc_b16", 4096, 128, 4, 64, 16),
    ("tc_b10_rows200_L90", 3000, 200, 5, 45, 10),
    ("tc_b40_groups", 1024, 13, 3, 32, 40),
    ("L2048_max_length", 96, 5, 3, 1024, 9),  # the longest transform (N_t = 1024, one pair per CTA)
    ("b9_Nm_not_mult4", 333, 7, 2, 20, 9),    # B >= 8 but N_m % 4 != 0: CUDA-core FP16 products
    ("tc_R1100_b20", 512, 1100, 3, 12, 20),    # tensor-core forward over 9 row tiles; adjoint on CUDA cores
    # lengths 2^a 5^b: the (8, 4, 2, 5) radix-set FFT kernels
    ("L250_radix_2_5", 700, 6, 3, 125, 2),     # plan 2, 5, 5, 5 (no radix-8 first pass)
    ("L1000_radix_8_5", 96, 5, 3, 500, 3),     # plan 8, 5, 5, 5 (half-zero radix-8 first pass)
    ("L100_radix_4_5_b16", 300, 7, 2, 50, 16), # plan 4, 5, 5; B = 16 (tensor cores in the FP16 tier)
]


@pytest.mark.parametrize("store", [bti.F64, bti.F32, bti.DF64, bti.F16], ids=["f64", "f32", "df64", "f16"])
@pytest.mark.parametrize("name,Nm,Nd,Nq,Nt,B", CASES, ids=[c[0] for c in CASES])
def test_apply_F_FT_Fq_match_oracle(name, Nm, Nd, Nq, Nt, B, store):
    p = synthetic.small(name, 1, Nm, Nd, Nt, Nq=Nq)
    F = p.blocks_F()
    Fq = p.blocks_Fq()
    m = p.vectors_m(B)
    d = p.vectors_d(B)
    h = make_handle(F, Fq, store)
    dt = torch.float32 if store in (bti.F32, bti.F16) else torch.float64
    m_g, d_g = cuda(m, dt), cuda(d, dt)
    out_d = torch.empty((B, Nt, Nd), dtype=dt, device="cuda")
    out_m = torch.empty((B, Nt, Nm), dtype=dt, device="cuda")
    out_q = torch.empty((B, Nt, Nq), dtype=dt, device="cuda")
    h.apply_F(m_g, out_d)
    h.apply_FT(d_g, out_m)
    h.apply_Fq(m_g, out_q)
    h.sync()
    # the oracle sees the inputs exactly as the GPU does (rounded to the io type)
    m_in, d_in = host(m_g), host(d_g)
    tol = TOL[store]
    check(relb(host(out_d), oracle.p2o_apply(F, m_in)), tol)
    check(relb(host(out_m), oracle.p2o_apply_adjoint(F, d_in)), tol)
    check(relb(host(out_q), oracle.p2o_apply(Fq, m_in)), tol)
    h.close()


@pytest.mark.parametrize("store,io", [(bti.F64, torch.float32), (bti.F32, torch.float64),
                                      (bti.DF64, torch.float32)],
                         ids=["f64tier_f32io", "f32tier_f64io", "df64tier_f32io"])
def test_mixed_io_types(store, io):
    p = synthetic.small("mixed_io", 40, 50, 9, 32)
    F = p.blocks_F()
    m = p.vectors_m(2)
    h = make_handle(F, None, store)
    m_g = cuda(m, io)
    d = torch.empty((2, 32, 9), dtype=io, device="cuda")
    h.apply_F(m_g, d)
    check(relb(host(d), oracle.p2o_apply(F, host(m_g))), 1e-5)


@pytest.mark.parametrize("store", [bti.F64, bti.F32, bti.DF64, bti.F16], ids=["f64", "f32", "df64", "f16"])
def test_tuned_launch_shapes_serve_every_batch_size(store):
    """Shapes tuned for single vectors (a forward chunk of up to 4,096 columns) and for
    groups of four are kept apart: after tuning at B = 1 and at B = 8, calls with 1, 5
    and 16 right-hand sides all launch and match the oracle."""
    p = synthetic.small("tuned_batches", 1, 5000, 16, 32)
    F = p.blocks_F()
    h = make_handle(F, None, store)
    dt = torch.float32 if store in (bti.F32, bti.F16) else torch.float64
    h.autotune(bti.OP_F, 1)
    for B in (1, 5, 16):
        if B == 5:
            h.autotune(bti.OP_F, 8)
        m_g = cuda(p.vectors_m(B), dt)
        d_g = cuda(p.vectors_d(B), dt)
        od = torch.empty((B, 32, 16), dtype=dt, device="cuda")
        om = torch.empty((B, 32, 5000), dtype=dt, device="cuda")
        h.apply_F(m_g, od)
        h.apply_FT(d_g, om)
        check(relb(host(od), oracle.p2o_apply(F, host(m_g))), TOL[store], str(B))
        check(relb(host(om), oracle.p2o_apply_adjoint(F, host(d_g))), TOL[store], str(B))
    h.close()


@pytest.mark.parametrize("B", [8, 16, 33])
def test_tensor_core_products_match_cuda_core_path(B):
    """The tcgen05 FP16 forward and adjoint products against the CUDA-core FP16 kernels and
    the oracle: all within the FP16 tier's 1e-3, and the two paths within 1e-3 of each
    other (they differ by the rounding of the vectors' spectra to FP16)."""
    p = synthetic.small("tc_vs_cuda", 1, 2048, 130, 48, Nq=4)
    F = p.blocks_F()
    h = make_handle(F, None, bti.F16)
    m = cuda(p.vectors_m(B), torch.float32)
    d = cuda(p.vectors_d(B), torch.float32)
    out = {}
    for tc in (True, False):
        h.set_tensor_cores(tc)
        od = torch.empty((B, 48, 130), dtype=torch.float32, device="cuda")
        om = torch.empty((B, 48, 2048), dtype=torch.float32, device="cuda")
        h.apply_F(m, od)
        h.apply_FT(d, om)
        h.sync()  # also reports a tensor-core wait that gave up
        out[tc] = (host(od), host(om))
    h.close()
    ref_d = oracle.p2o_apply(F, host(m))
    ref_m = oracle.p2o_apply_adjoint(F, host(d))
    for tc in (True, False):
        check(relb(out[tc][0], ref_d), 1e-3, str(tc))
        check(relb(out[tc][1], ref_m), 1e-3, str(tc))
    for k in (0, 1):
        assert 0.0 < relb(out[True][k], out[False][k]) < 1e-3  # the tensor-core path really ran


def test_impulse_response_and_causality():
    p = synthetic.small("impulse", 8, 8, 4, 24)
    F = p.blocks_F()
    h = make_handle(F)
    Nt, Nd, Nm = F.shape
    m = np.zeros((1, Nt, Nm))
    s, j = 5, 17
    m[0, s, j] = 1.0
    d = torch.empty((1, Nt, Nd), dtype=torch.float64, device="cuda")
    h.apply_F(cuda(m), d)
    dh = host(d)[0]
    scale = np.abs(F).max()
    np.testing.assert_allclose(dh[:s], 0.0, atol=1e-14 * scale)
    for t in range(s, Nt):
        np.testing.assert_allclose(dh[t], F[t - s][:, j], rtol=0, atol=1e-14 * scale)


def test_adjoint_identity_on_gpu():
    p = synthetic.small("adjoint", 32, 32, 16, 100)
    F = p.blocks_F()
    h = make_handle(F)
    m = cuda(p.vectors_m(1))
    dv = cuda(p.vectors_d(1))
    Fm = torch.empty((1, 100, 16), dtype=torch.float64, device="cuda")
    FTd = torch.empty((1, 100, 1024), dtype=torch.float64, device="cuda")
    h.apply_F(m, Fm)
    h.apply_FT(dv, FTd)
    lhs = float((Fm * dv).sum())
    rhs = float((m * FTd).sum())
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), float(Fm.abs().sum() * dv.abs().max()))


def test_zero_batch_is_noop_and_errors_are_reported():
    p = synthetic.small("errs", 4, 4, 3, 8)
    F = p.blocks_F()
    h = bti.Handle(16, 3, 2, 8)
    m = torch.zeros((1, 8, 16), dtype=torch.float64, device="cuda")
    d = torch.zeros((1, 8, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(bti.BtiError) as e:
        h.apply_F(m, d)  # blocks not set
    assert e.value.status == 3
    with pytest.raises(bti.BtiError) as e:
        h.build_K()
    assert e.value.status == 3
    with pytest.raises(bti.BtiError) as e:
        h.infer_map(d, m)
    assert e.value.status == 3
    h.set_blocks(bti.OP_F, cuda(F))
    L = bti.lib()
    assert L.bti_apply_F(h.raw, m.data_ptr(), d.data_ptr(), 0, 0) == 0
    assert L.bti_apply_F(h.raw, m.data_ptr(), d.data_ptr(), -1, 0) == 1
    assert L.bti_apply_F(h.raw, m.data_ptr(), d.data_ptr(), 1, 7) == 1
    assert L.bti_apply_F(h.raw, None, d.data_ptr(), 1, 0) == 1
    assert L.bti_set_prior_se_grid(h.raw, 3, 3, 3.0, 1.0, 0) == 2  # 3 x 3 != 16
    assert "gx * gy" in h.last_error
    h.close()


def tiny_problem():
    p = synthetic.TINY
    F = p.blocks_F()
    Fq = p.blocks_Fq()
    Cs = oracle.se_covariance(p.gx, p.gy, p.ell, p.sigma_p)
    G = oracle.prior_blocks(F, Cs)
    m_true = oracle.prior_sample(p.z_true(1), p.gx, p.gy, p.ell, p.sigma_p)
    d_obs = oracle.p2o_apply(F, m_true) + np.sqrt(p.sigma2) * p.noise(1)
    return p, F, Fq, G, d_obs


@pytest.mark.parametrize("store", [bti.F64, bti.DF64], ids=["f64", "df64"])
def test_tiny_inversion_end_to_end(store):
    p, F, Fq, G, d_obs = tiny_problem()
    h = make_handle(F, Fq, store)
    h.set_prior_se_grid(p.gx, p.gy, p.ell, p.sigma_p, store)
    # G^* from the device-built SE prior matches Gamma_prior F^T
    dv = p.vectors_d(2)
    mg = torch.empty((2, p.Nt, p.Nm), dtype=torch.float64, device="cuda")
    h.apply_Gstar(cuda(dv), mg)
    check(relb(host(mg), oracle.p2o_apply_adjoint(G, dv)), 1e-12)
    h.set_noise(p.sigma2)
    h.build_K()
    K_gpu = host(h.copy_K())
    K_or = oracle.assemble_K(F, G, p.sigma2)
    low = np.tril_indices(K_or.shape[0])
    check(rel(K_gpu[low], K_or[low]), 1e-12)
    h.factor_K()
    L_gpu = host(h.copy_K())
    L_or = oracle.cholesky_lower(K_or)
    check(rel(L_gpu[low], L_or[low]), 1e-12)
    m_map = torch.empty((1, p.Nt, p.Nm), dtype=torch.float64, device="cuda")
    h.infer_map(cuda(d_obs), m_map)
    q_map = torch.empty((1, p.Nt, p.Nq), dtype=torch.float64, device="cuda")
    h.predict_qoi(m_map, q_map)
    m_or = oracle.map_point(F, G, p.sigma2, d_obs)
    check(relb(host(m_map), m_or), 1e-12)
    check(relb(host(q_map), oracle.qoi_map(Fq, m_or)), 1e-12)
    # iterative refinement keeps the answer (and is exercised)
    m_ref = torch.empty_like(m_map)
    h.infer_map(cuda(d_obs), m_ref, refine_iters=2)
    check(relb(host(m_ref), m_or), 1e-12)


def test_diagonal_noise_and_batched_obs():
    p = synthetic.small("diagnoise", 6, 6, 5, 30, Nq=3)
    F = p.blocks_F()
    Cs = oracle.se_covariance(6, 6, 2.0, 1.0)
    G = oracle.prior_blocks(F, Cs)
    var = 1e-3 * (1.0 + np.arange(30 * 5).reshape(30, 5) % 7)
    d_obs = p.vectors_d(5)
    h = make_handle(F, p.blocks_Fq())
    h.set_prior_se_grid(6, 6, 2.0, 1.0)
    h.set_noise(0.0, cuda(var))
    h.build_K(col_block=37)
    h.factor_K()
    m_map = torch.empty((5, 30, 36), dtype=torch.float64, device="cuda")
    h.infer_map(cuda(d_obs), m_map, refine_iters=1)
    b = solve_bounds(oracle_K("diagnoise", F, G, var), d_obs, parity.U_F64)
    check(relb(host(m_map), b.m), b.tol_m, "FP64 solves and residual; " + b.info)


def test_not_spd_is_reported_with_pivot():
    """A negative noise variance injected on the host makes K indefinite."""
    p = synthetic.small("notspd", 4, 4, 3, 10)
    F = p.blocks_F() * 1e-3
    var = np.full((10, 3), 1e-4)
    var[4, 1] = -10.0  # data index 4 * 3 + 1 = 13 -> pivot 14 (1-based) or earlier
    h = make_handle(F)
    h.set_prior_se_grid(4, 4, 3.0, 1.0)
    h.set_noise(0.0, cuda(var))
    h.build_K()
    with pytest.raises(bti.BtiError) as e:
        h.factor_K()
    assert e.value.status == 6
    assert "pivot 14" in e.value.message
    # the handle stays usable: a valid noise makes it factorable again
    h.set_noise(1e-4)
    h.build_K()
    h.factor_K()
    h.sync()


def test_autograd_gradient_matches_oracle_and_fd():
    p = synthetic.small("grad", 8, 16, 6, 32)
    F = p.blocks_F()
    h = make_handle(F)
    m0 = p.vectors_m(1)
    dobs = p.vectors_d(1)
    s2 = 0.05
    m = cuda(m0).requires_grad_(True)
    d = cuda(dobs)
    r = bti.apply_F_autograd(h, m) - d
    loss = 0.5 * (r * r).sum() / s2
    loss.backward()
    g_or = oracle.loss_gradient(F, m0[0], dobs[0], s2)
    check(relb(host(m.grad), g_or[None]), 1e-12)
    v = np.random.default_rng(0).standard_normal(m0.shape)
    hstep = 1e-6
    lp = oracle.loss(F, (m0 + hstep * v)[0], dobs[0], s2)
    lm = oracle.loss(F, (m0 - hstep * v)[0], dobs[0], s2)
    fd = (lp - lm) / (2 * hstep)
    assert abs(fd - float(np.vdot(host(m.grad), v))) <= 1e-6 * abs(fd) + 1e-8 * abs(float(loss))


def test_df64_is_not_an_io_type():
    p = synthetic.small("df64io", 4, 4, 3, 8)
    h = make_handle(p.blocks_F(), None, bti.DF64)
    m = torch.zeros((1, 8, 16), dtype=torch.float64, device="cuda")
    d = torch.zeros((1, 8, 3), dtype=torch.float64, device="cuda")
    assert bti.lib().bti_apply_F(h.raw, m.data_ptr(), d.data_ptr(), 1, bti.DF64) == 1
    h.close()


def test_online_graph_matches_separate_calls_and_replays():
    p, F, Fq, G, d_obs = tiny_problem()
    h = make_handle(F, Fq, bti.DF64)
    h.set_prior_se_grid(p.gx, p.gy, p.ell, p.sigma_p, bti.DF64)
    h.set_noise(p.sigma2)
    h.build_K()
    h.factor_K()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        h.set_stream(stream)
        d = cuda(np.concatenate([d_obs, 2.0 * d_obs]))
        m = torch.empty((2, p.Nt, p.Nm), dtype=torch.float64, device="cuda")
        q = torch.empty((2, p.Nt, p.Nq), dtype=torch.float64, device="cuda")
        h.online(d, m, q)  # capture + first launch
        m_or = oracle.map_point(F, G, p.sigma2, np.concatenate([d_obs, 2.0 * d_obs]))
        check(relb(host(m), m_or), 1e-12)
        check(relb(host(q), oracle.qoi_map(Fq, m_or)), 1e-12)
        d.mul_(-0.5)  # same buffers, new contents: the graph is replayed
        h.online(d, m, q)
        check(relb(host(m), -0.5 * m_or), 1e-12)
        check(relb(host(q), oracle.qoi_map(Fq, -0.5 * m_or)), 1e-12)
        m2 = torch.empty_like(m)
        h.online(d, m2, None, refine_iters=1)  # other arguments: a new capture
        check(relb(host(m2), -0.5 * m_or), 1e-12)
    torch.cuda.synchronize()
    h.set_stream(torch.cuda.current_stream())
    h.close()


def test_online_graph_refuses_the_legacy_stream():
    p, F, Fq, G, d_obs = tiny_problem()
    h = make_handle(F, Fq)
    h.set_prior_se_grid(p.gx, p.gy, p.ell, p.sigma_p)
    h.set_noise(p.sigma2)
    h.build_K()
    h.factor_K()
    d = cuda(d_obs)
    m = torch.empty((1, p.Nt, p.Nm), dtype=torch.float64, device="cuda")
    L = bti.lib()
    assert L.bti_set_stream(h.raw, None) == 0
    assert L.bti_online(h.raw, d.data_ptr(), m.data_ptr(), None, 1, 0) == 3
    h.close()


@pytest.mark.parametrize("store", [bti.DF64, bti.F32], ids=["df64", "f32"])
def test_autotune_keeps_results(store):
    p = synthetic.small("tune", 8, 300, 13, 45, Nq=3)
    F = p.blocks_F()
    h = make_handle(F, None, store)
    rep = h.autotune(bti.OP_F, 1)
    assert rep["op"] == 0 and rep["fft_p_chosen"] >= 1 and rep["jc_chosen"] >= 512 and rep["vpt_chosen"] in (2, 4, 8)
    dt = torch.float32 if store == bti.F32 else torch.float64
    m = p.vectors_m(1)
    d = p.vectors_d(1)
    od = torch.empty((1, p.Nt, p.Nd), dtype=dt, device="cuda")
    om = torch.empty((1, p.Nt, p.Nm), dtype=dt, device="cuda")
    mg, dg = cuda(m, dt), cuda(d, dt)
    h.apply_F(mg, od)
    h.apply_FT(dg, om)
    check(relb(host(od), oracle.p2o_apply(F, host(mg))), TOL[store])
    check(relb(host(om), oracle.p2o_apply_adjoint(F, host(dg))), TOL[store])
    h.close()


@pytest.mark.parametrize("case", ["tiny", "diagnoise"])
def test_mixed_precision_solve_recovers_fp64(case):
    """K assembled with FP32 products, FP64 Cholesky, refinement with double-FP32
    operators: m_map and q_map reach the FP64 tolerance against the oracle."""
    if case == "tiny":
        p, F, Fq, G, d_obs = tiny_problem()
        noise = p.sigma2
        h = make_handle(F, Fq, bti.DF64)
        h.set_prior_se_grid(p.gx, p.gy, p.ell, p.sigma_p, bti.DF64)
        h.set_noise(p.sigma2)
    else:
        p = synthetic.small("mixed_solve", 6, 6, 5, 30, Nq=3)
        F, Fq = p.blocks_F(), p.blocks_Fq()
        G = oracle.prior_blocks(F, oracle.se_covariance(6, 6, 2.0, 1.0))
        noise = 1e-3 * (1.0 + np.arange(30 * 5).reshape(30, 5) % 7)
        d_obs = p.vectors_d(3)
        h = make_handle(F, Fq, bti.DF64)
        h.set_prior_se_grid(6, 6, 2.0, 1.0, bti.DF64)
        h.set_noise(0.0, cuda(noise))
    h.build_K_prec(0, bti.F32)
    K_low = host(h.copy_K())
    K_or = oracle.assemble_K(F, G, noise)
    low = np.tril_indices(K_or.shape[0])
    err_K = np.linalg.norm(K_low[low] - K_or[low]) / np.linalg.norm(K_or[low])
    assert 1e-12 < err_K < 1e-5  # genuinely low precision, but close
    h.factor_K()
    B = d_obs.shape[0]
    m0 = torch.empty((B, p.Nt, p.Nm), dtype=torch.float64, device="cuda")
    h.infer_map(cuda(d_obs), m0, refine_iters=0)
    m_or = oracle.map_point(F, G, noise, d_obs)
    assert relb(host(m0), m_or) > 1e-11  # without refinement the assembly error shows
    m = torch.empty_like(m0)
    q = torch.empty((B, p.Nt, p.Nq), dtype=torch.float64, device="cuda")
    h.infer_map(cuda(d_obs), m, refine_iters=4)
    h.predict_qoi(m, q)
    check(relb(host(m), m_or), 1e-12)
    check(relb(host(q), oracle.qoi_map(Fq, m_or)), 1e-12)
    h.close()


def test_dense_double_fp32_path():
    """K assembly, Cholesky and solves in double-FP32 arithmetic: K and L close to the
    oracle's, and m_map / q_map at the FP64 tolerance after one refinement step."""
    p, F, Fq, G, d_obs = tiny_problem()
    h = make_handle(F, Fq, bti.DF64)
    h.set_prior_se_grid(p.gx, p.gy, p.ell, p.sigma_p, bti.DF64)
    h.set_noise(p.sigma2)
    h.set_dense_precision(bti.DF64)
    h.build_K()
    K_gpu = host(h.copy_K())
    K_or = oracle.assemble_K(F, G, p.sigma2)
    low = np.tril_indices(K_or.shape[0])
    check(rel(K_gpu[low], K_or[low]), 1e-12)
    h.factor_K()
    L_gpu = host(h.copy_K())
    c = oracle_K("tiny", F, G, p.sigma2, Fq)
    # the factor's updates run in digit planes on the tensor cores (the default)
    check(rel(L_gpu[low], c.L[low]), parity.tol_solve(c.kappa, parity.U_DIGITS),
          f"double-FP32 and digit-plane factor; kappa(K) = {c.kappa:.0f}")
    m = torch.empty((1, p.Nt, p.Nm), dtype=torch.float64, device="cuda")
    q = torch.empty((1, p.Nt, p.Nq), dtype=torch.float64, device="cuda")
    h.infer_map(cuda(d_obs), m, refine_iters=1)
    h.predict_qoi(m, q)
    m_or = oracle.map_point(F, G, p.sigma2, d_obs)
    check(relb(host(m), m_or), 1e-12)
    check(relb(host(q), oracle.qoi_map(Fq, m_or)), 1e-12)
    assert bti.lib().bti_set_dense_precision(h.raw, bti.F32) == 1
    h.close()


def test_elliptic_prior_operator_and_full_map_loss_gradient():
    """A_s m (Eq. (5.1) operator) and the gradient of the full negative log-posterior
    (misfit + elliptic prior term) through the library kernels, against the oracle."""
    p = synthetic.small("elliptic", 6, 9, 4, 12)
    F = p.blocks_F()
    h = make_handle(F, None, bti.DF64)
    A = oracle.elliptic_operator(p.gx, p.gy, 1.3, 0.7)
    m = p.vectors_m(2)
    out = torch.empty((2, p.Nt, p.Nm), dtype=torch.float64, device="cuda")
    h.apply_elliptic(p.gx, p.gy, 1.3, 0.7, cuda(m), out)
    ref = (A @ m.reshape(-1, p.Nm).T).T.reshape(m.shape)
    check(relb(host(out), ref), 1e-14)
    h.apply_elliptic(p.gx, p.gy, 1.3, 0.7, cuda(m), out, squared=True)
    ref2 = (A @ (A @ m.reshape(-1, p.Nm).T)).T.reshape(m.shape)
    check(relb(host(out), ref2), 1e-14)
    # full loss with the prior term, alpha1 = alpha2 = 1 (reading R13)
    A1 = oracle.elliptic_operator(p.gx, p.gy, 1.0, 1.0)
    d = p.vectors_d(1)
    s2 = 0.05
    mg = cuda(m[:1]).requires_grad_(True)
    loss = bti.map_loss(h, mg, cuda(d), s2, p.gx, p.gy)
    loss.backward()
    g_or = oracle.loss_gradient(F, m[0], d[0], s2, A1)
    check(relb(host(mg.grad), g_or[None]), 1e-12)
    assert abs(float(loss.detach()) - oracle.loss(F, m[0], d[0], s2, A1)) <= 1e-12 * abs(float(loss.detach()))
    h.close()


def test_non_finite_input_is_reported_not_spd():
    """A NaN injected on the host (in the noise variances) reaches the first Cholesky
    pivot it touches, which the factorisation reports instead of producing NaN factors."""
    p = synthetic.small("nan_noise", 4, 4, 3, 10)
    F = p.blocks_F()
    var = np.full((10, 3), 1e-2)
    var[2, 0] = np.nan  # data index 6 -> pivot 7
    h = make_handle(F)
    h.set_prior_se_grid(4, 4, 3.0, 1.0)
    h.set_noise(0.0, cuda(var))
    h.build_K()
    with pytest.raises(bti.BtiError) as e:
        h.factor_K()
    assert e.value.status == 6 and "pivot 7" in e.value.message
    h.close()


@pytest.mark.parametrize("dense", ["f64", "df64"])
def test_d2q_map_and_qoi_covariance(dense):
    """Q (Eq. (4.11)) and Gamma_post(q) (Eq. (4.10)) against the oracle; q_map = Q d_obs
    (Eq. (4.14)) equals the push-forward F_q m_map."""
    p, F, Fq, G, d_obs = tiny_problem()
    h = make_handle(F, Fq, bti.DF64)
    h.set_prior_se_grid(p.gx, p.gy, p.ell, p.sigma_p, bti.DF64)
    h.set_noise(p.sigma2)
    if dense == "df64":
        h.set_dense_precision(bti.DF64)
    h.build_K()
    h.factor_K()
    h.build_Q(with_covariance=True)
    Q, C = h.copy_Q(covariance=True)
    Cs = oracle.se_covariance(p.gx, p.gy, p.ell, p.sigma_p)
    Q_or = oracle.d2q_map(Fq, F, G, p.sigma2)
    C_or = oracle.qoi_posterior_covariance(Fq, oracle.prior_blocks(Fq, Cs), F, G, p.sigma2)
    d = cuda(np.concatenate([d_obs, p.vectors_d(2)]))
    q = torch.empty((3, p.Nt, p.Nq), dtype=torch.float64, device="cuda")
    h.apply_Q(d, q)
    q_or = oracle.qoi_map(Fq, oracle.map_point(F, G, p.sigma2, host(d)))
    h.close()
    # rows of Q are solves with K; Gamma_post(q) = X_qq - Q X^T cancels, q = Q d amplifies
    t = d2q_bounds(oracle_K("tiny", F, G, p.sigma2, Fq), Fq, G, Q_or, C_or, host(d),
                   parity.U_F64 if dense == "f64" else parity.U_DIGITS)
    check(rel(host(Q), Q_or), t.tol_Q, t.info)
    check(rel(host(C), C_or), t.tol_C, t.info)
    check(relb(host(q), q_or), t.tol_q, t.info)


def test_d2q_map_through_the_explicit_inverse():
    """With bti_invert_K first (K^{-1} = W^T W, W = L^{-1} from forward solves on the identity,
    the product on the tensor cores), bti_build_Q applies K^{-1} on the tensor cores instead
    of the two triangular solves: Q and Gamma_post(q) still match the oracle."""
    p, F, Fq, G, _ = tiny_problem()
    h = make_handle(F, Fq, bti.DF64)
    h.set_prior_se_grid(p.gx, p.gy, p.ell, p.sigma_p, bti.DF64)
    h.set_noise(p.sigma2)
    h.set_dense_precision(bti.DF64)
    h.build_K()
    h.factor_K()
    h.invert_K()
    h.build_Q(with_covariance=True)
    Q, C = h.copy_Q(covariance=True)
    Cs = oracle.se_covariance(p.gx, p.gy, p.ell, p.sigma_p)
    Q_or = oracle.d2q_map(Fq, F, G, p.sigma2)
    C_or = oracle.qoi_posterior_covariance(Fq, oracle.prior_blocks(Fq, Cs), F, G, p.sigma2)
    h.close()
    t = d2q_bounds(oracle_K("tiny", F, G, p.sigma2, Fq), Fq, G, Q_or, C_or, None, parity.U_DIGITS, kind="inverse")
    check(rel(host(Q), Q_or), t.tol_Q, t.info)
    check(rel(host(C), C_or), t.tol_C, t.info)


@pytest.mark.parametrize("B", [1, 3, 70], ids=["b1", "b3", "b70"])
def test_online_qoi_via_d2q_map_on_tensor_cores(B):
    """bti_set_online_qoi: q_map = Q d_obs (Eq. (4.14)) with Q in FP16 digit planes on the
    tensor cores for B >= 16 (the stream-K product of the explicit inverse, rectangular here:
    N_q N_t = 256 rows against N_d N_t = 512 columns), in bti_apply_Q and in the online graph;
    the dense GEMM for fewer vectors and with tensor cores off, and for one or two vectors the
    matrix-vector product over Q's float pairs; errors for a missing Q."""
    p, F, Fq, G, _ = tiny_problem()
    h = make_handle(F, Fq, bti.DF64)
    h.set_prior_se_grid(p.gx, p.gy, p.ell, p.sigma_p, bti.DF64)
    h.set_noise(p.sigma2)
    h.set_dense_precision(bti.DF64)
    h.build_K()
    h.factor_K()
    with pytest.raises(bti.BtiError) as e:
        h.set_online_qoi(True)
    assert e.value.status == 3
    h.build_Q()
    h.set_online_qoi(True)
    d = p.vectors_d(B)
    m_or = oracle.map_point(F, G, p.sigma2, d)
    q_or = oracle.qoi_map(Fq, m_or)
    # Q from double-FP32 solves with the digit-plane factor (reading R20); the digit-plane and
    # GEMM products of the same Q differ by the products' rounding only
    Q_or = oracle.d2q_map(Fq, F, G, p.sigma2)
    t = d2q_bounds(oracle_K("tiny", F, G, p.sigma2, Fq), Fq, G, Q_or, Q_or, d, parity.U_DIGITS)
    tol_prod = max(parity.FLOOR, parity.C_BOUND * parity.U_DIGITS * t.alpha)
    q = torch.empty((B, p.Nt, p.Nq), dtype=torch.float64, device="cuda")
    h.profile_enable(True)
    h.profile_read()
    h.apply_Q(cuda(d), q)
    n_tc = h.profile_read()[0]["dense"][1]
    if B >= 16:
        assert n_tc == 3 * ((B + 63) // 64)  # per 64 vectors: their planes, MMAs, sum
    elif B <= 2:
        assert n_tc == 2  # the vectors as float pairs, then the matrix-vector product
    else:
        assert n_tc == 1  # fewer than 16 vectors: one dense GEMM (memory-bound)
    check(relb(host(q), q_or), t.tol_q, t.info)
    h.set_tensor_cores(False)
    q2 = torch.empty_like(q)
    h.apply_Q(cuda(d), q2)
    assert h.profile_read()[0]["dense"][1] == (2 if B <= 2 else 1)
    h.set_tensor_cores(True)
    check(relb(host(q), host(q2)), tol_prod, t.info)
    h.profile_enable(False)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        h.set_stream(stream)
        m = torch.empty((B, p.Nt, p.Nm), dtype=torch.float64, device="cuda")
        q3 = torch.empty_like(q)
        h.online(cuda(d), m, q3, refine_iters=1)
        check(relb(host(m), m_or), 1e-12)
        check(relb(host(q3), q_or), t.tol_q, t.info)
        # a new Q (here the same map rebuilt, in a new buffer) is picked up by the online graph
        h.build_Q()
        h.online(cuda(d), m, q3, refine_iters=1)
        check(relb(host(q3), q_or), t.tol_q, t.info)
        h.set_online_qoi(False)
        h.online(cuda(d), m, q3, refine_iters=1)  # back to the push-forward F_q m_map
        check(relb(host(q3), q_or), 1e-12)
    torch.cuda.synchronize()
    h.set_stream(torch.cuda.current_stream())
    h.close()


ONLINE_LATENCY_TOL = 1e-6  # the online latency metric's relative error


@pytest.mark.parametrize("via_Q", [True, False], ids=["via_Q", "push_forward"])
def test_online_fp32_level_form(via_Q):
    """bti_set_online_precision(BTI_P_F32): the online graph with its digit-plane products cut
    to their most significant planes (five for K^{-1}, four for G^*, F_q and Q).  B = 20
    vectors on the tensor cores; m_map and q_map against the oracle within the online latency
    metric's 1e-6; the truncation takes effect (the result differs from the FP64-level form's);
    refinement is refused; switching back restores the FP64-level graph."""
    p, F, Fq, G, _ = tiny_problem()
    B = 20
    d = p.vectors_d(B)
    m_or = oracle.map_point(F, G, p.sigma2, d)
    q_or = oracle.qoi_map(Fq, m_or)
    h = make_handle(F, Fq, bti.DF64)
    h.set_prior_se_grid(p.gx, p.gy, p.ell, p.sigma_p, bti.DF64)
    h.set_noise(p.sigma2)
    h.set_dense_precision(bti.DF64)
    h.build_K()
    h.factor_K()
    h.invert_K()
    h.set_digit_planes(bti.OP_G, True)
    h.set_digit_planes(bti.OP_FQ, True)
    if via_Q:
        h.build_Q()
        h.set_online_qoi(True)
    with pytest.raises(bti.BtiError) as e:
        h.set_online_precision(bti.F16)
    assert e.value.status == 1
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        h.set_stream(stream)
        m = torch.empty((B, p.Nt, p.Nm), dtype=torch.float64, device="cuda")
        q = torch.empty((B, p.Nt, p.Nq), dtype=torch.float64, device="cuda")
        h.online(cuda(d), m, q)
        m64, q64 = host(m), host(q)
        h.set_online_precision(bti.F32)
        with pytest.raises(bti.BtiError) as e:
            h.online(cuda(d), m, q, refine_iters=1)
        assert e.value.status == 1
        h.online(cuda(d), m, q)
        m32, q32 = host(m), host(q)
        h.set_online_precision(bti.DF64)
        h.online(cuda(d), m, q)
        m64b = host(m)
    torch.cuda.synchronize()
    h.set_stream(torch.cuda.current_stream())
    h.close()
    check(relb(m32, m_or), ONLINE_LATENCY_TOL, "m_map, FP32-level online form")
    check(relb(q32, q_or), ONLINE_LATENCY_TOL, "q_map, FP32-level online form")
    assert relb(m32, m64) > 1e-12  # the truncated planes took effect
    assert np.array_equal(m64b, m64)  # the FP64-level graph is back, bit for bit


def test_replacing_blocks_drops_what_was_derived_from_them():
    """bti_set_blocks on an operator that is already set must take effect everywhere:
    - the old blocks' digit planes go, so B >= 16 products use the new blocks;
    - Q goes when any operator or the noise changes;
    - a G that a prior formed from the old F goes;
    - calls that need what was dropped return BTI_ERR_STATE until it is rebuilt."""
    p, F, Fq, G, _ = tiny_problem()
    B = 16
    rng = np.random.default_rng(5)
    F2 = F * (1.0 + 0.5 * rng.standard_normal(F.shape))
    Fq2 = Fq * (1.0 + 0.5 * rng.standard_normal(Fq.shape))
    m = p.vectors_m(B)
    d = p.vectors_d(B)
    h = make_handle(F, Fq, bti.DF64)
    h.set_prior_se_grid(p.gx, p.gy, p.ell, p.sigma_p, bti.DF64)
    h.set_noise(p.sigma2)
    h.set_dense_precision(bti.DF64)
    for op in (bti.OP_F, bti.OP_G, bti.OP_FQ):
        h.set_digit_planes(op, True)
    h.build_K()
    h.factor_K()
    h.build_Q()
    out_d = torch.empty((B, p.Nt, p.Nd), dtype=torch.float64, device="cuda")
    out_q = torch.empty((B, p.Nt, p.Nq), dtype=torch.float64, device="cuda")
    h.apply_F(cuda(m), out_d)
    check(relb(host(out_d), oracle.p2o_apply(F, m)), 1e-12)

    def state_error(fn, *args):
        with pytest.raises(bti.BtiError) as e:
            fn(*args)
        assert e.value.status == 3

    h.set_blocks(bti.OP_F, cuda(F2), bti.DF64)
    h.apply_F(cuda(m), out_d)
    check(relb(host(out_d), oracle.p2o_apply(F2, m)), 1e-12)
    state_error(h.apply_Q, cuda(d), out_q)
    state_error(h.build_K)  # G was formed from the old F
    state_error(h.apply_Gstar, cuda(d), torch.empty((B, p.Nt, p.Nm), dtype=torch.float64, device="cuda"))
    h.set_prior_se_grid(p.gx, p.gy, p.ell, p.sigma_p, bti.DF64)
    h.set_digit_planes(bti.OP_F, True)
    h.set_digit_planes(bti.OP_G, True)
    h.profile_enable(True)
    h.profile_read()
    h.apply_F(cuda(m), out_d)
    assert h.profile_read()[0]["prod_fwd"][1] == 3  # the digit-plane path again, on the new planes
    h.profile_enable(False)
    check(relb(host(out_d), oracle.p2o_apply(F2, m)), 1e-12)
    Cs = oracle.se_covariance(p.gx, p.gy, p.ell, p.sigma_p)
    G2 = oracle.prior_blocks(F2, Cs)
    h.build_K()
    h.factor_K()
    h.build_Q()
    h.apply_Q(cuda(d), out_q)
    Q2 = oracle.d2q_map(Fq, F2, G2, p.sigma2)
    q_or = (d.reshape(B, -1) @ Q2.T).reshape(B, p.Nt, p.Nq)
    t = d2q_bounds(oracle_K("tiny_F2", F2, G2, p.sigma2, Fq), Fq, G2, Q2, Q2, d, parity.U_F64)
    check(relb(host(out_q), q_or), t.tol_q, t.info)

    h.set_blocks(bti.OP_FQ, cuda(Fq2), bti.DF64)
    state_error(h.apply_Q, cuda(d), out_q)
    h.apply_Fq(cuda(m), out_q)
    check(relb(host(out_q), oracle.p2o_apply(Fq2, m)), 1e-12)
    h.build_Q()
    h.set_noise(2.0 * p.sigma2)
    state_error(h.apply_Q, cuda(d), out_q)
    h.close()


def test_posterior_covariance_actions_and_prior_mean():
    """Gamma_prior v, Gamma_post(m) v (Eq. (4.7)), pointwise posterior variances from unit
    vectors, and m_map with a nonzero prior mean (Eq. (4.13) with Eq. (4.8))."""
    p, F, Fq, G, d_obs = tiny_problem()
    Cs = oracle.se_covariance(p.gx, p.gy, p.ell, p.sigma_p)
    h = make_handle(F, Fq, bti.DF64)
    h.set_prior_se_grid(p.gx, p.gy, p.ell, p.sigma_p, bti.DF64)
    h.set_noise(p.sigma2)
    h.build_K()
    h.factor_K()
    v = p.vectors_m(3)
    out = torch.empty((3, p.Nt, p.Nm), dtype=torch.float64, device="cuda")
    h.apply_prior(cuda(v), out)
    check(relb(host(out), oracle.prior_apply(Cs, v)), 1e-13)
    h.apply_postcov(cuda(v), out)
    tol, info = postcov_bound(oracle_K("tiny", F, G, p.sigma2, Fq), Cs, v, parity.U_F64)
    check(relb(host(out), oracle.posterior_cov_apply(F, G, Cs, p.sigma2, v)), tol, info)
    # two pointwise variances: e^T Gamma_post(m) e for unit vectors e
    E = np.zeros((2, p.Nt, p.Nm))
    E[0, 5, 17] = 1.0
    E[1, 60, 200] = 1.0
    col = torch.empty((2, p.Nt, p.Nm), dtype=torch.float64, device="cuda")
    h.apply_postcov(cuda(E), col)
    col = host(col)
    ref = oracle.posterior_cov_apply(F, G, Cs, p.sigma2, E)
    for b, (t, j) in enumerate(((5, 17), (60, 200))):
        var = col[b, t, j]
        assert abs(var - ref[b, t, j]) <= 1e-11 * abs(ref[b, t, j])
        assert 0.0 < var <= p.sigma_p ** 2  # the data can only reduce the prior variance
    m0 = 0.3 * p.vectors_m(1)
    mm = torch.empty((1, p.Nt, p.Nm), dtype=torch.float64, device="cuda")
    h.infer_map_prior(cuda(d_obs), cuda(m0), mm)
    check(relb(host(mm), oracle.map_point_with_prior_mean(F, G, p.sigma2, d_obs, m0)), 1e-12)
    h.close()


@pytest.mark.parametrize("probes", ["unit", "signs"])
def test_posterior_variance_probe(probes):
    """bti_postcov_diag_probe against the oracle's estimator on the same probes: all unit
    vectors (the exact diagonal of Gamma_post(m), 128 probes in two batches) and 100 random
    sign vectors (a batch of 64 and one of 36); every estimated variance lies in (0, sigma_p^2]."""
    p = synthetic.small("var_probe", 4, 4, 3, 8, Nq=2)
    F = p.blocks_F()
    Cs = oracle.se_covariance(4, 4, 2.0, 1.0)
    G = oracle.prior_blocks(F, Cs)
    h = make_handle(F, None, bti.DF64)
    h.set_prior_se_grid(4, 4, 2.0, 1.0, bti.DF64)
    h.set_noise(1e-2)
    h.build_K()
    h.factor_K()
    N = p.Nt * p.Nm
    if probes == "unit":
        V = np.eye(N).reshape(N, p.Nt, p.Nm)
    else:
        V = np.sign(np.random.default_rng(7).standard_normal((100, p.Nt, p.Nm)))
    out = torch.empty((p.Nt, p.Nm), dtype=torch.float64, device="cuda")
    h.postcov_diag_probe(cuda(V), out)
    ref = oracle.posterior_variance_probe(F, G, Cs, 1e-2, V)
    got = host(out)
    tol, info = postcov_bound(oracle_K("var_probe", F, G, 1e-2), Cs, V, parity.U_F64, probe=True)
    check(rel(got, ref), tol, info)
    if probes == "unit":
        assert np.all(got > 0.0) and np.all(got <= 1.0 + 1e-12)
    h.close()


@pytest.mark.parametrize("stride", [4, 16])
def test_coarse_qoi_grid(stride):
    """QoIs on every stride-th time step (the Remark after Eq. (2.15); the Sec. 5 example
    reads them at 1 Hz from a 10 Hz grid): F_q m, predict_qoi, the online graph, Q,
    Gamma_post(q) and Q d_obs on the coarse grid against the oracle's selected rows."""
    p, F, Fq, G, d_obs = tiny_problem()
    steps = oracle.qoi_time_steps(p.Nt, stride)
    rows = oracle.qoi_rows(p.Nt, p.Nq, stride)
    Ntq = p.Nt // stride
    h = make_handle(F, Fq, bti.DF64)
    h.set_prior_se_grid(p.gx, p.gy, p.ell, p.sigma_p, bti.DF64)
    h.set_noise(p.sigma2)
    h.build_K()
    h.factor_K()
    h.set_qoi_stride(stride)
    m = p.vectors_m(2)
    q = torch.empty((2, Ntq, p.Nq), dtype=torch.float64, device="cuda")
    h.apply_Fq(cuda(m), q)
    check(relb(host(q), oracle.qoi_map(Fq, m)[:, steps]), 1e-12)
    c = oracle_K("tiny", F, G, p.sigma2, Fq)
    b = solve_bounds(c, d_obs, parity.U_F64)
    q_or = b.q[:, steps]
    # the kept steps carry the whole vector's error: relative to their own norm it grows by
    # ||q|| / ||q_kept||
    tol_q = b.tol_q * float(np.linalg.norm(b.q) / np.linalg.norm(q_or))
    mm = torch.empty((1, p.Nt, p.Nm), dtype=torch.float64, device="cuda")
    q1 = torch.empty((1, Ntq, p.Nq), dtype=torch.float64, device="cuda")
    h.infer_map(cuda(d_obs), mm)
    h.predict_qoi(mm, q1)
    check(relb(host(q1), q_or), tol_q, b.info)
    stream = torch.cuda.Stream()  # graph capture needs a non-default stream
    with torch.cuda.stream(stream):
        h.set_stream(stream)
        q1.zero_()
        h.online(cuda(d_obs), mm, q1)
        check(relb(host(q1), q_or), tol_q, b.info)
    torch.cuda.synchronize()
    h.set_stream(torch.cuda.current_stream())
    h.build_Q(with_covariance=True)
    Q, C = h.copy_Q(covariance=True)
    assert tuple(Q.shape) == (Ntq * p.Nq, p.Nt * p.Nd) and tuple(C.shape) == (Ntq * p.Nq,) * 2
    Cs = oracle.se_covariance(p.gx, p.gy, p.ell, p.sigma_p)
    Q_or = oracle.d2q_map(Fq, F, G, p.sigma2)[rows]
    C_or = oracle.qoi_posterior_covariance(Fq, oracle.prior_blocks(Fq, Cs), F, G, p.sigma2)[np.ix_(rows, rows)]
    t = d2q_bounds(c, Fq, G, Q_or, C_or, d_obs, parity.U_F64, rows=rows)
    check(rel(host(Q), Q_or), t.tol_Q, t.info)
    check(rel(host(C), C_or), t.tol_C, t.info)
    q1.zero_()
    h.apply_Q(cuda(d_obs), q1)
    check(relb(host(q1), q_or), t.tol_q, t.info)
    # back to the full grid: Q must be rebuilt, and F_q writes every step again
    h.set_qoi_stride(1)
    with pytest.raises(bti.BtiError):
        h.apply_Q(cuda(d_obs), torch.empty((1, p.Nt, p.Nq), dtype=torch.float64, device="cuda"))
    qf = torch.empty((2, p.Nt, p.Nq), dtype=torch.float64, device="cuda")
    h.apply_Fq(cuda(m), qf)
    check(relb(host(qf), oracle.qoi_map(Fq, m)), 1e-12)
    with pytest.raises(bti.BtiError):
        h.set_qoi_stride(3)  # does not divide N_t = 64
    h.close()


@pytest.mark.parametrize("form", ["plain_df64", "refined_f16", "refined_f32_f64store", "flexible_f16",
                                  "plain_df64_pc", "flexible_f16_pc"])
def test_matrix_free_solve_matches_dense_oracle(form):
    """m_map = G^* K^{-1} d_obs by conjugate gradients without forming K, against the
    oracle's dense Cholesky solve: FP64 CG with double-FP32 operators, and FP64
    refinement around FP32 CG with FP16 (or FP32) shadow operators."""
    p, F, Fq, G, d_obs = tiny_problem()
    d = np.concatenate([d_obs, p.vectors_d(2)])
    store = bti.F64 if form == "refined_f32_f64store" else bti.DF64
    h = make_handle(F, None, store)
    h.set_noise(p.sigma2)
    if form.startswith("plain_df64"):
        h.set_prior_se_grid(p.gx, p.gy, p.ell, p.sigma_p, bti.DF64)
    else:
        low = bti.F32 if form == "refined_f32_f64store" else bti.F16
        h.set_prior_se_grid(p.gx, p.gy, p.ell, p.sigma_p, low)
        h.set_shadow(bti.OP_F, low)
    if form.endswith("_pc"):
        h.set_matfree_precond(1)
    m = torch.empty((3, p.Nt, p.Nm), dtype=torch.float64, device="cuda")
    x = torch.empty((3, p.Nt, p.Nd), dtype=torch.float64, device="cuda")
    refine = {"plain_df64": 0, "flexible_f16": 2, "plain_df64_pc": 0, "flexible_f16_pc": 2}.get(form, 1)
    info = h.solve_matfree(cuda(d), m, x, refine=refine, tol=1e-12, max_outer=100, max_inner=2000,
                           inner_tol=0.2 if refine == 2 else 1e-3)
    h.close()
    # stopped at ||d - K x|| <= 1e-12 ||d|| with the FP64-accurate operator (FP64 with the F64
    # store, else double-FP32): the CG bound of reading R20
    u = parity.U_F64 if store == bti.F64 else parity.U_DF64
    b = solve_bounds(oracle_K("tiny", F, G, p.sigma2, Fq), d, u, kind="cg", eta=1e-12)
    check(relb(host(x), b.x), b.tol_x, b.info + " " + str(info))
    check(relb(host(m), b.m), b.tol_m, b.info + " " + str(info))
    assert info["rel_residual"] <= 1e-12
    if refine == 1:  # each refinement step gains about -log10(kappa(K) ||K - K~|| / ||K||) digits
        assert 1 <= info["outer_iters"] <= 30, info


def test_block_jacobi_preconditioner_cuts_iterations():
    """With the block-Jacobi preconditioner the FP64 CG of the matrix-free solve needs fewer
    iterations for the same residual, and the answer is unchanged (against the oracle)."""
    p, F, Fq, G, d_obs = tiny_problem()
    h = make_handle(F, None, bti.DF64)
    h.set_noise(p.sigma2)
    h.set_prior_se_grid(p.gx, p.gy, p.ell, p.sigma_p, bti.DF64)
    m = torch.empty((1, p.Nt, p.Nm), dtype=torch.float64, device="cuda")
    plain = h.solve_matfree(cuda(d_obs), m, refine=0, tol=1e-12, max_inner=3000)
    h.set_matfree_precond(1)
    pcg = h.solve_matfree(cuda(d_obs), m, refine=0, tol=1e-12, max_inner=3000)
    h.set_noise(p.sigma2)  # drops the preconditioner: the plain count again
    again = h.solve_matfree(cuda(d_obs), m, refine=0, tol=1e-12, max_inner=3000)
    h.close()
    assert pcg["inner_iters"] < plain["inner_iters"], (pcg, plain)
    assert again["inner_iters"] == plain["inner_iters"]
    b = solve_bounds(oracle_K("tiny", F, G, p.sigma2, Fq), d_obs, parity.U_DF64, kind="cg", eta=1e-12)
    check(relb(host(m), b.m), b.tol_m, b.info)


def test_matrix_free_solve_reports_no_convergence():
    """An iteration limit too small for the tolerance returns BTI_ERR_NO_CONVERGENCE,
    with the statistics of the iterations taken and the last iterate written."""
    p, F, Fq, G, d_obs = tiny_problem()
    h = make_handle(F, None, bti.DF64)
    h.set_noise(p.sigma2)
    h.set_prior_se_grid(p.gx, p.gy, p.ell, p.sigma_p, bti.DF64)
    m = torch.full((1, p.Nt, p.Nm), float("nan"), dtype=torch.float64, device="cuda")
    with pytest.raises(bti.BtiError) as e:
        h.solve_matfree(cuda(d_obs), m, refine=False, tol=1e-14, max_inner=3)
    assert e.value.status == 8
    assert h.last_solve["inner_iters"] == 3 and h.last_solve["rel_residual"] > 1e-14
    assert torch.isfinite(m).all()
    with pytest.raises(bti.BtiError) as e:  # F in a low tier cannot give the FP64 residual
        h2 = make_handle(F, None, bti.F32)
        h2.set_noise(p.sigma2)
        h2.set_prior_se_grid(p.gx, p.gy, p.ell, p.sigma_p, bti.F32)
        h2.solve_matfree(cuda(d_obs), m)
    assert e.value.status == 3
    h2.close()
    h.close()


def test_tensor_core_wait_timeout_is_reported_and_recoverable():
    """Failure handling without a fault: with one pipeline stage withheld (test hook), the
    tensor-core forward's bounded waits run out; bti_sync reports BTI_ERR_TIMEOUT once, and
    the same handle then computes correct products again."""
    p = synthetic.small("tc_timeout", 1, 2048, 64, 32, Nq=4)
    F = p.blocks_F()
    h = make_handle(F, None, bti.F16)
    m = cuda(p.vectors_m(16), torch.float32)
    d = torch.empty((16, 32, 64), dtype=torch.float32, device="cuda")
    h.test_withhold_tc_stage(2)
    h.apply_F(m, d)
    with pytest.raises(bti.BtiError) as e:
        h.sync()
    assert e.value.status == 7  # BTI_ERR_TIMEOUT
    h.sync()  # reported once
    h.test_withhold_tc_stage(-1)
    h.apply_F(m, d)
    h.sync()
    h.close()
    check(relb(host(d), oracle.p2o_apply(F, host(m))), 1e-3)


@pytest.mark.parametrize("which", ["adjoint", "forward"])
def test_digit_plane_wait_timeout_is_reported_and_recoverable(which):
    """The same failure handling in the digit-plane kernels (adjoint: adj_tc_kernel; forward:
    the stream-K kernel shared with the explicit inverse and Q): with one TMA stage withheld
    the bounded waits run out, the whole MMA warp agrees on the abort, the kernel drains,
    frees its tensor memory and sets the status word; bti_sync reports BTI_ERR_TIMEOUT once
    and the handle computes correct products afterwards."""
    p = synthetic.small("dig_timeout", 1, 512, 20, 16, Nq=2)
    F = p.blocks_F()
    h = make_handle(F, None, bti.DF64)
    h.set_digit_planes(bti.OP_F, True)
    if which == "adjoint":
        x = cuda(p.vectors_d(16))
        y = torch.empty((16, 16, 512), dtype=torch.float64, device="cuda")
        run, ref = h.apply_FT, lambda: oracle.p2o_apply_adjoint(F, host(x))
    else:
        x = cuda(p.vectors_m(16))
        y = torch.empty((16, 16, 20), dtype=torch.float64, device="cuda")
        run, ref = h.apply_F, lambda: oracle.p2o_apply(F, host(x))
    h.test_withhold_tc_stage(1)  # the second 32-column box: every CTA here loads at least two
    run(x, y)
    with pytest.raises(bti.BtiError) as e:
        h.sync()
    assert e.value.status == 7  # BTI_ERR_TIMEOUT
    h.sync()  # reported once
    h.test_withhold_tc_stage(-1)
    run(x, y)
    h.sync()
    check(relb(host(y), ref()), 1e-12)
    h.close()


@pytest.mark.parametrize("store", [bti.F64, bti.DF64], ids=["f64", "df64"])
def test_elliptic_prior_full_inversion(store):
    """The elliptic prior of Eq. (5.1), Gamma_prior = (alpha1 I - alpha2 Delta_h)^{-2},
    applied by DCT on each axis: Gamma_prior v, K, m_map, q_map, Gamma_post(m) v and the
    matrix-free solve against the oracle with the dense inverse of A_s^2."""
    p = synthetic.small("elliptic_inv", 8, 12, 5, 24, Nq=3)
    F, Fq = p.blocks_F(), p.blocks_Fq()
    A = oracle.elliptic_operator(p.gx, p.gy, 1.3, 0.7).toarray()
    Cs = np.linalg.inv(A @ A)
    Cs = 0.5 * (Cs + Cs.T)
    G = oracle.prior_blocks(F, Cs)
    h = make_handle(F, Fq, store)
    h.set_prior_elliptic_grid(p.gx, p.gy, 1.3, 0.7, store)
    h.set_noise(p.sigma2)
    v = p.vectors_m(2)
    out = torch.empty((2, p.Nt, p.Nm), dtype=torch.float64, device="cuda")
    h.apply_prior(cuda(v), out)
    check(relb(host(out), oracle.prior_apply(Cs, v)), 1e-12)
    d = p.vectors_d(2)
    h.build_K()
    h.factor_K()
    m = torch.empty((2, p.Nt, p.Nm), dtype=torch.float64, device="cuda")
    q = torch.empty((2, p.Nt, p.Nq), dtype=torch.float64, device="cuda")
    h.infer_map(cuda(d), m)
    h.predict_qoi(m, q)
    c = oracle_K("elliptic_inv", F, G, p.sigma2, Fq)
    b = solve_bounds(c, d, parity.U_F64)
    check(relb(host(m), b.m), b.tol_m, b.info)
    check(relb(host(q), b.q), b.tol_q, b.info)
    h.apply_postcov(cuda(v), out)
    tol, info = postcov_bound(c, Cs, v, parity.U_F64)
    check(relb(host(out), oracle.posterior_cov_apply(F, G, Cs, p.sigma2, v, L=c.L)), tol, info)
    m.zero_()
    h.solve_matfree(cuda(d), m, refine=0, tol=1e-12, max_inner=4000)
    h.close()
    bc = solve_bounds(c, d, parity.U_F64 if store == bti.F64 else parity.U_DF64, kind="cg", eta=1e-12)
    check(relb(host(m), bc.m), bc.tol_m, bc.info)


@pytest.mark.parametrize("B", [1, 5, 20, 70], ids=["b1", "b5", "b20", "b70"])
def test_explicit_inverse_online_solve(B):
    """bti_invert_K: x = K^{-1} d as one product with the explicit inverse, on the tensor
    cores (six FP16 digit planes, exact per accumulation period) and, with tensor cores off,
    in double-FP32 on the CUDA cores (4-, 16- and 64-wide right-hand-side tiles); stream-K
    partials summed in CTA order; a second 64-chunk at B = 70.  m_map matches the oracle,
    refinement brings it to the FP64 tolerance, a new factorisation returns to the
    triangular solves until the inverse is formed again, and release works."""
    p, F, Fq, G, _ = tiny_problem()
    d = p.vectors_d(B)
    m_or = oracle.map_point(F, G, p.sigma2, d)
    # the inverse is W^T W on the tensor cores (47-bit digit planes): the explicit-inverse
    # bound of reading R20.  The two products of the same inverse differ by the rounding of its
    # two images only: each entry within 2^-47 of its row's largest, so the outputs differ by
    # at most 2 2^-47 ||r|| with r_i = max_j |K^{-1}_ij| ||d||_1 (per vector), times C = 10 slack
    c = oracle_K("tiny", F, G, p.sigma2, Fq)
    bi = solve_bounds(c, d, parity.U_DIGITS, kind="inverse")
    Kinv = oracle.solve_K(c.L, np.eye(c.K.shape[0]))
    rowmax = np.abs(Kinv).max(axis=1)
    dflat = d.reshape(B, -1)
    tol_prod = max(parity.FLOOR, float(np.max(
        parity.C_BOUND * 2 * parity.U_DIGITS * np.linalg.norm(rowmax) * np.abs(dflat).sum(axis=1)
        / np.linalg.norm(bi.x.reshape(B, -1), axis=1))))
    h = make_handle(F, Fq, bti.DF64)
    h.set_prior_se_grid(p.gx, p.gy, p.ell, p.sigma_p, bti.DF64)
    h.set_noise(p.sigma2)
    with pytest.raises(bti.BtiError) as e:
        h.invert_K()
    assert e.value.status == 3
    h.build_K()
    h.factor_K()
    m = torch.empty((B, p.Nt, p.Nm), dtype=torch.float64, device="cuda")
    h.profile_enable(True)
    h.profile_read()
    h.infer_map(cuda(d), m)
    n_trsm = h.profile_read()[0]["dense"][1]
    check(relb(host(m), m_or), 1e-12)
    h.invert_K()
    h.profile_read()  # drop the launches of forming the inverse
    m.zero_()
    h.infer_map(cuda(d), m)
    n_inv = h.profile_read()[0]["dense"][1]
    assert n_inv + 20 < n_trsm  # a few launches per 64 vectors, not 2 n / 64 blocked steps
    check(relb(host(m), m_or), bi.tol_m, bi.info)
    # the same product in double-FP32 on the CUDA cores (tensor cores off)
    h.set_tensor_cores(False)
    m_dd = torch.empty_like(m)
    h.infer_map(cuda(d), m_dd)
    h.set_tensor_cores(True)
    check(relb(host(m_dd), m_or), bi.tol_m, bi.info)
    check(relb(host(m), host(m_dd)), tol_prod, bi.info)
    h.infer_map(cuda(d), m, refine_iters=1)
    check(relb(host(m), m_or), 1e-12)
    # the online graph applies the inverse too, and with G's digit planes its G^* (B >= 16)
    # runs on the tensor cores as well
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        h.set_stream(stream)
        q = torch.empty((B, p.Nt, p.Nq), dtype=torch.float64, device="cuda")
        m2 = torch.empty_like(m)
        h.online(cuda(d), m2, q, refine_iters=1)
        check(relb(host(m2), m_or), 1e-12)
        check(relb(host(q), oracle.qoi_map(Fq, m_or)), 1e-12)
        h.set_digit_planes(bti.OP_G, True)
        h.set_digit_planes(bti.OP_FQ, True)
        h.online(cuda(d), m2, q)
        check(relb(host(m2), m_or), bi.tol_m, bi.info)
        check(relb(host(q), bi.q), bi.tol_q, bi.info)
        h.set_digit_planes(bti.OP_G, False)
        h.set_digit_planes(bti.OP_FQ, False)
    torch.cuda.synchronize()
    h.set_stream(torch.cuda.current_stream())
    # a new factor: the stale inverse is not used
    h.set_noise(2.0 * p.sigma2)
    h.build_K()
    h.factor_K()
    h.profile_read()
    h.infer_map(cuda(d), m)
    assert h.profile_read()[0]["dense"][1] == n_trsm
    check(relb(host(m), oracle.map_point(F, G, 2.0 * p.sigma2, d)), 1e-12)
    h.invert_K()
    h.infer_map(cuda(d), m)
    b2 = solve_bounds(oracle_K("tiny_2s", F, G, 2.0 * p.sigma2, Fq), d, parity.U_DIGITS, kind="inverse")
    check(relb(host(m), b2.m), b2.tol_m, b2.info)
    h.invert_K(False)
    h.infer_map(cuda(d), m)
    check(relb(host(m), oracle.map_point(F, G, 2.0 * p.sigma2, d)), 1e-12)
    h.profile_enable(False)
    h.close()


def test_explicit_inverse_ragged_size():
    """n = 150 (two 128-row tiles, the second ragged; rows padded to 160 columns) with a
    diagonal noise covariance."""
    p = synthetic.small("kinv_ragged", 6, 6, 5, 30, Nq=3)
    F = p.blocks_F()
    Cs = oracle.se_covariance(6, 6, 2.0, 1.0)
    G = oracle.prior_blocks(F, Cs)
    var = 1e-3 * (1.0 + np.arange(30 * 5).reshape(30, 5) % 7)
    d_obs = p.vectors_d(7)
    h = make_handle(F, p.blocks_Fq())
    h.set_prior_se_grid(6, 6, 2.0, 1.0)
    h.set_noise(0.0, cuda(var))
    h.build_K(col_block=37)
    h.factor_K()
    h.invert_K()
    m_map = torch.empty((7, 30, 36), dtype=torch.float64, device="cuda")
    h.infer_map(cuda(d_obs), m_map, refine_iters=1)
    # one refinement step with FP64 residuals after the explicit inverse: the solve bound
    b = solve_bounds(oracle_K("kinv_ragged", F, G, var), d_obs, parity.U_F64)
    check(relb(host(m_map), b.m), b.tol_m, b.info)
    # one vector: the symmetric product over the inverse's lower triangle (n = 150: a full
    # 128-row panel and a ragged one of 22 rows), no refinement
    m1 = torch.empty((1, 30, 36), dtype=torch.float64, device="cuda")
    h.infer_map(cuda(d_obs[2:3]), m1)
    b1 = solve_bounds(oracle_K("kinv_ragged", F, G, var), d_obs[2:3], parity.U_DIGITS, kind="inverse")
    check(relb(host(m1), b1.m), b1.tol_m, b1.info)
    h.close()


DIGIT_CASES = [
    # (name, Nm, Nd, Nt, B): ragged row tiles (N_m % 128 != 0), one or two column groups,
    # one or many 128-wide accumulation chunks (2 R up to 2,200), ragged vector groups
    ("b16_R13_ragged", 1000, 13, 45, 16),
    ("b40_two_groups", 700, 6, 64, 40),
    ("b20_R1100_chunks", 300, 1100, 8, 20),
    ("b64_Nm512", 512, 20, 30, 64),
]


@pytest.mark.parametrize("name,Nm,Nd,Nt,B", DIGIT_CASES, ids=[c[0] for c in DIGIT_CASES])
def test_digit_plane_products_match_oracle(name, Nm, Nd, Nt, B):
    """bti_set_digit_planes: the double-FP32 tier's products for B >= 16 on the tensor cores,
    exact in FP16 digit planes -- the adjoint (row tiles of N_m, K = 2 N_d) and the forward
    products F and F_q (stream-K over K = 2 N_m; 32- or 64-row groups of F, 18 of them at
    N_d = 1,100) -- match the oracle at the FP64 tolerance and the CUDA-core double-FP32
    kernels closely; releasing the planes returns to the CUDA cores."""
    p = synthetic.small(name, 1, Nm, Nd, Nt, Nq=2)
    F = p.blocks_F()
    Fq = p.blocks_Fq()
    d = p.vectors_d(B)
    m = p.vectors_m(B)
    h = make_handle(F, Fq, bti.DF64)
    h.set_digit_planes(bti.OP_F, True)
    h.set_digit_planes(bti.OP_FQ, True)
    out_m = torch.empty((B, Nt, Nm), dtype=torch.float64, device="cuda")
    out_d = torch.empty((B, Nt, Nd), dtype=torch.float64, device="cuda")
    out_q = torch.empty((B, Nt, 2), dtype=torch.float64, device="cuda")
    h.profile_enable(True)
    h.profile_read()
    h.apply_FT(cuda(d), out_m)
    h.apply_F(cuda(m), out_d)
    h.apply_Fq(cuda(m), out_q)
    prof = h.profile_read()[0]
    ngroups = (B + 63) // 64
    assert prof["prod_adj"][1] == 2  # vector planes + the tensor-core kernel
    assert prof["prod_fwd"][1] == 2 * 3 * ngroups  # per 64 vectors: planes, stream-K kernel, sum
    assert prof["reduce"][1] == 0
    check(relb(host(out_m), oracle.p2o_apply_adjoint(F, d)), 1e-12)
    check(relb(host(out_d), oracle.p2o_apply(F, m)), 1e-12)
    check(relb(host(out_q), oracle.p2o_apply(Fq, m)), 1e-12)
    h.set_digit_planes(bti.OP_F, False)
    h.set_digit_planes(bti.OP_FQ, False)
    out_m2, out_d2 = torch.empty_like(out_m), torch.empty_like(out_d)
    h.apply_FT(cuda(d), out_m2)
    h.apply_F(cuda(m), out_d2)
    prof = h.profile_read()[0]
    assert prof["prod_adj"][1] == 1 and prof["prod_fwd"][1] == 1
    check(relb(host(out_m), host(out_m2)), 1e-12)
    check(relb(host(out_d), host(out_d2)), 1e-12)
    h.profile_enable(False)
    h.close()


def test_digit_planes_need_the_double_fp32_tier():
    p = synthetic.small("dig_state", 1, 64, 3, 8)
    h = make_handle(p.blocks_F(), None, bti.F64)
    with pytest.raises(bti.BtiError) as e:
        h.set_digit_planes(bti.OP_F, True)
    assert e.value.status == 3
    h.close()


def _df64_products_both_paths(F, m, d):
    """F m and F^T d in the double-FP32 tier: 3 vectors per call (the CUDA-core float-pair
    kernels) and all of them per call with digit planes on the tensor cores (B >= 16)."""
    Nt, Nd, Nm = F.shape
    B = m.shape[0]
    h = make_handle(F, None, bti.DF64)
    out = {}
    for path in ("cuda_cores", "digit_planes"):
        if path == "digit_planes":
            h.set_digit_planes(bti.OP_F, True)
        nb = 3 if path == "cuda_cores" else B
        od = torch.empty((nb, Nt, Nd), dtype=torch.float64, device="cuda")
        om = torch.empty((nb, Nt, Nm), dtype=torch.float64, device="cuda")
        h.apply_F(cuda(m[:nb]), od)
        h.apply_FT(cuda(d[:nb]), om)
        out[path] = (host(od), host(om), nb)
    h.close()
    return out


@pytest.mark.parametrize("scale", [1e-20, 1e-30, 1e30], ids=["1e-20", "1e-30", "1e+30"])
def test_double_fp32_tier_holds_fp64_accuracy_for_blocks_in_any_units(scale):
    """The paper's operators come from PDE solves in physical units (Sec. 3, Sec. 5), so their
    entries may sit anywhere in FP64's range.  Float pairs have FP32's exponent range (a pair
    near 1e-30 would lose its low part to underflow; products near 1e30 overflow), so the
    double-FP32 tier stores F-hat divided by a power of two that puts its largest entry in
    [1/2, 1) and multiplies the outputs back, exactly.  Blocks scaled by 1e-20, 1e-30 and 1e+30
    keep the FP64 tolerance on the CUDA cores and through the digit planes."""
    p = synthetic.small("df64_units", 20, 30, 7, 24, Nq=2)
    F = p.blocks_F() * scale
    m, d = p.vectors_m(16), p.vectors_d(16)
    for path, (od, om, nb) in _df64_products_both_paths(F, m, d).items():
        check(relb(od, oracle.p2o_apply(F, m[:nb])), 1e-12, path)
        check(relb(om, oracle.p2o_apply_adjoint(F, d[:nb])), 1e-12, path)


def test_double_fp32_tier_rows_spanning_twelve_decades():
    """Rows whose entries span twelve decades (row 1: 10^(-12 j / (N_m - 1)) along j) and a
    whole row 1e-12 below the others (row 4).  The digit planes keep a 47-bit image of each row
    of their operand relative to the row's (or column's) largest entry, so the smallest
    entries keep only a few bits; normwise, the error stays at the FP64 level."""
    p = synthetic.small("df64_rows", 20, 30, 7, 24, Nq=2)
    F = p.blocks_F()
    F[:, 1, :] *= 10.0 ** (-12.0 * np.arange(p.Nm) / (p.Nm - 1))
    F[:, 4, :] *= 1e-12
    m, d = p.vectors_m(16), p.vectors_d(16)
    for path, (od, om, nb) in _df64_products_both_paths(F, m, d).items():
        check(relb(od, oracle.p2o_apply(F, m[:nb])), 1e-12, path)
        check(relb(om, oracle.p2o_apply_adjoint(F, d[:nb])), 1e-12, path)


def test_double_fp32_tier_refuses_non_finite_blocks():
    p = synthetic.small("df64_nan", 4, 4, 3, 8)
    F = p.blocks_F()
    F[3, 1, 5] = np.inf
    h = bti.Handle(p.Nm, p.Nd, 0, p.Nt)
    with pytest.raises(bti.BtiError) as e:
        h.set_blocks(bti.OP_F, cuda(F), bti.DF64)
    assert e.value.status == 1 and "non-finite" in e.value.message
    h.set_blocks(bti.OP_F, cuda(p.blocks_F()), bti.DF64)  # the handle stays usable
    h.close()


FACTOR_CASES = [
    # (name, gx, gy, Nd, Nt, panel): n = N_d N_t over several panels; ragged last panels and
    # trailing matrices ragged against the 128-row tiles, or exact multiples of them
    ("n770_panel128", 6, 6, 11, 70, 128),    # 6 panels + 2 columns; trailing 642, 514, ..., 2
    ("n720_panel64", 6, 6, 24, 30, 64),      # 11 panels + 16 columns; K = 64: half a digit chunk
    ("n640_panel128_exact", 8, 8, 10, 64, 128),  # trailing 512, 384, 256, 128 rows: whole tiles
    ("n1200_panel512", 8, 8, 12, 100, 512),  # two panels and a ragged third
    ("n1200_recursive", 8, 8, 12, 100, 1 << 20),  # one panel: the whole factor by recursive halves
]


@pytest.mark.parametrize("name,gx,gy,Nd,Nt,panel", FACTOR_CASES, ids=[c[0] for c in FACTOR_CASES])
def test_tensor_core_cholesky_matches_oracle(name, gx, gy, Nd, Nt, panel):
    """bti_factor_K under BTI_P_DF64 with tensor cores on: panels of `panel` columns, each
    factored by recursive halves, whose updates A22 -= L21 L21^T (inside the panel and of the
    trailing matrix) run in exact digit planes on tcgen05 (lower-trapezoid tiles only,
    subtracted in place).  L against the oracle's factor, and m_map through the blocked solves
    that use its diagonal-block inverses, at the solve bound 10 kappa(K) 2^-47 (reading R20;
    noise variance 1 gives kappa(K) of a few thousand, as in the batched workload)."""
    p = synthetic.small(name, gx, gy, Nd, Nt, Nq=3, sigma2=1.0)
    F, Fq = p.blocks_F(), p.blocks_Fq()
    G = oracle.prior_blocks(F, oracle.se_covariance(gx, gy, 2.0, 1.0))
    h = make_handle(F, Fq, bti.DF64)
    h.set_prior_se_grid(gx, gy, 2.0, 1.0, bti.DF64)
    h.set_noise(p.sigma2)
    h.set_dense_precision(bti.DF64)
    h.set_factor_panel(panel)
    h.build_K()
    h.factor_K()
    L_gpu = host(h.copy_K())
    d = p.vectors_d(3)
    m = torch.empty((3, Nt, gx * gy), dtype=torch.float64, device="cuda")
    h.infer_map(cuda(d), m, refine_iters=0)
    h.close()
    c = oracle_K(name, F, G, p.sigma2, Fq)
    low = np.tril_indices(Nd * Nt)
    tol = parity.tol_solve(c.kappa, parity.U_DIGITS)
    check(rel(L_gpu[low], c.L[low]), tol, f"L, panel {panel}; kappa(K) = {c.kappa:.0f}")
    b = solve_bounds(c, d, parity.U_DIGITS)
    check(relb(host(m), b.m), b.tol_m, "m_map, blocked solves; " + b.info)


def test_tensor_core_cholesky_reports_pivot_and_timeout():
    """Failure handling of the tensor-core factorisation and inverse, injected on the host: a
    negative noise variance past the first panel gives BTI_ERR_NOT_SPD with its pivot; a
    withheld TMA stage (test hook) makes the digit-plane products' bounded waits run out, and
    factor_K, then invert_K, return BTI_ERR_TIMEOUT; the same handle then builds, factors and
    inverts K correctly."""
    name, gx, gy, Nd, Nt = "chol_tc_fail", 6, 6, 10, 40
    p = synthetic.small(name, gx, gy, Nd, Nt, Nq=3, sigma2=1.0)
    F = p.blocks_F()
    G = oracle.prior_blocks(F, oracle.se_covariance(gx, gy, 2.0, 1.0))
    var = np.full((Nt, Nd), 1.0)
    var[30, 3] = -1e4  # data index 303 (third panel of 128) -> pivot 304 (1-based)
    h = make_handle(F, None, bti.DF64)
    h.set_prior_se_grid(gx, gy, 2.0, 1.0, bti.DF64)
    h.set_dense_precision(bti.DF64)
    h.set_factor_panel(128)
    h.set_noise(0.0, cuda(var))
    h.build_K()
    with pytest.raises(bti.BtiError) as e:
        h.factor_K()
    assert e.value.status == 6
    assert "pivot 304" in e.value.message, e.value.message
    h.set_noise(p.sigma2)
    h.build_K()
    h.test_withhold_tc_stage(1)
    with pytest.raises(bti.BtiError) as e:
        h.factor_K()
    assert e.value.status == 7  # BTI_ERR_TIMEOUT
    h.test_withhold_tc_stage(-1)
    h.build_K()
    h.factor_K()
    L_gpu = host(h.copy_K())
    h.test_withhold_tc_stage(1)
    with pytest.raises(bti.BtiError) as e:
        h.invert_K()
    assert e.value.status == 7
    h.test_withhold_tc_stage(-1)
    h.invert_K()
    d = p.vectors_d(2)
    m = torch.empty((2, Nt, gx * gy), dtype=torch.float64, device="cuda")
    h.infer_map(cuda(d), m)
    h.close()
    c = oracle_K(name, F, G, p.sigma2)
    low = np.tril_indices(Nd * Nt)
    check(rel(L_gpu[low], c.L[low]), parity.tol_solve(c.kappa, parity.U_DIGITS),
          f"L after a timeout; kappa(K) = {c.kappa:.0f}")
    b = solve_bounds(c, d, parity.U_DIGITS, kind="inverse")
    check(relb(host(m), b.m), b.tol_m, "m_map, explicit inverse after a timeout; " + b.info)
