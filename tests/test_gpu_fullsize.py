"""Parity at the workloads' full sizes, in the launch configuration the bench times.

- Matvec sweep (N_m = 65,536, N_d = 128, N_t = 256): single-vector F and F^T
  calls on every tier; the oracle computes sampled output blocks one by one.
- Batched online (N_m = 4,096, N_d = 100, N_t = 200, K = 20,000^2, 64
  observation vectors): K (sampled entries and the whole lower triangle), the
  Cholesky factor, m_map and q_map against the oracle's complete inversion, in
  every solve form (FP64, double-FP32, the explicit inverse, refined, with K
  assembled in FP32).
- Differentiation (N_m = 8,192, N_d = 64, N_t = 256): the autograd gradient of
  the data misfit against the oracle gradient.
- The mixed-precision workload's products (N_d = 600, N_t = 420, L = 840) in the
  FP16, FP32 and double-FP32 tiers, its matrix-free m_map at full size (residual
  recomputed by the oracle), and at its first 42 time steps (K 25,200^2) m_map and
  q_map against the oracle's dense solve, for one vector and for 16 at once.

Tolerances follow reading R20 (tests/parity.py): 1e-12 for products, and for results
that pass through a solve with K a bound from kappa(K), which the oracle measures at
the test's size, and the unit roundoff of the arithmetic.  Minutes of host time for
the oracle; GPU only.
"""

import numpy as np
import pytest

import oracle
from paper_2501_14911_gb300 import synthetic
import parity
from parity import check, rel, relb

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

import paper_2501_14911_gb300 as bti  # noqa: E402


@pytest.fixture(scope="module")
def sweep():
    p = synthetic.SWEEP
    return p, p.blocks_F(), p.vectors_m(2), p.vectors_d(2)


@pytest.mark.parametrize("store,tol", [(bti.DF64, 1e-12), (bti.F64, 1e-12), (bti.F32, 1e-5), (bti.F16, 1e-3)],
                         ids=["df64", "f64", "f32", "f16"])
def test_sweep_sampled_outputs(sweep, store, tol):
    p, F, m, d = sweep
    dt = torch.float32 if store in (bti.F32, bti.F16) else torch.float64
    h = bti.Handle(p.Nm, p.Nd, 0, p.Nt)
    Fd = torch.from_numpy(F).cuda()
    h.set_blocks(bti.OP_F, Fd, store)
    torch.cuda.synchronize()
    del Fd
    torch.cuda.empty_cache()
    m_g = torch.from_numpy(m).cuda().to(dt)
    d_g = torch.from_numpy(d).cuda().to(dt)
    outd = torch.empty((2, p.Nt, p.Nd), dtype=dt, device="cuda")
    outm = torch.empty((2, p.Nt, p.Nm), dtype=dt, device="cuda")
    for b in range(2):  # one vector per call, as the bench runs it
        h.apply_F(m_g[b], outd[b])
        h.apply_FT(d_g[b], outm[b])
    torch.cuda.synchronize()
    m_in = m_g.double().cpu().numpy()
    d_in = d_g.double().cpu().numpy()
    od = outd.double().cpu().numpy()
    om = outm.double().cpu().numpy()
    h.close()
    for b in range(2):
        for t in (0, 1, 97, 255):
            check(rel(od[b, t], oracle.p2o_apply_block(F, m_in[b], t)), tol, str((b, t)))
        for s in (0, 128, 255):
            check(rel(om[b, s], oracle.p2o_apply_adjoint_block(F, d_in[b], s)), tol, str((b, s)))


@pytest.fixture(scope="module")
def batched():
    """The batched workload's oracle inversion, computed once for the module: G = F C_s, K and
    its Cholesky factor, kappa(K), and x = K^{-1} d_obs, m_map = G^* x, q_map = F_q m_map for
    the 64 observation vectors, with rho = ||K^{-1}|| ||d_obs|| / ||x|| (max over vectors)."""
    p = synthetic.BATCHED
    o = type("BatchedOracle", (), {})()
    o.p = p
    o.F, o.Fq, o.d_obs = p.blocks_F(), p.blocks_Fq(), p.vectors_d()
    o.G = oracle.prior_blocks(o.F, oracle.se_covariance(p.gx, p.gy, p.ell, p.sigma_p))
    o.K = oracle.assemble_K(o.F, o.G, p.sigma2)
    o.L = oracle.cholesky_lower(o.K)
    o.lmin, o.lmax = parity.spd_extremes(o.K, o.L)
    o.kappa = o.lmax / o.lmin
    B = o.d_obs.shape[0]
    o.x = oracle.solve_K(o.L, o.d_obs.reshape(B, -1)).reshape(o.d_obs.shape)
    o.m = oracle.p2o_apply_adjoint(o.G, o.x)
    o.q = oracle.qoi_map(o.Fq, o.m)
    o.rho = parity.rho_inverse(o.lmin, o.d_obs, o.x)
    return o


def _batched_handle(o):
    p = o.p
    h = bti.Handle(p.Nm, p.Nd, p.Nq, p.Nt)
    h.set_blocks(bti.OP_F, torch.from_numpy(o.F).cuda(), bti.DF64)
    h.set_blocks(bti.OP_FQ, torch.from_numpy(o.Fq).cuda(), bti.DF64)
    h.set_prior_se_grid(p.gx, p.gy, p.ell, p.sigma_p, bti.DF64)
    h.set_noise(p.sigma2)
    return h


def test_batched_inversion_full_size(batched):
    """Plain FP64 dense work (Gram product, Cholesky, triangular solves) with double-FP32
    spectral products: K against its block definition (sampled) and the oracle's (whole
    lower triangle) at 1e-12; the factor, m_map, q_map, q_map = Q d_obs through the FP64
    d2q map and through its digit planes at the FP64 solve bound 10 kappa(K) 2^-53."""
    o = batched
    p = o.p
    h = _batched_handle(o)
    h.build_K(p.col_block)
    K_gpu = h.copy_K().cpu().numpy()
    h.factor_K()
    L_gpu = h.copy_K().cpu().numpy()
    m_map = torch.empty((p.n_vectors, p.Nt, p.Nm), dtype=torch.float64, device="cuda")
    q_map = torch.empty((p.n_vectors, p.Nt, p.Nq), dtype=torch.float64, device="cuda")
    h.infer_map(torch.from_numpy(o.d_obs).cuda(), m_map)
    h.predict_qoi(m_map, q_map)
    m_gpu = m_map.cpu().numpy()
    q_gpu = q_map.cpu().numpy()
    # the d2q map (Eq. (4.11)) and q_map = Q d_obs (Eq. (4.14)) at full size
    h.build_Q()
    q_d2q = torch.empty_like(q_map)
    h.apply_Q(torch.from_numpy(o.d_obs).cuda(), q_d2q)
    q_d2q = q_d2q.cpu().numpy()
    # the same through Q's digit planes on the tensor cores (6,400 x 20,000)
    h.set_online_qoi(True)
    q_tc = torch.empty_like(q_map)
    h.apply_Q(torch.from_numpy(o.d_obs).cuda(), q_tc)
    q_tc = q_tc.cpu().numpy()
    # one vector: the matrix-vector product over Q's float pairs
    q_1 = torch.empty((1, p.Nt, p.Nq), dtype=torch.float64, device="cuda")
    h.apply_Q(torch.from_numpy(o.d_obs[7:8]).cuda(), q_1)
    q_1 = q_1.cpu().numpy()
    h.close()

    # sampled entries of K one by one from the block definition
    rng = np.random.default_rng(0)
    n = p.Nt * p.Nd
    for _ in range(200):
        r, c = sorted(rng.integers(0, n, size=2))[::-1]
        t, i = divmod(int(r), p.Nd)
        tp, ip = divmod(int(c), p.Nd)
        v = sum(float(o.F[t - s, i] @ o.G[tp - s, ip]) for s in range(min(t, tp) + 1))
        if r == c:
            v += p.sigma2
        assert abs(K_gpu[r, c] - v) <= 1e-12 * abs(K_gpu[r, r]), (r, c)
    low = np.tril_indices(n)
    check(rel(K_gpu[low], o.K[low]), 1e-12, "K")
    del K_gpu
    tol = parity.tol_solve(o.kappa, parity.U_F64)
    kinfo = f"kappa(K) = {o.kappa:.0f}"
    check(rel(L_gpu[low], o.L[low]), tol, "L " + kinfo)
    del L_gpu, low
    check(relb(m_gpu, o.m), tol, "m_map " + kinfo)
    check(relb(q_gpu, o.q), tol, "q_map " + kinfo)
    check(relb(q_d2q, o.q), tol, "Q d_obs " + kinfo)
    check(relb(q_tc, o.q), tol, "Q d_obs, digit planes " + kinfo)
    check(relb(q_1, o.q[7:8]), tol, "Q d_obs, one vector, float pairs " + kinfo)


def test_diff_gradient_full_size():
    """The differentiation workload: loss 0.5 ||F m - d||^2 / sigma^2 plus the elliptic
    prior term (reading R13, alpha1 = alpha2 = 1) through autograd, against the oracle
    gradient; the misfit-only gradient as well."""
    p = synthetic.DIFF
    F = p.blocks_F()
    m0 = p.vectors_m(1)
    dobs = p.vectors_d(1)
    h = bti.Handle(p.Nm, p.Nd, 0, p.Nt)
    h.set_blocks(bti.OP_F, torch.from_numpy(F).cuda(), bti.DF64)
    m = torch.from_numpy(m0).cuda().requires_grad_(True)
    r = bti.apply_F_autograd(h, m) - torch.from_numpy(dobs).cuda()
    loss = 0.5 * (r * r).sum() / p.sigma2
    loss.backward()
    g = m.grad.detach().cpu().numpy()
    m2 = torch.from_numpy(m0).cuda().requires_grad_(True)
    full = bti.map_loss(h, m2, torch.from_numpy(dobs).cuda(), p.sigma2, p.gx, p.gy)
    full.backward()
    g_full = m2.grad.detach().cpu().numpy()
    h.close()
    g_or = oracle.loss_gradient(F, m0[0], dobs[0], p.sigma2)
    check(relb(g, g_or[None]), 1e-12)
    A = oracle.elliptic_operator(p.gx, p.gy, 1.0, 1.0)
    g_full_or = oracle.loss_gradient(F, m0[0], dobs[0], p.sigma2, A)
    check(relb(g_full, g_full_or[None]), 1e-12)


def test_batched_double_fp32_dense_without_refinement_full_size(batched):
    """The batched workload with K's Gram product and the Cholesky's trailing updates in
    exact digit planes on the tensor cores (panels of 4,096, each by recursive halves), the panel steps and triangular
    solves in double-FP32 arithmetic, and no refinement step: the online form for the 1e-6
    latency target.  L and the solves are held to the solve bound 10 kappa(K) 2^-47 of the
    digit planes.  The same through the explicit inverse
    of bti_invert_K (K^{-1} = W^T W, W = L^{-1}) in the online graph, with the inverse, G^* and
    F_q products on the tensor cores in exact digit planes: the inverse adds its formation
    error to every product, so it is held to 10 kappa(K) rho 2^-47; one refinement step, its
    residual from the digit-plane products, brings it back to the solve bound 10 kappa(K) 2^-47."""
    o = batched
    p = o.p
    h = _batched_handle(o)
    h.set_dense_precision(bti.DF64)
    h.build_K(p.col_block)
    h.factor_K()
    L_gpu = h.copy_K().cpu().numpy()
    low = np.tril_indices(p.Nt * p.Nd)
    err_L = rel(L_gpu[low], o.L[low])
    del L_gpu, low
    m_map = torch.empty((p.n_vectors, p.Nt, p.Nm), dtype=torch.float64, device="cuda")
    q_map = torch.empty((p.n_vectors, p.Nt, p.Nq), dtype=torch.float64, device="cuda")
    h.infer_map(torch.from_numpy(o.d_obs).cuda(), m_map, refine_iters=0)
    h.predict_qoi(m_map, q_map)
    m_gpu = m_map.cpu().numpy()
    q_gpu = q_map.cpu().numpy()
    # the explicit inverse (bti_invert_K): n = 20,000 gives 157 row tiles of 1,250 k-steps,
    # so stream-K CTAs span two or three row tiles; B = 64 and a 1-vector call
    h.invert_K()
    h.set_digit_planes(bti.OP_G, True)
    h.set_digit_planes(bti.OP_FQ, True)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        h.set_stream(stream)
        h.online(torch.from_numpy(o.d_obs).cuda(), m_map, q_map, refine_iters=0)
        torch.cuda.synchronize()
        m_inv = m_map.cpu().numpy()
        q_inv = q_map.cpu().numpy()
        h.online(torch.from_numpy(o.d_obs).cuda(), m_map, q_map, refine_iters=1)
        torch.cuda.synchronize()
        m_ref = m_map.cpu().numpy()
        q_ref = q_map.cpu().numpy()
    h.set_stream(torch.cuda.current_stream())
    m1 = torch.empty((1, p.Nt, p.Nm), dtype=torch.float64, device="cuda")
    h.infer_map(torch.from_numpy(o.d_obs[5:6]).cuda(), m1, refine_iters=0)
    m1 = m1.cpu().numpy()
    # q_map = Q d_obs (Eq. (4.14)) with Q = X K^{-1} formed by the tile products (the Gram X =
    # F_q G^* and the product with the explicit inverse, both in digit planes) and applied in
    # digit planes in the online graph
    h.build_Q()
    h.set_online_qoi(True)
    with torch.cuda.stream(stream):
        h.set_stream(stream)
        h.online(torch.from_numpy(o.d_obs).cuda(), m_map, q_map, refine_iters=0)
        torch.cuda.synchronize()
        q_Q = q_map.cpu().numpy()
        # the FP32-level online form (bti_set_online_precision): five digit planes for K^{-1},
        # four for G^* and Q; 64 vectors, and one (which takes the FP64-level kernels)
        h.set_online_precision(bti.F32)
        h.online(torch.from_numpy(o.d_obs).cuda(), m_map, q_map, refine_iters=0)
        torch.cuda.synchronize()
        m_32, q_32 = m_map.cpu().numpy(), q_map.cpu().numpy()
        m_1 = torch.empty((1, p.Nt, p.Nm), dtype=torch.float64, device="cuda")
        q_1 = torch.empty((1, p.Nt, p.Nq), dtype=torch.float64, device="cuda")
        h.online(torch.from_numpy(o.d_obs[5:6].copy()).cuda(), m_1, q_1, refine_iters=0)
        torch.cuda.synchronize()
        m_32_1, q_32_1 = m_1.cpu().numpy(), q_1.cpu().numpy()
        h.set_online_precision(bti.DF64)
    h.set_stream(torch.cuda.current_stream())
    h.close()
    kinfo = f"kappa(K) = {o.kappa:.0f}, rho = {o.rho:.1f}"
    tol = parity.tol_solve(o.kappa, parity.U_DIGITS)
    check(err_L, tol, "L, tensor-core trailing updates " + kinfo)
    check(relb(m_gpu, o.m), tol, "m_map, double-FP32 solves " + kinfo)
    check(relb(q_gpu, o.q), tol, "q_map, double-FP32 solves " + kinfo)
    tol = parity.tol_inverse(o.kappa, parity.U_DIGITS, o.rho)
    check(relb(m_inv, o.m), tol, "m_map, explicit inverse " + kinfo)
    check(relb(q_inv, o.q), tol, "q_map, explicit inverse " + kinfo)
    check(relb(m1, o.m[5:6]), tol, "m_map, explicit inverse, one vector " + kinfo)
    check(relb(q_Q, o.q), tol, "q_map = Q d_obs, Q from the explicit inverse " + kinfo)
    # the FP32-level form, against the online latency metric's 1e-6
    check(relb(m_32, o.m), 1e-6, "m_map, FP32-level online form " + kinfo)
    check(relb(q_32, o.q), 1e-6, "q_map, FP32-level online form " + kinfo)
    check(relb(m_32_1, o.m[5:6]), 1e-6, "m_map, FP32-level online form, one vector " + kinfo)
    check(relb(q_32_1, o.q[5:6]), 1e-6, "q_map, FP32-level online form, one vector " + kinfo)
    tol = parity.tol_solve(o.kappa, parity.U_DIGITS)
    check(relb(m_ref, o.m), tol, "m_map, inverse + one refinement step " + kinfo)
    check(relb(q_ref, o.q), tol, "q_map, inverse + one refinement step " + kinfo)


@pytest.mark.parametrize("dense", ["f64", "df64"])
def test_batched_mixed_precision_solve_full_size(batched, dense):
    """The batched workload with K assembled in FP32, Cholesky and solves in FP64 (or
    double-FP32), and four refinement steps whose residuals use double-FP32 operators:
    m_map and q_map at the refinement bound 10 kappa(K) 2^-48."""
    o = batched
    p = o.p
    h = _batched_handle(o)
    if dense == "df64":
        h.set_dense_precision(bti.DF64)
    h.build_K_prec(p.col_block, bti.F32)
    h.factor_K()
    m_map = torch.empty((p.n_vectors, p.Nt, p.Nm), dtype=torch.float64, device="cuda")
    q_map = torch.empty((p.n_vectors, p.Nt, p.Nq), dtype=torch.float64, device="cuda")
    h.infer_map(torch.from_numpy(o.d_obs).cuda(), m_map, refine_iters=4)
    h.predict_qoi(m_map, q_map)
    m_gpu = m_map.cpu().numpy()
    q_gpu = q_map.cpu().numpy()
    h.close()
    tol = parity.tol_solve(o.kappa, parity.U_DF64)
    kinfo = f"kappa(K) = {o.kappa:.0f}"
    check(relb(m_gpu, o.m), tol, "m_map " + kinfo)
    check(relb(q_gpu, o.q), tol, "q_map " + kinfo)


@pytest.fixture(scope="module")
def mixed():
    p = synthetic.MIXED
    return p, p.blocks_F(), p.vectors_m(1), p.vectors_d(1)


@pytest.mark.parametrize("store,tol", [(bti.F16, 1e-3), (bti.F32, 1e-5), (bti.DF64, 1e-12)],
                         ids=["f16", "f32", "df64"])
def test_mixed_workload_products_full_size(mixed, store, tol):
    """The mixed-precision workload's operators (N_m = 16,384, N_d = 600, N_t = 420, so
    L = 840 = 8 * 7 * 5 * 3): F and F^T on one vector per call against the oracle's
    complete products, normwise over the whole vector (the tolerance metric).  The FP16
    tier is that workload's low-precision product tier, the double-FP32 tier its FP64
    refinement operator."""
    p, F, m, d = mixed
    dt = torch.float32 if store in (bti.F32, bti.F16) else torch.float64
    h = bti.Handle(p.Nm, p.Nd, 0, p.Nt)
    Fd = torch.from_numpy(F).cuda()
    h.set_blocks(bti.OP_F, Fd, store)
    torch.cuda.synchronize()
    del Fd
    torch.cuda.empty_cache()
    m_g = torch.from_numpy(m).cuda().to(dt)
    d_g = torch.from_numpy(d).cuda().to(dt)
    od = torch.empty((1, p.Nt, p.Nd), dtype=dt, device="cuda")
    om = torch.empty((1, p.Nt, p.Nm), dtype=dt, device="cuda")
    h.apply_F(m_g, od)
    h.apply_FT(d_g, om)
    torch.cuda.synchronize()
    m_in = m_g.double().cpu().numpy()
    d_in = d_g.double().cpu().numpy()
    od = od.double().cpu().numpy()
    om = om.double().cpu().numpy()
    h.close()
    check(relb(od, oracle.p2o_apply(F, m_in)), tol)
    check(relb(om, oracle.p2o_apply_adjoint(F, d_in)), tol)


def test_mixed_workload_matrix_free_map_full_size(mixed):
    """The mixed-precision workload's m_map at full size, where K (252,000^2, 508 GB in FP64)
    cannot be formed: flexible FP64 conjugate gradients preconditioned by FP32 conjugate
    gradients with FP16 spectral blocks of F and G, to ||d - K x|| <= 1e-10 ||d|| for white
    N(0,1) data.  A convergence check: the oracle recomputes the residual of the returned
    x = K^{-1} d with its direct convolution sums and the SE prior and confirms the solver's
    own (the rounding of the double-FP32 operator lets the two differ by far less than the
    factor 1.5 allowed).  The forward error of m_map against the oracle's solution is checked
    at the workload's first 42 time steps, where the oracle can factor K (below)."""
    p, F, m, d = mixed
    h = bti.Handle(p.Nm, p.Nd, 0, p.Nt)
    Fd = torch.from_numpy(F).cuda()
    h.set_blocks(bti.OP_F, Fd, bti.DF64)
    torch.cuda.synchronize()
    del Fd
    torch.cuda.empty_cache()
    h.set_prior_se_grid(p.gx, p.gy, p.ell, p.sigma_p, bti.F16)
    h.set_shadow(bti.OP_F, bti.F16)
    h.set_noise(p.sigma2)
    mm = torch.empty((1, p.Nt, p.Nm), dtype=torch.float64, device="cuda")
    x = torch.empty((1, p.Nt, p.Nd), dtype=torch.float64, device="cuda")
    info = h.solve_matfree(torch.from_numpy(d).cuda(), mm, x, refine=2, tol=1e-10, max_outer=400,
                           max_inner=2000, inner_tol=0.1)
    h.close()
    x = x.cpu().numpy()[0]
    w = oracle.prior_blocks_separable(oracle.p2o_apply_adjoint(F, x), p.gx, p.gy, p.ell, p.sigma_p)  # G^* x
    r = d[0] - (p.sigma2 * x + oracle.p2o_apply(F, w))
    check(np.linalg.norm(r) / np.linalg.norm(d[0]), 1.5e-10, "oracle residual of the returned x " + str(info))


@pytest.fixture(scope="module")
def mixed42():
    """The mixed-precision workload truncated to its first 42 time steps (synthetic.MIXED_NT42,
    K 25,200^2): 16 observation vectors d = F m_true + sigma noise with m_true drawn from the
    prior (reading R12), the oracle's dense inversion for them, kappa(K) and rho."""
    p = synthetic.MIXED_NT42
    o = type("MixedOracle", (), {})()
    o.p = p
    o.F, o.Fq = p.blocks_F(), p.blocks_Fq()
    m_true = oracle.prior_sample(p.z_true(), p.gx, p.gy, p.ell, p.sigma_p)
    o.d = oracle.p2o_apply(o.F, m_true) + np.sqrt(p.sigma2) * p.noise()
    o.G = oracle.prior_blocks_separable(o.F, p.gx, p.gy, p.ell, p.sigma_p)
    K = oracle.assemble_K(o.F, o.G, p.sigma2)
    L = oracle.cholesky_lower(K)
    o.lmin, o.lmax = parity.spd_extremes(K, L)
    del K
    o.kappa = o.lmax / o.lmin
    B = o.d.shape[0]
    o.x = oracle.solve_K(L, o.d.reshape(B, -1)).reshape(o.d.shape)
    del L
    o.m = oracle.p2o_apply_adjoint(o.G, o.x)
    o.q = oracle.qoi_map(o.Fq, o.m)
    o.rho = parity.rho_inverse(o.lmin, o.d, o.x)
    return o


@pytest.mark.parametrize("B", [1, 16], ids=["one_vector", "16_vectors_tensor_cores"])
def test_mixed_truncated_matrix_free_map_against_oracle(mixed42, B):
    """The matrix-free mixed-precision solve (flexible FP64 CG with the double-FP32 operator,
    preconditioned by FP32 CG on FP16 spectral blocks of F and G, block-Jacobi in both) at the
    mixed workload's first 42 time steps, where the oracle factors K: x = K^{-1} d, m_map and
    q_map against the oracle's dense solve, element by element.  With 16 observation vectors
    per call the inner FP16 products run on the tensor cores (tcgen05, B >= 8): the forward
    chunk sums then launch only from the outer FP64 products, far fewer than the inner
    iterations.  Tolerance: the CG bound of reading R20, rho eta + 10 kappa(K) 2^-48, for x,
    m_map and q_map."""
    o = mixed42
    p = o.p
    h = bti.Handle(p.Nm, p.Nd, p.Nq, p.Nt)
    h.set_blocks(bti.OP_F, torch.from_numpy(o.F).cuda(), bti.DF64)
    h.set_blocks(bti.OP_FQ, torch.from_numpy(o.Fq).cuda(), bti.DF64)
    h.set_prior_se_grid(p.gx, p.gy, p.ell, p.sigma_p, bti.F16)
    h.set_shadow(bti.OP_F, bti.F16)
    h.set_noise(p.sigma2)
    h.set_matfree_precond(1)
    eta = 1e-11
    d = torch.from_numpy(o.d[:B].copy()).cuda()
    mm = torch.empty((B, p.Nt, p.Nm), dtype=torch.float64, device="cuda")
    x = torch.empty((B, p.Nt, p.Nd), dtype=torch.float64, device="cuda")
    q = torch.empty((B, p.Nt, p.Nq), dtype=torch.float64, device="cuda")
    h.profile_enable(True)
    h.profile_read()
    info = h.solve_matfree(d, mm, x, refine=2, tol=eta, max_outer=400, max_inner=2000, inner_tol=0.1)
    prof = h.profile_read()[0]
    h.profile_enable(False)
    h.predict_qoi(mm, q)
    x, mm, q = x.cpu().numpy(), mm.cpu().numpy(), q.cpu().numpy()
    h.close()
    if B >= 8:
        # inner products on the tensor cores: no chunk-sum kernel per inner iteration
        assert prof["reduce"][1] < info["inner_iters"], (prof, info)
    tol = parity.tol_cg(o.kappa, parity.U_DF64, o.rho, eta)
    what = f"kappa(K) = {o.kappa:.0f}, rho = {o.rho:.1f} {info}"
    check(relb(x, o.x[:B]), tol, "x " + what)
    check(relb(mm, o.m[:B]), tol, "m_map " + what)
    check(relb(q, o.q[:B]), tol, "q_map " + what)
