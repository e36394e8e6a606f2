"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances are normwise relative errors per right-hand side, the maximum over
the batch: 1e-12 for the FP64 tier, 1e-5 for the FP32 tier (products and FFTs
in FP32), 1e-12 for K, its factor, m_map and q_map at the tiny inversion
(kappa(K) is a few hundred, so FP64 rounding stays far below that bound).
"""

import numpy as np
import pytest

import oracle
from paper_2501_14911_gb300 import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2501_14911_gb300 as bti  # noqa: E402

TOL = {bti.F64: 1e-12, bti.F32: 1e-5, bti.DF64: 1e-12, bti.F16: 1e-3}


def relb(a, b):
    """max over the leading batch axis of ||a_b - b_b|| / ||b_b||."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    a = a.reshape(a.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    num = np.linalg.norm(a - b, axis=1)
    den = np.maximum(np.linalg.norm(b, axis=1), 1e-300)
    return float(np.max(num / den))


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
    assert relb(host(out_d), oracle.p2o_apply(F, m_in)) < tol
    assert relb(host(out_m), oracle.p2o_apply_adjoint(F, d_in)) < tol
    assert relb(host(out_q), oracle.p2o_apply(Fq, m_in)) < tol
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
    assert relb(host(d), oracle.p2o_apply(F, host(m_g))) < 1e-5


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
        assert relb(host(od), oracle.p2o_apply(F, host(m_g))) < TOL[store], B
        assert relb(host(om), oracle.p2o_apply_adjoint(F, host(d_g))) < TOL[store], B
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
        assert relb(out[tc][0], ref_d) < 1e-3, tc
        assert relb(out[tc][1], ref_m) < 1e-3, tc
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
    assert relb(host(mg), oracle.p2o_apply_adjoint(G, dv)) < 1e-12
    h.set_noise(p.sigma2)
    h.build_K()
    K_gpu = host(h.copy_K())
    K_or = oracle.assemble_K(F, G, p.sigma2)
    low = np.tril_indices(K_or.shape[0])
    assert np.linalg.norm(K_gpu[low] - K_or[low]) / np.linalg.norm(K_or[low]) < 1e-12
    h.factor_K()
    L_gpu = host(h.copy_K())
    L_or = oracle.cholesky_lower(K_or)
    assert np.linalg.norm(L_gpu[low] - L_or[low]) / np.linalg.norm(L_or[low]) < 1e-12
    m_map = torch.empty((1, p.Nt, p.Nm), dtype=torch.float64, device="cuda")
    h.infer_map(cuda(d_obs), m_map)
    q_map = torch.empty((1, p.Nt, p.Nq), dtype=torch.float64, device="cuda")
    h.predict_qoi(m_map, q_map)
    m_or = oracle.map_point(F, G, p.sigma2, d_obs)
    assert relb(host(m_map), m_or) < 1e-12
    assert relb(host(q_map), oracle.qoi_map(Fq, m_or)) < 1e-12
    # iterative refinement keeps the answer (and is exercised)
    m_ref = torch.empty_like(m_map)
    h.infer_map(cuda(d_obs), m_ref, refine_iters=2)
    assert relb(host(m_ref), m_or) < 1e-12


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
    assert relb(host(m_map), oracle.map_point(F, G, var, d_obs)) < 1e-11


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
    assert relb(host(m.grad), g_or[None]) < 1e-12
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
        assert relb(host(m), m_or) < 1e-12
        assert relb(host(q), oracle.qoi_map(Fq, m_or)) < 1e-12
        d.mul_(-0.5)  # same buffers, new contents: the graph is replayed
        h.online(d, m, q)
        assert relb(host(m), -0.5 * m_or) < 1e-12
        assert relb(host(q), oracle.qoi_map(Fq, -0.5 * m_or)) < 1e-12
        m2 = torch.empty_like(m)
        h.online(d, m2, None, refine_iters=1)  # other arguments: a new capture
        assert relb(host(m2), -0.5 * m_or) < 1e-12
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
    assert relb(host(od), oracle.p2o_apply(F, host(mg))) < TOL[store]
    assert relb(host(om), oracle.p2o_apply_adjoint(F, host(dg))) < TOL[store]
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
    assert relb(host(m), m_or) < 1e-12
    assert relb(host(q), oracle.qoi_map(Fq, m_or)) < 1e-12
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
    assert np.linalg.norm(K_gpu[low] - K_or[low]) / np.linalg.norm(K_or[low]) < 1e-12
    h.factor_K()
    L_gpu = host(h.copy_K())
    L_or = oracle.cholesky_lower(K_or)
    assert np.linalg.norm(L_gpu[low] - L_or[low]) / np.linalg.norm(L_or[low]) < 1e-11
    m = torch.empty((1, p.Nt, p.Nm), dtype=torch.float64, device="cuda")
    q = torch.empty((1, p.Nt, p.Nq), dtype=torch.float64, device="cuda")
    h.infer_map(cuda(d_obs), m, refine_iters=1)
    h.predict_qoi(m, q)
    m_or = oracle.map_point(F, G, p.sigma2, d_obs)
    assert relb(host(m), m_or) < 1e-12
    assert relb(host(q), oracle.qoi_map(Fq, m_or)) < 1e-12
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
    assert relb(host(out), ref) < 1e-14
    h.apply_elliptic(p.gx, p.gy, 1.3, 0.7, cuda(m), out, squared=True)
    ref2 = (A @ (A @ m.reshape(-1, p.Nm).T)).T.reshape(m.shape)
    assert relb(host(out), ref2) < 1e-14
    # full loss with the prior term, alpha1 = alpha2 = 1 (reading R13)
    A1 = oracle.elliptic_operator(p.gx, p.gy, 1.0, 1.0)
    d = p.vectors_d(1)
    s2 = 0.05
    mg = cuda(m[:1]).requires_grad_(True)
    loss = bti.map_loss(h, mg, cuda(d), s2, p.gx, p.gy)
    loss.backward()
    g_or = oracle.loss_gradient(F, m[0], d[0], s2, A1)
    assert relb(host(mg.grad), g_or[None]) < 1e-12
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
    tol = 1e-12 if dense == "f64" else 1e-11
    assert np.linalg.norm(host(Q) - Q_or) / np.linalg.norm(Q_or) < tol
    assert np.linalg.norm(host(C) - C_or) / np.linalg.norm(C_or) < 1e-10
    d = cuda(np.concatenate([d_obs, p.vectors_d(2)]))
    q = torch.empty((3, p.Nt, p.Nq), dtype=torch.float64, device="cuda")
    h.apply_Q(d, q)
    q_or = oracle.qoi_map(Fq, oracle.map_point(F, G, p.sigma2, host(d)))
    assert relb(host(q), q_or) < tol
    h.close()


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
    assert np.linalg.norm(host(Q) - Q_or) / np.linalg.norm(Q_or) < 1e-10
    assert np.linalg.norm(host(C) - C_or) / np.linalg.norm(C_or) < 1e-9
    h.close()


@pytest.mark.parametrize("B", [3, 70], ids=["b3", "b70"])
def test_online_qoi_via_d2q_map_on_tensor_cores(B):
    """bti_set_online_qoi: q_map = Q d_obs (Eq. (4.14)) with Q in FP16 digit planes on the
    tensor cores for B >= 16 (the stream-K product of the explicit inverse, rectangular here:
    N_q N_t = 256 rows against N_d N_t = 512 columns), in bti_apply_Q and in the online graph;
    the dense GEMM for fewer vectors and with tensor cores off; errors for a missing Q."""
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
    q = torch.empty((B, p.Nt, p.Nq), dtype=torch.float64, device="cuda")
    h.profile_enable(True)
    h.profile_read()
    h.apply_Q(cuda(d), q)
    n_tc = h.profile_read()[0]["dense"][1]
    if B >= 16:
        assert n_tc == 4 * ((B + 63) // 64)  # per 64 vectors: their planes (2 kernels), MMAs, sum
    else:
        assert n_tc == 1  # fewer than 16 vectors: one dense GEMM (memory-bound)
    assert relb(host(q), q_or) < 1e-10
    h.set_tensor_cores(False)
    q2 = torch.empty_like(q)
    h.apply_Q(cuda(d), q2)
    assert h.profile_read()[0]["dense"][1] == 1
    h.set_tensor_cores(True)
    assert relb(host(q), host(q2)) < 1e-10
    h.profile_enable(False)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        h.set_stream(stream)
        m = torch.empty((B, p.Nt, p.Nm), dtype=torch.float64, device="cuda")
        q3 = torch.empty_like(q)
        h.online(cuda(d), m, q3, refine_iters=1)
        assert relb(host(m), m_or) < 1e-12
        assert relb(host(q3), q_or) < 1e-10
        # a new Q (here the same map rebuilt, in a new buffer) is picked up by the online graph
        h.build_Q()
        h.online(cuda(d), m, q3, refine_iters=1)
        assert relb(host(q3), q_or) < 1e-10
        h.set_online_qoi(False)
        h.online(cuda(d), m, q3, refine_iters=1)  # back to the push-forward F_q m_map
        assert relb(host(q3), q_or) < 1e-12
    torch.cuda.synchronize()
    h.set_stream(torch.cuda.current_stream())
    h.close()


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
    assert relb(host(out_d), oracle.p2o_apply(F, m)) < 1e-12

    def state_error(fn, *args):
        with pytest.raises(bti.BtiError) as e:
            fn(*args)
        assert e.value.status == 3

    h.set_blocks(bti.OP_F, cuda(F2), bti.DF64)
    h.apply_F(cuda(m), out_d)
    assert relb(host(out_d), oracle.p2o_apply(F2, m)) < 1e-12
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
    assert relb(host(out_d), oracle.p2o_apply(F2, m)) < 1e-12
    Cs = oracle.se_covariance(p.gx, p.gy, p.ell, p.sigma_p)
    G2 = oracle.prior_blocks(F2, Cs)
    h.build_K()
    h.factor_K()
    h.build_Q()
    h.apply_Q(cuda(d), out_q)
    q_or = (d.reshape(B, -1) @ oracle.d2q_map(Fq, F2, G2, p.sigma2).T).reshape(B, p.Nt, p.Nq)
    assert relb(host(out_q), q_or) < 1e-10

    h.set_blocks(bti.OP_FQ, cuda(Fq2), bti.DF64)
    state_error(h.apply_Q, cuda(d), out_q)
    h.apply_Fq(cuda(m), out_q)
    assert relb(host(out_q), oracle.p2o_apply(Fq2, m)) < 1e-12
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
    assert relb(host(out), oracle.prior_apply(Cs, v)) < 1e-13
    h.apply_postcov(cuda(v), out)
    assert relb(host(out), oracle.posterior_cov_apply(F, G, Cs, p.sigma2, v)) < 1e-11
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
    assert relb(host(mm), oracle.map_point_with_prior_mean(F, G, p.sigma2, d_obs, m0)) < 1e-12
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
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-11
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
    assert relb(host(q), oracle.qoi_map(Fq, m)[:, steps]) < 1e-12
    m_or = oracle.map_point(F, G, p.sigma2, d_obs)
    q_or = oracle.qoi_map(Fq, m_or)[:, steps]
    mm = torch.empty((1, p.Nt, p.Nm), dtype=torch.float64, device="cuda")
    q1 = torch.empty((1, Ntq, p.Nq), dtype=torch.float64, device="cuda")
    h.infer_map(cuda(d_obs), mm)
    h.predict_qoi(mm, q1)
    assert relb(host(q1), q_or) < 1e-11
    stream = torch.cuda.Stream()  # graph capture needs a non-default stream
    with torch.cuda.stream(stream):
        h.set_stream(stream)
        q1.zero_()
        h.online(cuda(d_obs), mm, q1)
        assert relb(host(q1), q_or) < 1e-11
    torch.cuda.synchronize()
    h.set_stream(torch.cuda.current_stream())
    h.build_Q(with_covariance=True)
    Q, C = h.copy_Q(covariance=True)
    assert tuple(Q.shape) == (Ntq * p.Nq, p.Nt * p.Nd) and tuple(C.shape) == (Ntq * p.Nq,) * 2
    Cs = oracle.se_covariance(p.gx, p.gy, p.ell, p.sigma_p)
    Q_or = oracle.d2q_map(Fq, F, G, p.sigma2)[rows]
    C_or = oracle.qoi_posterior_covariance(Fq, oracle.prior_blocks(Fq, Cs), F, G, p.sigma2)[np.ix_(rows, rows)]
    assert np.linalg.norm(host(Q) - Q_or) / np.linalg.norm(Q_or) < 1e-11
    assert np.linalg.norm(host(C) - C_or) / np.linalg.norm(C_or) < 1e-10
    q1.zero_()
    h.apply_Q(cuda(d_obs), q1)
    assert relb(host(q1), q_or) < 1e-11
    # back to the full grid: Q must be rebuilt, and F_q writes every step again
    h.set_qoi_stride(1)
    with pytest.raises(bti.BtiError):
        h.apply_Q(cuda(d_obs), torch.empty((1, p.Nt, p.Nq), dtype=torch.float64, device="cuda"))
    qf = torch.empty((2, p.Nt, p.Nq), dtype=torch.float64, device="cuda")
    h.apply_Fq(cuda(m), qf)
    assert relb(host(qf), oracle.qoi_map(Fq, m)) < 1e-12
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
    L = oracle.cholesky_lower(oracle.assemble_K(F, G, p.sigma2))
    x_or = oracle.solve_K(L, d.reshape(3, -1)).reshape(x.shape)
    assert relb(host(x), x_or) < 1e-10, info
    assert relb(host(m), oracle.map_point(F, G, p.sigma2, d, L=L)) < 1e-10, info
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
    assert relb(host(m), oracle.map_point(F, G, p.sigma2, d_obs)) < 1e-10


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
    assert relb(host(d), oracle.p2o_apply(F, host(m))) < 1e-3


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
    h.test_withhold_tc_stage(3)
    run(x, y)
    with pytest.raises(bti.BtiError) as e:
        h.sync()
    assert e.value.status == 7  # BTI_ERR_TIMEOUT
    h.sync()  # reported once
    h.test_withhold_tc_stage(-1)
    run(x, y)
    h.sync()
    assert relb(host(y), ref()) < 1e-12
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
    assert relb(host(out), oracle.prior_apply(Cs, v)) < 1e-12
    d = p.vectors_d(2)
    h.build_K()
    h.factor_K()
    m = torch.empty((2, p.Nt, p.Nm), dtype=torch.float64, device="cuda")
    q = torch.empty((2, p.Nt, p.Nq), dtype=torch.float64, device="cuda")
    h.infer_map(cuda(d), m)
    h.predict_qoi(m, q)
    L = oracle.cholesky_lower(oracle.assemble_K(F, G, p.sigma2))
    m_or = oracle.map_point(F, G, p.sigma2, d, L=L)
    assert relb(host(m), m_or) < 1e-11
    assert relb(host(q), oracle.qoi_map(Fq, m_or)) < 1e-11
    h.apply_postcov(cuda(v), out)
    assert relb(host(out), oracle.posterior_cov_apply(F, G, Cs, p.sigma2, v, L=L)) < 1e-10
    m.zero_()
    h.solve_matfree(cuda(d), m, refine=0, tol=1e-12, max_inner=4000)
    h.close()
    assert relb(host(m), m_or) < 1e-10


@pytest.mark.parametrize("B", [1, 5, 20, 70], ids=["b1", "b5", "b20", "b70"])
def test_explicit_inverse_online_solve(B):
    """bti_invert_K: x = K^{-1} d as one product with the explicit inverse, on the tensor
    cores (six FP16 digit planes, exact per 128-column chunk) and, with tensor cores off,
    in double-FP32 on the CUDA cores (4-, 16- and 64-wide right-hand-side tiles); stream-K
    partials summed in CTA order; a second 64-chunk at B = 70.  m_map matches the oracle,
    refinement brings it to the FP64 tolerance, a new factorisation returns to the
    triangular solves until the inverse is formed again, and release works."""
    p, F, Fq, G, _ = tiny_problem()
    d = p.vectors_d(B)
    m_or = oracle.map_point(F, G, p.sigma2, d)
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
    assert relb(host(m), m_or) < 1e-12
    h.invert_K()
    h.profile_read()  # drop the launches of forming the inverse
    m.zero_()
    h.infer_map(cuda(d), m)
    n_inv = h.profile_read()[0]["dense"][1]
    assert n_inv + 20 < n_trsm  # a few launches per 64 vectors, not 2 n / 64 blocked steps
    assert relb(host(m), m_or) < 1e-10
    # the same product in double-FP32 on the CUDA cores (tensor cores off)
    h.set_tensor_cores(False)
    m_dd = torch.empty_like(m)
    h.infer_map(cuda(d), m_dd)
    h.set_tensor_cores(True)
    assert relb(host(m_dd), m_or) < 1e-10
    assert relb(host(m), host(m_dd)) < 1e-10
    h.infer_map(cuda(d), m, refine_iters=1)
    assert relb(host(m), m_or) < 1e-12
    # the online graph applies the inverse too, and with G's digit planes its G^* (B >= 16)
    # runs on the tensor cores as well
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        h.set_stream(stream)
        q = torch.empty((B, p.Nt, p.Nq), dtype=torch.float64, device="cuda")
        m2 = torch.empty_like(m)
        h.online(cuda(d), m2, q, refine_iters=1)
        assert relb(host(m2), m_or) < 1e-12
        assert relb(host(q), oracle.qoi_map(Fq, m_or)) < 1e-12
        h.set_digit_planes(bti.OP_G, True)
        h.set_digit_planes(bti.OP_FQ, True)
        h.online(cuda(d), m2, q)
        assert relb(host(m2), m_or) < 1e-10
        assert relb(host(q), oracle.qoi_map(Fq, m_or)) < 1e-10
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
    assert relb(host(m), oracle.map_point(F, G, 2.0 * p.sigma2, d)) < 1e-12
    h.invert_K()
    h.infer_map(cuda(d), m)
    assert relb(host(m), oracle.map_point(F, G, 2.0 * p.sigma2, d)) < 1e-10
    h.invert_K(False)
    h.infer_map(cuda(d), m)
    assert relb(host(m), oracle.map_point(F, G, 2.0 * p.sigma2, d)) < 1e-12
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
    assert relb(host(m_map), oracle.map_point(F, G, var, d_obs)) < 1e-11
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
    assert relb(host(out_m), oracle.p2o_apply_adjoint(F, d)) < 1e-12
    assert relb(host(out_d), oracle.p2o_apply(F, m)) < 1e-12
    assert relb(host(out_q), oracle.p2o_apply(Fq, m)) < 1e-12
    h.set_digit_planes(bti.OP_F, False)
    h.set_digit_planes(bti.OP_FQ, False)
    out_m2, out_d2 = torch.empty_like(out_m), torch.empty_like(out_d)
    h.apply_FT(cuda(d), out_m2)
    h.apply_F(cuda(m), out_d2)
    prof = h.profile_read()[0]
    assert prof["prod_adj"][1] == 1 and prof["prod_fwd"][1] == 1
    assert relb(host(out_m), host(out_m2)) < 1e-12
    assert relb(host(out_d), host(out_d2)) < 1e-12
    h.profile_enable(False)
    h.close()


def test_digit_planes_need_the_double_fp32_tier():
    p = synthetic.small("dig_state", 1, 64, 3, 8)
    h = make_handle(p.blocks_F(), None, bti.F64)
    with pytest.raises(bti.BtiError) as e:
        h.set_digit_planes(bti.OP_F, True)
    assert e.value.status == 3
    h.close()
