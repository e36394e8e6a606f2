/*
 * bti.h -- C ABI of libbti, a single-GPU (NVIDIA GB300, sm_103a) implementation
 * of the data-parallel hot path of goal-oriented real-time Bayesian inversion
 * for linear autonomous dynamical systems (Henneking, Venkat, Ghattas,
 * arXiv 2501.14911).
 *
 * Problem (Sec. 2): the parameter-to-observable map F and the parameter-to-QoI
 * map F_q are block lower-triangular Toeplitz in time (Eq. (2.5), Eq. (2.16)):
 * block (t, s) of F is F_{t-s} (t >= s), with F_0 the diagonal block.  With a
 * time-invariant prior Gamma_prior = I_t (x) C_s and diagonal noise
 * Gamma_noise, the library forms G^* = Gamma_prior F^T (Sec. 4, Phase 2),
 * K = Gamma_noise + F G^* and its Cholesky factor, and computes the MAP point
 * m_map = G^* K^{-1} d_obs (Eq. (4.13) with zero prior mean, simplified using
 * K - F G^* = Gamma_noise) and the QoI prediction q_map = F_q m_map (Eq. (4.2)).
 *
 * Conventions for every call:
 *  - Indices are 0-based.  A parameter vector is m[b][t][j] (b < B, t < N_t,
 *    j < N_m), a data vector d[b][t][i] (i < N_d), a QoI vector q[b][t][l]
 *    (l < N_q); all dense row-major.  The data-space index of (t, i) is
 *    t * N_d + i, so K is (N_t N_d) x (N_t N_d).
 *  - Every pointer argument is a DEVICE pointer on the handle's device unless
 *    stated otherwise.  The caller owns all pointers it passes; the library
 *    copies what it keeps (set_blocks copies) and owns every buffer it
 *    allocates, freeing them in bti_destroy.
 *  - Calls are asynchronous on the handle's CUDA stream (the stream passed to
 *    bti_create, which the caller may change with bti_set_stream).  Argument,
 *    shape and call-order errors are detected on the host and returned at once;
 *    nothing is launched in that case.  Device-side failures (a non-positive
 *    pivot in the Cholesky factorisation) are recorded in a device status word
 *    and returned by bti_sync, and by bti_factor_K, which synchronises.
 *  - A handle must not be used from two host threads at the same time.
 *  - bti_last_error returns a message for the last non-OK status (valid until
 *    the next call on the handle).
 */
#ifndef BTI_H
#define BTI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bti_ctx* bti_handle;

typedef enum {
  BTI_OK = 0,
  BTI_ERR_ARG = 1,      /* null pointer, negative or unsupported size or enum */
  BTI_ERR_SHAPE = 2,    /* sizes inconsistent with the handle */
  BTI_ERR_STATE = 3,    /* call order violated (e.g. apply before set_blocks) */
  BTI_ERR_CUDA = 4,     /* a CUDA runtime call failed */
  BTI_ERR_OOM = 5,      /* device allocation failed */
  BTI_ERR_NOT_SPD = 6,  /* Cholesky met a non-positive or non-finite pivot */
  BTI_ERR_TIMEOUT = 7,  /* a bounded device wait gave up (reported by bti_sync) */
  BTI_ERR_NO_CONVERGENCE = 8  /* an iterative solve missed its tolerance within its iteration limit */
} bti_status;

/* Which block-Toeplitz operator a call refers to.
 * BTI_OP_F : p2o map F, blocks F_k (N_d x N_m), Eq. (2.5).
 * BTI_OP_G : blocks G_k = F_k C_s of G^* = Gamma_prior F^T (Sec. 4, Phase 2).
 * BTI_OP_FQ: p2q map F_q, blocks (N_q x N_m), Eq. (2.15)-(2.16). */
typedef enum { BTI_OP_F = 0, BTI_OP_G = 1, BTI_OP_FQ = 2 } bti_op;

/* Storage / arithmetic tier of the spectral blocks, and (F64, F32 only) vector precision.
 * BTI_P_F64 : spectral blocks complex FP64, FFTs and products FP64.
 * BTI_P_F32 : spectral blocks complex FP32, FFTs and products FP32 (so blocks
 *             and vectors within FP32's range, about 1e-30 .. 1e30 in magnitude).
 * BTI_P_DF64: spectral blocks as pairs of FP32 (hi + lo, about 48 significant
 *             bits; 16 bytes per complex like FP64), products in double-FP32
 *             arithmetic on the FP32 pipes with error-free accumulation; the
 *             FFTs in float pairs as well; input and output vectors FP64.
 *             FP64-level accuracy (well inside 1e-12) at the HBM rate, where
 *             GB300's FP64 pipe would bind first.  Valid as a storage tier
 *             only, not as an io type.  Range: float pairs have FP32's exponent
 *             range, so the spectral blocks are stored divided by the power of
 *             two that puts their largest entry in [1/2, 1), and every output
 *             is multiplied back (both exact): operators in any units within
 *             FP64's range keep the FP64-level accuracy.  Input vectors must
 *             have their entries within about 2^-90 .. 2^90 (1e-27 .. 1e27) of
 *             one: below that their low parts underflow, above it the float-pair
 *             sums can overflow.  set_blocks returns BTI_ERR_ARG for blocks
 *             holding a non-finite value.
 * BTI_P_F16 : spectral blocks as FP16 complex pairs (4 bytes per complex) with one
 *             power-of-two FP32 scale per frequency row; products with FP32
 *             accumulation, FFTs and vectors FP32.  About 1e-3 relative: the
 *             low-precision operator of mixed-precision solves.  Storage tier only.
 */
typedef enum { BTI_P_F64 = 0, BTI_P_F32 = 1, BTI_P_DF64 = 2, BTI_P_F16 = 3 } bti_prec;

/* Create a handle for N_m spatial parameters, N_d sensors, N_q QoI points and
 * N_t time steps on CUDA device `device`, issuing work on `cuda_stream`
 * (a cudaStream_t, or NULL for the legacy default stream).  N_q may be 0 when
 * no QoI map is used.  The circulant embedding length is L = 2 N_t (any
 * L >= 2 N_t - 1 is exact, Sec. 4 "FFT-based ... matvecs"); L must factor into
 * 2, 3, 5 and 7 and be at most 2048 (N_t <= 1024).  Returns BTI_ERR_ARG for sizes <= 0 or an
 * unsupported L. */
bti_status bti_create(int64_t Nm, int64_t Nd, int64_t Nq, int64_t Nt, int device,
                      void* cuda_stream, bti_handle* out);

/* Free every device buffer of the handle (synchronises its stream first). */
bti_status bti_destroy(bti_handle h);

/* Replace the stream subsequent calls are issued on. */
bti_status bti_set_stream(bti_handle h, void* cuda_stream);

/* Store operator `op` from its time-domain blocks and precompute its spectral
 * blocks once (Sec. 4: "the DFT only needs to be done once for each matrix").
 * blocks: device, FP64, [N_t][R][N_m] row-major, R = N_d for F and G, N_q for
 * FQ; block k is F_k.  The spectral blocks hat_F_w = sum_k F_k e^{-2 pi i k w / L}
 * (w = 0..N_t) are kept in `store` precision, layout [N_t+1][R][N_m] complex.
 * The caller's buffer is read during the call's stream work only.  Calling
 * again replaces the operator and releases its digit planes (bti_set_digit_planes).
 * It invalidates Q and Gamma_post(q) (rebuild with bti_build_Q), and for OP_F / OP_G
 * also K with its factor and inverse.  Replacing OP_F also releases a G that
 * bti_set_prior_* formed from the old F; calls that need G return BTI_ERR_STATE
 * until the prior is set again. */
bti_status bti_set_blocks(bti_handle h, bti_op op, const double* blocks, bti_prec store);

/* Build the G operator from the stored F time-domain blocks and a squared-
 * exponential spatial prior on a gx x gy grid (gx * gy = N_m, node index
 * j = ix * gy + iy, unit cell spacing):
 *   C_s[a, b] = sigma^2 exp(-|x_a - x_b|^2 / (2 ell^2)),   G_k = F_k C_s.
 * Requires a prior bti_set_blocks(BTI_OP_F, ...); G is stored in `store`
 * precision.  The separable structure C_s = C_x (x) C_y is used on the device. */
bti_status bti_set_prior_se_grid(bti_handle h, int gx, int gy, double ell, double sigma,
                                 bti_prec store);

/* The elliptic prior of Eq. (5.1) instead: Gamma_prior = I_t (x) (alpha1 I - alpha2 Delta_h)^{-2}
 * on the gx x gy grid (node index ix * gy + iy), Delta_h the 5-point Laplacian with
 * Neumann boundaries in graph form (the paper's Robin coefficient is not given).  The
 * operator is diagonalised by the orthonormal DCT-II on each axis, so the prior is applied
 * exactly: X -> D_x^T [ (D_x X D_y^T) o W ] D_y with W = (alpha1 + alpha2 (lx + ly))^{-2} and
 * lx_k = 2 - 2 cos(pi k / gx).  G = F Gamma_prior and its spectral blocks (tier `store`)
 * replace any previous prior; everything that uses the prior (K, Q, Gamma_post, the
 * matrix-free solve) then uses this one.  alpha1 > 0, alpha2 >= 0.  Synchronises. */
bti_status bti_set_prior_elliptic_grid(bti_handle h, int gx, int gy, double alpha1, double alpha2,
                                       bti_prec store);

/* Arithmetic of the dense data-space work that follows (the Gram product of
 * bti_build_K, the panel and trailing updates of bti_factor_K, and the block
 * updates of the triangular solves): BTI_P_F64 (default; FP64 FMA) or BTI_P_DF64
 * (float pairs on the FP32 pipes, about 48 significant bits; GB300 issues FP32 at
 * 64x its FP64 rate).  The 64 x 64 diagonal-block factorisations and inverses are
 * FP64 either way.  With BTI_P_DF64 one refinement step (refine_iters = 1)
 * restores the last digits of m_map for ill-conditioned K. */
bti_status bti_set_dense_precision(bti_handle h, bti_prec arith);

/* Gamma_noise: sigma2 * I if `diag` is NULL, otherwise diag (device, FP64,
 * [N_t][N_d] variances, all > 0).  Invalidates K, Q and Gamma_post(q). */
bti_status bti_set_noise(bti_handle h, double sigma2, const double* diag);

/* d = F m for B vectors: m [B][N_t][N_m] -> d [B][N_t][N_d] (Eq. (2.6)),
 * computed as zero-padded FFT along time, per-frequency block product
 * hat_d_w = hat_F_w hat_m_w, inverse FFT truncated to the first N_t steps.
 * `io` is the element type of m and d (BTI_P_F64: double, BTI_P_F32: float);
 * the arithmetic follows the stored tier of F.  m and d must not overlap. */
bti_status bti_apply_F(bti_handle h, const void* m, void* d, int64_t B, bti_prec io);

/* m = F^T d (the exact transpose of bti_apply_F) using the conjugate-transposed
 * spectral blocks (Sec. 4): d [B][N_t][N_d] -> m [B][N_t][N_m]. */
bti_status bti_apply_FT(bti_handle h, const void* d, void* m, int64_t B, bti_prec io);

/* q = F_q m (Eq. (2.15)): m [B][N_t][N_m] -> q [B][N_t^q][N_q] (N_t^q = N_t unless
 * bti_set_qoi_stride). */
bti_status bti_apply_Fq(bti_handle h, const void* m, void* q, int64_t B, bti_prec io);

/* m = G^* d = Gamma_prior F^T d using the G spectral blocks:
 * d [B][N_t][N_d] -> m [B][N_t][N_m]. */
bti_status bti_apply_Gstar(bti_handle h, const void* d, void* m, int64_t B, bti_prec io);

/* Assemble K = Gamma_noise + F G^* on the device (Sec. 4, Phase 2), lower
 * triangle only (the strict upper triangle is left undefined), stored in FP64.
 * The Gram product W = F_stack G_stack^T that holds the work runs in the dense
 * arithmetic of bti_set_dense_precision: FP64 FMA by default; under BTI_P_DF64
 * float pairs (about 48 significant bits), or, with tensor cores also on, exact
 * FP16 digit planes on tcgen05 (a 47-bit image of each row); the block-diagonal
 * prefix sums and the noise are FP64 either way.
 * Requires F and G (either tier; the FP64 time-domain blocks kept by
 * set_blocks are used) and set_noise.  col_block (> 0) is the column-panel
 * width of the assembly; 512 is the default when 0 is passed. */
bti_status bti_build_K(bti_handle h, int64_t col_block);

/* As bti_build_K, with the Gram product that assembles K computed in `assembly`
 * precision: BTI_P_F64 (same as bti_build_K) or BTI_P_F32 (FP32 products and
 * accumulation over N_m, about 1e-6 relative; K itself, its block-diagonal
 * accumulation and the noise stay FP64).  The FP32 form is the low-precision half
 * of a mixed-precision solve: factor it with bti_factor_K and call bti_infer_map
 * with refine_iters > 0 and FP64-level (BTI_P_DF64 or BTI_P_F64) F and G operators,
 * which recovers FP64-level m_map when kappa(K) times the assembly error is well
 * below one. */
bti_status bti_build_K_prec(bti_handle h, int64_t col_block, bti_prec assembly);

/* Cholesky-factor K = L L^T in place (lower triangle, stored in FP64; Sec. 4,
 * Phase 2).  The 64 x 64 diagonal-block factorisations are FP64; the panel and
 * trailing updates run in the arithmetic of bti_set_dense_precision: FP64 FMA by
 * default; float pairs (about 48 significant bits) under BTI_P_DF64 with tensor
 * cores off; under BTI_P_DF64 with tensor cores on (bti_set_tensor_cores, the
 * default) and N_d N_t > 64, blocked by panels of the width of
 * bti_set_factor_panel, each factored recursively by halves, with every update
 * A22 -= L21 L21^T (within the panels and of the trailing matrix) on tcgen05 in
 * exact FP16 digit planes of L21's rows (a 47-bit image of each row); the solves
 * of the 64-row panels below each diagonal block stay in float pairs.  Synchronises;
 * returns BTI_ERR_NOT_SPD (message names the 1-based pivot) if a pivot is <= 0 or
 * not finite, and BTI_ERR_TIMEOUT if a bounded wait of the tensor-core update gave
 * up (K is then no longer valid: build it again). */
bti_status bti_factor_K(bti_handle h);

/* Panel width of the tensor-core form of bti_factor_K: a positive multiple of 64 (at
 * most 2^30), or 0 for the default (4096).  It sets the contraction length of the
 * trailing updates and the depth of the recursion inside each panel (a width of at
 * least N_d N_t factors K by recursive halves alone); the flop count does not depend
 * on it.  The planes take 12 ceil128(N_d N_t) ceil128(min(width, N_d N_t)) bytes
 * during the call. */
bti_status bti_set_factor_panel(bti_handle h, int64_t width);

/* Copy the (N_t N_d) x (N_t N_d) row-major K buffer to dst (device, double):
 * its lower triangle holds K after bti_build_K and the Cholesky factor L after
 * bti_factor_K; the strict upper triangle is undefined.  Requires build_K. */
bti_status bti_copy_K(bti_handle h, double* dst);

/* Explicit inverse of K for the online phase (Sec. 4, Phase 4: the triangular solves
 * of Eq. (4.13) moved offline).  enable = 1, after bti_factor_K: forms K^{-1} by
 * solving with the factor against the identity (double-FP32 GEMMs, 2 n^3 flops for
 * n = N_t N_d) and keeps it on the device as float pairs (hi, lo), 8 n^2 bytes.
 * bti_infer_map and bti_online then apply K^{-1} as one dense product instead of the n / 64
 * sequential blocked solves: for B >= 16 vectors with tensor cores on, as exact FP16
 * digit-plane MMAs on tcgen05 (K^{-1} formed as W^T W with W = L^{-1}, the product on the
 * tensor cores too); otherwise in double-FP32 arithmetic (about 48 significant bits), for a
 * single vector by a symmetric product that reads K^{-1}'s lower triangle only.  The inverse belongs to the factor it was formed from: after a new
 * bti_factor_K the solves return to the factor until this is called again.
 * enable = 0 releases the inverse.  Requires factor_K for enable = 1 (BTI_ERR_STATE);
 * BTI_ERR_OOM if the 16 n^2-byte peak (inverse plus FP64 temporary) does not fit.
 * Synchronises. */
bti_status bti_invert_K(bti_handle h, int enable);

/* m_map = G^* K^{-1} d_obs for B observation vectors (Eq. (4.13), zero prior
 * mean): d_obs [B][N_t][N_d] (double) -> m_map [B][N_t][N_m] (double).
 * K^{-1} is applied by the two triangular solves with the factor (or, after
 * bti_invert_K, by one product with the explicit inverse); with
 * refine_iters > 0 that many steps of iterative refinement x += K^{-1}(d - K x)
 * follow, the residual evaluated with the FP64 spectral operators.
 * Requires factor_K. */
bti_status bti_infer_map(bti_handle h, const double* d_obs, double* m_map, int64_t B,
                         int refine_iters);

/* The online phase of Sec. 4, Phase 4 as one CUDA graph launch: m_map = G^* K^{-1}
 * d_obs (with refine_iters refinement steps, as bti_infer_map) followed, when q_map
 * is not NULL, by q_map = F_q m_map (as bti_predict_qoi), for B observation
 * vectors.  The first call for a given (d_obs, m_map, q_map, B, refine_iters,
 * stream) captures every launch of that sequence into a CUDA graph on the handle's
 * stream, which must not be the legacy default stream (BTI_ERR_STATE otherwise);
 * later calls with the same arguments replay it with a single graph launch.  The
 * graph is rebuilt automatically after the operators, the noise or K change.  The
 * buffers' contents may change between calls; their addresses may not (a new
 * address triggers a new capture).  Kernel launches inside the graph are not
 * counted or timed by bti_profile_read. */
bti_status bti_online(bti_handle h, const double* d_obs, double* m_map, double* q_map, int64_t B,
                      int refine_iters);

/* QoI time grid (Sec. 2, the Remark on separate time discretisations): keep every
 * stride-th step of the QoI, q_k at fine step stride (k + 1) - 1, k < N_t^q = N_t /
 * stride (stride must divide N_t; 1 restores the full grid).  Affects the QoI vectors
 * of bti_apply_Fq, bti_predict_qoi, bti_online and bti_apply_Q, which become
 * [B][N_t^q][N_q], and the rows of Q and Gamma_post(q) (bti_build_Q, rebuild after
 * a change), which then hold N_q N_t^q rows. */
bti_status bti_set_qoi_stride(bti_handle h, int stride);

/* out = Gamma_prior v with the SE prior of bti_set_prior_se_grid applied to each
 * time block (Gamma_prior = I_t (x) C_s): v, out [B][N_t][N_m] device doubles, not
 * aliased.  Synchronises. */
bti_status bti_apply_prior(bti_handle h, const double* v, double* out, int64_t B);

/* Action of the parameter posterior covariance, Eq. (4.7):
 * out = Gamma_post(m) v = (I - G^* K^{-1} F) Gamma_prior v, for B vectors
 * [B][N_t][N_m] (device doubles, not aliased).  Columns of Gamma_post(m) and its
 * pointwise variances (Sec. 4, Phase 2) follow from unit vectors.  Requires the SE
 * prior and factor_K; synchronises. */
bti_status bti_apply_postcov(bti_handle h, const double* v, double* out, int64_t B);

/* Probe estimate of the pointwise posterior variances, diag(Gamma_post(m)) (Sec. 4, Phase 2):
 * diag[e] = sum_s V[s][e] (Gamma_post(m) V[s])[e] / sum_s V[s][e]^2 over S caller-drawn probe
 * vectors V [S][N_t][N_m] (device doubles; e.g. random signs), 0 where no probe touches an
 * entry; diag [N_t][N_m] (device double, not aliased with V).  The actions run in batches of
 * up to 64 probes (bti_apply_postcov, so the explicit inverse and digit planes apply when
 * set).  Exact for the unit vectors and for Hadamard sign vectors.  Requires the prior and
 * factor_K; synchronises. */
bti_status bti_postcov_diag_probe(bti_handle h, const double* V, int64_t S, double* diag);

/* m_map with a nonzero prior mean, Eq. (4.13) with the term of Eq. (4.8):
 * m_map = G^* K^{-1} d_obs + (I - G^* K^{-1} F) m_prior
 *       = m_prior + G^* K^{-1} (d_obs - F m_prior).
 * d_obs [B][N_t][N_d], m_prior and m_map [B][N_t][N_m] (device doubles; m_prior and
 * m_map not aliased).  refine_iters as bti_infer_map.  Synchronises. */
bti_status bti_infer_map_prior(bti_handle h, const double* d_obs, const double* m_prior, double* m_map, int64_t B,
                               int refine_iters);

/* Exact tensor-core products for the double-FP32 tier (enable = 1; 0 releases).  Forms,
 * once, digit planes of op's spectral blocks: each F-hat_w[i][j] (re and im) as six FP16
 * planes of balanced base-256 digits with a power-of-two scale per (w, j) for the adjoint and
 * per (w, i) for the forward product, a 47-bit fixed-point image (about 24 n_f N_m (2R
 * rounded up to 128) bytes in all: 5 GB for the batched workload's G, 1.9 GB for its F_q).
 * Calls with B >= 16 vectors and tensor cores on then run the per-frequency products of
 * Sec. 4 as tcgen05 FP16 MMAs whose FP32 sums are exact: adjoint-type calls (bti_apply_FT,
 * bti_apply_Gstar, G^* inside infer_map and online) and forward-type calls (bti_apply_F,
 * bti_apply_Fq, predict_qoi, F_q inside online).  Results match the double-FP32 CUDA-core
 * kernels to FP64 level.  Requires the operator set in BTI_P_DF64 (BTI_ERR_STATE); new
 * blocks or a new prior drop the planes.  Synchronises. */
bti_status bti_set_digit_planes(bti_handle h, bti_op op, int enable);

/* Tensor-core products (on = 1, the default): with FP16 spectral blocks and B >= 8
 * vectors per call (N_m a multiple of 4), the forward products F, F_q run as tcgen05
 * FP16 GEMMs with FP32 accumulation; the vectors' spectra are rounded to FP16 with a
 * power-of-two scale per vector and chunk (about 1e-3 relative in total, like the
 * tier).  on = 0 keeps the CUDA-core FP16 kernels for every B.  A bounded wait that
 * gives up inside the tensor-core kernel is reported by bti_sync as BTI_ERR_TIMEOUT. */
bti_status bti_set_tensor_cores(bti_handle h, int on);

/* Failure-handling test hook: while stage >= 0, the tensor-core kernels that stream an
 * operand by TMA (the FP16 tier's forward product, and the digit-plane products of
 * bti_set_digit_planes, bti_invert_K and bti_set_online_qoi) withhold the stage-th tile load
 * (counting from 0; a 32-column box of all digit planes in the digit-plane kernels) in every
 * CTA that issues that many, so their bounded waits (about a second) run out; the kernel then
 * stops, drains what it issued, frees its tensor memory and sets the device status word
 * that bti_sync reports as BTI_ERR_TIMEOUT.  The handle and the CUDA context stay usable.
 * -1 (the default) turns it off. */
bti_status bti_test_withhold_tc_stage(bti_handle h, int stage);

/* ---------------------------------------------------------------- matrix-free solve
 * When K = Gamma_noise + F G^* is too large to form (N_d N_t = 252,000 makes it
 * 508 GB in FP64), K x = d_obs is solved by conjugate gradients with K applied as
 * Gamma_noise x + F (G^* x) through the spectral operators, and m_map = G^* x
 * (Eq. (4.13) with the simplification m_map = G^* K^{-1} d_obs, Sec. 4).  K is
 * symmetric positive definite (Gamma_noise > 0), so CG applies. */

/* A second, lower-tier copy of the spectral blocks of F or G (from the FP64
 * time-domain blocks kept by set_blocks / set_prior_se_grid), used by the inner
 * iteration of bti_solve_matfree with refine = 1.  store: any tier (BTI_P_F16 or
 * BTI_P_F32 in practice).  A later set_blocks of F or set_prior_se_grid drops the
 * copy.  Synchronises. */
bti_status bti_set_shadow(bti_handle h, bti_op op, bti_prec store);

/* Block-Jacobi preconditioner for bti_solve_matfree (kind = 1; 0 removes it): the inverses
 * of K's N_t time-diagonal blocks K(t,t) = Gamma_noise(t) + sum_{k <= t} F_k G_k^T
 * (N_d x N_d each, N_t N_d^2 doubles), from the time-domain blocks of F and G (Gram
 * blocks in double-FP32 arithmetic, Cholesky and inverse per block).  Every CG
 * iteration of the matrix-free solve (the FP64 one and the FP32 inner one) is then
 * preconditioned.  Requires F, G (set_prior_se_grid) and set_noise; a later change of
 * any of them drops it.  Returns BTI_ERR_NOT_SPD if a block fails to factor.
 * Synchronises. */
bti_status bti_set_matfree_precond(bti_handle h, int kind);

typedef struct {
  int outer_iters;     /* refinement steps or flexible-CG iterations (0 for refine = 0) */
  int inner_iters;     /* conjugate-gradient iterations in total */
  double rel_residual; /* max over the batch of ||d - K x|| / ||d|| with the FP64-accurate operators */
} bti_solve_info;

/* m_map = G^* K^{-1} d_obs for B observation vectors without forming K.
 * d_obs [B][N_t][N_d] -> m_map [B][N_t][N_m] (device doubles); x_out (device, may be
 * NULL) receives x = K^{-1} d_obs [B][N_t][N_d].
 * The FP64-accurate operator is K x = Gamma_noise x + F (G^* x) with F stored in
 * BTI_P_F64 or BTI_P_DF64 and G^* from the G store when that is also FP64-accurate,
 * else Gamma_prior F^T with the SE prior applied separably in FP64.
 *   refine = 0: conjugate gradients in FP64 with that operator until
 *     ||d - K x|| <= tol ||d|| for every vector (at most max_inner iterations).
 * For refine = 0 and 2 the returned residual is recomputed from x, not the recursive one.
 *   refine = 1: FP64 iterative refinement (at most max_outer steps): the residual
 *     r = d - K x with the FP64-accurate operator, then K~ delta = r / ||r|| by FP32
 *     conjugate gradients with the inner operator K~ (the shadow copies of F and G
 *     where set, else their stores) until the inner residual drops by inner_tol (or
 *     max_inner iterations), and x += ||r|| delta.  Each step gains about
 *     -log10(kappa(K) ||K - K~|| / ||K|| + inner_tol) digits.
 *   refine = 2: the same inner solve as the preconditioner of flexible conjugate
 *     gradients in FP64 with the FP64-accurate operator (at most max_outer outer
 *     iterations; beta in the Polak-Ribiere form, which tolerates the inner solve's
 *     variation).  The Krylov outer iteration keeps converging where plain
 *     refinement stalls on kappa(K) ||K - K~|| / ||K||, so a loose inner_tol
 *     (0.1 - 0.3) suffices.
 * Requires F, the SE prior (set_prior_se_grid, which also sets G) and set_noise.
 * Returns BTI_ERR_NO_CONVERGENCE (m_map and x_out still written from the last
 * iterate) when the tolerance is not reached; info (may be NULL) is filled in every
 * case.  Synchronises. */
bti_status bti_solve_matfree(bti_handle h, const double* d_obs, double* m_map, double* x_out, int64_t B,
                             int refine, double tol, int max_outer, int max_inner, double inner_tol,
                             bti_solve_info* info);

/* Elliptic prior operator of Eq. (5.1), per time block: out = A_s m with
 * A_s = alpha1 I - alpha2 Delta_h on the gx x gy grid (gx * gy = N_m, node
 * ix * gy + iy, unit spacing), Delta_h the 5-point Laplacian with homogeneous
 * Neumann boundaries in graph form (the paper's Robin coefficient is not given).
 * Eq. (5.1) takes A_s^{-2} as the prior covariance, so 0.5 ||A_s m_t||^2 summed over
 * t is the prior term of the negative log-posterior and A_s^2 m its gradient.
 * m, out: device, double, [B][N_t][N_m], not aliased.  squared != 0 returns A_s^2 m
 * (A_s is symmetric); that form allocates and frees one temporary and synchronises. */
bti_status bti_apply_elliptic(bti_handle h, int gx, int gy, double alpha1, double alpha2, const double* m,
                              double* out, int64_t B, int squared);

/* Precompute the data-to-QoI map Q of Eq. (4.11) (zero prior mean), and with
 * with_covariance != 0 also the QoI posterior covariance Gamma_post(q) of Eq. (4.10)
 * (Sec. 4, Phase 3).  Since F G^* = K - Gamma_noise, Eq. (4.11) reduces to
 * Q = F_q G^* K^{-1}: the block-Toeplitz product F_q G^* is a Gram product of the
 * stacked time-domain blocks with block-diagonal prefix sums, and its rows are solved
 * with the Cholesky factor.  Gamma_post(q) = F_q Gamma_prior F_q^T - Q (F_q G^*)^T,
 * with the stored SE prior applied to F_q.  Q is (N_q N_t) x (N_d N_t), the
 * covariance (N_q N_t)^2, both FP64 and owned by the handle (arithmetic per
 * bti_set_dense_precision).  Requires factor_K, F_q and G; synchronises when the
 * covariance is built. */
bti_status bti_build_Q(bti_handle h, int with_covariance);

/* q_map = Q d_obs (Eq. (4.14) with zero prior mean) for B observation vectors:
 * d_obs [B][N_t][N_d] -> q_map [B][N_t][N_q], device doubles.  Requires build_Q. */
bti_status bti_apply_Q(bti_handle h, const double* d_obs, double* q_map, int64_t B);

/* Copy Q (row-major [N_q N_t][N_d N_t]) and/or Gamma_post(q) ([N_q N_t]^2) to device
 * buffers; either pointer may be NULL. */
bti_status bti_copy_Q(bti_handle h, double* Q_out, double* cov_out);

/* Precision of the online phase that bti_online captures (Sec. 4, Phase 4), for latency
 * targets looser than FP64.  BTI_P_DF64 (the default): FP64-level m_map and q_map, the same
 * arithmetic as bti_infer_map and bti_predict_qoi / bti_apply_Q.  BTI_P_F32: for B >= 16
 * vectors with tensor cores on, the digit-plane products (bti_invert_K, bti_set_digit_planes,
 * bti_set_online_qoi) use only the most significant of the six planes of each operand: five
 * for K^{-1} (a 39-bit image, error about kappa(K) 2^-38 relative to ||K^{-1} d||) and four
 * for G^*, F_q and Q (31 bits, about 2^-30 of each output's row scale); the transforms keep
 * FP64 level.  m_map and q_map then stay within about 1e-8 of the FP64 result (relative,
 * 2-norm) for kappa(K) up to about 1e4; fewer vectors, and the other entry points, keep FP64
 * level.  refine_iters must be 0 under BTI_P_F32 (BTI_ERR_ARG from bti_online).  Any other
 * prec: BTI_ERR_ARG.  A change drops the captured online graph. */
bti_status bti_set_online_precision(bti_handle h, bti_prec prec);

/* How bti_online gives q_map.  via_Q = 1: q_map = Q d_obs with the d2q map of bti_build_Q
 * (Eq. (4.14), the paper's online QoI prediction; requires build_Q, BTI_ERR_STATE
 * otherwise), and Q is also formed as six FP16 digit planes (12 (N_q N_t^q rounded up to
 * 128)(N_t N_d rounded up to 128) bytes), so that bti_apply_Q and the online graph apply
 * it on the tensor cores with FP64-level accuracy for B >= 16 while tensor cores are on.  via_Q = 0
 * (the default): q_map = F_q m_map (push-forward, as bti_predict_qoi); the planes are
 * released.  via_Q = 1 also keeps Q as float pairs (8 (N_q N_t^q) (N_t N_d) bytes), which
 * bti_apply_Q and the online graph read for one or two vectors per call (a matrix-vector
 * product at the HBM rate, double-FP32 arithmetic).  A later bti_build_Q makes the planes
 * and pairs stale: apply_Q falls back to the dense GEMM until this is called again.
 * Synchronises. */
bti_status bti_set_online_qoi(bti_handle h, int via_Q);

/* q_map = F_q m_map (Eq. (4.2)): m_map [B][N_t][N_m] -> q_map [B][N_t][N_q],
 * both double.  Requires FQ. */
bti_status bti_predict_qoi(bti_handle h, const double* m_map, double* q_map, int64_t B);

/* Project autotuner: time candidate launch shapes of the hot kernels for operator
 * `op` with B vectors per call, on this handle's stored operator and device, and
 * keep the fastest for every later call of the same storage tier: column pairs per
 * FFT CTA, columns per CTA of the forward product, columns per thread of the
 * single-vector adjoint product (coordinate search, median of 3 timed runs).
 * Uses zeroed stand-in vectors it allocates and frees itself; synchronises.
 * report (host, may be NULL) receives a JSON summary of the timings and choices,
 * truncated to report_len - 1 bytes. */
bti_status bti_autotune(bti_handle h, bti_op op, int64_t B, char* report, int64_t report_len);

/* Kernel classes for bti_profile_read. */
typedef enum {
  BTI_K_RFFT = 0,      /* forward zero-padded FFT of input columns (and spectral blocks) */
  BTI_K_PROD_FWD = 1,  /* per-frequency product hat_F hat_m (reduction over N_m) */
  BTI_K_REDUCE = 2,    /* fixed-order sum of the forward product's chunk partials */
  BTI_K_IRFFT = 3,     /* inverse FFT with truncation to N_t steps */
  BTI_K_PROD_ADJ = 4,  /* per-frequency product hat_F^H hat_d */
  BTI_K_DENSE = 5,     /* dense FP64 work: K assembly, Cholesky, triangular solves */
  BTI_K_NCLASS = 6
} bti_kclass;

/* Measurement hook.  Every kernel launch of the handle is counted per class
 * (library kernels only; device-to-device copies are not counted).  While
 * enabled (enable != 0), the library also records a CUDA event pair on its
 * stream around each launch of the first five classes (up to 4096 pairs
 * between reads; later launches are counted but not timed).  bti_profile_read
 * synchronises the stream and writes, per class, the summed device
 * milliseconds (ms[BTI_K_NCLASS], may be NULL) and the launch count
 * (launches[BTI_K_NCLASS], may be NULL) since the previous read, then resets
 * both.  *timed_all (may be NULL) is set to 1 if every counted launch of the
 * timed classes was timed.  Host pointers. */
bti_status bti_profile_enable(bti_handle h, int enable);
bti_status bti_profile_read(bti_handle h, double* ms, int64_t* launches, int* timed_all);

/* Wait for the handle's stream and return any device-side error status. */
bti_status bti_sync(bti_handle h);

/* Message for the last non-OK status on this handle ("" if none). */
const char* bti_last_error(bti_handle h);

/* Size of the device scratch array used by bti_apply_F_noalloc (64 MiB). */
#define BTI_NOALLOC_SCRATCH_BYTES (64ull << 20)

/* d = F m (FP64) without allocating any device memory.  The paper has no
 * counterpart: this entry point exists for callers that may not call
 * cudaMalloc / cudaFree -- code whose device memory belongs to another
 * allocator (a framework's pool or a budget fixed at start-up), and online
 * callers with latency deadlines, for which cudaFree's device-wide
 * synchronisation and cudaMalloc's unbounded cost are unacceptable.
 *
 * No handle: blocks (device, FP64, [N_t][N_d][N_m], block k = F_k), m (device,
 * FP64, [B][N_t][N_m]) and d (device, FP64, [B][N_t][N_d]) are the caller's;
 * the work is queued on cuda_stream (a cudaStream_t, or NULL).  The spectral
 * blocks are recomputed on every call.  All intermediates live in one static
 * device array of BTI_NOALLOC_SCRATCH_BYTES that the library holds on every
 * GPU where it is loaded until the process exits; a problem needing more
 * (about 16 (N_t+1) N_m (N_d + B) bytes plus small terms) returns
 * BTI_ERR_SHAPE before anything is launched.  The first call on a device
 * resolves that array's device address (cudaGetSymbolAddress, with the device
 * current) and keeps it with the current context; a later call in another
 * context on that device (after cudaDeviceReset, or under a caller's own
 * context) resolves it again, since each context holds its own copy of the
 * array.  Make the first call in each context before any stream capture.  Every call on a
 * device shares the array, so calls that overlap on the GPU (other streams or
 * host threads) race and must be serialised by the caller.  Returns BTI_ERR_ARG
 * for null pointers, sizes <= 0 or an unsupported L = 2 N_t, BTI_ERR_CUDA if a
 * launch fails. */
bti_status bti_apply_F_noalloc(const double* blocks, const double* m, double* d, int64_t Nm,
                               int64_t Nd, int64_t Nt, int64_t B, void* cuda_stream);

/* Library version string. */
const char* bti_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BTI_H */
