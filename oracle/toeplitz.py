"""Time-domain block lower-triangular Toeplitz operators (oracle, FP64).

Test infrastructure only; see the package docstring.
"""

import numpy as np


def p2o_apply(blocks, m):
    """d = F m by the convolution sum of Eq. (2.3)/(2.5).

    Eq. (2.3) gives d_{k+1} = sum_{i=0}^{k} B A^i C m_{k-i}; with F_i := B A^i C
    and 0-based data blocks this is d[t] = sum_{k=0}^{t} F_k m[t-k], i.e. block
    (t, s) of F is F_{t-s} for t >= s and zero above the diagonal (Eq. (2.5)).

    blocks: [N_t][R][N_m] float64; m: [..., N_t, N_m].  Returns [..., N_t, R].
    The sum over k runs in increasing k; for each k every output block t >= k
    receives F_k m[t-k] (one matmul per k).
    """
    blocks = np.asarray(blocks, dtype=np.float64)
    m = np.asarray(m, dtype=np.float64)
    Nt, R, Nm = blocks.shape
    if m.shape[-2:] != (Nt, Nm):
        raise ValueError(f"m has shape {m.shape}, expected [..., {Nt}, {Nm}]")
    d = np.zeros(m.shape[:-2] + (Nt, R), dtype=np.float64)
    for k in range(Nt):
        # d[t] += F_k m[t - k] for t = k .. N_t - 1
        d[..., k:, :] += m[..., : Nt - k, :] @ blocks[k].T
    return d


def p2o_apply_adjoint(blocks, d):
    """m = F^T d, the exact transpose of p2o_apply (Eq. (2.5) transposed).

    Block (s, t) of F^T is F_{t-s}^T for t >= s, so m[s] = sum_{t=s}^{N_t-1}
    F_{t-s}^T d[t] = sum_{k=0}^{N_t-1-s} F_k^T d[s+k].  The adjoint in the
    Euclidean inner product is the transpose (the paper's F^* in Eq. (2.12)).

    blocks: [N_t][R][N_m]; d: [..., N_t, R].  Returns [..., N_t, N_m].
    """
    blocks = np.asarray(blocks, dtype=np.float64)
    d = np.asarray(d, dtype=np.float64)
    Nt, R, Nm = blocks.shape
    if d.shape[-2:] != (Nt, R):
        raise ValueError(f"d has shape {d.shape}, expected [..., {Nt}, {R}]")
    m = np.zeros(d.shape[:-2] + (Nt, Nm), dtype=np.float64)
    for k in range(Nt):
        # m[s] += F_k^T d[s + k] for s = 0 .. N_t - 1 - k
        m[..., : Nt - k, :] += d[..., k:, :] @ blocks[k]
    return m


def p2o_dense(blocks):
    """The explicit (R N_t) x (N_m N_t) matrix of Eq. (2.5).

    Row block t, column block s holds F_{t-s} when t >= s and zeros otherwise.
    Only for tiny sizes (brute-force pin).
    """
    blocks = np.asarray(blocks, dtype=np.float64)
    Nt, R, Nm = blocks.shape
    P = np.zeros((Nt * R, Nt * Nm), dtype=np.float64)
    for t in range(Nt):
        for s in range(t + 1):
            P[t * R:(t + 1) * R, s * Nm:(s + 1) * Nm] = blocks[t - s]
    return P


def lti_blocks(A, B, C, Nt):
    """F_k = B A^k C, k = 0 .. N_t - 1 (the block definition after Eq. (2.5))."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    out = np.empty((Nt, B.shape[0], C.shape[1]), dtype=np.float64)
    AkC = C.copy()
    for k in range(Nt):
        out[k] = B @ AkC
        AkC = A @ AkC
    return out


def lti_simulate(A, B, C, m):
    """Run the discrete LTI recursion Eq. (2.2) from w_0 = 0 and observe Eq. (2.3).

    w_{k+1} = A w_k + C m_k, d_{k+1} = B w_{k+1}; returns the data blocks
    d_1 .. d_{N_t} as a 0-based array [N_t][N_d] (row t holds d_{t+1}).
    """
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    m = np.asarray(m, dtype=np.float64)
    Nt = m.shape[0]
    w = np.zeros(A.shape[0], dtype=np.float64)
    d = np.empty((Nt, B.shape[0]), dtype=np.float64)
    for k in range(Nt):
        w = A @ w + C @ m[k]
        d[k] = B @ w
    return d


def p2o_apply_block(blocks, m, t):
    """Output block d[t] = sum_{k=0}^{t} F_k m[t-k] alone (Eq. (2.3)); m: [N_t, N_m].

    For spot checks of large problems, where the whole product is too costly.
    """
    blocks = np.asarray(blocks)
    m = np.asarray(m, dtype=np.float64)
    out = np.zeros(blocks.shape[1], dtype=np.float64)
    for k in range(t + 1):
        out += blocks[k].astype(np.float64) @ m[t - k]
    return out


def p2o_apply_adjoint_block(blocks, d, s):
    """Output block m[s] = sum_{k=0}^{N_t-1-s} F_k^T d[s+k] alone; d: [N_t, R]."""
    blocks = np.asarray(blocks)
    d = np.asarray(d, dtype=np.float64)
    Nt = blocks.shape[0]
    out = np.zeros(blocks.shape[2], dtype=np.float64)
    for k in range(Nt - s):
        out += d[s + k] @ blocks[k].astype(np.float64)
    return out
