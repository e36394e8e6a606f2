"""bti_apply_F_noalloc against the handle-based bti_apply_F, through the C ABI.

The no-allocation entry point serves callers that may not call cudaMalloc or
cudaFree (device memory owned by another allocator, or online code with
latency deadlines).  It keeps every intermediate in a fixed static device
array, so this test checks that two calls in a row (different sizes and data,
so the second reuses scratch the first left behind) both agree with the
regular entry point to the FP64 tolerance of the other parity tests, that a
ragged case matches the oracle's direct time-domain convolution, that a call
after a warm first one leaves the device's free memory and torch's reserved
memory unchanged (it allocates nothing), and that an oversized problem is
refused before anything runs.  The file is named to be collected last and
passes alone in a fresh process as well.
"""

import ctypes

import numpy as np
import pytest

import oracle
from paper_2501_14911_gb300 import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2501_14911_gb300 as bti  # noqa: E402

TOL = 1e-12  # FP64 tier tolerance used by the parity tests


def relb(a, b):
    a = a.reshape(a.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    return float(torch.max(torch.linalg.norm(a - b, dim=1) / torch.linalg.norm(b, dim=1)))


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def run_both(name, gx, gy, Nd, Nt, B):
    p = synthetic.small(name, gx, gy, Nd, Nt)
    F = dev(p.blocks_F())
    m = dev(p.vectors_m(B))
    h = bti.Handle(p.Nm, Nd, 0, Nt)
    h.set_blocks(bti.OP_F, F)
    d_ref = torch.empty((B, Nt, Nd), dtype=torch.float64, device="cuda")
    h.apply_F(m, d_ref)
    d_new = torch.full((B, Nt, Nd), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    st = bti.lib().bti_apply_F_noalloc(F.data_ptr(), m.data_ptr(), d_new.data_ptr(), p.Nm, Nd, Nt, B,
                                       ctypes.c_void_p(stream))
    torch.cuda.synchronize()
    h.close()
    assert st == 0
    return relb(d_new, d_ref)


def test_noalloc_matches_apply_F_on_two_calls_in_a_row():
    # first call: ragged sizes (N_m not a multiple of the chunk, odd N_d, L = 90)
    assert run_both("noalloc_a", 30, 100, 13, 45, 3) < TOL
    # second call: other sizes and data; scratch still holds the first call's values
    assert run_both("noalloc_b", 16, 16, 8, 64, 5) < TOL


def test_noalloc_matches_oracle_and_allocates_nothing():
    """A ragged case (N_m = 3,000, N_d = 13, L = 90, 3 vectors) against the oracle's direct
    convolution sums, called twice: the second call, after a warm first one, must leave
    cudaMemGetInfo's free bytes and torch's reserved bytes exactly as they were."""
    p = synthetic.small("noalloc_oracle", 30, 100, 13, 45)
    B = 3
    F_h, m_h = p.blocks_F(), p.vectors_m(B)
    F, m = dev(F_h), dev(m_h)
    d1 = torch.full((B, p.Nt, p.Nd), float("nan"), dtype=torch.float64, device="cuda")
    d2 = torch.full_like(d1, float("nan"))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    L = bti.lib()
    assert L.bti_apply_F_noalloc(F.data_ptr(), m.data_ptr(), d1.data_ptr(), p.Nm, p.Nd, p.Nt, B, stream) == 0
    torch.cuda.synchronize()
    free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
    assert L.bti_apply_F_noalloc(F.data_ptr(), m.data_ptr(), d2.data_ptr(), p.Nm, p.Nd, p.Nt, B, stream) == 0
    torch.cuda.synchronize()
    free1, reserved1 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
    assert (free1, reserved1) == (free0, reserved0)
    ref = torch.as_tensor(oracle.p2o_apply(F_h, m_h), device="cuda")
    assert relb(d1, ref) < TOL
    assert relb(d2, ref) < TOL


def test_noalloc_rejects_oversized_problems_before_launching():
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    L = bti.lib()
    # 256 x 65536 x (128 + 1) complex FP64 far exceeds the static scratch
    st = L.bti_apply_F_noalloc(x.data_ptr(), x.data_ptr(), x.data_ptr(), 65536, 128, 256, 1, None)
    assert st == 2  # BTI_ERR_SHAPE
    assert L.bti_apply_F_noalloc(None, x.data_ptr(), x.data_ptr(), 16, 2, 8, 1, None) == 1
    assert L.bti_apply_F_noalloc(x.data_ptr(), x.data_ptr(), x.data_ptr(), 16, 2, 11, 1, None) == 1  # L = 22
