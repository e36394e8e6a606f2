"""Handle lifetime through the C ABI: bti_destroy returns every byte the handle allocated.

Each cycle takes a handle through the whole offline and online phase on the tensor cores and
then destroys it. The phase covers:
- double-FP32 spectral blocks with digit planes for F, G and F_q;
- K built, factored and inverted (float pairs and digit planes);
- Q and its digit planes;
- the online graph.

After the first cycle, which also loads the library's kernels, the device's free memory must not
drift. Each cycle allocates several hundred MiB, so a leak of any one buffer shows.
"""

import pytest

from paper_2501_14911_gb300 import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2501_14911_gb300 as bti  # noqa: E402


def _free_bytes():
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return torch.cuda.mem_get_info()[0]


def test_destroy_releases_every_buffer():
    p = synthetic.small("lifecycle", 32, 64, 32, 64, Nq=4)  # N_m = 2,048; K is 2,048 x 2,048
    B = 16
    F = torch.as_tensor(p.blocks_F(), device="cuda")
    Fq = torch.as_tensor(p.blocks_Fq(), device="cuda")
    d = torch.as_tensor(p.vectors_d(B), device="cuda")
    m = torch.empty((B, p.Nt, p.Nm), dtype=torch.float64, device="cuda")
    q = torch.empty((B, p.Nt, p.Nq), dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()

    def cycle():
        with torch.cuda.stream(stream):
            h = bti.Handle(p.Nm, p.Nd, p.Nq, p.Nt, stream=stream)
            h.set_blocks(bti.OP_F, F, bti.DF64)
            h.set_blocks(bti.OP_FQ, Fq, bti.DF64)
            h.set_prior_se_grid(p.gx, p.gy, p.ell, p.sigma_p, bti.DF64)
            h.set_noise(p.sigma2)
            h.set_dense_precision(bti.DF64)
            for op in (bti.OP_F, bti.OP_G, bti.OP_FQ):
                h.set_digit_planes(op, True)
            h.build_K()
            h.factor_K()
            h.invert_K()
            h.build_Q()
            h.set_online_qoi(True)
            h.online(d, m, q, refine_iters=1)
            h.close()
        torch.cuda.synchronize()
        assert torch.isfinite(m).all() and torch.isfinite(q).all()

    cycle()
    base = _free_bytes()
    for _ in range(3):
        cycle()
    drift = base - _free_bytes()
    assert drift <= 8 << 20, f"{drift / 2**20:.1f} MiB not returned after three create/destroy cycles"
