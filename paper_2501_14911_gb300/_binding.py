"""ctypes marshalling for libbti's C ABI (include/bti.h).  No arithmetic here."""

from __future__ import annotations

import ctypes
import os
import re

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
HEADER = os.path.join(ROOT, "include", "bti.h")

OP_F, OP_G, OP_FQ = 0, 1, 2
# kernel classes of bti_profile_read
KCLASSES = ("rfft", "prod_fwd", "reduce", "irfft", "prod_adj", "dense")
F64, F32, DF64, F16 = 0, 1, 2, 3

STATUS = {
    0: "BTI_OK", 1: "BTI_ERR_ARG", 2: "BTI_ERR_SHAPE", 3: "BTI_ERR_STATE", 4: "BTI_ERR_CUDA",
    5: "BTI_ERR_OOM", 6: "BTI_ERR_NOT_SPD", 7: "BTI_ERR_TIMEOUT", 8: "BTI_ERR_NO_CONVERGENCE",
}


class SolveInfo(ctypes.Structure):
    """bti_solve_info: refinement steps, CG iterations, final relative residual."""

    _fields_ = [("outer_iters", ctypes.c_int), ("inner_iters", ctypes.c_int), ("rel_residual", ctypes.c_double)]

    def as_dict(self):
        return {"outer_iters": self.outer_iters, "inner_iters": self.inner_iters, "rel_residual": self.rel_residual}

_lib = None


class BtiError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status
        self.message = message


def lib_path():
    return os.path.join(PKG, "libbti.so")


def header_symbols():
    """Names of every function the public header declares."""
    with open(HEADER) as f:
        text = f.read()
    return sorted(set(re.findall(r"^\s*(?:bti_status|const char\*)\s+(bti_\w+)\s*\(", text, re.M)))


def lib():
    """The loaded libbti (ctypes.CDLL) with argument types set.  Raises if not built."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libbti.so is not built ({path}); run __graft_entry__.build() first")
    L = ctypes.CDLL(path)
    i64, vp, dp, ip = ctypes.c_int64, ctypes.c_void_p, ctypes.c_double, ctypes.c_int
    st = ctypes.c_int
    sig = {
        "bti_create": ([i64, i64, i64, i64, ip, vp, ctypes.POINTER(vp)], st),
        "bti_destroy": ([vp], st),
        "bti_set_stream": ([vp, vp], st),
        "bti_set_blocks": ([vp, ip, vp, ip], st),
        "bti_set_prior_se_grid": ([vp, ip, ip, dp, dp, ip], st),
        "bti_set_prior_elliptic_grid": ([vp, ip, ip, dp, dp, ip], st),
        "bti_set_noise": ([vp, dp, vp], st),
        "bti_set_dense_precision": ([vp, ip], st),
        "bti_apply_F": ([vp, vp, vp, i64, ip], st),
        "bti_apply_FT": ([vp, vp, vp, i64, ip], st),
        "bti_apply_Fq": ([vp, vp, vp, i64, ip], st),
        "bti_apply_Gstar": ([vp, vp, vp, i64, ip], st),
        "bti_build_K": ([vp, i64], st),
        "bti_build_K_prec": ([vp, i64, ip], st),
        "bti_factor_K": ([vp], st),
        "bti_invert_K": ([vp, ip], st),
        "bti_set_online_qoi": ([vp, ip], st),
        "bti_set_online_precision": ([vp, ip], st),
        "bti_set_digit_planes": ([vp, ip, ip], st),
        "bti_copy_K": ([vp, vp], st),
        "bti_infer_map": ([vp, vp, vp, i64, ip], st),
        "bti_predict_qoi": ([vp, vp, vp, i64], st),
        "bti_online": ([vp, vp, vp, vp, i64, ip], st),
        "bti_build_Q": ([vp, ip], st),
        "bti_apply_prior": ([vp, vp, vp, i64], st),
        "bti_set_qoi_stride": ([vp, ip], st),
        "bti_apply_postcov": ([vp, vp, vp, i64], st),
        "bti_postcov_diag_probe": ([vp, vp, i64, vp], st),
        "bti_infer_map_prior": ([vp, vp, vp, vp, i64, ip], st),
        "bti_set_shadow": ([vp, ip, ip], st),
        "bti_set_tensor_cores": ([vp, ip], st),
        "bti_set_factor_panel": ([vp, i64], st),
        "bti_set_matfree_precond": ([vp, ip], st),
        "bti_test_withhold_tc_stage": ([vp, ip], st),
        "bti_solve_matfree": ([vp, vp, vp, vp, i64, ip, dp, ip, ip, dp, ctypes.POINTER(SolveInfo)], st),
        "bti_apply_Q": ([vp, vp, vp, i64], st),
        "bti_copy_Q": ([vp, vp, vp], st),
        "bti_apply_elliptic": ([vp, ip, ip, dp, dp, vp, vp, i64, ip], st),
        "bti_autotune": ([vp, ip, i64, ctypes.c_char_p, i64], st),
        "bti_sync": ([vp], st),
        "bti_profile_enable": ([vp, ip], st),
        "bti_profile_read": ([vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                              ctypes.POINTER(ctypes.c_int)], st),
        "bti_last_error": ([vp], ctypes.c_char_p),
        "bti_version": ([], ctypes.c_char_p),
        "bti_apply_F_noalloc": ([vp, vp, vp, i64, i64, i64, i64, vp], st),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _ptr(x):
    """Device pointer of a torch tensor (or an int address)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


class Handle:
    """One problem instance on one GPU: owns the library handle (bti_create/destroy).

    Methods mirror the C entry points (set_blocks, apply_F, apply_FT, apply_Fq,
    apply_Gstar, build_K, factor_K, infer_map, predict_qoi, sync) and take torch
    CUDA tensors; they check dtype, device, contiguity and shape, pass raw
    pointers, and raise BtiError on a non-OK status.
    """

    def __init__(self, Nm, Nd, Nq, Nt, device=0, stream=None):
        import torch

        self.Nm, self.Nd, self.Nq, self.Nt = int(Nm), int(Nd), int(Nq), int(Nt)
        self.Ntq = self.Nt  # QoI time steps (bti_set_qoi_stride)
        self.device = torch.device("cuda", device) if isinstance(device, int) else torch.device(device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self._stream = stream
        h = ctypes.c_void_p()
        st = lib().bti_create(self.Nm, self.Nd, self.Nq, self.Nt, self.device.index or 0,
                              ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h))
        if st != 0:
            raise BtiError(st, f"bti_create({Nm}, {Nd}, {Nq}, {Nt}) failed")
        self._h = h

    # -- plumbing
    @property
    def raw(self):
        return self._h

    def _check(self, st):
        if st != 0:
            msg = lib().bti_last_error(self._h)
            raise BtiError(st, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().bti_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        self._stream = stream
        self._check(lib().bti_set_stream(self._h, ctypes.c_void_p(stream.cuda_stream)))

    def _tensor(self, x, shape_tail, name, dtypes=None):
        import torch

        if not isinstance(x, torch.Tensor):
            raise TypeError(f"{name} must be a torch tensor")
        if x.device != self.device:
            raise ValueError(f"{name} is on {x.device}, handle is on {self.device}")
        if not x.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        dtypes = dtypes or (torch.float64,)
        if x.dtype not in dtypes:
            raise TypeError(f"{name} has dtype {x.dtype}, expected one of {dtypes}")
        tail = tuple(shape_tail)
        if tuple(x.shape[-len(tail):]) != tail:
            raise ValueError(f"{name} has shape {tuple(x.shape)}, expected [..., {', '.join(map(str, tail))}]")
        return x

    @staticmethod
    def _io(x):
        import torch

        return F64 if x.dtype == torch.float64 else F32

    def _batch(self, x, tail_len):
        n = 1
        for s in x.shape[:-tail_len]:
            n *= int(s)
        return n

    # -- operators
    def set_blocks(self, op, blocks, store=F64):
        R = self.Nq if op == OP_FQ else self.Nd
        self._tensor(blocks, (self.Nt, R, self.Nm), "blocks")
        self._check(lib().bti_set_blocks(self._h, op, _ptr(blocks), store))

    def set_prior_se_grid(self, gx, gy, ell, sigma, store=F64):
        self._check(lib().bti_set_prior_se_grid(self._h, gx, gy, float(ell), float(sigma), store))

    def set_prior_elliptic_grid(self, gx, gy, alpha1=1.0, alpha2=1.0, store=F64):
        """The elliptic prior (alpha1 I - alpha2 Delta_h)^{-2} of Eq. (5.1), applied exactly by DCT."""
        self._check(lib().bti_set_prior_elliptic_grid(self._h, int(gx), int(gy), float(alpha1), float(alpha2),
                                                      int(store)))

    def set_dense_precision(self, arith=F64):
        """Arithmetic of K assembly, Cholesky and solves: F64 (FP64 FMA) or DF64 (float pairs)."""
        self._check(lib().bti_set_dense_precision(self._h, int(arith)))

    def set_noise(self, sigma2, diag=None):
        if diag is not None:
            self._tensor(diag, (self.Nt, self.Nd), "diag")
        self._check(lib().bti_set_noise(self._h, float(sigma2), _ptr(diag)))

    def _apply(self, fn, x, y, tin, tout):
        import torch

        dts = (torch.float64, torch.float32)
        self._tensor(x, tin, "input", dts)
        self._tensor(y, tout, "output", dts)
        if x.dtype != y.dtype:
            raise TypeError("input and output must have the same dtype")
        B = self._batch(x, len(tin))
        if self._batch(y, len(tout)) != B:
            raise ValueError("input and output batch sizes differ")
        self._check(fn(self._h, _ptr(x), _ptr(y), B, self._io(x)))
        return y

    def apply_F(self, m, d):
        return self._apply(lib().bti_apply_F, m, d, (self.Nt, self.Nm), (self.Nt, self.Nd))

    def apply_FT(self, d, m):
        return self._apply(lib().bti_apply_FT, d, m, (self.Nt, self.Nd), (self.Nt, self.Nm))

    def apply_Fq(self, m, q):
        return self._apply(lib().bti_apply_Fq, m, q, (self.Nt, self.Nm), (self.Ntq, self.Nq))

    def set_qoi_stride(self, stride):
        """QoI on every stride-th time step (N_t^q = N_t / stride)."""
        self._check(lib().bti_set_qoi_stride(self._h, int(stride)))
        self.Ntq = self.Nt // int(stride)

    def apply_Gstar(self, d, m):
        return self._apply(lib().bti_apply_Gstar, d, m, (self.Nt, self.Nd), (self.Nt, self.Nm))

    def build_K(self, col_block=512):
        self._check(lib().bti_build_K(self._h, int(col_block)))

    def build_K_prec(self, col_block=512, assembly=F64):
        self._check(lib().bti_build_K_prec(self._h, int(col_block), int(assembly)))

    def factor_K(self):
        self._check(lib().bti_factor_K(self._h))

    def set_digit_planes(self, op, enable=True):
        """Exact tensor-core adjoint products (B >= 16) for a double-FP32 operator."""
        self._check(lib().bti_set_digit_planes(self._h, int(op), int(bool(enable))))

    def set_online_precision(self, prec):
        """online() at FP64 level (DF64, the default) or at FP32 level (F32: the tensor-core
        products on their most significant digit planes only, about 1e-8 relative)."""
        self._check(lib().bti_set_online_precision(self._h, int(prec)))

    def set_online_qoi(self, via_Q=True):
        """online() takes q_map = Q d_obs (needs build_Q; Q on the tensor cores) or F_q m_map."""
        self._check(lib().bti_set_online_qoi(self._h, int(bool(via_Q))))

    def invert_K(self, enable=True):
        """Form K^{-1} from the factor (or release it) so infer_map / online apply it as one product."""
        self._check(lib().bti_invert_K(self._h, int(bool(enable))))

    def copy_K(self, out=None):
        import torch

        n = self.Nt * self.Nd
        if out is None:
            out = torch.empty((n, n), dtype=torch.float64, device=self.device)
        self._tensor(out, (n, n), "out")
        self._check(lib().bti_copy_K(self._h, _ptr(out)))
        return out

    def infer_map(self, d_obs, m_map, refine_iters=0):
        self._tensor(d_obs, (self.Nt, self.Nd), "d_obs")
        self._tensor(m_map, (self.Nt, self.Nm), "m_map")
        B = self._batch(d_obs, 2)
        if self._batch(m_map, 2) != B:
            raise ValueError("d_obs and m_map batch sizes differ")
        self._check(lib().bti_infer_map(self._h, _ptr(d_obs), _ptr(m_map), B, int(refine_iters)))
        return m_map

    def apply_prior(self, v, out):
        """out = Gamma_prior v (the SE prior per time block)."""
        return self._param_op(lib().bti_apply_prior, v, out, "apply_prior")

    def apply_postcov(self, v, out):
        """out = Gamma_post(m) v (Eq. (4.7))."""
        return self._param_op(lib().bti_apply_postcov, v, out, "apply_postcov")

    def postcov_diag_probe(self, V, out):
        """Probe estimate of diag(Gamma_post(m)) from S probe vectors V [S][N_t][N_m] into out [N_t][N_m]."""
        self._check(lib().bti_postcov_diag_probe(self._h, _ptr(V), int(V.shape[0]), _ptr(out)))

    def _param_op(self, fn, v, out, name):
        self._tensor(v, (self.Nt, self.Nm), name + " input")
        self._tensor(out, (self.Nt, self.Nm), name + " output")
        B = self._batch(v, 2)
        if self._batch(out, 2) != B:
            raise ValueError("batch sizes differ")
        self._check(fn(self._h, _ptr(v), _ptr(out), B))
        return out

    def set_tensor_cores(self, on=True):
        """Tensor-core FP16 forward products for B >= 8 vectors (on by default)."""
        self._check(lib().bti_set_tensor_cores(self._h, 1 if on else 0))

    def set_factor_panel(self, width=0):
        """Panel width of the tensor-core Cholesky (a multiple of 64; 0: the default, 4096)."""
        self._check(lib().bti_set_factor_panel(self._h, int(width)))

    def test_withhold_tc_stage(self, stage):
        """Failure-handling test hook: the tensor-core forward withholds one pipeline stage."""
        self._check(lib().bti_test_withhold_tc_stage(self._h, int(stage)))

    def set_matfree_precond(self, kind=1):
        """Block-Jacobi preconditioner (time-diagonal blocks of K) for solve_matfree; 0 removes it."""
        self._check(lib().bti_set_matfree_precond(self._h, int(kind)))

    def set_shadow(self, op, store):
        """A lower-tier copy of F's or G's spectral blocks for the inner solve."""
        self._check(lib().bti_set_shadow(self._h, int(op), int(store)))

    def solve_matfree(self, d_obs, m_map, x=None, refine=1, tol=1e-12, max_outer=20, max_inner=500,
                      inner_tol=1e-3):
        """m_map = G^* K^{-1} d_obs by conjugate gradients without forming K: FP64 CG
        (refine=0), FP64 iterative refinement around FP32 CG with the shadow operators
        (refine=1), or that inner solve preconditioning flexible FP64 CG (refine=2).
        Returns the solve statistics as a dict; raises BtiError (status
        BTI_ERR_NO_CONVERGENCE) when tol is not reached."""
        self._tensor(d_obs, (self.Nt, self.Nd), "d_obs")
        self._tensor(m_map, (self.Nt, self.Nm), "m_map")
        B = self._batch(d_obs, 2)
        if self._batch(m_map, 2) != B:
            raise ValueError("d_obs and m_map batch sizes differ")
        if x is not None:
            self._tensor(x, (self.Nt, self.Nd), "x")
            if self._batch(x, 2) != B:
                raise ValueError("d_obs and x batch sizes differ")
        info = SolveInfo()
        st = lib().bti_solve_matfree(self._h, _ptr(d_obs), _ptr(m_map), _ptr(x) if x is not None else None, B,
                                     int(refine), float(tol), int(max_outer), int(max_inner),
                                     float(inner_tol), ctypes.byref(info))
        self.last_solve = info.as_dict()
        self._check(st)
        return self.last_solve

    def infer_map_prior(self, d_obs, m_prior, m_map, refine_iters=0):
        """m_map with a nonzero prior mean (Eq. (4.13) with Eq. (4.8))."""
        self._tensor(d_obs, (self.Nt, self.Nd), "d_obs")
        self._tensor(m_prior, (self.Nt, self.Nm), "m_prior")
        self._tensor(m_map, (self.Nt, self.Nm), "m_map")
        B = self._batch(d_obs, 2)
        if self._batch(m_prior, 2) != B or self._batch(m_map, 2) != B:
            raise ValueError("batch sizes differ")
        self._check(lib().bti_infer_map_prior(self._h, _ptr(d_obs), _ptr(m_prior), _ptr(m_map), B,
                                              int(refine_iters)))
        return m_map

    def build_Q(self, with_covariance=False):
        """Precompute the d2q map Q (Eq. (4.11)) and optionally Gamma_post(q) (Eq. (4.10))."""
        self._check(lib().bti_build_Q(self._h, 1 if with_covariance else 0))

    def apply_Q(self, d_obs, q_map):
        """q_map = Q d_obs (Eq. (4.14))."""
        self._tensor(d_obs, (self.Nt, self.Nd), "d_obs")
        self._tensor(q_map, (self.Ntq, self.Nq), "q_map")
        B = self._batch(d_obs, 2)
        if self._batch(q_map, 2) != B:
            raise ValueError("d_obs and q_map batch sizes differ")
        self._check(lib().bti_apply_Q(self._h, _ptr(d_obs), _ptr(q_map), B))
        return q_map

    def copy_Q(self, covariance=False):
        """(Q, Gamma_post(q) or None) as new device tensors."""
        import torch

        nq, n = self.Ntq * self.Nq, self.Nt * self.Nd
        Q = torch.empty((nq, n), dtype=torch.float64, device=self.device)
        C = torch.empty((nq, nq), dtype=torch.float64, device=self.device) if covariance else None
        self._check(lib().bti_copy_Q(self._h, _ptr(Q), _ptr(C)))
        return Q, C

    def predict_qoi(self, m_map, q_map):
        self._tensor(m_map, (self.Nt, self.Nm), "m_map")
        self._tensor(q_map, (self.Ntq, self.Nq), "q_map")
        B = self._batch(m_map, 2)
        if self._batch(q_map, 2) != B:
            raise ValueError("m_map and q_map batch sizes differ")
        self._check(lib().bti_predict_qoi(self._h, _ptr(m_map), _ptr(q_map), B))
        return q_map

    def online(self, d_obs, m_map, q_map=None, refine_iters=0):
        """m_map (and q_map) for a batch of observations as one CUDA-graph launch (bti_online)."""
        self._tensor(d_obs, (self.Nt, self.Nd), "d_obs")
        self._tensor(m_map, (self.Nt, self.Nm), "m_map")
        B = self._batch(d_obs, 2)
        if self._batch(m_map, 2) != B:
            raise ValueError("d_obs and m_map batch sizes differ")
        if q_map is not None:
            self._tensor(q_map, (self.Ntq, self.Nq), "q_map")
            if self._batch(q_map, 2) != B:
                raise ValueError("m_map and q_map batch sizes differ")
        self._check(lib().bti_online(self._h, _ptr(d_obs), _ptr(m_map), _ptr(q_map), B, int(refine_iters)))
        return m_map

    def apply_elliptic(self, gx, gy, alpha1, alpha2, m, out, squared=False):
        """out = A_s m (or A_s^2 m) per time block: the elliptic prior operator of Eq. (5.1)."""
        self._tensor(m, (self.Nt, self.Nm), "m")
        self._tensor(out, (self.Nt, self.Nm), "out")
        B = self._batch(m, 2)
        self._check(lib().bti_apply_elliptic(self._h, int(gx), int(gy), float(alpha1), float(alpha2), _ptr(m),
                                             _ptr(out), B, 1 if squared else 0))
        return out

    def autotune(self, op=OP_F, B=1):
        """Pick launch shapes for operator `op` with B vectors per call; returns the timing report."""
        import json

        buf = ctypes.create_string_buffer(4096)
        self._check(lib().bti_autotune(self._h, int(op), int(B), buf, len(buf)))
        return json.loads(buf.value.decode())

    def sync(self):
        self._check(lib().bti_sync(self._h))

    def profile_enable(self, on=True):
        self._check(lib().bti_profile_enable(self._h, 1 if on else 0))

    def profile_read(self):
        """{class: (milliseconds, launches)} since the last read, and whether all were timed."""
        n = len(KCLASSES)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int64 * n)()
        ok = ctypes.c_int()
        self._check(lib().bti_profile_read(self._h, ms, cnt, ctypes.byref(ok)))
        return {k: (ms[i], cnt[i]) for i, k in enumerate(KCLASSES)}, bool(ok.value)

    @property
    def last_error(self):
        return lib().bti_last_error(self._h).decode()
