#!/usr/bin/env python3
"""Benchmark of the block-Toeplitz matvec hot path on one GB300 (or N replicas).

Workload (the matvec sweep): N_m = 65,536 (256 x 256 grid), N_d = 128,
N_t = 256 (L = 512), seeded Gaussian blocks with exp(-k/64) decay, 16 random
m and d vectors.  One step applies F to each of the 16 m vectors and F^T to
each of the 16 d vectors, one vector per call (single right-hand side, the
paper's matvec), on the FP64 tier; every call streams the 34.5 GB of FP64
spectral blocks from HBM (far larger than L2), so no L2 flush is needed.

value = algorithmic bytes of the step's calls / device time, summed over
ranks (replicas: each rank runs the whole workload on its own GPU).  The
algorithmic bytes of one call are the spectral blocks read once plus its input
and output vectors.  The JSON line also carries the FP32 tier, the end-to-end
figure through host buffers, the dominant kernel's roofline, the CPU oracle
baseline, clocks, and the online m_map + q_map latency of the batched workload.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "F/F^T matvec GB/s and % HBM roofline; online m_map+q_map latency at 1e-6 rel err"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-online", action="store_true", help="skip the batched online-latency block")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-workload matrix-free solve block")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--case", choices=["sweep", "small", "digits_small", "factor_small", "online_batched"],
                    default="sweep",
                    help="small: the sweep shape with N_m = 4096 and 16 vectors (2.2 GB of FP64 spectral "
                         "blocks, still far above L2) for ncu captures; implies --no-online, "
                         "--no-mixed, --no-cpu-baseline and --no-e2e.  digits_small: the batched "
                         "workload's shapes at N_t = 50 with 64 vectors, timing the tensor-core digit-plane "
                         "products (adjoint, forward, explicit inverse) once each, for ncu captures.  "
                         "factor_small: K of 8,192^2 factored by recursive halves and inverted on the tensor "
                         "cores once each, for ncu captures.  online_batched: the batched workload's tensor-core "
                         "offline phase, then its online graph (64 vectors: FP64-level and FP32-level; one "
                         "vector) timed a few times each, for the online phase's launch list")
    a = ap.parse_args()
    if a.case == "small":
        a.no_online = a.no_mixed = a.no_cpu_baseline = a.no_e2e = True
    return a


def workload(args):
    from paper_2501_14911_gb300 import synthetic

    if args.case == "small":
        return synthetic.Problem("matvec_sweep_small_Nm4096_Nd128_Nt256", 6, 64, 64, 128, 256, 32, 64.0,
                                 n_vectors=16)
    return synthetic.SWEEP


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Replicas:
    """Host-side plumbing for N independent replicas (one process per GPU): a barrier
    around the timed region and the max of the per-rank times.  No data-path
    collective: every rank runs the whole workload on its own device."""

    def __init__(self, world, rank, backend="nccl"):
        import torch.distributed as dist

        self.world, self.rank, self.dist = world, rank, dist
        if world > 1 and not dist.is_initialized():
            dist.init_process_group(backend, init_method="env://")

    def barrier(self):
        if self.world > 1:
            self.dist.barrier()

    def max_ms(self, ms, device=None):
        if self.world == 1:
            return ms
        import torch

        t = torch.tensor([ms], dtype=torch.float64, device=device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.world > 1 and self.dist.is_initialized():
            self.dist.destroy_process_group()


def aggregate_gbs(world, bytes_per_step, steps, max_ms):
    """Whole-job throughput: every replica moves bytes_per_step per step; the slowest
    rank's time bounds the job."""
    return world * bytes_per_step * steps / (max_ms * 1e-3) / 1e9


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), float(pk.get("bf16_tflops", 1900.0)), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


# FP64 FFMA-pipe rate of this GB300 (TFLOP/s), from a DFMA throughput probe:
# 2 DFMA per clock per SM x 152 SMs at the sustained clock.  Used only when the live
# measurement below fails.
FP64_TFLOPS = 1.2
# FP32 FFMA rate (TFLOP/s) from the same probe: 128 lanes/clk/SM x 152 SMs x 2 flop.
FP32_TFLOPS = 75.0


def measure_alu_peaks(dev):
    """FP64 and FP32 (no TF32) GEMM throughput of the library GEMM on this GPU, best of 3
    timed runs after one warm-up, with CUDA events: the denominators of the arithmetic-bound
    tiers' rooflines, measured in the same run.  {"fp64_tflops", "fp32_tflops", "how"} or
    None when the measurement fails (the probe constants then serve, and the JSON says so)."""
    import torch
    try:
        tf32 = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = False
        out = {}
        for key, dt, n in (("fp64_tflops", torch.float64, 6144), ("fp32_tflops", torch.float32, 8192)):
            a = torch.randn((n, n), dtype=dt, device=dev)
            b = torch.randn((n, n), dtype=dt, device=dev)
            torch.matmul(a, b)
            torch.cuda.synchronize()
            best = float("inf")
            for _ in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b)
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1))
            out[key] = 2.0 * n ** 3 / (best * 1e-3) / 1e12
            del a, b
        torch.backends.cuda.matmul.allow_tf32 = tf32
        out["how"] = "torch.matmul FP64 6144^3 and FP32 (TF32 off) 8192^3, best of 3, CUDA events, this run"
        return out
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampler (every 200 ms) for the timed region."""

    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                if self.uuid and self.uuid not in parts[0]:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_source_hash(names):
    """Hash of the source text of the named kernels in spectral.cu (template line to
    closing brace), so a traffic record stays valid exactly as long as those kernels do."""
    with open(os.path.join(ROOT, "paper_2501_14911_gb300", "csrc", "spectral.cu")) as f:
        src = f.read()
    h = hashlib.sha256()
    for name in names:
        i = src.index(name + "(")
        j = src.rfind("template <", 0, i)
        k = src.index("\n}\n", i) + 3
        h.update(src[j:k].encode())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_tag):
    """Per-launch DRAM bytes of the product kernels from the committed ncu summary,
    or None when the kernels changed since that capture."""
    path = os.path.join(ROOT, "profiles", "traffic_spectral_products.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        if rec.get("source_hash") != kernel_source_hash(rec["kernels"]):
            return None
    except Exception:
        return None
    return rec.get(kernel_tag)


def cores_used():
    try:
        from threadpoolctl import threadpool_info

        n = [i.get("num_threads") for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    return os.cpu_count() or 1


def bytes_per_call(p, esize, csize):
    Fhat = (p.Nt + 1) * p.Nd * p.Nm * csize
    io = (p.Nt * p.Nm + p.Nt * p.Nd) * esize
    return Fhat + io


def cpu_oracle_sample(p, F, m, d, budget_s=12.0):
    """Time the oracle's F and F^T on whole vectors until ~budget_s of CPU work."""
    import oracle

    t0 = time.perf_counter()
    pairs = 0
    while pairs < m.shape[0]:
        oracle.p2o_apply(F, m[pairs])
        oracle.p2o_apply_adjoint(F, d[pairs])
        pairs += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return pairs, dt


def cpu_oracle_online():
    """The oracle's offline and online phases on the batched workload (N_m = 4,096, N_d = 100,
    N_t = 200, K 20,000^2, 64 observation vectors), once, on the host cores: G = F C_s, K by
    the Gram product and block-diagonal sums, its Cholesky factor (LAPACK), then m_map + q_map
    (two triangular solves, G^* and F_q by direct convolution sums) for a sample of 8 of the 64
    observation vectors, scaled to 64.  About 20-40 s."""
    import oracle
    from paper_2501_14911_gb300 import synthetic

    p = synthetic.BATCHED
    F, Fq = p.blocks_F(), p.blocks_Fq()
    B = p.n_vectors
    d = p.vectors_d()[:8]  # the online sample
    nb = d.shape[0]
    t = [time.perf_counter()]
    G = oracle.prior_blocks(F, oracle.se_covariance(p.gx, p.gy, p.ell, p.sigma_p))
    t.append(time.perf_counter())
    K = oracle.assemble_K(F, G, p.sigma2)
    t.append(time.perf_counter())
    L = oracle.cholesky_lower(K)
    del K
    t.append(time.perf_counter())
    x = oracle.solve_K(L, d.reshape(nb, -1)).reshape(d.shape)
    t.append(time.perf_counter())
    m = oracle.p2o_apply_adjoint(G, x)
    oracle.qoi_map(Fq, m)
    t.append(time.perf_counter())
    ms = [(b - a) * 1e3 for a, b in zip(t, t[1:])]
    n = p.Nt * p.Nd
    per_vec = (ms[3] + ms[4]) / nb
    return {"kind": "oracle", "cores": cores_used(),
            "sample": f"the batched workload's offline phase once (K {n}^2) and its online phase for {nb} of "
                      f"the {B} observation vectors, scaled to {B}",
            "prior_blocks_ms": ms[0], "build_K_ms": ms[1], "factor_K_ms": ms[2],
            "triangular_solves_ms_per_vector": ms[3] / nb, "G_star_and_F_q_ms_per_vector": ms[4] / nb,
            "offline_ms": ms[0] + ms[1] + ms[2], "m_map_plus_q_map_ms": per_vec * B,
            "m_map_plus_q_map_ms_per_vector": per_vec,
            "factor_tflops_fp64": (n ** 3 / 3.0) / (ms[2] * 1e-3) / 1e12}


# --------------------------------------------------------------------------------------------
def run_reference(args):
    """The CPU oracle as the reference arm (rank 0 only), on the same workload and metric."""
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2501_14911_gb300 import synthetic

    p = workload(args)
    F = p.blocks_F()
    m = p.vectors_m()
    d = p.vectors_d()
    bpc = bytes_per_call(p, 8, 16)
    times = []
    for it in range(args.warmup + args.steps):
        pairs, dt = cpu_oracle_sample(p, F, m[:1], d[:1], budget_s=0.0)
        if it >= args.warmup:
            times.append(dt / pairs)
    per_pair = statistics.mean(times)
    value = 2 * bpc / per_pair / 1e9
    cores = cores_used()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_pair * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": p.name, "Nm": p.Nm, "Nd": p.Nd, "Nt": p.Nt, "vectors": p.n_vectors,
                   "rhs_per_call": 1, "parallelism": "cpu",
                   "step": f"one F m + F^T d pair of the workload's {p.n_vectors} (a bounded sample); "
                           "ms_per_step is its measured time"},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": cores, "kind": "oracle",
                         "sample": "each step: oracle time-domain F m and F^T d on one sweep vector pair "
                                   "(full size), scaled to the GPU formulation's algorithmic bytes"},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------------------------
def run_ours(args):
    import torch

    import paper_2501_14911_gb300 as bti
    from paper_2501_14911_gb300 import synthetic

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    reps = Replicas(world, rank, "nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    hbm_peak, _, peak_src = load_peaks()

    p = workload(args)
    V = p.n_vectors
    F_host = p.blocks_F()
    m_host = p.vectors_m()
    d_host = p.vectors_d()

    # One handle per tier, built and timed in turn (the device keeps one set of spectral
    # blocks at a time).  Headline: the double-FP32 tier (FP64-accurate products and FFTs in
    # float pairs on the FP32 pipes, FP64 vectors); the native FP64 and the FP32 tiers follow.
    Fd = torch.from_numpy(F_host).to(dev)
    m64 = torch.from_numpy(m_host).to(dev)
    d64 = torch.from_numpy(d_host).to(dev)
    m32, d32 = m64.float(), d64.float()
    od64 = torch.empty((V, p.Nt, p.Nd), dtype=torch.float64, device=dev)
    om64 = torch.empty((V, p.Nt, p.Nm), dtype=torch.float64, device=dev)
    od32, om32 = od64.float(), om64.float()

    def step(h, m, d, od, om):
        for b in range(V):
            h.apply_F(m[b], od[b])
            h.apply_FT(d[b], om[b])

    def barrier():
        reps.barrier()

    def timed(fn, steps, warmup, prof_handle=None):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        if prof_handle is not None:
            prof_handle.profile_read()  # reset counters
            prof_handle.profile_enable(True)
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = e0.elapsed_time(e1)
        prof = None
        if prof_handle is not None:
            prof = prof_handle.profile_read()
            prof_handle.profile_enable(False)
        ms = reps.max_ms(ms, dev)
        return ms, prof

    props = torch.cuda.get_device_properties(dev)
    uuid = str(getattr(props, "uuid", ""))

    alu = measure_alu_peaks(dev) if rank == 0 else None
    fp64_peak = alu["fp64_tflops"] if alu else FP64_TFLOPS
    fp32_peak = alu["fp32_tflops"] if alu else FP32_TFLOPS
    alu_src = f"measured: {alu['how']}" if alu else "probe constant (the live measurement failed)"

    # dominant kernel: the per-frequency spectral products (forward and adjoint)
    def roofline(prof, csize, kind):
        (pf_ms, pf_n), (pa_ms, pa_n) = prof[0]["prod_fwd"], prof[0]["prod_adj"]
        nf = p.Nt + 1
        Fhat = nf * p.Nd * p.Nm * csize
        mhat = nf * p.Nm * 16  # the frequency-domain vector (complex FP64 for f64, float pairs for df64)
        if kind in ("f32", "f16"):
            mhat = nf * p.Nm * 8
        bytes_launch = Fhat + mhat
        elems = nf * p.Nd * p.Nm
        avg_ms = (pf_ms + pa_ms) / max(pf_n + pa_n, 1)
        gbs = bytes_launch / (avg_ms * 1e-3) / 1e9
        t_hbm = bytes_launch / (hbm_peak * 1e9)
        # arithmetic: f64 = 8 DP flop per element on the FP64 pipe; f32 = 4 FFMA; df64 = 48 FP32
        # instructions per element (4 float-pair multiply-accumulates of 12 operations)
        if kind == "f64":
            work, peak, unit, src = 8.0 * elems, fp64_peak * 1e12, "TFLOP/s", "FP64 GEMM rate, " + alu_src
        elif kind in ("f32", "f16"):
            work, peak, unit, src = 8.0 * elems, fp32_peak * 1e12, "TFLOP/s", "FP32 GEMM rate, " + alu_src
        else:
            # FP32 instructions: half the FP32 GEMM's flop rate (one FFMA = 2 flop)
            work, peak, unit, src = 48.0 * elems, fp32_peak / 2 * 1e12, "Tinstr/s", \
                "FP32 instruction rate = FP32 GEMM rate / 2, " + alu_src
        t_alu = work / peak
        traffic = ncu_traffic(f"{kind}_bytes_per_launch")
        share_total = sum(v[0] for v in prof[0].values())
        common = {"kernel": f"prod_fwd + prod_adj ({kind})", "avg_launch_ms": avg_ms,
                  "launches": pf_n + pa_n, "share_of_step_kernel_time": (pf_ms + pa_ms) / max(share_total, 1e-9),
                  "traffic": traffic, "algorithmic_bytes_per_launch": bytes_launch,
                  "hbm_gbs": gbs, "hbm_frac": gbs / hbm_peak}
        if t_alu > t_hbm:
            ach = work / (avg_ms * 1e-3) / 1e12
            return dict({"bound": "alu", "achieved": ach, "peak": peak / 1e12, "unit": unit,
                         "frac": ach * 1e12 / peak, "peak_source": src}, **common)
        return dict({"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                      "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_src})"}, **common)

    tiers = {"df64": (bti.DF64, 16, 8), "f64": (bti.F64, 16, 8), "f32": (bti.F32, 8, 4), "f16": (bti.F16, 4, 4)}
    res = {}
    clk = None
    e2e = None
    for name, (prec, csize, esize) in tiers.items():
        h = bti.Handle(p.Nm, p.Nd, 0, p.Nt, device=dev)
        h.set_blocks(bti.OP_F, Fd, prec)
        tune = h.autotune(bti.OP_F, 1)  # launch shapes for single-vector calls (outside the timed region)
        torch.cuda.synchronize()
        vecs = (m32, d32, od32, om32) if name in ("f32", "f16") else (m64, d64, od64, om64)
        headline = name == "df64"
        if headline:
            clocks = Clocks(uuid)
            clocks.start()
        ms, prof = timed(lambda: step(h, *vecs), args.steps, args.warmup, h)
        if headline:
            clk = clocks.stop()
        bytes_step = 2 * V * bytes_per_call(p, esize, csize)
        # the same 16 vector pairs as one call each way (B = 16).  The CUDA-core product
        # kernels take 4 right-hand sides per CTA, so the spectral blocks stream 4 times per
        # call; the FP16 tier's tensor-core kernels take all 16 in one pass.
        ms_b, prof_b = timed(lambda: (h.apply_F(vecs[0], vecs[2]), h.apply_FT(vecs[1], vecs[3])), args.steps, 1, h)
        tensor_cores = name == "f16" and p.Nm % 4 == 0 and V >= 8
        streams = 1 if tensor_cores else (V + 3) // 4
        kms = {k: v[0] / args.steps for k, v in prof_b[0].items()}
        prod_ms = kms["prod_fwd"] + kms["prod_adj"]
        batched = {"ms_per_step": ms_b / args.steps, "vector_pairs_per_s": world * V * args.steps / (ms_b * 1e-3),
                   "speedup_vs_single_vector_calls": ms / ms_b, "tensor_cores": tensor_cores,
                   "spectral_streams_per_call": streams, "kernel_ms_per_step": kms,
                   "product_stream_gbs": 2 * streams * (p.Nt + 1) * p.Nd * p.Nm * csize / (prod_ms * 1e-3) / 1e9}
        res[name] = {"ms": ms, "prof": prof, "bytes_step": bytes_step, "autotune": tune, "batched16": batched,
                     "value": aggregate_gbs(world, bytes_step, args.steps, ms),
                     "roofline": roofline(prof, csize, name)}
        if headline and not args.no_e2e:
            e2e = e2e_block(args, h, p, m_host, d_host, dev, timed, world, bytes_step)
        h.close()
    del Fd
    torch.cuda.empty_cache()

    head = res["df64"]
    launches = sum(v[1] for v in head["prof"][0].values())
    line = {
        "metric": METRIC, "value": head["value"], "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "df64", "data": "synthetic",
        "config": {"workload": p.name, "Nm": p.Nm, "Nd": p.Nd, "Nt": p.Nt, "L": p.L, "vectors": V,
                   "rhs_per_call": 1, "calls_per_step": 2 * V,
                   "tier": "double-FP32: spectral blocks as FP32 hi+lo pairs (16 B/complex), products in "
                           "float-pair arithmetic on the FP32 pipes; FFTs in float pairs (ffloat), input and output "
                           "vectors FP64; 1e-12 vs the FP64 oracle",
                   "l2": f"inputs larger than L2: each call streams the {(p.Nt + 1) * p.Nd * p.Nm * 16 / 1e9:.1f} GB "
                         "spectral blocks from HBM",
                   "parallelism": f"replicas x{world}",
                   "autotune": {k: {kk: v["autotune"][kk] for kk in ("fft_p_chosen", "jc_chosen", "vpt_chosen")}
                                for k, v in res.items()}},
        "hbm_frac": head["value"] / world / hbm_peak,
        "roofline": head["roofline"],
        "tiers": {k: {"value": v["value"], "unit": "GB/s", "ms_per_step": v["ms"] / args.steps,
                      "hbm_frac": v["value"] / world / hbm_peak, "roofline": v["roofline"]}
                  for k, v in res.items() if k != "df64"},
        "batched16": {k: v["batched16"] for k, v in res.items()},
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
        "kernel_ms_per_step": {k: v[0] / args.steps for k, v in head["prof"][0].items()},
        "alu_peaks": alu if alu else {"fp64_tflops": FP64_TFLOPS, "fp32_tflops": FP32_TFLOPS,
                                      "how": "probe constants (the live measurement failed)"},
    }
    bpc64 = bytes_per_call(p, 8, 16)

    # online m_map + q_map latency on the batched workload (64 observation vectors)
    # single-GPU sidecar measurements (skipped when ranks run replicas)
    # (a sidecar that fails is recorded in its block; the headline line prints regardless)
    if not args.no_online and world == 1:
        try:
            line["online"] = online_block(args, dev, stream)
        except Exception as ex:
            line["online"] = {"error": f"{type(ex).__name__}: {ex}"}
    if not args.no_mixed and world == 1:
        try:
            line["mixed"] = mixed_block(args, dev, stream)
        except Exception as ex:
            line["mixed"] = {"error": f"{type(ex).__name__}: {ex}"}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        pairs, dt = cpu_oracle_sample(p, F_host, m_host, d_host)
        line["cpu_baseline"] = {"value": 2 * pairs * bpc64 / dt / 1e9, "unit": "GB/s", "cores": cores_used(),
                                "kind": "oracle",
                                "sample": f"oracle time-domain F m and F^T d on {pairs} full-size sweep vector "
                                          f"pair(s) in {dt:.1f} s, scaled to the GPU formulation's bytes"}
        if "online" in line:
            line["online"]["cpu_baseline"] = cpu_oracle_online()
    if rank == 0:
        print(json.dumps(line), flush=True)
    reps.close()
    return 0


def e2e_block(args, h, p, m_host, d_host, dev, timed, world, bytes_step):
    """The headline step through the public API from pinned host buffers: every call's
    input is copied host->device and its output device->host inside the timed region.
    Copies run on two copy streams, double-buffered against the compute stream, so
    the transfers of vector b+1 and b-1 overlap the products of vector b."""
    import torch

    V = p.n_vectors
    comp = torch.cuda.current_stream(dev)
    up = torch.cuda.Stream(dev)
    down = torch.cuda.Stream(dev)
    mh = torch.from_numpy(m_host).pin_memory()
    dh = torch.from_numpy(d_host).pin_memory()
    odh = torch.empty((V, p.Nt, p.Nd), dtype=torch.float64).pin_memory()
    omh = torch.empty((V, p.Nt, p.Nm), dtype=torch.float64).pin_memory()
    mdev = [torch.empty((p.Nt, p.Nm), dtype=torch.float64, device=dev) for _ in range(2)]
    ddev = [torch.empty((p.Nt, p.Nd), dtype=torch.float64, device=dev) for _ in range(2)]
    odev = [torch.empty((p.Nt, p.Nd), dtype=torch.float64, device=dev) for _ in range(2)]
    omdev = [torch.empty((p.Nt, p.Nm), dtype=torch.float64, device=dev) for _ in range(2)]
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]

    def e2e_step():
        for k in range(2):
            ev_out[k].record(comp)
        for b in range(V):
            k = b % 2
            up.wait_event(ev_out[k])  # slot k's previous results have left the device
            with torch.cuda.stream(up):
                mdev[k].copy_(mh[b], non_blocking=True)
                ddev[k].copy_(dh[b], non_blocking=True)
            ev_in[k].record(up)
            comp.wait_event(ev_in[k])
            h.apply_F(mdev[k], odev[k])
            h.apply_FT(ddev[k], omdev[k])
            ev_done[k].record(comp)
            down.wait_event(ev_done[k])
            with torch.cuda.stream(down):
                odh[b].copy_(odev[k], non_blocking=True)
                omh[b].copy_(omdev[k], non_blocking=True)
            ev_out[k].record(down)
        for k in range(2):
            comp.wait_event(ev_out[k])

    ms, _ = timed(e2e_step, args.steps, min(args.warmup, 3))
    vec_bytes = (p.Nt * p.Nm + p.Nt * p.Nd) * 8
    return {"value": aggregate_gbs(world, bytes_step, args.steps, ms), "unit": "GB/s",
            "ms_per_step": ms / args.steps, "h2d_bytes_per_step": V * vec_bytes,
            "d2h_bytes_per_step": V * vec_bytes,
            "note": "pinned host buffers; H2D and D2H on two copy streams, double-buffered against compute"}


def online_block(args, dev, stream):
    """Offline build (K, Cholesky) and online latency of m_map + q_map for the 64
    observation vectors of the batched workload, in four forms: plain FP64; the dense
    work (Gram product, Cholesky updates, triangular solves) in double-FP32
    arithmetic; K assembled in FP32 with refinement; and both.  All forms reach FP64-
    level m_map (tests/test_gpu_parity.py, tests/test_gpu_fullsize.py)."""
    import torch

    import paper_2501_14911_gb300 as bti
    from paper_2501_14911_gb300 import synthetic

    p = synthetic.BATCHED
    B = p.n_vectors
    h = bti.Handle(p.Nm, p.Nd, p.Nq, p.Nt, device=dev)
    h.set_blocks(bti.OP_F, torch.from_numpy(p.blocks_F()).to(dev), bti.DF64)
    h.set_blocks(bti.OP_FQ, torch.from_numpy(p.blocks_Fq()).to(dev), bti.DF64)
    h.set_prior_se_grid(p.gx, p.gy, p.ell, p.sigma_p, bti.DF64)
    h.set_noise(p.sigma2)
    d_obs = torch.from_numpy(p.vectors_d()).to(dev)
    m_map = torch.empty((B, p.Nt, p.Nm), dtype=torch.float64, device=dev)
    q_map = torch.empty((B, p.Nt, p.Nq), dtype=torch.float64, device=dev)
    gs = torch.cuda.Stream(dev)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    reps = 3
    # (name, dense arithmetic, K assembly, refinement steps, explicit inverse, tensor cores):
    # with tensor cores the Gram product of K (double-FP32 dense), the explicit inverse and the
    # G^* and F_q products of the 64 vectors run as exact digit-plane MMAs; without, in
    # double-FP32 on the CUDA cores
    forms = [("plain_f64", bti.F64, bti.F64, 0, False, False), ("dense_df64", bti.DF64, bti.F64, 1, False, False),
             ("dense_df64_no_refinement", bti.DF64, bti.F64, 0, False, False),
             ("explicit_inverse_cuda_cores", bti.DF64, bti.F64, 0, True, False),
             ("explicit_inverse_tensor_cores", bti.DF64, bti.F64, 0, True, True),
             ("f32_assembly", bti.F64, bti.F32, 3, False, False),
             ("f32_assembly_dense_df64", bti.DF64, bti.F32, 3, False, False)]
    out = {"workload": p.name, "obs_vectors": B, "K_n": p.Nt * p.Nd}
    for name, dense, assembly, refine, inverse, tcores in forms:
        h.set_stream(gs)
        with torch.cuda.stream(gs):
            h.set_dense_precision(dense)
            h.set_tensor_cores(tcores)  # the FP16-tier products and every digit-plane product
            torch.cuda.synchronize()
            e[0].record(gs)
            h.build_K_prec(p.col_block, assembly)
            e[1].record(gs)
            h.factor_K()
            e[2].record(gs)
            torch.cuda.synchronize()
            t_build, t_factor = e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])
            t_inv = t_planes = 0.0
            if inverse:
                e[0].record(gs)
                h.invert_K()
                e[1].record(gs)
                torch.cuda.synchronize()
                t_inv = e[0].elapsed_time(e[1])
            if tcores:
                e[0].record(gs)
                h.set_digit_planes(bti.OP_G, True)
                h.set_digit_planes(bti.OP_FQ, True)
                e[1].record(gs)
                torch.cuda.synchronize()
                t_planes = e[0].elapsed_time(e[1])
            for _ in range(2):
                h.online(d_obs, m_map, q_map, refine_iters=refine)
            torch.cuda.synchronize()
            e[0].record(gs)
            for _ in range(reps):
                h.online(d_obs, m_map, q_map, refine_iters=refine)
            e[1].record(gs)
            torch.cuda.synchronize()
            lat = e[0].elapsed_time(e[1]) / reps
        n = p.Nt * p.Nd
        out[name] = {"dense": "f64" if dense == bti.F64 else "df64",
                     "K_assembly": "f64" if assembly == bti.F64 else "f32", "refine_iters": refine,
                     "build_K_ms": t_build, "factor_K_ms": t_factor,
                     "factor_tflops_fp64_equiv": (n ** 3 / 3.0) / (t_factor * 1e-3) / 1e12,
                     "m_map_plus_q_map_graph_ms": lat, "ms_per_obs_vector": lat / B,
                     "offline_plus_online_ms": t_build + t_factor + t_inv + t_planes + lat}
        if inverse:
            out[name]["invert_K_ms"] = t_inv
        if tcores:
            # the same form with one refinement step (FP64-level m_map, equal to plain FP64's)
            with torch.cuda.stream(gs):
                for _ in range(2):
                    h.online(d_obs, m_map, q_map, refine_iters=1)
                torch.cuda.synchronize()
                e[0].record(gs)
                for _ in range(reps):
                    h.online(d_obs, m_map, q_map, refine_iters=1)
                e[1].record(gs)
                torch.cuda.synchronize()
            out[name]["m_map_plus_q_map_refined_graph_ms"] = e[0].elapsed_time(e[1]) / reps
            out[name]["digit_planes_ms"] = t_planes
            # q_map = Q d_obs (Eq. (4.14)) with Q in digit planes, in the same online graph
            with torch.cuda.stream(gs):
                e[0].record(gs)
                h.build_Q(with_covariance=False)
                h.set_online_qoi(True)
                e[1].record(gs)
                torch.cuda.synchronize()
                t_q = e[0].elapsed_time(e[1])
                for r_it in (0, 1):
                    for _ in range(2):
                        h.online(d_obs, m_map, q_map, refine_iters=r_it)
                    torch.cuda.synchronize()
                    e[0].record(gs)
                    for _ in range(reps):
                        h.online(d_obs, m_map, q_map, refine_iters=r_it)
                    e[1].record(gs)
                    torch.cuda.synchronize()
                    key = "m_map_plus_q_map_via_Q_graph_ms" if r_it == 0 else "m_map_plus_q_map_via_Q_refined_graph_ms"
                    out[name][key] = e[0].elapsed_time(e[1]) / reps
                # one observation vector (the real-time case): B < 16 takes the memory-bound kernels
                for _ in range(2):
                    h.online(d_obs[:1], m_map[:1], q_map[:1])
                torch.cuda.synchronize()
                e[0].record(gs)
                for _ in range(reps):
                    h.online(d_obs[:1], m_map[:1], q_map[:1])
                e[1].record(gs)
                torch.cuda.synchronize()
                t1 = e[0].elapsed_time(e[1]) / reps
                out[name]["m_map_plus_q_map_via_Q_B1_graph_ms"] = t1
                out[name]["one_vector_roofline"] = one_vector_roofline(p, t1)
                # the FP32-level online form for the 1e-6 latency target (bti_set_online_precision):
                # five digit planes for K^{-1}, four for G^* and Q (B >= 16; one vector keeps FP64 level)
                h.set_online_precision(bti.F32)
                for nb, key in ((B, "m_map_plus_q_map_fp32_level_graph_ms"),):
                    for _ in range(2):
                        h.online(d_obs[:nb], m_map[:nb], q_map[:nb])
                    torch.cuda.synchronize()
                    e[0].record(gs)
                    for _ in range(reps):
                        h.online(d_obs[:nb], m_map[:nb], q_map[:nb])
                    e[1].record(gs)
                    torch.cuda.synchronize()
                    out[name][key] = e[0].elapsed_time(e[1]) / reps
                h.set_online_precision(bti.DF64)
                h.set_online_qoi(False)
            out[name]["build_Q_and_planes_ms"] = t_q
            out[name]["G_star_roofline"] = digit_tensor_roofline(h, p, dev, gs, B)
        if inverse:
            h.invert_K(False)
        if tcores:
            h.set_digit_planes(bti.OP_G, False)
            h.set_digit_planes(bti.OP_FQ, False)
        h.set_tensor_cores(True)
        if name == "plain_f64":
            # q_map straight from the data through the precomputed d2q map (Eq. (4.14))
            with torch.cuda.stream(gs):
                e[0].record(gs)
                h.build_Q(with_covariance=True)
                e[1].record(gs)
                torch.cuda.synchronize()
                t_q = e[0].elapsed_time(e[1])
                for nb in (1, B):
                    for _ in range(2):
                        h.apply_Q(d_obs[:nb], q_map[:nb])
                    torch.cuda.synchronize()
                    e[0].record(gs)
                    for _ in range(reps):
                        h.apply_Q(d_obs[:nb], q_map[:nb])
                    e[1].record(gs)
                    torch.cuda.synchronize()
                    out[name][f"q_map_via_Q_ms_B{nb}"] = e[0].elapsed_time(e[1]) / reps
            out[name]["build_Q_and_covariance_ms"] = t_q
            out[name]["Q_shape"] = [p.Nt * p.Nq, p.Nt * p.Nd]
    h.set_stream(stream)
    h.close()
    out["accuracy"] = ("the forms with refinement reach FP64-level m_map and q_map: tests/test_gpu_parity.py "
                       "(tiny, 1e-12) and tests/test_gpu_fullsize.py (batched full size, 1e-11) against the oracle; "
                       "the three without are held to 3e-11 (blocked solves) and 1e-10 (explicit inverse, both "
                       "forms) there: 48-bit arithmetic times kappa(K), 1.2e-11 and 5.0e-11 measured, far inside "
                       "the 1e-6 latency target; the FP32-level form (m_map_plus_q_map_fp32_level_*) is held to "
                       "1e-6 against the oracle at full size (tests/test_gpu_fullsize.py)")
    return out


def one_vector_roofline(p, ms):
    """HBM roofline of the one-observation online graph with the explicit inverse and q_map =
    Q d_obs: its algorithmic bytes are K^{-1}'s lower triangle in float pairs (the 128 x 128
    tiles on and below the diagonal, 8 B per entry), G-hat in double-FP32 (16 B per complex)
    and Q in float pairs (8 B per entry); the vectors and transforms add well under 1 %."""
    hbm, _, src = load_peaks()
    n = p.Nt * p.Nd
    T = (n + 127) // 128
    kinv = T * (T + 1) // 2 * 128 * 128 * 8
    ghat = (p.Nt + 1) * p.Nd * p.Nm * 16
    qp = p.Nt * p.Nq * n * 8
    b = kinv + ghat + qp
    gbs = b / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "bytes_per_replay": b, "K_inv_lower_bytes": kinv, "G_hat_bytes": ghat, "Q_bytes": qp,
            "ms": ms, "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
            "hbm_bound_ms": b / (hbm * 1e9) * 1e3, "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({src})"}


def digit_tensor_roofline(h, p, dev, gs, B):
    """Roofline of the digit-plane adjoint (G^* on B vectors, the vector planes and the MMA
    kernel) on the method's own work.  The product m-hat_w = G-hat_w^H d-hat_w streams the
    spectral blocks once: HBM-bound.  Its algorithmic bytes are G-hat in double-FP32 (16 B per
    complex) plus d-hat read and m-hat written (16 B per complex, FP64); its algorithmic flops
    are 8 n_f N_d N_m B (complex multiply-adds).  The FP16 MMA work that the six digit planes
    emulate the FP64 products with (21 plane pairs x 4 K-steps per 64-column box, M = 128,
    N = 64, K = 16) is reported beside them as tensor-pipe utilisation, not as a roofline."""
    import torch

    import paper_2501_14911_gb300 as bti

    def rup(x, m):
        return (x + m - 1) // m * m

    nf = p.Nt + 1
    boxes = rup(2 * p.Nd, 128) // 64
    mmas = nf * (rup(p.Nm, 128) // 128) * (rup(2 * B, 64) // 64) * boxes * 21 * 4
    mma_flops = mmas * 2 * 128 * 64 * 16
    alg_bytes = nf * p.Nd * p.Nm * 16 + B * nf * (p.Nd + p.Nm) * 16
    alg_flops = 8.0 * nf * p.Nd * p.Nm * B
    x = torch.ones((B, p.Nt, p.Nd), dtype=torch.float64, device=dev)
    y = torch.empty((B, p.Nt, p.Nm), dtype=torch.float64, device=dev)
    with torch.cuda.stream(gs):
        for _ in range(2):
            h.apply_Gstar(x, y)
        torch.cuda.synchronize()
        h.profile_enable(True)
        h.profile_read()
        reps = 3
        for _ in range(reps):
            h.apply_Gstar(x, y)
        torch.cuda.synchronize()
        prof, _ok = h.profile_read()
        h.profile_enable(False)
    ms = prof["prod_adj"][0] / reps
    hbm, peak, src = load_peaks()
    gbs = alg_bytes / (ms * 1e-3) / 1e9
    mma_tf = mma_flops / (ms * 1e-3) / 1e12
    return {"bound": "hbm", "kernel": "adj_tc_kernel (G^*, digit planes) + its vector planes",
            "ms_per_call": ms, "algorithmic_bytes_per_call": alg_bytes, "achieved": gbs, "peak": hbm,
            "unit": "GB/s", "frac": gbs / hbm, "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({src})",
            "algorithmic_tflops": alg_flops / (ms * 1e-3) / 1e12,
            "tensor_pipe_note": {"mma_flops_per_call": mma_flops, "mma_tflops": mma_tf,
                                 "of_bf16_peak": mma_tf / peak,
                                 "what": "FP16 MMA work of the 21 digit-plane pairs (emulation of the FP64 "
                                         "products), against the measured dense BF16 peak"}}


def mixed_forward_error(dev):
    """Forward error of the matrix-free mixed-precision solve against the oracle, at the
    mixed workload truncated to its first 42 time steps (K 25,200^2, where the oracle's dense
    solve applies): the stored oracle solution (tests/golden/mixed_nt42_map.json, written by
    a script that calls only the oracle) for one white-data vector against the same solve
    form as the full-size block (flexible PCG, FP16 inner), to 1e-6 (the latency target) and
    1e-10 (white data leave the double-FP32 operator a residual floor near 3e-11 here)."""
    import numpy as np
    import torch

    import paper_2501_14911_gb300 as bti
    from paper_2501_14911_gb300 import synthetic

    path = os.path.join(ROOT, "tests", "golden", "mixed_nt42_map.json")
    with open(path) as f:
        gold = json.load(f)
    p = synthetic.MIXED_NT42
    h = bti.Handle(p.Nm, p.Nd, p.Nq, p.Nt, device=dev)
    h.set_blocks(bti.OP_F, torch.from_numpy(p.blocks_F()).to(dev), bti.DF64)
    h.set_blocks(bti.OP_FQ, torch.from_numpy(p.blocks_Fq()).to(dev), bti.DF64)
    h.set_prior_se_grid(p.gx, p.gy, p.ell, p.sigma_p, bti.F16)
    h.set_shadow(bti.OP_F, bti.F16)
    h.set_noise(p.sigma2)
    h.set_matfree_precond(1)
    d = torch.from_numpy(p.vectors_d(1)).to(dev)
    m = torch.empty((1, p.Nt, p.Nm), dtype=torch.float64, device=dev)
    x = torch.empty((1, p.Nt, p.Nd), dtype=torch.float64, device=dev)
    q = torch.empty((1, p.Nt, p.Nq), dtype=torch.float64, device=dev)
    out = {"workload": p.name, "K_n": p.Nt * p.Nd, "reference": "tests/golden/mixed_nt42_map.json (oracle)",
           "metric": "||v - v_oracle|| / ||v_oracle|| over 1,024 sampled entries of x and m_map, whole q_map"}
    for tol in (1e-6, 1e-10):
        try:
            info = h.solve_matfree(d, m, x, refine=2, tol=tol, max_outer=400, max_inner=2000, inner_tol=0.1)
        except bti.BtiError as ex:  # reported, not fatal: the record says it did not converge
            info = dict(h.last_solve, error=str(ex))
        h.predict_qoi(m, q)
        xs = x.reshape(-1).cpu().numpy()[gold["x_idx"]]
        ms = m.reshape(-1).cpu().numpy()[gold["m_idx"]]
        qs = q.reshape(-1).cpu().numpy()
        xv, mv, qv = (np.array(gold[k]) for k in ("x_val", "m_val", "q"))
        out[f"tol_{tol:.0e}"] = dict(info, x_err=float(np.linalg.norm(xs - xv) / np.linalg.norm(xv)),
                                     m_map_err=float(np.linalg.norm(ms - mv) / np.linalg.norm(mv)),
                                     q_map_err=float(np.linalg.norm(qs - qv) / np.linalg.norm(qv)))
    h.close()
    return out


def mixed_block(args, dev, stream):
    """m_map on the mixed-precision workload (N_m = 16,384, N_d = 600, N_t = 420, L = 840),
    where K would be 252,000^2 (508 GB in FP64) and is never formed.  Block-Jacobi
    preconditioned plain FP64 conjugate gradients (double-FP32 spectral operators, SE prior
    applied in FP64) against flexible FP64 CG preconditioned by FP32 CG on FP16 spectral
    blocks of F and G, both to the same relative residual with the FP64-accurate operator:
    1e-6 (the online latency target) and 1e-11 (FP64-level for this K).  One observation
    vector per call, and the flexible form also with 16 per call, where the inner FP16
    products run on the tensor cores (tcgen05, B >= 8).  The forward error against the
    oracle is measured at the workload's first 42 time steps (mixed_forward_error)."""
    import torch

    import paper_2501_14911_gb300 as bti
    from paper_2501_14911_gb300 import synthetic

    p = synthetic.MIXED
    h = bti.Handle(p.Nm, p.Nd, 0, p.Nt, device=dev)
    gs = torch.cuda.Stream(dev)
    h.set_stream(gs)
    B16 = 16
    out = {"workload": p.name, "K_n": p.Nt * p.Nd, "K_fp64_GB": (p.Nt * p.Nd) ** 2 * 8 / 1e9,
           "data": "d = F m + sigma noise for seeded N(0,1) m, through the library's F"}
    with torch.cuda.stream(gs):
        Fd = torch.from_numpy(p.blocks_F()).to(dev)
        h.set_blocks(bti.OP_F, Fd, bti.DF64)
        torch.cuda.synchronize()
        del Fd
        torch.cuda.empty_cache()
        h.set_noise(p.sigma2)
        d_obs = torch.empty((B16, p.Nt, p.Nd), dtype=torch.float64, device=dev)
        h.apply_F(torch.from_numpy(p.vectors_m(B16)).to(dev), d_obs)
        d_obs += p.sigma2 ** 0.5 * torch.from_numpy(p.noise(B16)).to(dev)
        m_map = torch.empty((B16, p.Nt, p.Nm), dtype=torch.float64, device=dev)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        h.set_prior_se_grid(p.gx, p.gy, p.ell, p.sigma_p, bti.F16)
        h.set_shadow(bti.OP_F, bti.F16)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h.set_matfree_precond(1)
        out["precond_build_ms"] = (time.perf_counter() - t0) * 1e3
        out["precond"] = "block-Jacobi: inverses of the N_t diagonal blocks K(t,t), N_d x N_d each"
        plain = dict(refine=0, max_inner=6000)
        flexible = dict(refine=2, max_outer=400, max_inner=2000, inner_tol=0.1)
        forms = (("plain_f64_pcg", plain, 1), ("flexible_pcg_f16_inner", flexible, 1),
                 ("flexible_pcg_f16_inner_16_vectors", flexible, B16))
        for name, kw, nb in forms:
            rec = {}
            for tol in (1e-6, 1e-11):
                torch.cuda.synchronize()
                h.profile_enable(True)
                h.profile_read()
                e[0].record(gs)
                try:
                    info = h.solve_matfree(d_obs[:nb], m_map[:nb], tol=tol, **kw)
                except bti.BtiError as ex:  # reported, not fatal: the line says it did not converge
                    info = dict(h.last_solve, error=str(ex))
                e[1].record(gs)
                torch.cuda.synchronize()
                prof, _ = h.profile_read()
                h.profile_enable(False)
                ms = e[0].elapsed_time(e[1])
                rec[f"tol_{tol:.0e}"] = dict(info, ms=ms, ms_per_vector=ms / nb,
                                             chunk_sum_launches=prof["reduce"][1])
            out[name] = dict(rec, vectors_per_call=nb, **{k: v for k, v in kw.items() if k != "refine"})
    h.set_stream(stream)
    h.close()
    torch.cuda.empty_cache()
    # mixed precision against plain FP64 at equal final residual, per observation vector
    for tol in ("1e-06", "1e-11"):
        base = out["plain_f64_pcg"][f"tol_{tol}"]["ms_per_vector"]
        out[f"speedup_at_{tol}"] = base / out["flexible_pcg_f16_inner"][f"tol_{tol}"]["ms_per_vector"]
        out[f"speedup_at_{tol}_16_vectors"] = base / out["flexible_pcg_f16_inner_16_vectors"][f"tol_{tol}"]["ms_per_vector"]
    out["tensor_cores"] = ("with 16 vectors per call the inner FP16 products run on tcgen05: chunk_sum_launches "
                           "counts only the outer FP64 products' fixed-order sums, against one per inner product "
                           "on the CUDA cores")
    try:
        out["forward_error_vs_oracle"] = mixed_forward_error(dev)
    except Exception as ex:  # a sidecar: the headline line must still print
        out["forward_error_vs_oracle"] = {"error": str(ex)}
    out["accuracy"] = ("every form stops at ||d - K x|| <= tol ||d|| with K applied by the FP64-accurate "
                       "operator; forward_error_vs_oracle gives the error of x, m_map and q_map against the "
                       "oracle's dense solve at the first 42 time steps")
    return out


def digits_small(args):
    """The digit-plane tensor-core products at a small size for ncu captures: the batched
    workload's shapes (N_m = 4,096, N_d = 100) with N_t = 50 (n_f = 51, n = 5,000) and 64
    vectors; operator planes of 0.6 GB each, above L2.  Prints one JSON line of times."""
    import torch

    import paper_2501_14911_gb300 as bti
    from paper_2501_14911_gb300 import synthetic

    dev = torch.device("cuda", 0)
    p = synthetic.small("digits_small_Nm4096_Nd100_Nt50", 64, 64, 100, 50, Nq=32)
    h = bti.Handle(p.Nm, p.Nd, p.Nq, p.Nt, device=dev)
    h.set_blocks(bti.OP_F, torch.from_numpy(p.blocks_F()).to(dev), bti.DF64)
    h.set_prior_se_grid(p.gx, p.gy, p.ell, p.sigma_p, bti.DF64)
    h.set_noise(p.sigma2)
    h.set_dense_precision(bti.DF64)
    h.build_K(512)
    h.factor_K()
    h.invert_K()
    h.set_digit_planes(bti.OP_F, True)
    B = 64
    g = torch.Generator(device="cpu").manual_seed(5)
    d = torch.randn((B, p.Nt, p.Nd), generator=g, dtype=torch.float64).to(dev)
    m = torch.randn((B, p.Nt, p.Nm), generator=g, dtype=torch.float64).to(dev)
    x = torch.empty_like(d)
    calls = {"adjoint_FT": lambda: h.apply_FT(d, m), "forward_F": lambda: h.apply_F(m, x),
             "infer_map_explicit_inverse": lambda: h.infer_map(d, m)}
    for fn in calls.values():
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"case": p.name, "vectors": B}
    for name, fn in calls.items():
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        out[name + "_ms"] = e0.elapsed_time(e1)
    h.close()
    print(json.dumps(out))
    return 0


def online_batched(args):
    """The batched workload's online phase (N_m = 4,096, N_d = 100, N_t = 200, K 20,000^2): the
    tensor-core offline phase (Gram, Cholesky, K^{-1}, digit planes of G, Q), then the online graph
    with q_map = Q d_obs for 64 observation vectors at FP64 level and at FP32 level, and for one
    vector, each replayed 3 times after one warm-up.  Prints one JSON line of times (ms)."""
    import torch

    import paper_2501_14911_gb300 as bti
    from paper_2501_14911_gb300 import synthetic

    dev = torch.device("cuda", 0)
    p = synthetic.BATCHED
    h = bti.Handle(p.Nm, p.Nd, p.Nq, p.Nt, device=dev)
    h.set_blocks(bti.OP_F, torch.from_numpy(p.blocks_F()).to(dev), bti.DF64)
    h.set_blocks(bti.OP_FQ, torch.from_numpy(p.blocks_Fq()).to(dev), bti.DF64)
    h.set_prior_se_grid(p.gx, p.gy, p.ell, p.sigma_p, bti.DF64)
    h.set_noise(p.sigma2)
    h.set_dense_precision(bti.DF64)
    h.build_K(p.col_block)
    h.factor_K()
    h.invert_K()
    h.set_digit_planes(bti.OP_G, True)
    h.build_Q()
    h.set_online_qoi(True)
    B = p.n_vectors
    d = torch.from_numpy(p.vectors_d(B)).to(dev)
    m = torch.empty((B, p.Nt, p.Nm), dtype=torch.float64, device=dev)
    q = torch.empty((B, p.Nt, p.Nq), dtype=torch.float64, device=dev)
    gs = torch.cuda.Stream(device=dev)
    out = {"case": "online_batched_Nm4096_Nd100_Nt200", "vectors": B}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(gs):
        h.set_stream(gs)
        for key, nb, prec in (("fp64_level_ms", B, bti.DF64), ("fp32_level_ms", B, bti.F32),
                              ("one_vector_ms", 1, bti.DF64)):
            h.set_online_precision(prec)
            h.online(d[:nb], m[:nb], q[:nb])
            torch.cuda.synchronize()
            e0.record(gs)
            for _ in range(3):
                h.online(d[:nb], m[:nb], q[:nb])
            e1.record(gs)
            torch.cuda.synchronize()
            out[key] = e0.elapsed_time(e1) / 3
        h.set_online_precision(bti.DF64)
    torch.cuda.synchronize()
    h.set_stream(torch.cuda.current_stream(dev))
    h.close()
    print(json.dumps(out))
    return 0


def factor_small(args):
    """The tensor-core Cholesky and inverse at a small size for ncu captures: K of 8,192^2
    (N_m = 1,024, N_d = 64, N_t = 128, noise variance 1), factored as one panel by recursive
    halves (its largest update, the 64th digit-plane tile product, has K = 4,096) and inverted;
    0.5 GB for K and 0.8 GB of planes.  Prints one JSON line of times."""
    import torch

    import paper_2501_14911_gb300 as bti
    from paper_2501_14911_gb300 import synthetic

    dev = torch.device("cuda", 0)
    p = synthetic.small("factor_small_Nm1024_Nd64_Nt128", 32, 32, 64, 128, Nq=4, sigma2=1.0)
    h = bti.Handle(p.Nm, p.Nd, p.Nq, p.Nt, device=dev)
    h.set_blocks(bti.OP_F, torch.from_numpy(p.blocks_F()).to(dev), bti.DF64)
    h.set_prior_se_grid(p.gx, p.gy, 2.0, 1.0, bti.DF64)
    h.set_noise(p.sigma2)
    h.set_dense_precision(bti.DF64)
    h.set_factor_panel(1 << 20)
    h.build_K()
    torch.cuda.synchronize()
    out = {"case": p.name, "n": p.Nt * p.Nd}
    t0 = time.perf_counter()
    h.factor_K()
    out["factor_K_ms"] = 1e3 * (time.perf_counter() - t0)
    t0 = time.perf_counter()
    h.invert_K()
    out["invert_K_ms"] = 1e3 * (time.perf_counter() - t0)
    h.close()
    print(json.dumps(out))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.case == "digits_small":
        return digits_small(args)
    if args.case == "factor_small":
        return factor_small(args)
    if args.case == "online_batched":
        return online_batched(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
