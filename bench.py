"""Benchmark: seconds per CS decomposition (and TFLOP/s) at n = 4096, FP64.

Workload: real FP64 CSD of a 2n x n matrix with orthonormal columns, n = 4096,
theta half uniform on [0, pi/2], a quarter within 1e-8 of 0 and a quarter
within 1e-8 of pi/2, plus an additive 1e-14 Gaussian perturbation and
re-orthonormalisation (kappa(A_i) ~ 1e8 and beyond).  One step = one full
csd_polar call (two Zolo-pd polar decompositions, Zolo-eig of B = H2 - H1,
assembly of U1, U2, V1, theta) on device-resident inputs.  Throughput in
TFLOP/s counts the paper's 198 n^3 flops per CSD (Section 3, remark (v):
67 (m1 + m2) n^2 + 64 n^3 with m1 = m2 = n).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Multi-GPU (torchrun): every rank decomposes its own instance (replicas; the
path has no exchange step), value = total time / total CSDs.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FLOPS_PER_CSD = lambda n: 198.0 * n ** 3
WORKLOAD = lambda n: (f"real FP64 CSD n={n}, clustered theta (1/2 uniform, 1/4 within 1e-8 of 0, "
                      f"1/4 within 1e-8 of pi/2), 1e-14 noise, re-orthonormalised")
U = 2.0 ** -53


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sample-n", type=int, default=1024,
                    help="oracle sample size for the CPU baseline (about 20 s on 16 Grace cores)")
    ap.add_argument("--tc", type=int, default=1,
                    help="1 (default): real FP64 products on the tcgen05 tensor cores (exact BF16 slicing); 0: FP64 pipe")
    ap.add_argument("--compare-fp64", type=int, default=1,
                    help="with --tc 1, also time the FP64-pipe path (same workload, same accuracy checks)")
    ap.add_argument("--mixed-slices", type=int, default=6,
                    help="also time the mixed-precision path: Cholesky-iteration products with 5 or 6 BF16 slices "
                         "(0 = skip)")
    ap.add_argument("--mixed-scope", type=int, default=1,
                    help="bit 0: the two polar decompositions, bit 1: Zolo-eig's polar decompositions")
    ap.add_argument("--config", default="n4096", choices=list(CONFIGS),
                    help="n4096 (headline), n64 (median of 100 after 10), c2048 (complex rank 1536), n8192")
    ap.add_argument("--batch-count", type=int, default=1024, help="--mode batch: number of CSDs")
    ap.add_argument("--mode", default="csd", choices=["csd", "fp64-peak", "oracle-full", "gemm", "batch"],
                    help="fp64-peak: DFMA / mma.sync f64 microbenchmark; oracle-full: the CPU oracle once at full size")
    return ap.parse_args()


# workload configurations: (n, complex, rank or None, seed)
CONFIGS = {
    "n4096": dict(n=4096, cplx=False, rank=None, seed=2, kind="clustered"),
    "n64": dict(n=64, cplx=False, rank=None, seed=1, kind="haar"),
    "c2048": dict(n=2048, cplx=True, rank=1536, seed=3, kind="rankdef"),
    "n8192": dict(n=8192, cplx=False, rank=None, seed=4, kind="clustered"),
    "n1024": dict(n=1024, cplx=False, rank=None, seed=2, kind="clustered"),  # profiling case
}


def workload_name(cfg):
    n = cfg["n"]
    if cfg["kind"] == "clustered":
        return WORKLOAD(n)
    if cfg["kind"] == "haar":
        return f"real FP64 CSD n={n}, Haar U1, U2, V, theta i.i.d. U[0, pi/2]"
    return (f"complex128 partial isometry n={n}, rank {cfg['rank']} ({n - cfg['rank']} zero (C, S) pairs), "
            f"256 exactly repeated angles, the rest U[0, pi/2] (Algorithm 3)")


def make_inputs(cfg, rank_offset=0):
    from paper_1804_09002_gb300 import inputs as I
    n, seed = cfg["n"], cfg["seed"] + rank_offset
    if cfg["kind"] == "clustered":
        return I.clustered_csd(n, seed=seed)
    if cfg["kind"] == "haar":
        return I.haar_csd(n, seed=seed)
    return I.rankdef_csd(n, cfg["rank"], seed=seed, cplx=True, n_repeat=256)


def flops_per_csd(cfg):
    return FLOPS_PER_CSD(cfg["n"]) * (4.0 if cfg["cplx"] else 1.0)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def fp64_alu_peak_tflops():
    """FP64 FMA pipe peak from unit counts and clocks: 152 SMs x 2 DFMA/clk x
    2 flop x 2070 MHz = 1.2586 TFLOP/s (our DFMA microbenchmark measured
    1.195 TFLOP/s at 1995 MHz, i.e. 2.0 DFMA/clk/SM)."""
    return 152 * 2 * 2 * 2070e6 / 1e12


def max_over_ranks(value, dist, device="cpu"):
    """The largest value over the ranks: the slowest rank times the job."""
    if not dist:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def per_csd(ms, steps, ws):
    """Whole-job seconds per CSD: ws ranks each ran `steps` CSDs in `ms`
    (max over ranks) milliseconds."""
    return ms / 1e3 / (steps * ws)


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl"
        dist.init_process_group(backend=backend)
        return dist, dist.get_rank(), ws, int(os.environ.get("LOCAL_RANK", "0"))
    return None, 0, 1, 0


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def run_reference(args, rank, ws):
    """Reference arm: the CPU FP64 oracle (Jacobi SVD polar + cyclic Jacobi
    eig, OpenMP) on a bounded sample -- an instance of the same recipe at
    n = sample_n -- scaled to n by (n / sample_n)^3."""
    if rank != 0:
        return
    from oracle import csd as O
    from oracle import jacobi as OJ
    from paper_1804_09002_gb300 import inputs as I
    ns = args.sample_n
    A1, A2, _ = I.clustered_csd(ns, seed=2)
    for _ in range(args.warmup):
        O.csd(A1, A2)
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        O.csd(A1, A2)
        ts.append(time.perf_counter() - t0)
    scale = (args.n / ns) ** 3
    t = statistics.median(ts) * scale
    line = {
        "impl": "reference", "metric": "s/CSD at n=4096 (FP64)", "value": t, "unit": "s/CSD",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "tflops": FLOPS_PER_CSD(args.n) / t / 1e12,
        "config": {"workload": WORKLOAD(args.n), "n": args.n, "parallelism": "replicas x1",
                   "l2": "inputs larger than L2 (2 x 128 MiB)",
                   "products": "CPU oracle (one-sided Jacobi SVD polar, cyclic Jacobi eig), FP64"},
        "cpu_baseline": {"value": t, "unit": "s/CSD", "cores": OJ.threads(), "kind": "oracle",
                         "sample": f"oracle CSD of an n={ns} instance of the same recipe, median of {args.steps}, "
                                   f"scaled by (n/{ns})^3",
                         "full_size_measured": ORACLE_FULL if args.n == ORACLE_FULL["n"] else None},
        "e2e": {"value": t, "unit": "s/CSD", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(args):
    from oracle import csd as O
    from oracle import jacobi as OJ
    from paper_1804_09002_gb300 import inputs as I
    ns = args.sample_n
    A1, A2, _ = I.clustered_csd(ns, seed=2)
    t0 = time.perf_counter()
    O.csd(A1, A2)
    t = time.perf_counter() - t0
    return {"value": t * (args.n / ns) ** 3, "unit": "s/CSD", "cores": OJ.threads(), "kind": "oracle",
            "sample": f"oracle CSD of one n={ns} instance of the same recipe ({t:.2f} s), scaled by (n/{ns})^3",
            "extrapolated": True,
            "full_size_measured": ORACLE_FULL if args.n == ORACLE_FULL["n"] else None}


# The oracle timed once at full size on the GPU machine's host cores
# (`bench.py --mode oracle-full`, 16 Neoverse-V2 cores, aarch64): too long
# (about 19 minutes) to repeat inside every bench run.
ORACLE_FULL = {"n": 4096, "value": 1152.8, "unit": "s/CSD", "cores": 16, "cpu": "Neoverse-V2",
               "command": "python bench.py --mode oracle-full"}


def timed_run(args, B, ctx, A1, A2, out, dev, dist, local, profile, steps=None, warmup=None):
    """W untimed steps, then K steps between barrier + synchronize, timed with
    CUDA events on the launching stream (one event pair per step as well);
    returns (ms total, per-step ms, last result, profile, clocks, launches).
    With `profile`, every product launch is bracketed by CUDA events (the
    per-kernel accounting of the roofline); the headline runs without."""
    import torch
    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup

    def step():
        return ctx.csd_polar(A1, A2, out=out)

    R = None
    for _ in range(warmup):
        R = step()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    clocks = ClockSampler(local)
    if profile:
        B.lib.csd_profile_enable(ctx._h, 1)
    launches0 = B.lib.csd_launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev[0].record(stream)
    for i in range(steps):
        R = step()
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ck = clocks.stop()
    launches = B.lib.csd_launch_count() - launches0
    prof = B.csd_profile()
    if profile:
        B.lib.csd_profile_read(ctx._h, prof)
        B.lib.csd_profile_enable(ctx._h, 0)
    per = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
    ms = max_over_ranks(ev[0].elapsed_time(ev[steps]), dist, dev)
    return ms, per, R, prof, ck, launches


def _norm2_sym(E, iters=60):
    """2-norm of a Hermitian E by power iteration (matrix products only)."""
    import torch
    g = torch.Generator(device=E.device).manual_seed(0)
    v = torch.randn(E.shape[0], 1, dtype=torch.float64, device=E.device, generator=g).to(E.dtype)
    lam = 0.0
    for _ in range(iters):
        w = E @ v
        lam = float(torch.linalg.norm(w))
        if lam == 0.0:
            return 0.0
        v = w / lam
    return lam


def accuracy(R, A1, A2, th_known, n, dev):
    """Angles against the generator's, backward error and orthogonality
    (Frobenius and 2-norm), computed with torch on the GPU (not with the
    oracle)."""
    import torch
    rk = R["rank"]
    th = R["theta"][:rk]
    U1, U2, V1 = (R[k][:, :rk] for k in ("U1", "U2", "V1"))
    c, s_ = torch.cos(th).to(U1.dtype), torch.sin(th).to(U1.dtype)
    Vh = V1.conj().T
    num = torch.sqrt(torch.linalg.norm(A1 - (U1 * c) @ Vh) ** 2 + torch.linalg.norm(A2 - (U2 * s_) @ Vh) ** 2)
    den = torch.sqrt(torch.linalg.norm(A1) ** 2 + torch.linalg.norm(A2) ** 2)
    bwd = float(num / den)
    ang = float(np.max(np.abs(th.cpu().numpy() - th_known)))
    eye = torch.eye(rk, device=dev, dtype=U1.dtype)
    orth = max(float(torch.linalg.norm(X.conj().T @ X - eye)) for X in (U1, U2, V1))
    orth2 = max(_norm2_sym(X.conj().T @ X - eye) for X in (U1, U2, V1))
    return {"max_abs_theta_err_vs_known": ang, "backward_err_fro_over_u": bwd / U, "orth_fro_over_u": orth / U,
            "orth_2norm_over_u": orth2 / U, "rank": rk, "bar_over_u": 50 * n}


# DRAM traffic of the tensor-core product kernel per launch, from one ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum over every launch of
# the kernel in one step), with the hash of the kernel source it was taken
# at; reported only while tc_gemm.cu is unchanged since the capture.
TRAFFIC = {"tc_gemm": {"bytes_per_launch": 289092468, "src_hash": "60e10541738decac",
                      "profile": "profiles/tc_gemm_kernel_csd_n4096_traffic.md"}}


def _src_hash(name):
    import hashlib
    with open(os.path.join(ROOT, "paper_1804_09002_gb300", "csrc", name), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def traffic_for(kernel):
    t = TRAFFIC.get(kernel)
    if not t or t.get("src_hash") != _src_hash("tc_gemm.cu"):
        return None, None
    return t["bytes_per_launch"], t["profile"]


def run_fp64_peak(args):
    from paper_1804_09002_gb300 import binding as B
    ck = ClockSampler(0)
    ck.start()
    dfma, ms0 = B.fp64_peak(0)
    dmma, ms1 = B.fp64_peak(1)
    clocks = ck.stop()
    print(json.dumps({"mode": "fp64-peak", "dfma_tflops": dfma, "dmma_tflops": dmma, "dfma_best_ms": ms0,
                      "dmma_best_ms": ms1, "unit_count_peak_tflops": fp64_alu_peak_tflops(), "clocks": clocks}),
          flush=True)


def run_gemm(args):
    """The product kernels alone: C = A B with n x n x n real FP64 operands
    (N(0,1) entries, 3 x 8 n^2 bytes > L2 at n = 4096) through csd_gemm, on
    the tensor-core kernel (engine 1) and on the FP64 pipe (engine 0)."""
    import torch
    from paper_1804_09002_gb300 import binding as B
    n = args.n
    dev = torch.device("cuda", 0)
    g = torch.Generator(device=dev).manual_seed(1)
    A = torch.randn(n, n, dtype=torch.float64, device=dev, generator=g).t()
    Bm = torch.randn(n, n, dtype=torch.float64, device=dev, generator=g).t()
    C = torch.zeros(n, n, dtype=torch.float64, device=dev).t()
    ctx = B.Context(0)
    res = {}
    for engine in ([1, 0] if args.compare_fp64 else [1]):
        for _ in range(args.warmup):
            ctx.gemm(A, Bm, C, engine=engine)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        torch.cuda.synchronize()
        ev[0].record()
        for i in range(args.steps):
            ctx.gemm(A, Bm, C, engine=engine)
            ev[i + 1].record()
        torch.cuda.synchronize()
        ms = statistics.median(ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps))
        fl = 2.0 * n ** 3
        res["tensor_cores" if engine else "fp64_pipe"] = {
            "ms": ms, "fp64_equivalent_tflops": fl / ms / 1e9,
            **({"bf16_slice_tflops": 28 * fl / ms / 1e9,
                "frac_of_bf16_sustained": 28 * fl / ms / 1e9 / peaks().get("bf16_tflops_sustained", 1719.1)}
               if engine else {"frac_of_fp64_unit_peak": fl / ms / 1e9 / fp64_alu_peak_tflops()})}
    err = float(torch.max(torch.abs(C - A @ Bm)))
    ctx.close()
    print(json.dumps({"mode": "gemm", "n": n, "steps": args.steps, "max_abs_diff_vs_torch": err, **res}), flush=True)


def run_batch(args):
    """Config 5's forward: `--batch-count` real FP64 CSDs with n drawn from
    U{16..256} (theta uniform, seeds 5000 + i) in one autotuned,
    graph-captured batch (csd_batch_*); time per batch with CUDA events over
    K replays (inputs resident in HBM), Sigma 198 n_i^3 flops."""
    import torch
    from paper_1804_09002_gb300 import binding as B
    from paper_1804_09002_gb300 import inputs as I
    rng = np.random.default_rng(5)
    sizes = [int(v) for v in rng.integers(16, 257, args.batch_count)]
    dev = torch.device("cuda", 0)
    data = [I.haar_csd(n, seed=5000 + i) for i, n in enumerate(sizes)]
    ctx = B.Context(0)
    plan = B.Batch(ctx, sizes)
    plan.load([torch.from_numpy(np.ascontiguousarray(d[0].T)).to(dev).t() for d in data],
              [torch.from_numpy(np.ascontiguousarray(d[1].T)).to(dev).t() for d in data])
    t0 = time.perf_counter()
    plan.run()  # autotune + capture
    setup_s = time.perf_counter() - t0
    for _ in range(args.warmup):
        plan.run()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    clocks = ClockSampler(0)
    torch.cuda.synchronize()
    clocks.start()
    ev[0].record()
    for i in range(args.steps):
        plan.run()
        ev[i + 1].record()
    torch.cuda.synchronize()
    ck = clocks.stop()
    per = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    ms = statistics.median(per)
    fl = sum(198.0 * n ** 3 for n in sizes)
    worst_be = worst_th = 0.0
    for i, (n, d) in enumerate(zip(sizes, data)):
        R = plan.result(i)
        th = R["theta"]
        c, s_ = torch.cos(th), torch.sin(th)
        A1 = torch.from_numpy(d[0]).to(dev)
        A2 = torch.from_numpy(d[1]).to(dev)
        num = torch.sqrt(torch.linalg.norm(A1 - (R["U1"] * c) @ R["V1"].T) ** 2 +
                         torch.linalg.norm(A2 - (R["U2"] * s_) @ R["V1"].T) ** 2)
        worst_be = max(worst_be, float(num) / np.sqrt(n) / (n * U))
        worst_th = max(worst_th, float(np.max(np.abs(th.cpu().numpy() - d[2]))) / n)
    print(json.dumps({"mode": "batch", "metric": "s per batch of CSDs", "value": ms / 1e3, "unit": "s/batch",
                      "count": len(sizes), "sizes": "n ~ U{16..256}", "csd_per_s": len(sizes) / (ms / 1e3),
                      "tflops": fl / (ms / 1e3) / 1e12, "flops": fl, "steps": args.steps,
                      "setup_s_autotune_and_capture": setup_s, "autotuner": plan.stats(),
                      "status_ok": int(np.sum(plan.status == 0)),
                      "worst_backward_err_over_nu": worst_be, "worst_theta_err_vs_known_over_n": worst_th,
                      "clocks": ck}), flush=True)
    plan.close()
    ctx.close()


def run_oracle_full(args):
    """The CPU oracle once at the full size of --config (no extrapolation)."""
    import platform
    from oracle import csd as O
    from oracle import jacobi as OJ
    cfg = CONFIGS[args.config]
    A1, A2, _ = make_inputs(cfg)
    t0 = time.perf_counter()
    O.csd(A1, A2)
    t = time.perf_counter() - t0
    model = ""
    try:
        model = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        model = [ln.split(":", 1)[1].strip() for ln in model.splitlines() if ln.startswith("Model name")][0]
    except Exception:
        pass
    print(json.dumps({"mode": "oracle-full", "config": {"workload": workload_name(cfg), "n": cfg["n"]},
                      "value": t, "unit": "s/CSD", "cores": OJ.threads(), "nproc": os.cpu_count(),
                      "cpu_model": model, "machine": platform.machine()}), flush=True)


def main():
    args = parse()
    dist, rank, ws, local = dist_init()
    if args.impl == "reference":
        run_reference(args, rank, ws)
        if dist:
            dist.destroy_process_group()
        return
    if args.mode == "fp64-peak":
        run_fp64_peak(args)
        return
    if args.mode == "oracle-full":
        run_oracle_full(args)
        return
    if args.mode == "gemm":
        run_gemm(args)
        return
    if args.mode == "batch":
        run_batch(args)
        return
    import torch
    from paper_1804_09002_gb300 import binding as B

    cfg = CONFIGS[args.config]
    headline = args.config == "n4096"
    if args.config == "n64":  # latency case: median of 100 steps after 10 warm-up
        args.steps = max(args.steps, 100)
        args.warmup = max(args.warmup, 10)
    # the CPU baseline runs the oracle in worker threads: do it before the
    # first GPU call (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and headline:
        cpu = cpu_baseline(args)

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    n = cfg["n"]
    tdt = torch.complex128 if cfg["cplx"] else torch.float64
    A1h, A2h, th_known = make_inputs(cfg, rank)
    colmaj = lambda a: torch.from_numpy(np.ascontiguousarray(a.T)).to(dev).t()
    A1, A2 = colmaj(A1h), colmaj(A2h)
    ctx = B.Context(local)
    ctx.set_tensor_cores(bool(args.tc))
    out = {k: torch.empty((n, n), dtype=tdt, device=dev).t() for k in ("U1", "U2", "V1")}
    out["theta"] = torch.empty(n, dtype=torch.float64, device=dev)
    fl = flops_per_csd(cfg)

    # ---- headline: profiler off, inputs device-resident
    ms, per, R, _, ck, launches = timed_run(args, B, ctx, A1, A2, out, dev, dist, local, False)
    s_per_csd = per_csd(ms, args.steps, ws)
    if args.config == "n64":
        s_per_csd = statistics.median(per) / 1e3 / ws
    acc = accuracy(R, A1, A2, th_known, n, dev)
    # ---- one profiled step (CUDA events around every product launch): the
    # per-kernel and per-site accounting behind the roofline
    pms, _, _, prof, _, _ = timed_run(args, B, ctx, A1, A2, out, dev, dist, local, True, steps=1, warmup=0)
    # ---- the FP64-pipe path at the same backward-error bar, for comparison
    fp64 = None
    if args.tc and args.compare_fp64 and not cfg["cplx"]:
        ctx.set_tensor_cores(False)
        k64 = 1 if n >= 8192 else args.steps
        ms64, per64, R64, _, ck64, _ = timed_run(args, B, ctx, A1, A2, out, dev, dist, local, False,
                                               steps=k64, warmup=1)
        v64 = per_csd(ms64, k64, ws) if args.config != "n64" else statistics.median(per64) / 1e3 / ws
        fp64 = {"value": v64, "unit": "s/CSD", "tflops": fl / v64 / 1e12, "steps": k64,
                "accuracy": accuracy(R64, A1, A2, th_known, n, dev), "clocks": ck64}
        ctx.set_tensor_cores(bool(args.tc))
    # ---- mixed precision (fewer slices in the well-conditioned Cholesky
    # iteration), same workload and accuracy checks
    mixed = None
    if args.tc and args.mixed_slices in (5, 6) and not cfg["cplx"]:
        ctx.set_mixed_precision(args.mixed_slices, args.mixed_scope)
        kmx = 1 if n >= 8192 else args.steps
        msx, perx, Rx, _, ckx, _ = timed_run(args, B, ctx, A1, A2, out, dev, dist, local, False, steps=kmx,
                                             warmup=1)
        vx = per_csd(msx, kmx, ws) if args.config != "n64" else statistics.median(perx) / 1e3 / ws
        mixed = {"value": vx, "unit": "s/CSD", "tflops": fl / vx / 1e12, "steps": kmx,
                 "slices": args.mixed_slices, "scope": args.mixed_scope,
                 "accuracy": accuracy(Rx, A1, A2, th_known, n, dev), "clocks": ckx,
                 "what": "Gram and triangular-solve products of the Cholesky-form Zolo-pd iteration with "
                         f"{args.mixed_slices} BF16 slices; everything else FP64-accurate (7 slices)"}
        ctx.set_mixed_precision(7, 0)
    # ---- e2e: same call with pinned host buffers (copies inside the call)
    e2e = None
    if args.e2e_steps > 0:
        A1p = torch.from_numpy(np.ascontiguousarray(A1h.T)).pin_memory().t()
        A2p = torch.from_numpy(np.ascontiguousarray(A2h.T)).pin_memory().t()
        outp = {k: torch.empty((n, n), dtype=tdt).pin_memory().t() for k in ("U1", "U2", "V1")}
        outp["theta"] = torch.empty(n, dtype=torch.float64).pin_memory()
        ctx.csd_polar(A1p, A2p, out=outp)  # warm the host-buffer path
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            ctx.csd_polar(A1p, A2p, out=outp)
        torch.cuda.synchronize()
        # whole job: the slowest rank's wall time over all ranks' CSDs
        te = max_over_ranks(time.perf_counter() - t0, dist, dev) / (args.e2e_steps * ws)
        es = 16 if cfg["cplx"] else 8
        e2e = {"value": te, "unit": "s/CSD", "h2d_bytes_per_step": 2 * n * n * es,
               "d2h_bytes_per_step": 3 * n * n * es + n * 8}
    # ---- roofline of the dominant kernel (from the profiled step)
    kinds = ["gemm", "qr_panel", "potrf", "jacobi", "tc_gemm"]
    kms = {k: prof.ms[i] for i, k in enumerate(kinds)}
    dom = max(range(5), key=lambda i: prof.ms[i])
    avg_ms = prof.ms[dom] / max(prof.count[dom], 1)
    flops_per_launch = prof.flops[dom] / max(prof.count[dom], 1)
    pk = peaks()
    if kinds[dom] == "tc_gemm":
        # 28 BF16 slice products per FP64-equivalent product, against the
        # measured dense BF16 peak (slicing included in the kernel time)
        peak = pk.get("bf16_tflops_sustained", 1719.1)
        fp64eq = flops_per_launch / (avg_ms / 1e3) / 1e12 if avg_ms > 0 else 0.0
        achieved = 28.0 * fp64eq
        tr, tr_src = traffic_for("tc_gemm")
        roof = {"kernel": "tc_gemm", "bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": tr, "traffic_source": tr_src,
                "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (of measured)",
                "launches_per_step": prof.count[dom], "avg_launch_ms": avg_ms,
                "fp64_equivalent_tflops": fp64eq, "method_frac_of_bf16_peak": fp64eq / peak,
                "work_per_launch": "28 x 2mnk BF16 slice flops (2mnk FP64-equivalent) over the tiles executed"}
    else:
        peak = fp64_alu_peak_tflops()
        achieved = flops_per_launch / (avg_ms / 1e3) / 1e12 if avg_ms > 0 else 0.0
        roof = {"kernel": kinds[dom], "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None,
                "peak_source": "FP64 FMA pipe: 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz"}
    products = ("tcgen05 tensor cores, exact BF16 slicing (FP64-accurate), FP64 pipe for the rest" if args.tc
                and not cfg["cplx"] else "FP64 FMA pipe")
    metric = f"s/CSD at n={n} ({'complex128' if cfg['cplx'] else 'FP64'})"
    line = {
        "metric": metric, "value": s_per_csd, "unit": "s/CSD", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "c128" if cfg["cplx"] else "f64", "data": "synthetic",
        "tflops": fl / s_per_csd / 1e12,
        "tflops_frac_of_fp64_peak": fl / s_per_csd / 1e12 / fp64_alu_peak_tflops(),
        "config": {"workload": workload_name(cfg), "n": n, "parallelism": f"replicas x{ws}",
                   "l2": ("inputs larger than L2" if 2 * n * n * (16 if cfg["cplx"] else 8) > 129e6
                          else "inputs smaller than L2 (latency case)"),
                   "products": products, "timing": ("median of per-step CUDA-event times" if args.config == "n64"
                                                    else "CUDA events around K steps, profiler off")},
        "accuracy": acc,
        "roofline": roof,
        "profiled_step": {"value": pms / 1e3, "unit": "s/CSD",
                          "note": "one step with CUDA events around every product launch (roofline, sites)"},
        "kernel_ms_per_step": kms,
        "gemm_sites": {nm: {"ms_per_step": prof.site_ms[i],
                            "tflops": prof.site_flops[i] / max(prof.site_ms[i], 1e-9) / 1e9,
                            "launches_per_step": prof.site_count[i]}
                       for i, nm in enumerate(B.csd_profile.SITES) if prof.site_count[i]},
        "clocks": ck, "gpu_launches": int(launches), "launches_per_csd": launches / args.steps,
    }
    if fp64:
        line["fp64_pipe_path"] = fp64
    if mixed:
        line["mixed_precision_path"] = mixed
    if e2e:
        line["e2e"] = e2e
    if cpu:
        line["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
