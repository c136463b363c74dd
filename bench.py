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
    return ap.parse_args()


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
                                   f"scaled by (n/{ns})^3"},
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
            "sample": f"oracle CSD of one n={ns} instance of the same recipe ({t:.2f} s), scaled by (n/{ns})^3"}


def timed_run(args, B, ctx, A1, A2, out, dev, dist, local, profile):
    """W untimed steps, then K steps between barrier + synchronize, timed with
    CUDA events on the launching stream; returns (ms, last result, profile,
    clocks, launches)."""
    import torch

    def step():
        return ctx.csd_polar(A1, A2, out=out)

    R = None
    for _ in range(args.warmup):
        R = step()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    if profile:
        B.lib.csd_profile_enable(ctx._h, 1)
    launches0 = B.lib.csd_launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0.record(stream)
    for _ in range(args.steps):
        R = step()
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ck = clocks.stop()
    launches = B.lib.csd_launch_count() - launches0
    prof = B.csd_profile()
    if profile:
        B.lib.csd_profile_read(ctx._h, prof)
        B.lib.csd_profile_enable(ctx._h, 0)
    ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    return ms, R, prof, ck, launches


def accuracy(R, A1, A2, th_known, n, dev):
    """Angles against the generator's, backward error and orthogonality,
    computed with torch on the GPU (not with the oracle)."""
    import torch
    rk = R["rank"]
    th = R["theta"][:rk]
    c, s_ = torch.cos(th), torch.sin(th)
    U1, U2, V1 = (R[k][:, :rk] for k in ("U1", "U2", "V1"))
    num = torch.sqrt(torch.linalg.norm(A1 - (U1 * c) @ V1.T) ** 2 + torch.linalg.norm(A2 - (U2 * s_) @ V1.T) ** 2)
    bwd = float(num / np.sqrt(2.0 * n))  # ||A||_F = sqrt(n) for orthonormal columns
    ang = float(np.max(np.abs(th.cpu().numpy() - th_known)))
    # Frobenius norm (a plain reduction; the 2-norm would need torch's solver library)
    orth = max(float(torch.linalg.norm(X.T @ X - torch.eye(rk, device=dev, dtype=X.dtype))) for X in (U1, U2, V1))
    return {"max_abs_theta_err_vs_known": ang, "backward_err_fro_over_u": bwd / U, "orth_fro_over_u": orth / U,
            "rank": rk}


def main():
    args = parse()
    dist, rank, ws, local = dist_init()
    if args.impl == "reference":
        run_reference(args, rank, ws)
        if dist:
            dist.destroy_process_group()
        return
    import torch
    from paper_1804_09002_gb300 import binding as B
    from paper_1804_09002_gb300 import inputs as I

    # the CPU baseline runs the oracle in worker threads: do it before the
    # first GPU call (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args)

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    n = args.n
    A1h, A2h, th_known = I.clustered_csd(n, seed=2 + rank)
    colmaj = lambda a: torch.from_numpy(np.ascontiguousarray(a.T)).to(dev).t()
    A1, A2 = colmaj(A1h), colmaj(A2h)
    ctx = B.Context(local)
    ctx.set_tensor_cores(bool(args.tc))
    out = {k: torch.empty((n, n), dtype=torch.float64, device=dev).t() for k in ("U1", "U2", "V1")}
    out["theta"] = torch.empty(n, dtype=torch.float64, device=dev)

    # ---- headline path (inputs device-resident; A1, A2 = 256 MiB > L2)
    ms, R, prof, ck, launches = timed_run(args, B, ctx, A1, A2, out, dev, dist, local, True)
    s_per_csd = per_csd(ms, args.steps, ws)
    acc = accuracy(R, A1, A2, th_known, n, dev)
    # ---- the FP64-pipe path at the same backward-error bar, for comparison
    fp64 = None
    if args.tc and args.compare_fp64:
        ctx.set_tensor_cores(False)
        ms64, R64, _, ck64, _ = timed_run(args, B, ctx, A1, A2, out, dev, dist, local, False)
        fp64 = {"value": per_csd(ms64, args.steps, ws), "unit": "s/CSD",
                "tflops": FLOPS_PER_CSD(n) * args.steps * ws / (ms64 / 1e3) / 1e12,
                "accuracy": accuracy(R64, A1, A2, th_known, n, dev), "clocks": ck64}
        ctx.set_tensor_cores(True)
    # ---- e2e: same call with pinned host buffers (copies inside the call)
    e2e = None
    if args.e2e_steps > 0:
        A1p = torch.from_numpy(np.ascontiguousarray(A1h.T)).pin_memory().t()
        A2p = torch.from_numpy(np.ascontiguousarray(A2h.T)).pin_memory().t()
        outp = {k: torch.empty((n, n), dtype=torch.float64).pin_memory().t() for k in ("U1", "U2", "V1")}
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
        e2e = {"value": te, "unit": "s/CSD", "h2d_bytes_per_step": 2 * n * n * 8,
               "d2h_bytes_per_step": 3 * n * n * 8 + n * 8}
    # ---- roofline of the dominant kernel
    kinds = ["gemm", "qr_panel", "potrf", "jacobi", "tc_gemm"]
    kms = {k: prof.ms[i] for i, k in enumerate(kinds)}
    dom = max(range(5), key=lambda i: prof.ms[i])
    avg_ms = prof.ms[dom] / max(prof.count[dom], 1)
    flops_per_launch = prof.flops[dom] / max(prof.count[dom], 1)
    pk = peaks()
    if kinds[dom] == "tc_gemm":
        # 28 BF16 slice products per FP64-equivalent product, against the
        # measured dense BF16 peak (slicing and FP64 accumulation included in
        # the kernel time)
        peak = pk.get("bf16_tflops_sustained", 1719.1)
        achieved = 28.0 * flops_per_launch / (avg_ms / 1e3) / 1e12 if avg_ms > 0 else 0.0
        roof = {"kernel": "tc_gemm", "bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None,
                "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (of measured)",
                "fp64_equivalent_tflops": flops_per_launch / (avg_ms / 1e3) / 1e12 if avg_ms > 0 else 0.0}
    else:
        peak = fp64_alu_peak_tflops()
        achieved = flops_per_launch / (avg_ms / 1e3) / 1e12 if avg_ms > 0 else 0.0
        roof = {"kernel": kinds[dom], "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None,
                "peak_source": "FP64 FMA pipe: 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz"}
    products = ("tcgen05 tensor cores, exact BF16 slicing (FP64-accurate), FP64 pipe for the rest" if args.tc
                else "FP64 FMA pipe")
    line = {
        "metric": "s/CSD at n=4096 (FP64)", "value": s_per_csd, "unit": "s/CSD", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "tflops": FLOPS_PER_CSD(n) * args.steps * ws / (ms / 1e3) / 1e12,
        "tflops_frac_of_fp64_peak": FLOPS_PER_CSD(n) * args.steps * ws / (ms / 1e3) / 1e12 / fp64_alu_peak_tflops(),
        "config": {"workload": WORKLOAD(n),
                   "n": n, "parallelism": f"replicas x{ws}", "l2": "inputs larger than L2 (2 x 128 MiB)",
                   "products": products},
        "accuracy": acc,
        "roofline": roof,
        "kernel_ms_per_step": {k: v / args.steps for k, v in kms.items()},
        "gemm_sites": {nm: {"ms_per_step": prof.site_ms[i] / args.steps,
                            "tflops": prof.site_flops[i] / max(prof.site_ms[i], 1e-9) / 1e9,
                            "launches_per_step": prof.site_count[i] / args.steps}
                       for i, nm in enumerate(B.csd_profile.SITES) if prof.site_count[i]},
        "clocks": ck, "gpu_launches": int(launches),
    }
    if fp64:
        line["fp64_pipe_path"] = fp64
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
