"""Benchmark of the ADASAP hot path on B300 (one JSON line on rank 0).

A step is one full ADASAP iteration (Alg. 2: sample, Step I block residual,
Step II sketch, Alg. 4 Nystrom core, Alg. 5 stepsize, Step IV direction and
Alg. 6 update) on the regression workload: n = 2^20, d = 11, X ~ U[0,1]^11,
Matern-3/2, ell = 0.3, lambda = 1e-3, b = 10^4, r = 100, one right-hand side
(synthetic stand-in for the paper's regression datasets).

value: kernel entries k(x_i, x_j) evaluated per second over whole iterations
  (b n for Step I, b^2 for the sketch, N b^2 for the N powering products).
roofline: the fused kernel-row product (Step I's kernel) timed alone with CUDA
  events; its peak is the special-function-pipe bound at the issue rates
  measured on the GPU (adasap_measure_pipes), the SMs and the SM clock sampled
  during the kernel (Matern needs sqrt + ex2 per entry, RBF ex2 only).
e2e: the same entries through the C-ABI with host buffers (create + solve +
  copy-back inside the timed region).
cpu_baseline / --impl reference: the FP64 oracle's block-row product on a
  bounded row sample of the same workload, on the host.

Launch: python bench.py [--gpus N --steps K --warmup W]; for N > 1 under
torchrun each rank runs an independent replica ("replicas only": every box has
one GPU per call) and rank 0 reports the aggregate.
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

METRIC = "ADASAP s to rel-resid 1e-3 (mixed vs FP32); kernel-row Gentries/s, % roofline"
UNIT = "Gentries/s"


# DRAM bytes per kernel entry of k_rows_tc (Step I shape, s = 1): dram__bytes_read.sum +
# dram__bytes_write.sum of one ncu-captured launch at 10,000 x 262,144 entries, Matern-3/2
TC_DRAM_BYTES_PER_ENTRY = (39.048704e6 + 33.792e3) / (10000 * 262144)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-tol-run", action="store_true")
    p.add_argument("--no-multi-rhs", action="store_true", help="skip the many-right-hand-sides comparison")
    p.add_argument("--no-batched", action="store_true", help="skip the uneven batch of independent systems")
    p.add_argument("--batched-iters", type=int, default=40, help="iterations of the batched-systems timing")
    p.add_argument("--no-pathwise", action="store_true", help="skip the pathwise posterior-sampling timing")
    p.add_argument("--no-sap", action="store_true", help="skip the exact-block-solve SAP timing")
    p.add_argument("--no-taxi", action="store_true", help="skip the n = 2^25 mixed-vs-FP32 iteration timing")
    p.add_argument("--taxi-iters", type=int, default=3, help="timed iterations per precision at n = 2^25")
    p.add_argument("--mrhs-tol", type=float, default=0.8,
                   help="Frobenius relative residual of the many-right-hand-sides time-to-tolerance comparison")
    p.add_argument("--n", type=int, default=1 << 20, help="rows of the workload (default: full size)")
    p.add_argument("--kernel-launches", type=int, default=10, help="timed launches of the Step I kernel alone")
    p.add_argument("--tol-iters", type=int, default=6000, help="iteration cap of the time-to-1e-3 solves")
    p.add_argument("--only-kernel", action="store_true",
                   help="run only the Step I block-row product launches (profiling)")
    p.add_argument("--kern", choices=["rbf", "matern32", "matern52"], default="matern32",
                   help="covariance kernel of the --only-kernel launches (the workload's own: matern32)")
    p.add_argument("--only-workload", choices=["multirhs", "bo"],
                   help="run only --warmup + --steps iterations of that workload's solver (profiling)")
    return p.parse_args()


def workload(n):
    from paper_2505_13723_b300 import synth
    return synth.regress(n=n, b=min(10000, n // 4))


def entries_per_step(P, power_iters=10):
    n, b = P.X.shape[0], P.b
    return b * n + b * b + power_iters * b * b


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- CPU oracle
def host_cores():
    """Host cores this process may run on (its CPU affinity set)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_rows_rate(P, target_s=10.0, max_rows=None, threads=None):
    """Entries/s of the oracle's block-row product (FP64 NumPy) on sampled rows.

    The sampled rows are cut into one group per thread and each thread runs the
    oracle's kernel_rows on its group (NumPy releases the interpreter lock in the
    elementwise work, so the threads run on separate cores); BLAS is held to one
    thread inside each so that the host cores are not oversubscribed.
    Returns (entries/s, rows, seconds, threads)."""
    import contextlib
    from concurrent.futures import ThreadPoolExecutor

    try:
        from threadpoolctl import threadpool_limits
    except ImportError:   # not on every host: the oracle's one BLAS call is a small matrix-vector product
        def threadpool_limits(_):
            return contextlib.nullcontext()

    from oracle import kernels as OK
    X = P.X.astype(np.float64)
    W = P.Y.astype(np.float64)
    n = X.shape[0]
    threads = max(1, min(threads or host_cores(), 64))
    g = np.random.default_rng(0)
    with threadpool_limits(1), ThreadPoolExecutor(threads) as pool:
        probe = g.choice(n, size=threads, replace=False)
        t0 = time.perf_counter()
        list(pool.map(lambda r: OK.kernel_rows(X, [r], W, P.kernel, P.ell, P.sigma2), probe))
        per_row = (time.perf_counter() - t0) / threads     # wall time per row with all threads busy
        k = max(threads, int(target_s / max(per_row, 1e-6)))
        if max_rows:
            k = max(1, min(k, max_rows))
        rows = g.choice(n, size=k, replace=False)
        groups = [grp for grp in np.array_split(rows, min(threads, k)) if len(grp)]
        t0 = time.perf_counter()
        list(pool.map(lambda grp: OK.kernel_rows(X, grp, W, P.kernel, P.ell, P.sigma2), groups))
        dt = time.perf_counter() - t0
    return k * n / dt, k, dt, len(groups)


def run_reference(args, rank, world):
    if rank != 0:
        return
    P = workload(args.n)
    n = P.X.shape[0]
    for _ in range(args.warmup):
        oracle_rows_rate(P, target_s=0.5, max_rows=2)
    rates, tot_rows, tot_t, used = [], 0, 0.0, 1
    t_all = time.perf_counter()
    for _ in range(args.steps):
        rate, k, dt, used = oracle_rows_rate(P, target_s=5.0)
        rates.append(rate)
        tot_rows += k
        tot_t += dt
    value = tot_rows * n / tot_t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(P),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle",
                             "sample": "FP64 NumPy block-row product K(X_B, X) w on %d sampled rows x n=%d per "
                                       "step (%.1f s per step), rows split over %d threads (host affinity set: "
                                       "%d cores)" % (tot_rows // args.steps, n, tot_t / args.steps, used,
                                                      host_cores())},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t_all}
    print(json.dumps(line), flush=True)


# TF32 dense tensor rate relative to BF16 (nominal dense figures of this GPU: 1.1 and 2.25 PFLOP/s)
TF32_PER_BF16 = 1.1 / 2.25


def mrhs_roofline(entries, d, s, ms, pk, pk_src, pipes, sms, mhz):
    """Roofline of the multi-RHS block-row product (k_rows_tc_mrhs, RBF) at s right-hand sides.

    Algorithmic work per kernel entry: 2 d flops of distance and 2 s flops of contraction,
    both on the tensor pipe, plus one ex2 on the special-function pipe.  The tensor peak is
    TF32: the measured BF16 dense rate times the nominal TF32 / BF16 ratio.  The kernel
    executes more than the algorithmic flops: three TF32 passes (hi/lo split, FP32
    accuracy) of 2 (KP + s_pad) flops per entry with KP = 16 or 32 and s_pad = s rounded
    up to 16, or one pass in the single-pass TF32 mode; both are reported."""
    kp = 16 if d + 2 <= 16 else 32
    s_pad = (s + 15) // 16 * 16
    alg = 2.0 * d + 2.0 * s
    tf32_peak = pk["bf16_tflops"] * TF32_PER_BF16 * 1e12
    sfu_peak = sms * mhz * 1e6 * pipes["ex2"]
    t = ms["tf32x3"] * 1e-3
    out = {"bound": "tensor", "unit": "TFLOP/s",
           "achieved": alg * entries / t / 1e12, "peak": tf32_peak / 1e12,
           "frac": alg * entries / t / tf32_peak, "traffic": None,
           "kernel": "k_rows_tc_mrhs (tcgen05 TF32x3 distances and contraction), b x n = %d entries, s = %d"
                     % (entries, s),
           "ms_per_launch": ms["tf32x3"],
           "flops_per_entry_algorithmic": alg,
           "peak_basis": "TF32 dense = %s BF16 burst %.1f TFLOP/s x %.3f (nominal TF32 / BF16)"
                         % (pk_src, pk["bf16_tflops"], TF32_PER_BF16),
           "executed_tf32x3": {"flops_per_entry": 3 * 2.0 * (kp + s_pad),
                               "tflops": 3 * 2.0 * (kp + s_pad) * entries / t / 1e12,
                               "frac_of_tf32_peak": 3 * 2.0 * (kp + s_pad) * entries / t / tf32_peak},
           "special_function_pipe": {"entries_per_s": entries / t, "peak_entries_per_s": sfu_peak,
                                     "frac": entries / t / sfu_peak,
                                     "basis": "1 ex2 per entry at %.1f per SM per clock (adasap_measure_pipes)"
                                              % pipes["ex2"]}}
    if "tf32" in ms:
        t1 = ms["tf32"] * 1e-3
        out["single_pass_tf32"] = {"ms_per_launch": ms["tf32"],
                                   "flops_per_entry_executed": 2.0 * (3 * kp + s_pad),
                                   "frac_of_tf32_peak_executed": 2.0 * (3 * kp + s_pad) * entries / t1 / tf32_peak}
    return out


def config_dict(P):
    return {"workload": "regress: n=%d, d=11, X~U[0,1]^11, Matern-3/2 ell=0.3, lambda=1e-3, b=%d, r=100, s=1"
                        % (P.X.shape[0], P.b),
            "n": int(P.X.shape[0]), "d": 11, "kernel": "matern32", "b": int(P.b), "r": 100, "s": 1,
            "power_iters": 10, "l2": "flushed between timed steps",
            "parallelism": "replicas"}


def whole_job(t_local, units_local, dist, device):
    """(max over ranks of the timed seconds, sum over ranks of the units processed).

    Every rank is an independent replica (weak scaling), so the whole-job rate is
    the units all ranks processed over the slowest rank's time."""
    if dist is None:
        return t_local, units_local
    import torch
    t = torch.tensor([t_local], device=device, dtype=torch.float64)
    u = torch.tensor([units_local], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


# ----------------------------------------------------------------------------- GPU arm
def run_workload_only(args):
    """Iterations of one secondary workload alone (for launch lists under ncu): the multirhs
    solve (s = 64, split precision) or the bo batch (48 systems in one graph)."""
    import torch

    from paper_2505_13723_b300 import binding as lib
    from paper_2505_13723_b300 import synth
    dev = torch.device("cuda", 0)
    t0 = time.perf_counter()
    if args.only_workload == "multirhs":
        Q = synth.multirhs()
        cq = lib.Context(torch.from_numpy(Q.X).to(dev), Q.kernel, Q.ell, Q.sigma2, Q.lam)
        so = lib.Solver(cq, torch.from_numpy(Q.Y).to(dev),
                        opts=lib.default_opts(Q.X.shape[0], b=Q.b, r=Q.r, seed=3, check_every=0,
                                              max_iters=args.warmup + args.steps))
        so.step(args.warmup + args.steps)
        torch.cuda.synchronize()
        kernels = so.graph_kernels()
        so.close()
    else:
        systems = synth.bo_systems()
        ctxs = [lib.Context(torch.from_numpy(Q.X).to(dev), Q.kernel, Q.ell, Q.sigma2, Q.lam) for Q in systems]
        opts = [lib.default_opts(Q.X.shape[0], b=Q.b, r=Q.r, seed=40 + k, check_every=0,
                                 max_iters=args.warmup + args.steps) for k, Q in enumerate(systems)]
        lib.solve_batched(ctxs, [torch.from_numpy(Q.Y).to(dev) for Q in systems], opts=opts)
        torch.cuda.synchronize()
        kernels = None
    print(json.dumps({"workload": args.only_workload, "iterations": args.warmup + args.steps,
                      "kernels_per_iteration": kernels, "wall_s": time.perf_counter() - t0}), flush=True)


def run_kernel_only(args):
    """Only the fused block-row products with the benchmark's launch shapes (for ncu):
    Step I (b x n entries, s = 1), then the sketch (b x b entries, r right-hand sides)."""
    import torch

    from paper_2505_13723_b300 import binding as lib
    P = workload(args.n)
    P["kernel"] = {"rbf": 0, "matern32": 1, "matern52": 2}[args.kern]
    n, b = P.X.shape[0], P.b
    ctx = lib.Context(torch.from_numpy(P.X).cuda(), P.kernel, P.ell, P.sigma2, P.lam)
    g = np.random.default_rng(5)
    B = torch.from_numpy(g.choice(n, size=b, replace=False)).cuda()
    Wv = torch.from_numpy(g.standard_normal((n, 1)).astype(np.float32)).cuda()
    for _ in range(args.kernel_launches):
        ctx.kernel_rows(B, Wv)
    # the sketch shape K(X_B, X_B) Omega (b x b entries, r = 100 right-hand sides)
    cb = lib.Context(torch.from_numpy(np.ascontiguousarray(P.X[B.cpu().numpy()])).cuda(), P.kernel, P.ell,
                     P.sigma2, P.lam)
    Om = torch.from_numpy((g.standard_normal((b, P.r)) / np.sqrt(b)).astype(np.float32)).cuda()
    rows = torch.arange(b, device="cuda")
    for _ in range(args.kernel_launches):
        cb.kernel_rows(rows, Om)
    torch.cuda.synchronize()
    cb.close()
    ctx.close()
    print(json.dumps({"only_kernel": True, "kernel": args.kern, "n": n, "b": b, "r": P.r,
                      "launches": args.kernel_launches}))


def run_ours(args, rank, world, dist):
    import torch

    from paper_2505_13723_b300 import binding as lib

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    P = workload(args.n)
    n, b, r = P.X.shape[0], P.b, P.r
    stream = torch.cuda.current_stream()
    Xd = torch.from_numpy(P.X).to(dev)
    Yd = torch.from_numpy(P.Y).to(dev)
    ctx = lib.Context(Xd, P.kernel, P.ell, P.sigma2, P.lam)
    opts = lib.default_opts(n, b=b, r=r, seed=1, check_every=0, max_iters=args.steps)
    sol = lib.Solver(ctx, Yd, opts=opts)
    kernels_per_iter = sol.graph_kernels()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # 256 MB > 126 MB L2

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    sol.step(args.warmup)
    barrier()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        barrier()
        for i in range(args.steps):
            flush.zero_()
            starts[i].record(stream)
            sol.step(1)
            ends[i].record(stream)
        barrier()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    t_local = sum(step_ms) / 1e3
    rel = sol.residual()
    eta, rho, status = sol.scalars()
    diag = sol.diag()
    sol.close()
    ent = entries_per_step(P)
    t_max, units = whole_job(t_local, float(ent * args.steps), dist, dev)
    value = units / t_max / 1e9

    # ---- the dominant kernel alone: Step I block-row product, same launch shape
    g = np.random.default_rng(5)
    B = torch.from_numpy(g.choice(n, size=b, replace=False)).to(dev)
    Wv = torch.from_numpy(g.standard_normal((n, 1)).astype(np.float32)).to(dev)

    def time_kernel(prec):
        ctx.set_precision(prec)
        for _ in range(3):
            ctx.kernel_rows(B, Wv)
        ks = [torch.cuda.Event(enable_timing=True) for _ in range(args.kernel_launches)]
        ke = [torch.cuda.Event(enable_timing=True) for _ in range(args.kernel_launches)]
        with ClockSampler(local) as kc:
            torch.cuda.synchronize()
            for i in range(args.kernel_launches):
                flush.zero_()
                ks[i].record(stream)
                ctx.kernel_rows(B, Wv)
                ke[i].record(stream)
            torch.cuda.synchronize()
        return statistics.mean(s.elapsed_time(e) for s, e in zip(ks, ke)), kc

    default_prec = ctx.prec if hasattr(ctx, "prec") else lib.PREC_TF32X3
    fp32_ms, _ = time_kernel(lib.PREC_FP32)
    k_ms, kclk = time_kernel(default_prec)
    k_rate = b * n / (k_ms * 1e-3)
    pk, pk_src = peaks()
    # roofline of the block-row product: the special-function pipe, at the issue
    # rates measured on this GPU (ex2, sqrt per SM per cycle) and the SM clock
    # sampled while the kernel ran
    pipes = lib.measure_pipes()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    ksum = kclk.summary()
    mhz = float(ksum.get("sm_mhz") or pk.get("sm_max_mhz", 2032.0))
    clk_per_entry = 1.0 / pipes["ex2"] + (1.0 / pipes["sqrt"] if P.kernel != 0 else 0.0)
    peak_entries = sms * mhz * 1e6 / clk_per_entry

    # ---- the same Step I launch with the other covariance kernels (same points, rows and w):
    # RBF needs one ex2 per entry, Matern-5/2 the same sqrt + ex2 as Matern-3/2
    kernels_alt = {}
    for kname, kid in (("rbf", 0), ("matern52", 2)):
        ck = lib.Context(Xd, kid, P.ell, P.sigma2, P.lam)
        for _ in range(3):
            ck.kernel_rows(B, Wv)
        ks = [torch.cuda.Event(enable_timing=True) for _ in range(args.kernel_launches)]
        ke = [torch.cuda.Event(enable_timing=True) for _ in range(args.kernel_launches)]
        torch.cuda.synchronize()
        for i in range(args.kernel_launches):
            flush.zero_()
            ks[i].record(stream)
            ck.kernel_rows(B, Wv)
            ke[i].record(stream)
        torch.cuda.synchronize()
        ck.close()
        kms = statistics.mean(a.elapsed_time(e) for a, e in zip(ks, ke))
        kpeak = sms * mhz * 1e6 / (1.0 / pipes["ex2"] + (1.0 / pipes["sqrt"] if kid != 0 else 0.0))
        kernels_alt[kname] = {"ms_per_launch": kms, "gentries_per_s": b * n / (kms * 1e-3) / 1e9,
                              "entries_per_sm_per_clock": b * n / (kms * 1e-3) / (sms * mhz * 1e6),
                              "peak_gentries_per_s": kpeak / 1e9, "frac": b * n / (kms * 1e-3) / kpeak,
                              "peak_basis": "1 ex2" if kid == 0 else "1 ex2 + 1 sqrt"}

    # ---- time to relative residual 1e-3 (FP32), bounded
    tol_run = None
    if not args.no_tol_run and rank == 0:
        tol_run = {}
        for name, prec in (("fp32", lib.PREC_FP32), ("mixed", lib.PREC_TF32X3)):
            ctx.set_precision(prec)
            topts = lib.default_opts(n, b=b, r=r, seed=2, tol=1e-3, max_iters=args.tol_iters, check_every=50,
                                     check_rows=20000)
            W, st, stc = ctx.solve(Yd, opts=topts)
            # the stop was taken on 20,000 sampled rows; confirm on all n rows (adasap_residual)
            exact = ctx.residual(Yd, W)
            tol_run[name] = {"seconds": st["seconds"], "iters": st["iters"],
                             "rel_resid_sampled": st["rel_resid"], "resid_rows_sampled": 20000,
                             "rel_resid_exact": exact, "reached": bool(exact <= 1e-3)}
        ctx.set_precision(default_prec)

    # ---- many right-hand sides: the multirhs workload (n = 2^18, s = 64), device time per
    # iteration of the batched tensor-core solve of all 64 columns against the plain FP32
    # single-RHS solve of one column (the batched form replaces 64 such solves)
    multi = None
    if rank == 0 and not args.no_multi_rhs:
        from paper_2505_13723_b300 import synth
        Q = synth.multirhs()
        cq = lib.Context(torch.from_numpy(Q.X).to(dev), Q.kernel, Q.ell, Q.sigma2, Q.lam)
        Yq = torch.from_numpy(Q.Y).to(dev)

        def per_iter(prec, Yc, iters=40):
            cq.set_precision(prec)
            so = lib.Solver(cq, Yc, opts=lib.default_opts(Q.X.shape[0], b=Q.b, r=Q.r, seed=3, check_every=0,
                                                          max_iters=iters + 3))
            so.step(3)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            so.step(iters)
            e1.record(stream)
            torch.cuda.synchronize()
            so.close()
            return e0.elapsed_time(e1) / iters

        mixed_batched = per_iter(lib.PREC_TF32X3, Yq)
        tf32_batched = per_iter(lib.PREC_TF32, Yq)
        fp32_single = per_iter(lib.PREC_FP32, Yq[:, :1].contiguous())
        # the s = 64 Step I launch alone (b x n entries against 64 right-hand sides)
        nq, dq = Q.X.shape
        gq = np.random.default_rng(6)
        Bq = torch.from_numpy(gq.choice(nq, size=Q.b, replace=False)).to(dev)
        m_ms = {}
        for name, prec in (("tf32x3", lib.PREC_TF32X3), ("tf32", lib.PREC_TF32)):
            cq.set_precision(prec)
            for _ in range(3):
                cq.kernel_rows(Bq, Yq)
            es = [torch.cuda.Event(enable_timing=True) for _ in range(args.kernel_launches)]
            ee = [torch.cuda.Event(enable_timing=True) for _ in range(args.kernel_launches)]
            torch.cuda.synchronize()
            for i in range(args.kernel_launches):
                flush.zero_()
                es[i].record(stream)
                cq.kernel_rows(Bq, Yq)
                ee[i].record(stream)
            torch.cuda.synchronize()
            m_ms[name] = statistics.mean(a.elapsed_time(e) for a, e in zip(es, ee))
        cq.set_precision(lib.PREC_TF32X3)
        # seconds to a relative residual both forms reach: the batched split-TF32 solve of all 64
        # columns to a Frobenius residual tau, against 64 plain FP32 single-RHS solves each to tau
        # (column 0, the signal, and column 1, white noise, are solved; the other 62 white-noise
        # columns have column 1's distribution and are counted at its time).  The stepsize, the
        # preconditioner and the draws do not depend on Y, so every column follows the same
        # trajectory in both forms.
        tau = args.mrhs_tol
        tt = {"tol": tau, "check_every": 50, "resid_rows_sampled": 20000}
        cq.set_precision(lib.PREC_TF32X3)
        Wb, stb, _ = cq.solve(Yq, opts=lib.default_opts(nq, b=Q.b, r=Q.r, seed=3, tol=tau, max_iters=6000,
                                                        check_every=50, check_rows=20000))
        tt["mixed_batched_s64"] = {"seconds": stb["seconds"], "iters": stb["iters"],
                                   "rel_resid_sampled": stb["rel_resid"], "rel_resid_exact": cq.residual(Yq, Wb)}
        del Wb
        cq.set_precision(lib.PREC_FP32)
        single = {}
        for col in (0, 1):
            Yc = Yq[:, col:col + 1].contiguous()
            Wc, stc_, _ = cq.solve(Yc, opts=lib.default_opts(nq, b=Q.b, r=Q.r, seed=3, tol=tau, max_iters=6000,
                                                             check_every=50, check_rows=20000))
            single["column_%d" % col] = {"seconds": stc_["seconds"], "iters": stc_["iters"],
                                         "rel_resid_sampled": stc_["rel_resid"],
                                         "rel_resid_exact": cq.residual(Yc, Wc)}
        single["seconds_64_columns"] = single["column_0"]["seconds"] + 63 * single["column_1"]["seconds"]
        tt["fp32_single_rhs"] = single
        tt["speedup"] = single["seconds_64_columns"] / tt["mixed_batched_s64"]["seconds"]
        tt["note"] = ("rel-resid 1e-3 is out of reach here: after 3000 iterations the white-noise columns are at "
                      "0.73 (the stepsize stays near 0.09: r = 64 leaves much of this RBF spectrum outside the "
                      "preconditioner)")
        cq.set_precision(lib.PREC_TF32X3)
        cq.close()
        multi = {"workload": "multirhs: n=262144, d=16, X~N(0,I), RBF ell=2, lambda=1e-2, b=4096, r=64, s=64",
                 "ms_per_iteration_mixed_batched_s64": mixed_batched,
                 "ms_per_iteration_tf32_single_pass_contraction_s64": tf32_batched,
                 "ms_per_iteration_fp32_single_rhs": fp32_single,
                 "speedup_vs_64_fp32_single_rhs_solves": 64.0 * fp32_single / mixed_batched,
                 "roofline": mrhs_roofline(Q.b * nq, dq, Q.Y.shape[1], m_ms, pk, pk_src, pipes, sms, mhz),
                 "time_to_tol": tt}

    # ---- the uneven batch: 48 independent Matern-5/2 systems (n log-uniform in [4096, 65536],
    # b = n/50, r = 50) iterated together by adasap_solve_batched, against the same systems
    # solved one after another (device time per iteration of all 48)
    batched = None
    if rank == 0 and not args.no_batched:
        from paper_2505_13723_b300 import synth
        systems = synth.bo_systems()
        ctxs = [lib.Context(torch.from_numpy(Q.X).to(dev), Q.kernel, Q.ell, Q.sigma2, Q.lam) for Q in systems]
        Ys = [torch.from_numpy(Q.Y).to(dev) for Q in systems]
        it_b = args.batched_iters
        # one short batched solve first, so that the timed one does not carry the first
        # launches' one-time costs (as the other timings have their warm-up)
        lib.solve_batched(ctxs, Ys, opts=[lib.default_opts(Q.X.shape[0], b=Q.b, r=Q.r, seed=40 + k, check_every=0,
                                                           max_iters=3) for k, Q in enumerate(systems)])
        bopts = [lib.default_opts(Q.X.shape[0], b=Q.b, r=Q.r, seed=40 + k, check_every=0, max_iters=it_b)
                 for k, Q in enumerate(systems)]
        _, bst, bstatus = lib.solve_batched(ctxs, Ys, opts=bopts)
        t_batch = max(x["seconds"] for x in bst) / it_b
        it_s = max(3, it_b // 4)
        t_seq = 0.0
        for k, (Q, cq, Yq) in enumerate(zip(systems, ctxs, Ys)):
            _, sst, _ = cq.solve(Yq, opts=lib.default_opts(Q.X.shape[0], b=Q.b, r=Q.r, seed=40 + k,
                                                            check_every=0, max_iters=it_s))
            t_seq += sst["seconds"] / it_s
        for cq in ctxs:
            cq.close()
        ent_b = sum(Q.b * Q.X.shape[0] + 11 * Q.b * Q.b for Q in systems)
        batched = {"workload": "bo: 48 systems, n log-uniform in [4096, 65536] (sum %d), d in {4, 8, 12}, "
                               "X~U[-1,1]^d, Matern-5/2 ell~U[0.2,1], lambda=1e-3, b=n/50, r=50"
                               % sum(Q.X.shape[0] for Q in systems),
                   "ms_per_iteration_batched": 1e3 * t_batch,
                   "ms_per_iteration_one_after_another": 1e3 * t_seq,
                   "speedup": t_seq / t_batch,
                   "gentries_per_s_batched": ent_b / t_batch / 1e9,
                   "entries_per_iteration": ent_b, "status": bstatus,
                   "iterations_timed": {"batched": it_b, "one_after_another": it_s}}

    # ---- pathwise conditioning (Sec. 2.1) on the multirhs workload: 2048 random features,
    # 63 samples plus the posterior mean in one 64-column solve
    pathwise = None
    if rank == 0 and not args.no_pathwise:
        from paper_2505_13723_b300 import synth
        Q = synth.multirhs()
        nq, dq = Q.X.shape
        ns, q = 63, 2048
        z, u, phase, theta, zeta = synth.rf_draws(q, dq, None, ns, nq, Q.lam, seed=1)
        cq = lib.Context(torch.from_numpy(Q.X).to(dev), Q.kernel, Q.ell, Q.sigma2, Q.lam)
        Xq = torch.from_numpy(Q.X).to(dev)
        zt, pt, tt, zet = [torch.from_numpy(a).to(dev) for a in (z, phase, theta, zeta)]
        for _ in range(2):
            cq.rf_prior(Xq, zt, None, pt, tt)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(5):
            cq.rf_prior(Xq, zt, None, pt, tt)
        e1.record(stream)
        torch.cuda.synchronize()
        rf_ms = e0.elapsed_time(e1) / 5
        it_p = 40
        yq = torch.from_numpy(Q.Y[:, 0].copy()).to(dev)
        Xt = torch.from_numpy(Q.Xtest).to(dev)
        t0 = time.perf_counter()
        out, _, pst, pstatus = cq.pathwise(yq, Xt, zt, None, pt, tt, zet,
                                           opts=lib.default_opts(nq, b=Q.b, r=Q.r, seed=2, check_every=0,
                                                                 max_iters=it_p))
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        cq.close()
        pathwise = {"workload": "multirhs: n=262144, d=16, RBF ell=2, lambda=1e-2; q=2048 random features, "
                                "63 samples + posterior mean (s=64), 10000 test points, b=4096, r=64",
                    "rf_prior_ms_n262144_q2048_s63": rf_ms,
                    "rf_prior_gflops": 2.0 * nq * q * ns / (rf_ms * 1e-3) / 1e9,
                    "solve_ms_per_iteration": 1e3 * pst["seconds"] / it_p,
                    "seconds_total_%d_iterations" % it_p: wall, "status": pstatus}

    # ---- Alg. 1 (SAP) with the exact block solve at b = 4096 on the benchmark workload, against
    # ADASAP (Nystrom, r = 100) at the same block size: device time per iteration
    sap = None
    if rank == 0 and not args.no_sap:
        sap = {"workload": "regress (n=%d) with b=4096" % n}
        for name, extra in (("sap_exact", dict(precond=2)), ("adasap_r100", dict(r=100))):
            so = lib.Solver(ctx, Yd, opts=lib.default_opts(n, b=4096, seed=6, check_every=0, max_iters=20, **extra))
            so.step(2)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            so.step(8)
            e1.record(stream)
            torch.cuda.synchronize()
            sap[name + "_ms_per_iteration"] = e0.elapsed_time(e1) / 8
            sap[name + "_rel_resid_after_10"] = so.residual()
            so.close()
        sap["cholesky_flops_per_iteration"] = 4096 ** 3 / 3

    # ---- the largest workload (n = 2^25, d = 9, RBF, b = 10^5, r = 100): device time per iteration
    # in plain FP32 on the CUDA cores against the split-TF32 tensor-core path, and the relative
    # residual after the same iterations (sampled rows, exact on those rows) for both
    taxi = None
    if rank == 0 and not args.no_taxi:
        from paper_2505_13723_b300 import synth
        T5 = synth.taxi()
        n5 = T5.X.shape[0]
        c5 = lib.Context(torch.from_numpy(T5.X).to(dev), T5.kernel, T5.ell, T5.sigma2, T5.lam)
        Y5 = torch.from_numpy(T5.Y).to(dev)
        taxi = {"workload": "taxi: n=%d, d=9, X~U[0,1]^9, RBF ell=0.5, lambda=1e-2, b=%d, r=100, s=1" % (n5, T5.b),
                "iterations_timed": args.taxi_iters}
        for name, prec in (("mixed_tf32x3", lib.PREC_TF32X3), ("fp32", lib.PREC_FP32)):
            c5.set_precision(prec)
            so = lib.Solver(c5, Y5, opts=lib.default_opts(n5, b=T5.b, r=T5.r, seed=7, check_every=0,
                                                          max_iters=args.taxi_iters + 1))
            so.step(1)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            so.step(args.taxi_iters)
            e1.record(stream)
            torch.cuda.synchronize()
            ms5 = e0.elapsed_time(e1) / args.taxi_iters
            taxi[name] = {"ms_per_iteration": ms5,
                          "gentries_per_s": (T5.b * n5 + 11 * T5.b * T5.b) / (ms5 * 1e-3) / 1e9,
                          "rel_resid_after_%d_iterations_sampled_rows" % (args.taxi_iters + 1): so.residual()}
            so.close()
        taxi["speedup_mixed_vs_fp32"] = taxi["fp32"]["ms_per_iteration"] / taxi["mixed_tf32x3"]["ms_per_iteration"]
        c5.close()
        del Y5

    # ---- end to end through the C-ABI with host buffers
    e2e = None
    if rank == 0:
        # the inputs and the result buffer sit in pinned host memory before the timed region
        # (CPU tensors; the library sees host pointers and copies them)
        Xh = torch.from_numpy(P.X).pin_memory()
        Yh = torch.from_numpy(P.Y).pin_memory()
        Wh = torch.zeros(Yh.shape, dtype=torch.float32).pin_memory()
        eopts = lib.default_opts(n, b=b, r=r, seed=3, check_every=0, max_iters=args.steps)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c2 = lib.Context(Xh, P.kernel, P.ell, P.sigma2, P.lam)
        Wout, st2, _ = c2.solve(Yh, opts=eopts, W=Wh)
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        c2.close()
        nbytes = lambda t: t.numel() * t.element_size()
        e2e = {"value": ent * args.steps / te / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": int((nbytes(Xh) + nbytes(Yh) + nbytes(Wh)) / args.steps),
               "d2h_bytes_per_step": int(nbytes(Wh) / args.steps),
               "includes": "create (H2D of X from pinned host memory, centring) + solve (H2D of Y, W0; %d "
                           "iterations; final residual) + D2H of W into pinned host memory" % args.steps}

    ctx.close()
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline:
        try:
            rate, k, dt, used = oracle_rows_rate(P, target_s=12.0)
            cpu = {"value": rate / 1e9, "unit": UNIT, "cores": used, "kind": "oracle",
                   "sample": "FP64 NumPy block-row product K(X_B, X) w, %d sampled rows x n=%d (%.1f s), rows "
                             "split over %d threads (host affinity set: %d cores)" % (k, n, dt, used,
                                                                                       host_cores())}
        except Exception as ex:  # report, do not lose the GPU line
            cpu = {"value": None, "unit": UNIT, "cores": host_cores(), "kind": "oracle", "error": repr(ex)}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "tf32x3+f32" if default_prec == lib.PREC_TF32X3 else "f32", "data": "synthetic",
            "config": config_dict(P),
            "roofline": {"bound": "alu", "achieved": k_rate / 1e9, "peak": peak_entries / 1e9,
                         "unit": "Gentries/s", "frac": k_rate / peak_entries,
                         "traffic": (TC_DRAM_BYTES_PER_ENTRY * b * n if default_prec == lib.PREC_TF32X3 else None),
                         "traffic_basis": ("dram__bytes_read.sum + dram__bytes_write.sum of one ncu-captured "
                                           "k_rows_tc launch at 10,000 x 262,144 entries, scaled by the entries "
                                           "of this launch"),
                         "kernel": ("k_rows_tc (tcgen05 TF32x3 distances)" if default_prec == lib.PREC_TF32X3
                                    else "k_rows_narrow (FP32)")
                                   + " Step I block-row product, b=%d rows x n=%d" % (b, n),
                         "ms_per_launch": k_ms,
                         "fp32_cuda_core_kernel": {"ms_per_launch": fp32_ms,
                                                   "achieved": b * n / (fp32_ms * 1e-3) / 1e9},
                         "peak_basis": ("special-function pipe, measured on this GPU by adasap_measure_pipes: "
                                        "ex2 %.1f and sqrt %.1f per SM per clock; %s per entry; %d SMs x %.0f MHz "
                                        "(median SM clock sampled during the kernel)"
                                        % (pipes["ex2"], pipes["sqrt"],
                                           "1 ex2" if P.kernel == 0 else "1 ex2 + 1 sqrt", sms, mhz)),
                         "pipes_measured": pipes},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": kernels_per_iter * args.steps,
            "clocks": clk.summary(), "kernel_clocks": kclk.summary(),
            "step1_other_kernels": kernels_alt,
            "taxi_mixed_vs_fp32": taxi,
            "time_to_tol": tol_run,
            "multi_rhs": multi,
            "batched_systems": batched,
            "pathwise_sampling": pathwise,
            "sap_exact_block": sap,
            "step_ms": {"min": min(step_ms), "median": statistics.median(step_ms), "max": max(step_ms)},
            "solver_state": {"rel_resid_after": rel, "eta": eta, "rho": rho, "status": status,
                             "jacobi_sweeps": diag["jacobi_sweeps"], "chol_retries": diag["chol_retries"],
                             "delta": diag["delta"]}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        if args.impl == "reference":
            tdist = None
        else:
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
            tdist.init_process_group("nccl")
        dist = tdist
    if args.only_workload:
        run_workload_only(args)
    elif args.only_kernel:
        run_kernel_only(args)
    elif args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, dist)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
