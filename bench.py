#!/usr/bin/env python
"""Benchmark of the ASPOT solver (arXiv 2601.17196, Algorithm 2) on one GB300.

Workload (default ``cloud_32k``): n = m = 32768 BF16 points in R^128
(8-component Gaussian mixture, means ~ N(0, 4I), unit covariance, 5% uniform
outliers in [-6, 6]^128), uniform marginals of mass 1.0 and 1.25, s = 0.95,
gamma = 0.02, eps = 1e-2, squared-Euclidean cost normalised by its maximum
and never stored (tcgen05 on-the-fly passes).  One step = one whole solve:
setup, the accelerated loop to the stop threshold eps / (8 max C), rounding
to a feasible plan of mass s and the objective <C, X>.

Metric: ASPOT iterations per second at n = 32k (whole solve included), with
the time to epsilon per solve reported alongside; the block rule of
Algorithm 1 as printed (t mod 3) unless ``--block-rule greedy``, and the
greedy rule's solves measured beside the headline at N = 1.  Multi-GPU runs
are independent replicas (one instance per rank, seed = rank): weak scaling.

At N = 1 the line also carries, under ``workloads``, the other measured
configurations, each with its own warm-up, CUDA-event timing on the solve
stream, clocks sampled over its timed region and, where one applies, its
roofline: the 256-point dense configuration against the oracle (d1), the
dense 4096 gamma sweep and the 16384 HBM point (d2), the 512-instance
batched solve (d4), the learned warm start on 2000 training / 200 held-out
instances (d5), the appendix's runtime-vs-n study (d6) and the 64-pair
registration loop (f4).  ``--workload <name>`` runs one of them alone.

``--impl reference`` times the FP64 CPU oracle instead (the reference arm):
each step is a bounded sample, ASPOT iterations of the unmodified oracle in
one process per host core, each on its own seeded instance of the same
generator at n = m = 2048, the aggregate rate scaled to n = 32768 by the
number of cost entries.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_FULL = 32768
D_FULL = 128
# ncu DRAM bytes per launch of the current kernels (null once a kernel changes):
# dense_pass_kernel<0>, n = m = 16384 FP32 cost: 1.075126 GB read + 11.26 MB written
DENSE_16K_TRAFFIC = 1.075126e9 + 11.25888e6
# tc3_pass_kernel<0> (rows + columns), n = m = 32768, d = 128: 17.62 MB read (the BF16
# points) + 7.7 KB written per launch; the column partials (16.8 MB) stay in L2
TC3_32K_TRAFFIC = 17617152.0 + 7680.0


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_FULL, help="problem size (default: the 32k workload)")
    ap.add_argument("--max-iter", type=int, default=20000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--block-rule", default="cyclic", choices=["cyclic", "greedy"],
                    help="headline: Greenkhorn block rule of the timed solves (cyclic: t mod 3 as Algorithm 1 "
                         "prints it; greedy: the block with the largest decrease of phi)")
    ap.add_argument("--no-greedy", action="store_true",
                    help="headline: skip the greedy-block-rule solves measured beside the cyclic ones")
    ap.add_argument("--mode", default="solve", choices=["solve", "pass", "iters"],
                    help="'pass': time only the fused row+column pass (for ncu captures of that kernel); "
                         "'iters': ASPOT solves of exactly --max-iter iterations at size --n (for launch lists "
                         "of the solver loop)")
    ap.add_argument("--workload", default="cloud_32k",
                    choices=["cloud_32k", "dense_4096", "scaling_e4", "batch_3d", "warmstart", "small_dense",
                             "registration", "ws_train"],
                    help="cloud_32k: the headline line; dense_4096: the FP32 dense-cost path (gamma sweep, "
                         "HBM roofline of the CUDA-core pass); scaling_e4: the appendix's runtime-vs-n study; "
                         "batch_3d: 512 uneven 3-D instances; warmstart: the learned warm start (train + held-out); "
                         "small_dense: the 256-point configuration with the tuned-gamma Sinkhorn p sweep; "
                         "registration: batched rigid registration of 64 partial 3-D clouds; "
                         "ws_train: training-step throughput of the warm-start network kernels")
    ap.add_argument("--ws-train", type=int, default=20000, help="warmstart: training instances")
    ap.add_argument("--ws-eval", type=int, default=1000, help="warmstart: held-out seeds")
    ap.add_argument("--ws-epochs", type=int, default=12, help="warmstart: training epochs")
    ap.add_argument("--ws-small", type=int, default=2000,
                    help="training instances of the warm-start study in the headline line (0: skip)")
    ap.add_argument("--ws-small-eval", type=int, default=200,
                    help="held-out seeds of the warm-start study in the headline line")
    ap.add_argument("--no-workloads", action="store_true",
                    help="headline only: skip the other workloads' sub-objects (d1, d2, d4, d5, d6, f4)")
    return ap.parse_args()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["bf16_tflops"]), float(p["bf16_tflops_sustained"]), float(p["hbm_gbs"]), "measured"
    except Exception:
        return 1900.0, 1700.0, 6800.0, "fallback"


def _workload_desc(n):
    return (f"cloud_32k: n=m={n}, d=128 BF16 points, 8-component GMM (means~N(0,4I), unit cov) + 5% uniform "
            f"outliers in [-6,6]^128, |r|=1.0, |c|=1.25, s=0.95, gamma=0.02, eps=1e-2, sq-Euclidean cost / max, "
            f"never stored")


# ------------------------------------------------------------------ clocks --

class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in out.strip().splitlines():
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ oracle (CPU) --

_ORACLE_SAMPLE = {}


def _oracle_iters_per_s(n_sample, iters, seed=0, rule="cyclic"):
    """ASPOT iterations of the FP64 oracle, as it stands, at n = m = n_sample
    (the cost matrix is built once, outside the timed region)."""
    import pot_workloads as W
    from oracle import pot as O
    key = (n_sample, seed)
    if key not in _ORACLE_SAMPLE:
        pb = W.cloud_32k(seed, n=n_sample)
        _ORACLE_SAMPLE[key] = (pb, O.sqeuclid_cost(pb.X, pb.Y, 0.0))
    pb, C = _ORACLE_SAMPLE[key]
    t0 = time.perf_counter()
    O.aspot(C, pb.r, pb.c, pb.s, pb.eps, pb.gamma, max_iter=iters, no_stop=True, cmax=float(C.max()),
            block_rule=rule)
    dt = time.perf_counter() - t0
    return iters / dt, dt


def _oracle_worker(job):
    """One pool worker: `iters` oracle iterations on its own instance (seed),
    after one untimed warm-up iteration.  Pins numpy's threads to one core so
    that the workers together use each host core once."""
    n_sample, iters, seed, rule = job
    _oracle_iters_per_s(n_sample, 1, seed=seed, rule=rule)
    return _oracle_iters_per_s(n_sample, iters, seed=seed, rule=rule)


class OraclePool:
    """The oracle on every host core: one spawned process per core, each
    running the unmodified FP64 oracle on its own seeded instance of the
    sampled workload (independent replicas, like the GPU arm's ranks).  The
    aggregate rate is the sum over workers of its iterations over the time
    of its own timed region (the regions run at the same time).  'spawn'
    keeps the workers clear of the parent's CUDA state."""

    def __init__(self, cores=None):
        import multiprocessing as mp
        self.cores = cores or os.cpu_count() or 1
        env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in env:
            os.environ[k] = "1"
        try:
            self.pool = mp.get_context("spawn").Pool(self.cores)
        finally:
            for k, v in env.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def rate(self, n_sample, iters, rule="cyclic"):
        t0 = time.perf_counter()
        outs = self.pool.map(_oracle_worker, [(n_sample, iters, 100 + k, rule) for k in range(self.cores)])
        wall = time.perf_counter() - t0
        return sum(r for r, _ in outs), wall, max(dt for _, dt in outs)

    def close(self):
        self.pool.close()
        self.pool.join()


CPU_POOL_N = 2048
CPU_POOL_ITERS = 6


def cpu_baseline(n_full, rule="cyclic"):
    """The oracle as it stands on every host core (see OraclePool) at
    n = m = 2048 of the 32k generator, scaled to n_full by the number of cost
    entries; the single-core rate beside it."""
    pool = OraclePool()
    try:
        rate, wall, busy = pool.rate(CPU_POOL_N, CPU_POOL_ITERS, rule)
    finally:
        pool.close()
    scale = (CPU_POOL_N / n_full) ** 2
    single, dt1 = _oracle_iters_per_s(CPU_POOL_N, 2, rule=rule)
    return {"value": rate * scale, "unit": "it/s", "cores": pool.cores, "kind": "oracle",
            "sample": f"{pool.cores} concurrent processes (one per host core), each running {CPU_POOL_ITERS} FP64 "
                      f"oracle ASPOT iterations on its own seeded instance of the same generator at n=m={CPU_POOL_N} "
                      f"({wall:.1f} s wall); aggregate rate scaled by ({CPU_POOL_N}/{n_full})^2 to n={n_full}",
            "single_core_value": single * scale,
            "time_to_eps_note": ("a full oracle solve of this generator is out of reach at bench time: at n=512 it "
                                 "has not reached eps~ after 3000 iterations (82 s on one core); the GPU's "
                                 "time to eps at 32k divided by this rate's iteration time is the labelled "
                                 "extrapolation in time_to_eps_extrapolated_s")}


def run_reference(args, rank, world):
    if rank != 0:
        return
    scale = (CPU_POOL_N / args.n) ** 2
    pool = OraclePool()
    try:
        for _ in range(args.warmup):
            pool.rate(CPU_POOL_N, 1, args.block_rule)
        rates, secs = [], 0.0
        for _ in range(args.steps):
            r, wall, _ = pool.rate(CPU_POOL_N, 2, args.block_rule)
            rates.append(r * scale)
            secs += wall
    finally:
        pool.close()
    value = statistics.mean(rates)
    sample = (f"{pool.cores} concurrent processes (one per host core), 2 FP64 oracle ASPOT iterations each per step, "
              f"each on its own seeded instance of the same generator at n=m={CPU_POOL_N}; aggregate rate scaled by "
              f"({CPU_POOL_N}/{args.n})^2 to n={args.n}")
    line = {"metric": "ASPOT iterations/s at n=32k (time-to-epsilon alongside)", "value": value, "unit": "it/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": _workload_desc(args.n),
                       "parallelism": "single (rank 0 of the launch runs the oracle)", "block_rule": args.block_rule},
            "cpu_baseline": {"value": value, "unit": "it/s", "cores": pool.cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "it/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------- GPU arm --

def reduce_replicas(maxes, sums, device="cpu"):
    """Whole-job figures of independent replicas: the slowest rank's times
    (max over ranks) and the work of all ranks (sum over ranks).  Needs an
    initialised process group (nccl on GPUs, gloo in the CPU tests)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x) for x in maxes], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    s = torch.tensor([float(x) for x in sums], dtype=torch.float64, device=device)
    dist.all_reduce(s, op=dist.ReduceOp.SUM)
    return [float(x) for x in t], [float(x) for x in s]


def replica_throughput(total_units: float, max_ms: float) -> float:
    """value = units all ranks processed / the slowest rank's time."""
    return total_units / (max_ms / 1000.0)


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2601_17196_gb300 as pkg
    import pot_workloads as W

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    pb = W.cloud_32k(rank, n=args.n)
    dp = pkg.DeviceProblem.from_workload(pb, device=dev)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)     # > 129 MB L2
    flags = pkg.FLAG_PROFILE

    rule = pkg.BLOCK_GREEDY if args.block_rule == "greedy" else pkg.BLOCK_CYCLIC

    def solve(prob):
        return pkg.aspot_solve(prob, pb.gamma, pb.eps, max_iter=args.max_iter, flags=flags, check_every=24,
                               block_rule=rule)

    with torch.cuda.stream(stream):
        first_ms = None
        for w in range(args.warmup):
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            res = solve(dp)
            f1.record(stream)
            if w == 0:
                f1.synchronize()
                first_ms = f0.elapsed_time(f1)      # first call: graph capture / instantiation, cold caches
        torch.cuda.synchronize()

        # ---------------- device-resident inputs: the kernel-level value ----
        clk = Clocks(local_rank)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        clk.start()
        ev = []
        iters, pass_ms, pass_n, launches, conv = 0, 0.0, 0, 0, 0
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = solve(dp)
            e1.record(stream)
            ev.append((e0, e1))
            iters += res.iters
            pass_ms += res.pass_ms
            pass_n += res.pass_launches
            launches += res.kernel_launches
            conv += int(res.status == 0)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        clocks = clk.stop()
        ms = sum(a.elapsed_time(b) for a, b in ev)
        last = res

        # ---------------- end to end through host buffers -----------------
        hX = dp.X.cpu().pin_memory()
        hY = dp.Y.cpu().pin_memory()
        hr = dp.r.cpu().pin_memory()
        hc = dp.c.cpu().pin_memory()
        out = {k: torch.empty(getattr(last.plan, k).numel(), dtype=torch.float64).pin_memory()
               for k in ("f", "g", "p", "q", "kappa")}
        h2d = sum(t.numel() * t.element_size() for t in (hX, hY, hr, hc))
        d2h = sum(t.numel() * t.element_size() for t in out.values()) + 8
        dX, dY = torch.empty_like(dp.X), torch.empty_like(dp.Y)
        dr, dc = torch.empty_like(dp.r), torch.empty_like(dp.c)
        e2e_ms, e2e_iters = 0.0, 0
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            dX.copy_(hX, non_blocking=True)
            dY.copy_(hY, non_blocking=True)
            dr.copy_(hr, non_blocking=True)
            dc.copy_(hc, non_blocking=True)
            prob = pkg.DeviceProblem(dp.kind, dr, dc, dp.s, X=dX, Y=dY, cost_scale=dp.cost_scale)
            r2 = solve(prob)
            for k, t in out.items():
                t.copy_(getattr(r2.plan, k), non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            e2e_ms += e0.elapsed_time(e1)
            e2e_iters += r2.iters

        # ---------------- the greedy block rule, same workload and timing ---
        greedy = None
        if world == 1 and not args.no_greedy and args.block_rule == "cyclic":
            def solve_greedy(prob):
                return pkg.aspot_solve(prob, pb.gamma, pb.eps, max_iter=args.max_iter, flags=flags, check_every=24,
                                       block_rule=pkg.BLOCK_GREEDY)
            for _ in range(args.warmup):
                solve_greedy(dp)
            torch.cuda.synchronize()
            gclk = Clocks(local_rank)
            gclk.start()
            gev, g_iters, g_conv, g_pass_ms, g_pass_n = [], 0, 0, 0.0, 0
            for _ in range(args.steps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                rg = solve_greedy(dp)
                e1.record(stream)
                gev.append((e0, e1))
                g_iters += rg.iters
                g_conv += int(rg.status == 0)
                g_pass_ms += rg.pass_ms
                g_pass_n += rg.pass_launches
            torch.cuda.synchronize()
            g_clocks = gclk.stop()
            g_ms = sum(a.elapsed_time(b) for a, b in gev)
            greedy = {"block_rule": "greedy (the block with the largest exact decrease of phi, scored from a "
                                    "two-sided pass at z_grave and again at z^t)",
                      "value": g_iters / (g_ms / 1000.0), "unit": "it/s",
                      "time_to_eps_ms": g_ms / args.steps, "iters_per_solve": g_iters / args.steps,
                      "converged_steps": g_conv, "objective": rg.objective, "E_final": rg.err_final,
                      "avg_pass_ms": g_pass_ms / max(g_pass_n, 1), "clocks": g_clocks}

    # ---------------- reduce over ranks (replicas) -------------------------
    if world > 1:
        (ms, e2e_ms), (iters, e2e_iters, launches) = reduce_replicas([ms, e2e_ms], [iters, e2e_iters, launches], dev)
        iters, e2e_iters, launches = int(iters), int(e2e_iters), int(launches)
    if rank != 0:
        return

    burst, sustained, hbm, src = _peaks()
    n = args.n
    kernel_name = pkg.pass_kernel(dp, flags)          # the kernel the hot loop's passes ran
    flop_per_pass = 2.0 * n * n * D_FULL
    avg_pass_ms = pass_ms / max(pass_n, 1)
    achieved = flop_per_pass / (avg_pass_ms * 1e-3) / 1e12 if pass_n else None
    value = replica_throughput(iters, ms)
    line = {
        "metric": "ASPOT iterations/s at n=32k (time-to-epsilon alongside)",
        "value": value, "unit": "it/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16", "data": "synthetic",
        "config": {"workload": _workload_desc(n), "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs (16 MiB) fit in L2; a 256 MiB buffer is written before every step",
                   "stop": "E_t <= eps/(8 max C) = 1.25e-3", "max_iter": args.max_iter,
                   "block_rule": args.block_rule},
        "time_to_eps_ms": ms / args.steps,
        "first_call_ms": first_ms,
        "iters_per_solve": iters / (args.steps * world),
        "converged_steps": conv,
        "objective": last.objective,
        "e2e": {"value": e2e_iters / (e2e_ms / 1000.0), "unit": "it/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "time_to_eps_ms": e2e_ms / args.steps},
        "gpu_launches": launches,
        "clocks": clocks,
        "roofline": {"kernel": kernel_name, "bound": "tensor",
                     "achieved": achieved, "peak": sustained, "unit": "TFLOP/s",
                     "frac": (achieved / sustained) if achieved else None,
                     "traffic": TC3_32K_TRAFFIC if n == N_FULL else None,
                     "traffic_note": "ncu dram bytes of one two-sided launch at n=32768 (read + write)",
                     "peak_source": f"{src} bf16 dense, sustained (kernel timed inside a long step)",
                     "flop_per_launch": flop_per_pass, "avg_launch_ms": avg_pass_ms, "launches": pass_n},
    }
    if greedy is not None:
        greedy["time_to_eps_vs_cyclic"] = greedy["time_to_eps_ms"] / (ms / args.steps)
        line["greedy_rule"] = greedy
    if world == 1 and not args.no_workloads:
        # the other measured workloads, each timed the same way (warm-up, CUDA events on the solve stream,
        # clocks sampled over its own timed region); --workload <name> runs each one alone at full length
        wl = {}
        wl["d1_small_dense_256"] = small_study(args, quick=True, dev=dev)
        wl["d2_dense_4096"] = dense_study(args, quick=True, dev=dev)
        wl["d4_batch_3d_512"] = batched_study(args, quick=True, dev=dev)
        if args.ws_small > 0:
            ws = warm_start_study(args.ws_small, args.ws_small_eval, epochs=max(1, 80000 // args.ws_small),
                                  device=dev, greedy=not args.no_greedy)
            ws["note"] = (f"{args.ws_small} training instances / {args.ws_small_eval} held-out seeds inside the "
                          f"headline bench; --workload warmstart runs the 20000 / 1000 configuration")
            wl["d5_warm_start"] = ws
        wl["d6_scaling_e4"] = scaling_study(args, dev=dev)
        wl["f4_registration_64"] = registration_study(args, quick=True, dev=dev)
        line["workloads"] = wl
    if world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(n, rule=args.block_rule)
        cb["time_to_eps_extrapolated_s"] = (iters / (args.steps * world)) / cb["single_core_value"]
        cb["time_to_eps_extrapolated_note"] = ("labelled extrapolation: the GPU solve's iteration count times the "
                                               "oracle's single-core time per iteration at this n")
        line["cpu_baseline"] = cb
    print(json.dumps(line), flush=True)


def run_pass_only(args):
    """K fused row+column passes (pot_marginals) on the cloud workload (or,
    with --workload dense_4096, on a dense FP32 cost) at size n."""
    import numpy as np
    import torch
    import paper_2601_17196_gb300 as pkg
    import pot_workloads as W
    dense = args.workload == "dense_4096"
    pb = W.dense_4096(0, n=args.n, gamma=0.03) if dense else W.cloud_32k(0, n=args.n)
    dp = pkg.DeviceProblem.from_workload(pb, device="cuda")
    if not dense:
        dp.cost_scale = 1.0 / pkg.pot_cost_max(dp)
    rng = np.random.default_rng(0)
    u = torch.tensor(rng.uniform(-12, -9, dp.n), device="cuda")
    v = torch.tensor(rng.uniform(-12, -9, dp.m), device="cuda")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            pkg.pot_marginals(dp, pb.gamma, u, v, 5.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            pkg.pot_marginals(dp, pb.gamma, u, v, 5.0, check=False)     # enqueue only: device time
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    if dense:
        print(json.dumps({"mode": "pass", "workload": "dense", "n": args.n, "ms_per_pass_incl_combine": ms,
                          "GBps": 4.0 * args.n * args.n / (ms * 1e-3) / 1e9}), flush=True)
        return
    print(json.dumps({"mode": "pass", "n": args.n, "ms_per_pass_incl_combine": ms,
                      "tflops": 2.0 * args.n * args.n * D_FULL / (ms * 1e-3) / 1e12}), flush=True)


def run_iters_only(args):
    """--warmup untimed and --steps timed ASPOT solves of exactly --max-iter
    iterations (no stop test) on the cloud workload (or, with --workload
    dense_4096, the dense FP32 cost at gamma 0.03) at size n."""
    import torch
    import paper_2601_17196_gb300 as pkg
    import pot_workloads as W
    dense = args.workload == "dense_4096"
    pb = W.dense_4096(0, n=args.n, gamma=0.03) if dense else W.cloud_32k(0, n=args.n)
    dp = pkg.DeviceProblem.from_workload(pb, device="cuda")
    rule = 1 if args.block_rule == "greedy" else 0
    stream = torch.cuda.Stream()
    solve = lambda: pkg.aspot_solve(dp, pb.gamma, pb.eps, max_iter=args.max_iter, flags=pkg.FLAG_NO_STOP,
                                    block_rule=rule)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            solve()
        torch.cuda.synchronize()
        e0, e1 = _ev(), _ev()
        e0.record(stream)
        for _ in range(args.steps):
            res = solve()
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    print(json.dumps({"mode": "iters", "workload": "dense" if dense else "cloud", "n": args.n,
                      "block_rule": args.block_rule, "iters": res.iters, "ms_per_solve": ms,
                      "us_per_iter": 1e3 * ms / max(res.iters, 1), "launches_per_solve": res.kernel_launches,
                      "loop": "single-cluster" if res.cluster_loop else "staged"}), flush=True)


def _ev():
    import torch
    return torch.cuda.Event(enable_timing=True)


def _timed(stream, fn, warmup, steps, min_s=0.6, flush=None, gpu_index=0):
    """`warmup` untimed calls of fn, then at least `steps` timed calls, more
    until `min_s` seconds have passed (so that the clock sampler sees the
    region).  CUDA events on `stream` around each call; with `flush`, a
    buffer larger than L2 is written before each timed call.  Returns (last
    result, list of ms per call, clocks over the timed calls)."""
    import torch
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        clk = Clocks(gpu_index)
        clk.start()
        ev, out, t0 = [], None, time.perf_counter()
        while len(ev) < steps or time.perf_counter() - t0 < min_s:
            if flush is not None:
                flush.zero_()
            e0, e1 = _ev(), _ev()
            e0.record(stream)
            out = fn()
            e1.record(stream)
            ev.append((e0, e1))
            if len(ev) >= steps:
                e1.synchronize()
        torch.cuda.synchronize()
        clocks = clk.stop()
    return out, [a.elapsed_time(b) for a, b in ev], clocks


_FLUSH = {}


def _flush_buf(dev):
    import torch
    if dev not in _FLUSH:
        _FLUSH[dev] = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    return _FLUSH[dev]


def l2_copy_gbs(dev="cuda"):
    """Measured L2-resident copy bandwidth: b.copy_(a) on two 32 MiB buffers
    (both stay in the 129 MB L2), read + write bytes over CUDA-event time,
    best of 5 rounds of 50 copies.  The denominator of the passes whose
    operand sits in L2 (the 64 MiB cost of the 4096-point dense workload)."""
    import torch
    a = torch.empty(32 * 1024 * 1024, dtype=torch.uint8, device=dev)
    b = torch.empty_like(a)
    a.fill_(1)
    best = 0.0
    for _ in range(5):
        b.copy_(a)
        e0, e1 = _ev(), _ev()
        e0.record()
        for _ in range(50):
            b.copy_(a)
        e1.record()
        e1.synchronize()
        best = max(best, 50 * 2 * a.numel() / (e0.elapsed_time(e1) * 1e-3) / 1e9)
    return best


def dense_study(args, quick=False, dev="cuda"):
    """Dense FP32 cost, n = m = 4096 (and a 16384 point, 1 GiB of cost, for the
    HBM claim): ASPOT to eps at gamma in {0.1, 0.03, 0.01}; achieved bytes of
    the CUDA-core pass = 4 n m per launch over its CUDA-event time (in-loop
    passes, POT_FLAG_PROFILE), against the measured HBM copy bandwidth (1 GiB
    cost) or the measured L2 copy bandwidth (64 MiB cost, L2-resident during
    the solve).  Per iteration: the algorithmic bytes of three full passes
    (4 n m each) over the iteration's time."""
    import torch
    import paper_2601_17196_gb300 as pkg
    import pot_workloads as W
    burst, sustained, hbm, src = _peaks()
    l2 = l2_copy_gbs(dev)
    out = {"workload": "dense_4096: 64-D X~N(0,I), Y 90% N(0,I) + 10% N(4*1,I), FP32 cost / max, masses 1.0 / 1.3, "
                       "s=0.9, eps=1e-2; plus n=16384 (1 GiB cost) for the HBM point",
           "hbm_peak_gbs": hbm, "hbm_peak_source": src, "l2_copy_gbs_measured": l2, "rows": []}
    stream = torch.cuda.Stream(device=dev)
    warm, steps = (3, 5) if quick else (args.warmup, args.steps)
    flush = _flush_buf(dev)
    for n, gammas in ((4096, (0.1, 0.03, 0.01)), (16384, (0.03,))):
        for gam in gammas:
            pb = W.dense_4096(0, n=n, gamma=gam)
            dp = pkg.DeviceProblem.from_workload(pb, device=dev)
            res, ms, clocks = _timed(stream, lambda: pkg.aspot_solve(dp, gam, pb.eps, max_iter=args.max_iter),
                                     warm, steps, flush=flush)
            t = sum(ms) / len(ms)
            it = res.iters
            # one more solve with every main-loop pass timed by CUDA events (kept out of the timed solves)
            with torch.cuda.stream(stream):
                prof = pkg.aspot_solve(dp, gam, pb.eps, max_iter=args.max_iter, flags=pkg.FLAG_PROFILE)
            pms = prof.pass_ms / max(prof.pass_launches, 1)
            gbs = 4.0 * n * n / (pms * 1e-3) / 1e9
            peak = hbm if n == 16384 else l2
            iter_us = 1e3 * t / it
            row = {"n": n, "gamma": gam, "iters": it, "time_to_eps_ms": t, "it_per_s": it / (t / 1e3),
                   "kernel": pkg.pass_kernel(dp, pkg.FLAG_PROFILE), "clocks": clocks,
                   "pass_ms": pms, "passes_per_iter": prof.pass_launches / max(prof.iters, 1),
                   "launches_per_iter": res.kernel_launches / max(it, 1),
                   "roofline": {"bound": "hbm" if n == 16384 else "l2", "achieved": gbs, "peak": peak,
                                "unit": "GB/s", "frac": gbs / peak,
                                "peak_source": (f"{src} HBM copy" if n == 16384 else
                                                "measured L2-resident copy (64 MiB cost stays in L2)"),
                                "bytes_per_launch": 4.0 * n * n},
                   "per_iteration": {"us": iter_us, "algorithmic_bytes_3_passes": 12.0 * n * n,
                                     "achieved_GBps": 12.0 * n * n / (iter_us * 1e-6) / 1e9,
                                     "frac_of_peak": 12.0 * n * n / (iter_us * 1e-6) / 1e9 / peak},
                   "objective": res.objective, "converged": res.status == 0}
            if n == 16384:
                # DRAM bytes of one two-sided dense_pass_kernel launch at this size, from one ncu
                # capture of the current kernel (dram__bytes_read.sum + dram__bytes_write.sum)
                row["roofline"]["traffic"] = DENSE_16K_TRAFFIC
            if not args.no_greedy:
                rg, gms, gclk = _timed(stream, lambda: pkg.aspot_solve(dp, gam, pb.eps, max_iter=args.max_iter,
                                                                        block_rule=pkg.BLOCK_GREEDY),
                                       warm, steps, flush=flush)
                gt = sum(gms) / len(gms)
                row["greedy_rule"] = {"iters": rg.iters, "time_to_eps_ms": gt, "it_per_s": rg.iters / (gt / 1e3),
                                      "objective": rg.objective, "converged": rg.status == 0,
                                      "time_to_eps_vs_cyclic": gt / t, "clocks": gclk}
            out["rows"].append(row)
            del dp
            torch.cuda.empty_cache()
    return out


def scaling_study(args, dev="cuda"):
    """Runtime of 1500 fixed ASPOT iterations vs n (appendix scalability study):
    masses 5 / 3, s = 0.6, gamma = 1e-3, 2-D points, dense FP32 cost; the
    log-log slope is compared with the paper's ~2.27 (its hardware unstated)."""
    import numpy as np
    import torch
    import paper_2601_17196_gb300 as pkg
    import pot_workloads as W
    ns = [200, 300, 500, 1000, 1500, 2000, 2500, 3000, 3500, 4000]
    rows = []
    stream = torch.cuda.Stream(device=dev)
    clk = Clocks(0)
    clk.start()
    for n in ns:
        pb = W.scaling_e4(0, n=n)
        dp = pkg.DeviceProblem.from_workload(pb, device=dev)
        r, ms, _ = _timed(stream, lambda: pkg.aspot_solve(dp, pb.gamma, pb.eps, max_iter=1500,
                                                           flags=pkg.FLAG_NO_STOP),
                          1, 1, min_s=0.0)
        rows.append({"n": n, "ms": ms[0], "us_per_iter": 1e3 * ms[0] / 1500, "iters": r.iters,
                     "launches_per_iter": r.kernel_launches / 1500.0, "E": r.err_final,
                     "loop": "single-cluster" if r.cluster_loop else "staged"})
    clocks = clk.stop()
    x = np.log([q["n"] for q in rows])
    y = np.log([q["ms"] for q in rows])
    slope = float(np.polyfit(x, y, 1)[0])
    big = [q for q in rows if q["n"] >= 1500]
    slope_big = float(np.polyfit(np.log([q["n"] for q in big]), np.log([q["ms"] for q in big]), 1)[0])
    return {"workload": "scaling_e4: 2-D U[0,1]^2 points, masses 5/3, s=0.6, gamma=1e-3, 1500 fixed iterations",
            "rows": rows, "loglog_slope": slope, "loglog_slope_n_ge_1500": slope_big, "paper_slope": 2.27,
            "paper_slope_note": "the paper's slope is CPU-side context (hardware unstated), not a target",
            "clocks": clocks}


def batched_study(args, quick=False, dev="cuda"):
    """512 independent 3-D instances (n_k, m_k ~ U{64..2048}), solved in
    lockstep by aspot_solve_batched to each one's own threshold: default
    tiles, the autotuner (first call times the candidates, later calls hit
    the cache) and the greedy block rule."""
    import torch
    import paper_2601_17196_gb300 as pkg
    import pot_workloads as W
    insts = W.batch_3d(seed=0, count=512)
    probs = [pkg.DeviceProblem.from_workload(pb, device=dev) for pb in insts]
    elems = sum(p.n * p.m for p in probs)
    stream = torch.cuda.Stream(device=dev)
    warm, steps = (2, 3) if quick else (args.warmup, args.steps)
    flush = _flush_buf(dev)
    res, ms, clocks = _timed(stream, lambda: pkg.aspot_solve_batched(probs, 0.05, 1e-3, max_iter=args.max_iter),
                             warm, steps, flush=flush)
    t = sum(ms) / len(ms)
    its = [r.iters for r in res]
    out = {"workload": "batch_3d: 512 instances, n_k,m_k~U{64..2048}, U[0,1]^3 FP32 points, |r|=1, "
                       "|c|~U[1,1.5], s_k~U[0.5,0.95], gamma=0.05, eps=1e-3",
           "instances": len(probs), "cost_entries": elems,
           "ms_all_to_eps": t, "instances_per_s": len(probs) / (t / 1e3),
           "iters_max": max(its), "iters_mean": sum(its) / len(its),
           "launches_per_iter": res[0].kernel_launches / max(max(its), 1),
           "converged": sum(r.status == 0 for r in res), "kernel_launches": res[0].kernel_launches,
           "tile": [res[0].tile_rows, res[0].tile_cols], "clocks": clocks,
           "entry_sweeps_per_s": elems * max(its) / (t / 1e3)}
    pkg.autotune_clear()
    with torch.cuda.stream(stream):
        t0 = time.perf_counter()
        first = pkg.aspot_solve_batched(probs, 0.05, 1e-3, max_iter=args.max_iter, flags=pkg.FLAG_AUTOTUNE)
        torch.cuda.synchronize()
        first_ms = (time.perf_counter() - t0) * 1e3
    rt, tms, tclk = _timed(stream, lambda: pkg.aspot_solve_batched(probs, 0.05, 1e-3, max_iter=args.max_iter,
                                                                    flags=pkg.FLAG_AUTOTUNE),
                           warm, steps, flush=flush)
    tt = sum(tms) / len(tms)
    out["autotuned"] = {"tile": [rt[0].tile_rows, rt[0].tile_cols], "tune_ms": first[0].tune_ms,
                        "first_call_ms": first_ms, "ms_all_to_eps": tt,
                        "instances_per_s": len(probs) / (tt / 1e3), "vs_default_tile": tt / t,
                        "converged": sum(r.status == 0 for r in rt), "clocks": tclk}
    if not args.no_greedy:
        rg, gms, gclk = _timed(stream, lambda: pkg.aspot_solve_batched(probs, 0.05, 1e-3, max_iter=args.max_iter,
                                                                        flags=pkg.FLAG_AUTOTUNE,
                                                                        block_rule=pkg.BLOCK_GREEDY),
                               warm, steps, flush=flush)
        gt = sum(gms) / len(gms)
        gits = [r.iters for r in rg]
        out["greedy_rule_autotuned"] = {"ms_all_to_eps": gt, "instances_per_s": len(probs) / (gt / 1e3),
                                        "iters_max": max(gits), "iters_mean": sum(gits) / len(gits),
                                        "converged": sum(r.status == 0 for r in rg), "vs_default": gt / t,
                                        "clocks": gclk}
    return out


def small_study(args, quick=False, dev="cuda"):
    """The 256-point configuration (X ~ U[0,1]^2, Y ~ N((.5,.5), 0.1^2 I),
    masses 1.0 / 1.2, s = 0.8, gamma = 0.05, eps = 1e-3, dense FP32 cost):
    ASPOT and the feasible Sinkhorn baseline to their thresholds, and the
    tuned-gamma Sinkhorn of Theorem 2 for p in {1, 1.5, 2, 3, 4} (gamma =
    (2 eps / (49 H_min))^(1/p), eps' = H_min gamma^p; p = 1 only outside
    `quick`, it takes ~1e5 iterations), iterations, time to epsilon and
    <C, X>; the FP64 oracle's ASPOT on the same instance beside it."""
    import torch
    import paper_2601_17196_gb300 as pkg
    import pot_workloads as W
    from oracle import pot as O
    pb = W.small_dense(0)
    dp = pkg.DeviceProblem.from_workload(pb, device=dev)
    stream = torch.cuda.Stream(device=dev)
    warm, steps = (3, 10) if quick else (args.warmup, args.steps)
    rows = []
    r, ms, clocks = _timed(stream, lambda: pkg.aspot_solve(dp, pb.gamma, pb.eps, max_iter=args.max_iter),
                           warm, steps)
    t = sum(ms) / len(ms)
    # the same solve with the iterations as separate kernels (the single-cluster
    # loop's alternative), and the pass times from one extra, profiled solve
    # (profiling times each pass of the staged loop)
    rs, ms_s, _ = _timed(stream, lambda: pkg.aspot_solve(dp, pb.gamma, pb.eps, max_iter=args.max_iter,
                                                         flags=pkg.FLAG_STAGED), warm, steps)
    t_s = sum(ms_s) / len(ms_s)
    with torch.cuda.stream(stream):
        prof = pkg.aspot_solve(dp, pb.gamma, pb.eps, max_iter=args.max_iter, flags=pkg.FLAG_PROFILE)
    pms = prof.pass_ms / max(prof.pass_launches, 1)
    aspot = {"solver": "aspot", "gamma": r.gamma, "iters": r.iters, "time_to_eps_ms": t, "objective": r.objective,
             "converged": r.status == 0, "us_per_iter": 1e3 * t / r.iters, "clocks": clocks,
             "loop": "single-cluster" if r.cluster_loop else "staged",
             "staged_loop": {"iters": rs.iters, "time_to_eps_ms": t_s, "us_per_iter": 1e3 * t_s / rs.iters,
                             "launches_per_iter": rs.kernel_launches / rs.iters},
             "kernel": pkg.pass_kernel(dp, pkg.FLAG_PROFILE), "pass_us": 1e3 * pms,
             "launches_per_iter": r.kernel_launches / r.iters,
             "roofline": {"bound": "latency", "note": "0.25 MiB cost: a pass is a few microseconds of launch and "
                                                     "reduction latency; the HBM roofline of 3 passes (0.75 MiB) "
                                                     "is 0.1 us",
                          "achieved_pass_GBps": 4.0 * 256 * 256 / (pms * 1e-3) / 1e9}}
    rows.append(aspot)
    r, ms, clocks = _timed(stream, lambda: pkg.sinkhorn_pot_solve(dp, pb.gamma, pb.eps, max_iter=200000),
                           warm, steps)
    t = sum(ms) / len(ms)
    rows.append({"solver": "sinkhorn", "gamma": r.gamma, "iters": r.iters, "time_to_eps_ms": t,
                 "objective": r.objective, "converged": r.status == 0, "clocks": clocks})
    for p in ((1.5, 2.0, 3.0, 4.0) if quick else (1.0, 1.5, 2.0, 3.0, 4.0)):
        r, ms, clocks = _timed(stream, lambda: pkg.sinkhorn_pot_solve(dp, 0.0, pb.eps, max_iter=200000, p_tune=p),
                               1, 1, min_s=0.0)
        rows.append({"solver": f"tuned sinkhorn p={p}", "gamma": r.gamma, "eps_prime": r.eps_stop, "iters": r.iters,
                     "time_to_eps_ms": ms[0], "objective": r.objective, "converged": r.status == 0})
    t0 = time.time()
    C = O.sqeuclid_cost(pb.X, pb.Y, pb.cost_scale) if pb.C is None else pb.C.astype("float64")
    ora = O.solve_aspot(C, pb.r, pb.c, pb.s, pb.eps, pb.gamma)
    cpu_ms = (time.time() - t0) * 1e3
    return {"workload": "small_dense n=m=256 gamma=0.05 eps=1e-3 (masses 1.0/1.2, s=0.8)", "rows": rows,
            "oracle_aspot": {"iters": ora.iters, "ms": cpu_ms, "objective": ora.objective, "cores": 1,
                             "kind": "oracle"},
            "objective_rel_diff_gpu_vs_oracle": abs(aspot["objective"] - ora.objective) / ora.objective,
            "time_to_eps_gpu_over_oracle": aspot["time_to_eps_ms"] / cpu_ms}


def registration_study(args, quick=False, dev="cuda"):
    """Batched rigid registration (appendix, point cloud registration) of 64
    synthetic partial clouds: target n = 1024 points on three ellipsoid
    surfaces, source = half of it moved by up to 0.25 rad and 0.08, alpha =
    0.6, gamma 0.02 annealed by 0.83 to 0.002, eps = 1e-3; every outer step is
    one batched ASPOT solve of the pairs still moving plus the plan-moment /
    Procrustes kernel."""
    import numpy as np
    import torch
    from paper_2601_17196_gb300 import registration as PR
    import pot_workloads as W
    K = 64
    pairs, truth = [], []
    for seed in range(K):
        X, Y0, Rt, tt = W.registration_3d(seed, n=1024, frac=0.5, max_angle=0.25, max_shift=0.08)
        pairs.append((X, Y0))
        truth.append((Rt, tt))
    PR.register_batched(pairs[:2], alpha=0.6, max_reg=2, autotune=False)          # warm-up (build, caches)
    torch.cuda.synchronize()
    clk = Clocks(0)
    clk.start()
    t0 = time.time()
    out = PR.register_batched(pairs, alpha=0.6, gamma0=0.02, anneal=0.83, gamma_min=0.002, eps=1e-3, max_reg=40,
                              autotune=False)
    torch.cuda.synchronize()
    wall = time.time() - t0
    clocks = clk.stop()
    err = np.array([max(np.abs(r.R - Rt).max(), np.abs(r.t - tt).max()) for r, (Rt, tt) in zip(out, truth)])
    regs = np.array([r.registrations for r in out])
    inner = np.array([r.inner_iterations for r in out])
    res = {"workload": "registration: 64 pairs, target n=1024 (3 ellipsoid surfaces), source = half, "
                       "<=0.25 rad, <=0.08 shift, alpha=0.6, gamma 0.02*0.83^k >= 0.002, eps=1e-3",
           "wall_s": wall, "pairs": K, "registrations_mean": float(regs.mean()),
           "registrations_max": int(regs.max()), "aspot_iters_per_registration": float(inner.sum() / regs.sum()),
           "converged_pairs": int(sum(r.converged for r in out)),
           "motion_error_median": float(np.median(err)), "motion_error_p90": float(np.quantile(err, 0.9)),
           "pairs_within_0.06": int((err < 0.06).sum()), "clocks": clocks}
    if not quick:
        import paper_2601_17196_gb300 as pkg
        pkg.autotune_clear()
        tune = {}
        for leg in ("first_call_s", "wall_s"):
            torch.cuda.synchronize()
            t0 = time.time()
            PR.register_batched(pairs, alpha=0.6, gamma0=0.02, anneal=0.83, gamma_min=0.002, eps=1e-3, max_reg=40,
                                autotune=True)
            torch.cuda.synchronize()
            tune[leg] = time.time() - t0
        tune["vs_default_tile"] = tune["wall_s"] / wall
        res["autotuned"] = tune
    return res


def run_ws_train(args):
    """Training-step throughput of the warm-start network kernels: Adam steps
    on batches of 32 instances of 2048 points (random features of the
    network's shape, pot_workloads.ws_batch), BF16 tcgen05 and FP32 CUDA-core
    modes.  Tensor-core work per point and step: the 128 x 128 products of
    the forward pass, of training pass A (forward, dW2) and of pass B
    (forward, dH1) plus the N = 16 product of dW1: 2 * 128 * (5 * 128 + 16)
    FLOP."""
    import numpy as np
    import torch
    from paper_2601_17196_gb300 import warmstart as WS
    import pot_workloads as W
    burst, sustained, hbm, src = _peaks()
    K, npts = 256, 2048
    feats, extra, target, off = W.ws_batch([npts] * K, d=2, seed=0)
    fs = WS.FeatureSet(2, torch.from_numpy(feats).cuda(), torch.from_numpy(extra).cuda(), off,
                       torch.from_numpy(target).cuda())
    rows = []
    stream = torch.cuda.Stream()
    for mode in (WS.MODE_BF16, WS.MODE_FP32):
        net = WS.WarmStartNet(2, seed=0, mode=mode)
        with torch.cuda.stream(stream):
            for k in range(args.warmup):
                net.train_step(fs, list(range(32 * (k % 8), 32 * (k % 8) + 32)), lr=1e-3)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            steps = max(args.steps, 20)
            e0.record(stream)
            for k in range(steps):
                net.train_step(fs, list(range(32 * (k % 8), 32 * (k % 8) + 32)), lr=1e-3)
            e1.record(stream)
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        flop = 32 * npts * 2.0 * 128 * (5 * 128 + 16)
        rows.append({"mode": "bf16 tcgen05" if mode == WS.MODE_BF16 else "fp32 cuda cores", "ms_per_step": ms,
                     "points_per_step": 32 * npts, "points_per_s": 32 * npts / (ms / 1e3),
                     "contraction_tflops": flop / (ms * 1e-3) / 1e12,
                     "frac_of_bf16_peak": flop / (ms * 1e-3) / 1e12 / burst})
    print(json.dumps({"workload": "warm-start network training: Adam steps of 32 instances x 2048 points",
                      "rows": rows, "peak_bf16_tflops": burst, "peak_source": src}), flush=True)


def warm_start_study(n_train: int, n_eval: int, epochs: int, mode: int = 1, batch: int = 32, lr: float = 3e-3,
                     device="cuda", greedy: bool = False) -> dict:
    """Learned warm start on the 2-D mixture workload (n = m = 1024, 2-6
    Gaussians per cloud, masses U[1,1.5], s ~ U[0.6,0.95] x min mass,
    gamma = 0.02, eps = 1e-3): a training set of n_train instances (seeds
    10000 + k) labelled with the duals batched GPU ASPOT converges to, Adam on
    the GPU, then n_eval held-out seeds (0 .. n_eval-1) solved from zero and
    from the network's start (with the E(z_warm) > E(0) fallback).  Times are
    CUDA events on the solve stream; the warm time includes the warm start
    itself (features, network, shift step) and the fallback check.  With
    ``greedy`` the held-out seeds are also solved with the greedy block rule,
    from zero and from the same warm start."""
    import numpy as np
    import torch
    import paper_2601_17196_gb300 as pkg
    from paper_2601_17196_gb300 import warmstart as WS
    import pot_workloads as W
    gamma, eps = 0.02, 1e-3
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        t0 = time.time()
        train = [pkg.DeviceProblem.from_workload(W.mix_2d(10_000 + k), device=device, kind=pkg.COST_SQEUCLID_F32)
                 for k in range(n_train)]
        fs, iters = WS.build_training_set(train, gamma, eps)
        torch.cuda.synchronize()
        t1 = time.time()
        del train
        net = WS.WarmStartNet(2, seed=0, mode=mode, device=device)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        hist = net.fit(fs, epochs=epochs, batch=batch, lr=lr, lr_final=lr * 0.01, seed=0)
        e1.record(stream)
        torch.cuda.synchronize()
        train_ms = e0.elapsed_time(e1)
        steps = net.step
        del fs
        cold_it, warm_it, cold_ms, warm_ms, used, gap, g_rows = [], [], [], [], [], [], []
        clk = Clocks(0)
        clk.start()
        for k in range(n_eval):
            dp = pkg.DeviceProblem.from_workload(W.mix_2d(k), device=device, kind=pkg.COST_SQEUCLID_F32)
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            c = pkg.aspot_solve(dp, gamma, eps, max_iter=20000)
            a1.record(stream)
            b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            b0.record(stream)
            w = net.solve(dp, gamma, eps)
            b1.record(stream)
            torch.cuda.synchronize()
            cold_it.append(c.iters); warm_it.append(w.iters)
            cold_ms.append(a0.elapsed_time(a1)); warm_ms.append(b0.elapsed_time(b1))
            used.append(w.warm_used); gap.append(abs(w.objective - c.objective))
            if greedy:
                g0, g1, h0, h1 = (torch.cuda.Event(enable_timing=True) for _ in range(4))
                g0.record(stream)
                gc = pkg.aspot_solve(dp, gamma, eps, max_iter=20000, block_rule=pkg.BLOCK_GREEDY)
                g1.record(stream)
                h0.record(stream)
                gw = net.solve(dp, gamma, eps, block_rule=pkg.BLOCK_GREEDY)
                h1.record(stream)
                torch.cuda.synchronize()
                g_rows.append((gc.iters, gw.iters, g0.elapsed_time(g1), h0.elapsed_time(h1), gw.warm_used))
        clocks = clk.stop()
    ci, wi = np.array(cold_it, dtype=float), np.array(warm_it, dtype=float)
    cm, wm = np.array(cold_ms), np.array(warm_ms)
    greedy_out = None
    if g_rows:
        G = np.array(g_rows, dtype=float)
        greedy_out = {"cold_iters_mean": float(G[:, 0].mean()), "warm_iters_mean": float(G[:, 1].mean()),
                      "cold_ms_mean": float(G[:, 2].mean()), "warm_ms_mean": float(G[:, 3].mean()),
                      "iters_ratio_warm_over_cold": float(G[:, 1].mean() / G[:, 0].mean()),
                      "time_ratio_warm_over_cold": float(G[:, 3].mean() / G[:, 2].mean()),
                      "fallback_fraction": float(1.0 - G[:, 4].mean()),
                      "cold_greedy_over_cold_cyclic_time": float(G[:, 2].mean() / cm.mean())}
    return {"workload": "mix_2d n=m=1024 gamma=0.02 eps=1e-3", "train_instances": n_train, "eval_seeds": n_eval,
            "greedy_rule": greedy_out,
            "mode": "bf16 tcgen05" if mode == 1 else "fp32", "data_gen_s": t1 - t0,
            "train_iters_mean": float(iters.mean()), "train_steps": steps, "train_ms": train_ms,
            "train_ms_per_step": train_ms / max(steps, 1), "loss_first_epoch": hist[0], "loss_last_epoch": hist[-1],
            "cold_ms_mean": float(cm.mean()), "warm_ms_mean": float(wm.mean()),
            "time_ratio_warm_over_cold": float(wm.mean() / cm.mean()),
            "cold_iters_mean": float(ci.mean()), "warm_iters_mean": float(wi.mean()),
            "iters_ratio_warm_over_cold": float(wi.mean() / ci.mean()),
            "median_per_seed_iters_ratio": float(np.median(wi / ci)),
            "fallback_fraction": float(1.0 - np.mean(used)), "max_objective_gap": float(max(gap)),
            "clocks": clocks}


def run_warmstart(args):
    r = warm_start_study(args.ws_train, args.ws_eval, args.ws_epochs, greedy=not args.no_greedy)
    r.update({"metric": "time-to-epsilon (ms) of warm-started ASPOT, learned warm start vs cold start",
              "value": r["warm_ms_mean"], "unit": "ms", "higher_is_better": False, "n_gpus": 1,
              "dtype": "bf16 network, fp32 passes, fp64 duals", "data": "synthetic"})
    print(json.dumps(r), flush=True)


def main():
    args = _args()
    if args.workload == "warmstart":
        run_warmstart(args)
        return
    if args.workload == "small_dense":
        print(json.dumps(small_study(args)), flush=True)
        return
    if args.workload == "registration":
        print(json.dumps(registration_study(args)), flush=True)
        return
    if args.workload == "ws_train":
        run_ws_train(args)
        return
    if args.mode == "pass":
        run_pass_only(args)
        return
    if args.mode == "iters":
        run_iters_only(args)
        return
    if args.workload == "batch_3d":
        print(json.dumps(batched_study(args)), flush=True)
        return
    if args.workload == "dense_4096":
        print(json.dumps(dense_study(args)), flush=True)
        return
    if args.workload == "scaling_e4":
        print(json.dumps(scaling_study(args)), flush=True)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
