#!/usr/bin/env python
"""Benchmark of the Stokes boundary-integral hot path on one GB300 (or N replicas).

Default workload (the largest single-GPU configuration): helical pipe of helix radius 3,
pitch 2, 4 turns, tube radius 1, 2048 panels x 8 Gauss-Legendre x 64 trapezoid = 1,048,576
wall nodes plus two 16 x 64 end caps, and 100 rigid spheres of radius 0.2 (600 nodes each)
inside: 1,110,624 nodes.  Operator K = I/2 + D + eta S (paper Eq. stokes-bie-new) with
eta = 1/(2 eps log(1/eps)), eps = tube radius x centreline curvature.

One step = one operator apply K sigma in compensated FP32 (density pack, the combined-field
pair sum over all 1.23e12 node pairs, FP64 reduction with the diagonal term), the work of
every GMRES iteration.  Inputs are resident in HBM before the timed region; the tile shape
is autotuned once before it.  The L2 cache is flushed (256 MiB write) between steps,
outside the timed intervals.

metric: pair interactions per second of the apply.  Reported beside it: the pair-sum
kernel's fraction of the FP32 CUDA-core peak (roofline), the end-to-end rate of the same
apply through the host-buffer C-ABI call (stokes_apply_host: geometry and density copied
from pinned host memory, result copied back), the FP64 CPU oracle on sampled rows of the
same operator, and the GMRES solve times to 1e-10 (FP32-mixed vs plain FP64) of the
curved-pipe system and of the 64-segment batch.

Other workloads (--workload): curved_pipe (GMRES-IR solve as the timed step),
precision_sweep, batch, helix (the full solve of the helix system), laplace, mobility,
quadrature, peaks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "pair interactions/s and GMRES solve time at 1e-10 residual, FP32-mixed vs plain FP64"
UNIT = "pairs/s"
FLOPS_PER_PAIR = {"sl": 28, "dl": 29, "cf": 37}   # algorithmic FP32 flops per pair (FMA = 2)
WORKLOAD = "curved_pipe_arc90_Rc5_R1_16384wall_2048cap_gmres_ir_1e-10"
HEADLINE = ("helix_a3_pitch2_4turns_R1_1048576wall_2048cap_100spheres_1110624nodes_"
            "combined_field_apply_fp32c")
L2_FLUSH_BYTES = 256 << 20


def parse_args_for_test():
    """Default arguments, as `python bench.py` with no flags."""
    return parse([])


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sbq", choices=["sbq", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="CPU work bound of the oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--kernel-reps", type=int, default=20)
    ap.add_argument("--resid-prec", default="fp64", choices=["fp64", "df32"],
                    help="precision of the refinement residuals b - K x of the timed solve: "
                         "fp64 (default), or df32 (double-float, used where its rounding-error "
                         "bound certifies the tolerance); the other one is timed beside it and "
                         "the returned x is checked with an FP64 residual either way")
    ap.add_argument("--no-correction", action="store_true",
                    help="solve with the punctured sums alone (no double-layer singularity "
                         "subtraction)")
    ap.add_argument("--workload", default="headline",
                    choices=["headline", "curved_pipe", "precision_sweep", "batch", "helix",
                             "laplace", "mobility", "quadrature", "peaks", "tree"],
                    help="headline: the benchmark line (default, helix apply); curved_pipe: "
                         "GMRES-IR solves as the step; precision_sweep: FP32 vs compensated "
                         "FP32 vs FP64 pair sums on random loops of 64K/256K/1M nodes; batch: "
                         "64 independent capped arcs in one persistent launch")
    ap.add_argument("--no-extras", action="store_true",
                    help="headline: skip the curved-pipe and batch solves reported beside it")
    ap.add_argument("--sizes", default="512,2048,8192",
                    help="precision_sweep: panel counts of the random loops (x 128 nodes)")
    ap.add_argument("--helix-panels", type=int, default=2048,
                    help="headline and helix: axial panels of the helical wall (2048 -> "
                         "1,048,576 wall nodes; smaller values for profiler captures)")
    ap.add_argument("--helix-pitch", type=float, default=3.0,
                    help="helix: pitch (at 2 the tube surfaces of adjacent turns are 0.011 "
                         "apart, which the punctured sums cannot resolve)")
    ap.add_argument("--quad-panels", type=int, default=512,
                    help="quadrature: panels of the random loop (x 128 nodes)")
    ap.add_argument("--near-factor", type=float, default=1.0,
                    help="quadrature: near region of an element, radius + f max(length, 2 radius)")
    ap.add_argument("--tree-panels", default="8192,32768",
                    help="tree: loop panel counts (8 x 16 nodes each), comma separated")
    ap.add_argument("--tree-solve-panels", type=int, default=2048,
                    help="tree: loop panels of the GMRES-IR solve with treecode inner solves (0: none)")
    ap.add_argument("--build-only", action="store_true",
                    help="quadrature: only build the Stokes E of the random loop (--quad-panels), "
                         "--kernel-reps times inside the NVTX range 'kernel_only'")
    ap.add_argument("--iteration-study", action="store_true",
                    help="quadrature: also solve the corrected loop systems with plain FP64 "
                         "GMRES(100) and GMRES(256) and with the mixed solver at GMRES(256) "
                         "(minutes at 196K nodes)")
    ap.add_argument("--fp64-solve", action="store_true",
                    help="batch: also time the plain FP64 GMRES solve (minutes)")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch the Arnoldi steps from the host instead of the CUDA graph "
                         "(profilers cannot resolve kernels inside graphs with while nodes)")
    ap.add_argument("--kernel-only", default=None, choices=["fp32c", "fp32", "fp64", "df32"],
                    help="only time operator applies of this precision on the workload "
                         "(inside an NVTX range 'kernel_only', for profilers)")
    return ap.parse_args(argv)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(ms, world, device=None):
    """The slowest rank's time (the job's time): all-reduce MAX over the process group."""
    if world <= 1:
        return float(ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(pairs_per_step, ms, world):
    """Whole-job throughput of `world` independent replicas (weak scaling): every rank
    processes pairs_per_step per step, the job takes the slowest rank's ms."""
    return world * float(pairs_per_step) / (float(ms) * 1e-3)


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clk", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
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
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            if self.uuid and parts[1] != self.uuid:
                continue
            rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i] == "Active"})
        loaded = [v for v in sm if mx and v > 0.3 * max(mx)] or sm
        return {"sm_mhz": float(np.median(loaded)) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def gpu_uuid():
    import torch
    try:
        u = str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


# ---------------------------------------------------------------------------
# CPU oracle (baseline leg and the reference arm)
# ---------------------------------------------------------------------------
def oracle_rate(seconds, rows_per_call=1024):
    """FP64 CPU oracle on the curved-pipe operator: rows of K sigma evaluated in blocks of
    `rows_per_call` targets until `seconds` of CPU work have passed; pairs/s."""
    import oracle
    from paper_2310_00889_gb300 import inputs as I
    oracle.build()
    c = I.config2()
    s = c["surf"]
    eta = 1.0 / (2 * 0.2 * np.log(5.0))
    sig = I.density(s.size, seed=12)
    pairs, t0, k = 0.0, time.perf_counter(), 0
    while True:
        a = (k * rows_per_call) % s.size
        b = min(s.size, a + rows_per_call)
        oracle.combined(s.x, s.n, s.w, sig, s.x[:, a:b], eta, 1.0)
        pairs += float(b - a) * s.size
        k += 1
        dt = time.perf_counter() - t0
        if dt >= seconds:
            break
    return pairs / dt, oracle.num_threads(), dict(rows=int(pairs / s.size), seconds=dt)


def headline_inputs(panels=2048):
    """The headline workload's geometry, eps and density (seeded; shared by both arms)."""
    from paper_2310_00889_gb300 import inputs as I
    c = I.config5(panels=panels, pitch=2.0)
    s = c["surf"]
    return s, c["slenderness"], I.density(s.size, seed=12)


def oracle_rows(s, eps, sig, rows):
    """K sigma = sigma/2 + (D + eta S) sigma at the node rows `rows` (FP64 CPU oracle)."""
    import oracle
    eta = float(oracle.eta_slender(eps))
    return oracle.combined(s.x, s.n, s.w, sig, s.x[:, rows], eta, 1.0) + 0.5 * sig[:, rows]


def oracle_sample(s, eps, sig, seconds, rows_per_call=256, seed=4):
    """The cpu_baseline leg: the oracle evaluates random rows of the headline operator in
    blocks until `seconds` have passed.  Returns (pairs/s, threads, rows, values, seconds)."""
    import oracle
    oracle.build()
    n = s.size
    order = np.random.default_rng(seed).permutation(n)
    got_rows, vals, t0, k = [], [], time.perf_counter(), 0
    while True:
        r = np.sort(order[k * rows_per_call:(k + 1) * rows_per_call])
        vals.append(oracle_rows(s, eps, sig, r))
        got_rows.append(r)
        k += 1
        dt = time.perf_counter() - t0
        if dt >= seconds or (k + 1) * rows_per_call > n:
            break
    rows = np.concatenate(got_rows)
    return (float(rows.size) * n / dt, oracle.num_threads(), rows,
            np.concatenate(vals, axis=1), dt)


def run_reference(args):
    """The reference arm: the FP64 CPU oracle (the only other implementation: the paper
    ships no code) on the headline workload, each step a sample of operator rows."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    s, eps, sig = headline_inputs(args.helix_panels)
    n = s.size
    rows = 256
    order = np.random.default_rng(4).permutation(n)

    def step(k):
        r = np.sort(order[(k * rows) % (n - rows):][:rows])
        oracle_rows(s, eps, sig, r)

    for k in range(args.warmup):
        step(k)
    t0 = time.perf_counter()
    for k in range(args.steps):
        step(args.warmup + k)
    dt = (time.perf_counter() - t0) / args.steps
    value = rows * float(n) / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": HEADLINE, "nodes": n,
                   "sample": "%d random operator rows x %d sources per step" % (rows, n)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                         "kind": "oracle",
                         "sample": "%d rows of the combined-field operator per step" % rows},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _peak_tflops(info, clocks):
    """FP32 CUDA-core peak: SMs x FP32 lanes x 2 flops x the maximum SM clock (from
    MEASURED_PEAKS.json when present, else the sampled maximum, else 2070 MHz)."""
    sm_max = (clocks or {}).get("sm_max_mhz") or 2070.0
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(peaks_path):
        try:
            sm_max = float(json.load(open(peaks_path)).get("sm_max_mhz", sm_max))
        except Exception:
            pass
    return info["sms"] * info["fp32_lanes_per_sm"] * 2 * sm_max * 1e6 / 1e12, sm_max


def run_headline(args):
    """The benchmark line: compensated-FP32 operator applies on the helix with spheres."""
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    from paper_2310_00889_gb300 import build as b
    b.build()
    from paper_2310_00889_gb300 import sbq

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    t0 = time.perf_counter()
    s, eps, sig_h = headline_inputs(args.helix_panels)
    n = s.size
    gen_s = time.perf_counter() - t0
    eta = sbq.slender_eta(eps)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)
    if args.kernel_only:
        from paper_2310_00889_gb300 import inputs as I
        return kernel_only(args, sbq, I, t(s.x), t(s.n), t(s.w), eta, n, t, dev)
    t0 = time.perf_counter()
    op = sbq.StokesOp(t(s.x), t(s.n), t(s.w), eta)
    # explicit autotuning before the timed region; it also fills the process-wide tuning
    # cache from which the host-buffer call below takes its tile shape
    tune = op.autotune("fp32c")
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t0) * 1e3
    sig = t(sig_h)
    out = torch.empty_like(sig)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        op.matvec(sig, prec="fp32c", out=out)

    sampler = ClockSampler(gpu_uuid())
    sampler.start()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    kms, ams = [], []
    torch.cuda.nvtx.range_push("bench_timed")
    for _ in range(args.steps):
        flush.zero_()
        k, a = op.time_pairsum(sig, prec="fp32c", reps=1, out=out)
        kms.append(k)
        ams.append(a)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = max_over_ranks(float(np.mean(ams)), world, dev)
    pairs = float(n) * n
    value = replica_value(pairs, ms, world)
    kernel_ms = float(np.mean(kms))
    u = out.cpu().numpy()
    stats = op.stats("fp32c")

    info = sbq.device_info()
    peak, sm_max = _peak_tflops(info, clocks)
    achieved = FLOPS_PER_PAIR["cf"] * pairs / (kernel_ms * 1e-3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "traffic": _profiled_traffic("pairsum_f32_comp_helix_1110624.json"),
                "traffic_unit": "bytes per launch (ncu dram read + write, one-pass capture of "
                                "this launch, profiles/pairsum_f32_comp_helix_1110624.json)",
                "traffic_note": "the kernel is ALU-bound: 182 MB per 842 ms launch; reads are "
                                "1.4 x the packed sources and targets (88.8 MB), writes the "
                                "chunk partial sums that leave L2",
                "kernel": "pairsum_f32_kernel<combined field, compensated>",
                "flops_per_pair": FLOPS_PER_PAIR["cf"], "pairs_per_launch": pairs,
                "launch_ms": kernel_ms, "apply_ms": float(np.mean(ams)),
                "timing": "CUDA events on the launching stream around the kernel launch, "
                          "every timed step",
                "peak_basis": "%d SMs x %d FP32 lanes x 2 x %.0f MHz (sm_max_mhz)" % (
                    info["sms"], info["fp32_lanes_per_sm"], sm_max)}
    if clocks and clocks.get("sm_mhz"):
        roofline["frac_at_sampled_clock"] = achieved / (peak * clocks["sm_mhz"] / sm_max)

    # end to end through the host-buffer C-ABI call: geometry and density from pinned host
    # memory, operator build, apply, result back to pinned host memory
    pin = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).pin_memory()
    hsrc, hnrm, hw, hsig = pin(s.x), pin(s.n), pin(s.w), pin(sig_h)
    hout = torch.empty((3, n), dtype=torch.float64).pin_memory()
    e2e_times = []
    for k in range(max(2, min(args.steps, 3)) + 1):
        flush.zero_()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        sbq.apply_host(hsrc, hnrm, hw, hsig, eta, 0.5, prec="fp32c", out=hout)
        if k > 0:
            e2e_times.append(time.perf_counter() - t1)
    e2e_s = float(np.mean(e2e_times))
    h2d = sum(a.numel() * a.element_size() for a in (hsrc, hnrm, hw, hsig))
    d2h = hout.numel() * hout.element_size()
    e2e_vs_device = float(np.abs(hout.numpy() - u).max() / np.abs(u).max())

    cpu = None
    check = None
    if rank == 0 and not args.no_cpu_baseline:
        v, cores, rows, ref, secs = oracle_sample(s, eps, sig_h, args.cpu_seconds)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "FP64 oracle, %d random rows of the same operator x %d sources in "
                         "%.1f s" % (rows.size, n, secs)}
        check = {"rows": int(rows.size),
                 "max_rel_err_vs_oracle": float(np.abs(u[:, rows] - ref).max() / np.abs(ref).max())}

    extras = {}
    if not args.no_extras:
        extras["curved_pipe_solve"] = _guarded(lambda: pipe_solves(args, sbq, dev, flush))
        extras["batch_solve"] = _guarded(lambda: batch_solve_summary(args, sbq, dev))

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": HEADLINE, "nodes": n, "unknowns": 3 * n, "eta": eta,
                       "pairs_per_step": pairs, "precision": "FP32 pair arithmetic, "
                       "TwoSum-compensated accumulation, FP64 reduction",
                       "operator": "K = I/2 + D + eta S (no correction)",
                       "tune": tune, "kernels_per_apply": stats["kernels_per_matvec"],
                       "l2": "flushed between steps (256 MiB write, outside the timed intervals)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "setup": {"generation_s": gen_s, "operator_and_autotune_ms": setup_ms},
            "oracle_check": check,
            "clocks": clocks,
            "e2e": {"value": pairs / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_s * 1e3,
                    "call": "stokes_apply_host",
                    "includes": "H2D of geometry and density, operator build (node order, "
                                "packing), apply, D2H of K sigma; tile shape from the tuning "
                                "cache filled by the autotuning before the timed region",
                    "max_rel_diff_vs_device_apply": e2e_vs_device},
            "gpu_launches": stats["kernels_per_matvec"] * args.steps,
            "roofline": roofline,
            "cpu_baseline": cpu,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    op.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def _guarded(fn):
    try:
        return fn()
    except Exception as e:   # an extra measurement must not cost the benchmark line
        return {"error": "%s: %s" % (type(e).__name__, e)}


def pipe_solves(args, sbq, dev, flush):
    """Curved pipe (18,432 nodes): GMRES to 1e-10 with compensated-FP32 inner solves and FP64
    (and double-float) refinement residuals, against the plain FP64 GMRES solve; the
    end-to-end solve through stokes_solve_host."""
    import torch
    from paper_2310_00889_gb300 import inputs as I
    c = I.config2()
    s = c["surf"]
    n = s.size
    eta = sbq.slender_eta(c["slenderness"])
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)
    src, nrm, w, rhs = t(s.x), t(s.n), t(s.w), t(c["rhs"])
    stream = torch.cuda.current_stream()
    corr = sbq.dl_gauss_correction(src, nrm, w, prec="fp32c")
    op = sbq.StokesOp(src, nrm, w, eta, correction=corr)
    for p in ("fp32c", "fp64", "df32"):
        op.autotune(p)
    opts = dict(tol=1e-10, restart=100, inner_prec="fp32c", inner_tol=1e-5, max_outer=30,
                use_graph=True)

    def timed(reps, **kw):
        ts, rep, x = [], None, None
        for _ in range(reps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            x, rep = op.solve(rhs, **kw)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.min(ts[1:] if len(ts) > 1 else ts)), rep, x

    # the compensated-FP32 pair-sum kernel alone on this size (few target tiles per SM)
    sig = t(I.density(n, seed=12))
    out = torch.empty_like(sig)
    op.matvec(sig, prec="fp32c", out=out)
    kl = []
    for _ in range(20):
        flush.zero_()
        k, _ = op.time_pairsum(sig, prec="fp32c", reps=1, out=out)
        kl.append(k)
    kernel_ms = float(np.mean(kl))
    peak, _ = _peak_tflops(sbq.device_info(), None)
    kernel = {"fp32c_pairsum_kernel_ms": kernel_ms, "tune": op.tune("fp32c"),
              "achieved_tflops": FLOPS_PER_PAIR["cf"] * float(n) * n / (kernel_ms * 1e-3) / 1e12}
    kernel["frac_of_fp32_peak"] = kernel["achieved_tflops"] / peak
    mixed_ms, rep, x = timed(4, resid_prec="fp64", **opts)
    df_ms, repd, _ = timed(4, resid_prec="df32", **opts)
    fp64_ms, rep64, x64 = timed(2, tol=1e-10, restart=100, inner_prec="fp64", use_graph=True)
    for r in (rep, repd, rep64):
        if r["status"] != 0 or r["rel_res"] > 1e-10:
            raise RuntimeError("curved-pipe solve missed the tolerance: %s" % r)
    kx = op.matvec(x, prec="fp64")
    chk = float((rhs - kx).norm() / rhs.norm())
    xdiff = float((x - x64).abs().max() / x64.abs().max())
    pin = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).pin_memory()
    hsrc, hnrm, hw, hrhs = pin(s.x), pin(s.n), pin(s.w), pin(c["rhs"])
    e2e = []
    for k in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        xh, reph = sbq.solve_host(hsrc, hnrm, hw, hrhs, eta, corr_prec="fp32c", **opts)
        if k > 0:
            e2e.append(time.perf_counter() - t0)
    op.close()
    return {"nodes": n, "unknowns": 3 * n, "tol": 1e-10,
            "correction": "double-layer singularity subtraction, row sums in compensated FP32",
            "mixed_ms": mixed_ms, "mixed_iters": rep["iters"],
            "mixed_refinements": rep["outer_iters"], "mixed_rel_res": rep["rel_res"],
            "mixed_x_fp64_rel_res": chk,
            "mixed_with_df32_residuals_ms": df_ms, "df32_resid_fallbacks": repd["resid_fallbacks"],
            "fp64_ms": fp64_ms, "fp64_iters": rep64["iters"], "fp64_rel_res": rep64["rel_res"],
            "speedup_mixed_vs_fp64": fp64_ms / mixed_ms,
            "speedup_df32_resid_vs_fp64": fp64_ms / df_ms,
            "x_rel_diff_mixed_vs_fp64": xdiff,
            "e2e_solve_host_ms": 1e3 * float(np.mean(e2e)),
            "e2e_status": reph["status_name"], "e2e_rel_res": reph["rel_res"],
            "kernel": kernel}


def batch_solve_summary(args, sbq, dev):
    """64 capped arcs (1.28M nodes) in one block-diagonal operator: one mixed GMRES-IR solve
    to 1e-10 per segment (compensated FP32 inner, FP64 residuals); plain FP64 estimated from
    its apply time (the full FP64 solve takes minutes: --workload batch --fp64-solve)."""
    import torch
    from paper_2310_00889_gb300 import inputs as I
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)
    c = I.config4()
    segs = c["segments"]
    off = np.cumsum([0] + [g["surf"].size for g in segs])
    X = t(np.concatenate([g["surf"].x for g in segs], axis=1))
    Nn = t(np.concatenate([g["surf"].n for g in segs], axis=1))
    W = t(np.concatenate([g["surf"].w for g in segs]))
    rhs = t(np.concatenate([g["rhs"] for g in segs], axis=1))
    eta = sbq.slender_eta(c["slenderness"])
    plan = sbq.BatchPlan(off)
    corr = sbq.dl_gauss_correction(X, Nn, W, off, prec="df32")
    op = sbq.StokesOp(X, Nn, W, eta, correction=corr, plan=plan)
    op.autotune("fp32c")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    x, rep = op.solve(rhs, tol=1e-10, restart=100, inner_prec="fp32c", inner_tol=1e-5)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3
    kx = op.matvec(x, prec="fp64")
    worst = 0.0
    for i in range(len(segs)):
        a, b_ = int(off[i]), int(off[i + 1])
        worst = max(worst, float(((rhs[:, a:b_] - kx[:, a:b_]).norm() / rhs[:, a:b_].norm()).item()))
    sig = t(I.density(int(off[-1]), seed=7))
    o = torch.empty_like(sig)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    op.matvec(sig, prec="fp64", out=o)
    torch.cuda.synchronize()
    ms64 = (time.perf_counter() - t0) * 1e3
    op.close()
    plan.close()
    return {"segments": len(segs), "nodes": int(off[-1]),
            "pairs_per_matvec": float(np.sum(np.diff(off).astype(np.float64) ** 2)),
            "mixed_ms": ms, "iters": rep["iters"], "refinements": rep["outer_iters"],
            "status": rep["status_name"], "max_segment_fp64_rel_res": worst,
            "fp64_apply_ms": ms64,
            "fp64_solve_estimate_ms": ms64 * (rep["iters"] + 2),
            "fp64_solve_estimate_basis": "measured FP64 apply x (mixed iterations + 2); an "
                                         "estimate, not a measurement"}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_curved_pipe(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    from paper_2310_00889_gb300 import build as b
    b.build()
    from paper_2310_00889_gb300 import inputs as I
    from paper_2310_00889_gb300 import sbq

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    c = I.config2()
    s = c["surf"]
    n = s.size
    eta = sbq.slender_eta(c["slenderness"])
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)
    src, nrm, w, rhs = t(s.x), t(s.n), t(s.w), t(c["rhs"])
    stream = torch.cuda.current_stream()

    if args.kernel_only:
        return kernel_only(args, sbq, I, src, nrm, w, eta, n, t, dev)

    t_setup = time.perf_counter()
    # the correction is operator data; its row sums in compensated FP32 (1e-7) are far below
    # the discretisation error and cost a tenth of double-float ones
    corr = None if args.no_correction else sbq.dl_gauss_correction(src, nrm, w, prec="fp32c")
    op = sbq.StokesOp(src, nrm, w, eta, correction=corr)
    op.autotune("fp32c")
    op.autotune("fp64")
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t_setup) * 1e3
    opts = dict(tol=1e-10, restart=100, inner_prec="fp32c", inner_tol=1e-5, max_outer=30,
                use_graph=not args.no_graph, resid_prec=args.resid_prec)
    op.autotune(args.resid_prec)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    for _ in range(args.warmup):
        x, rep = op.solve(rhs, **opts)
    if rep["status"] != 0 or rep["rel_res"] > 1e-10:
        raise RuntimeError("mixed solve did not converge: %s" % rep)

    sampler = ClockSampler(gpu_uuid())
    sampler.start()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    times, reps = [], []
    torch.cuda.nvtx.range_push("bench_timed")
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        x, rep = op.solve(rhs, **opts)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        reps.append(rep)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = max_over_ranks(float(np.mean(times)), world, dev)
    rep = reps[-1]
    for r in reps:
        if r["status"] != 0 or r["rel_res"] > 1e-10:
            raise RuntimeError("a timed solve missed the tolerance: %s" % r)
    # the returned x, checked with an FP64 residual (outside the timed region)
    kx = op.matvec(x, prec="fp64")
    fp64_check = float((rhs - kx).norm() / rhs.norm())
    if fp64_check > 1e-10:
        raise RuntimeError("FP64 residual of the timed solve's x is %.3e" % fp64_check)
    # the other residual precision, same inner solve (for comparison)
    other = "fp64" if args.resid_prec == "df32" else "df32"
    oth_times = []
    for k in range(3):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        xo, repo = op.solve(rhs, **dict(opts, resid_prec=other))
        e1.record(stream)
        e1.synchronize()
        oth_times.append(e0.elapsed_time(e1))
    oth_ms = float(np.min(oth_times[1:]))
    pairs_step = float(rep["matvecs_fp64"] + rep["matvecs_low"]) * n * n
    value = replica_value(pairs_step, ms, world)
    kpm32 = op.stats("fp32c")["kernels_per_matvec"]
    launches = rep["kernel_launches"] * args.steps

    # plain FP64 GMRES solve of the same system (the comparison the metric names)
    fp64_times = []
    for k in range(2):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        flush.zero_()
        e0.record(stream)
        x64, rep64 = op.solve(rhs, tol=1e-10, restart=100, inner_prec="fp64", use_graph=True)
        e1.record(stream)
        e1.synchronize()
        fp64_times.append(e0.elapsed_time(e1))
    fp64_ms = float(np.min(fp64_times[1:] or fp64_times))
    xdiff = float((x - x64).abs().max() / x64.abs().max())

    # the dominant kernel on its own: compensated-FP32 combined-field pair sum, same launch
    # configuration as inside the solve, CUDA events on the launching stream
    sig = t(I.density(n, seed=12))
    out = torch.empty_like(sig)

    def time_matvec(prec, reps_):
        """(pair-sum kernel ms, whole apply ms): CUDA events recorded by the library on the
        launching stream around the kernel launch and around the apply; L2 flushed before
        each apply."""
        for _ in range(2):
            op.matvec(sig, prec=prec, out=out)
        kl, al = [], []
        for _ in range(reps_):
            flush.zero_()
            kms, ams = op.time_pairsum(sig, prec=prec, reps=1, out=out)
            kl.append(kms)
            al.append(ams)
        return float(np.mean(kl)), float(np.mean(al))

    kk32c, k32c = time_matvec("fp32c", args.kernel_reps)
    kk32, k32 = time_matvec("fp32", args.kernel_reps)
    kkdf, kdf = time_matvec("df32", max(3, args.kernel_reps // 2))
    kk64, k64 = time_matvec("fp64", max(3, args.kernel_reps // 4))
    info = sbq.device_info()
    sm_max = (clocks or {}).get("sm_max_mhz") or 2070.0
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(peaks_path):
        try:
            sm_max = float(json.load(open(peaks_path)).get("sm_max_mhz", sm_max))
        except Exception:
            pass
    peak = info["sms"] * info["fp32_lanes_per_sm"] * 2 * sm_max * 1e6 / 1e12   # TFLOP/s
    achieved = FLOPS_PER_PAIR["cf"] * float(n) * n / (kk32c * 1e-3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": _profiled_traffic("pairsum_f32_comp_curved_pipe.json"),
                "traffic_unit": "bytes per launch (ncu dram read + write)",
                "kernel": "pairsum_f32_kernel<combined field, compensated>",
                "flops_per_pair": FLOPS_PER_PAIR["cf"], "pairs_per_launch": float(n) * n,
                "launch_ms": kk32c, "apply_ms": k32c,
                "timing": "CUDA events on the launching stream around the kernel launch",
                "peak_basis": "%d SMs x %d FP32 lanes x 2 x %.0f MHz (sm_max_mhz)" % (
                    info["sms"], info["fp32_lanes_per_sm"], sm_max)}
    if clocks and clocks.get("sm_mhz"):
        roofline["frac_at_sampled_clock"] = achieved / (peak * clocks["sm_mhz"] / sm_max)

    # end to end through the public API from pinned host buffers
    hsrc, hnrm, hw, hrhs = (torch.as_tensor(np.ascontiguousarray(a)).pin_memory()
                            for a in (s.x, s.n, s.w, c["rhs"]))
    e2e_times = []
    for k in range(max(2, min(args.steps, 3)) + 1):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        xh, reph = sbq.solve_host(hsrc, hnrm, hw, hrhs, eta, tol=1e-10, inner_prec="fp32c",
                                  restart=100, inner_tol=1e-5, max_outer=30,
                                  corr_prec=None if args.no_correction else "fp32c",
                                  resid_prec=args.resid_prec)
        torch.cuda.synchronize()
        if k > 0:
            e2e_times.append(time.perf_counter() - t0)
    e2e_s = float(np.mean(e2e_times))
    pairs_e2e = float(reph["matvecs_fp64"] + reph["matvecs_low"]) * n * n
    h2d = sum(a.numel() * a.element_size() for a in (hsrc, hnrm, hw, hrhs))
    d2h = xh.numel() * xh.element_size()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        v, cores, smp = oracle_rate(args.cpu_seconds)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "FP64 oracle rows of the same combined-field operator, %d target rows x "
                         "%d sources in %.1f s" % (smp["rows"], n, smp["seconds"])}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nodes": n, "unknowns": 3 * n, "eta": eta,
                       "tol": 1e-10, "inner": "fp32 compensated GMRES inside iterative refinement",
                       "restart": 100, "graph": not args.no_graph,
                       "resid": args.resid_prec + (" (double-float, FP64-class)"
                                                   if args.resid_prec == "df32" else ""),
                       "correction": "none" if args.no_correction else
                       "double-layer singularity subtraction, row sums in compensated FP32",
                       "l2": "flushed between steps (256 MiB write, outside the timed intervals)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "solve": {"mixed_ms": ms, "fp64_ms": fp64_ms, "speedup_vs_fp64": fp64_ms / ms,
                      "mixed_iters": rep["iters"], "mixed_refinements": rep["outer_iters"],
                      "mixed_matvecs_fp32c": rep["matvecs_low"],
                      "mixed_matvecs_fp64": rep["matvecs_fp64"], "mixed_rel_res": rep["rel_res"],
                      "fp64_iters": rep64["iters"], "fp64_rel_res": rep64["rel_res"],
                      "x_rel_diff_mixed_vs_fp64": xdiff,
                      "mixed_x_fp64_rel_res": fp64_check,
                      "mixed_ms_with_%s_residuals" % other: oth_ms,
                      "mixed_iters_with_%s_residuals" % other: repo["iters"]},
            "kernels": {"fp32c_matvec_ms": k32c, "fp32_matvec_ms": k32, "fp64_matvec_ms": k64,
                        "fp32c_pairsum_kernel_ms": kk32c, "fp32_pairsum_kernel_ms": kk32,
                        "fp64_pairsum_kernel_ms": kk64, "df32_matvec_ms": kdf,
                        "df32_pairsum_kernel_ms": kkdf,
                        "df32_pairs_per_s": n * n / (kkdf * 1e-3),
                        "tune_df32": op.tune("df32"),
                        "fp32c_pairs_per_s": n * n / (k32c * 1e-3),
                        "fp32_pairs_per_s": n * n / (k32 * 1e-3),
                        "fp64_pairs_per_s": n * n / (k64 * 1e-3),
                        "tune_fp32c": op.tune("fp32c"), "tune_fp64": op.tune("fp64"),
                        "kernels_per_matvec_fp32c": kpm32},
            "setup_ms": setup_ms,
            "clocks": clocks,
            "e2e": {"value": pairs_e2e / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_s * 1e3,
                    "includes": "H2D of geometry and data, correction and operator build, "
                                "graph capture, solve, D2H of the solution"},
            "gpu_launches": launches,
            "roofline": roofline,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    op.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def kernel_only(args, sbq, I, src, nrm, w, eta, n, t, dev):
    """Operator applies of one precision on the workload, for profilers: the tile shape is
    autotuned first, then --kernel-reps applies run inside the NVTX range 'kernel_only'."""
    import torch
    op = sbq.StokesOp(src, nrm, w, eta)
    op.autotune(args.kernel_only)
    sig = t(I.density(n, seed=12))
    out = torch.empty_like(sig)
    for _ in range(2):
        op.matvec(sig, prec=args.kernel_only, out=out)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("kernel_only")
    e0.record(stream)
    for _ in range(args.kernel_reps):
        op.matvec(sig, prec=args.kernel_only, out=out)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / args.kernel_reps
    print(json.dumps({"kernel_only": args.kernel_only, "nodes": n, "ms_per_apply": ms,
                      "pairs_per_s": n * n / (ms * 1e-3), "tune": op.tune(args.kernel_only),
                      "stats": op.stats(args.kernel_only)}), flush=True)
    op.close()
    return 0


def _profiled_traffic(record):
    """DRAM bytes per launch of the compensated combined-field kernel on a workload, from a
    committed ncu record under profiles/, or None when the kernel's or the layout's sources
    changed since it was taken (the record keeps their SHA-256)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", record)
    try:
        d = json.load(open(path))
        h = hashlib.sha256()
        for f in d["sources"]:
            with open(os.path.join(ROOT, f), "rb") as fh:
                h.update(fh.read())
        if h.hexdigest() != d["sources_sha256"]:
            return None
        return int(d["dram_bytes_read"]) + int(d["dram_bytes_write"])
    except (OSError, ValueError, KeyError):
        return None


def _cuda_timer(fn, reps, stream, warm=True):
    import torch
    if warm:
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def run_precision_sweep(args):
    """Random closed slender loops (paper Sec. 5.2 recipe) of 64K/256K/1M nodes: the
    combined-field operator in FP64, FP32 and compensated FP32; error of each against the
    FP64 GPU result over all rows and against the FP64 CPU oracle on 4096 sampled rows."""
    import torch
    import oracle
    from paper_2310_00889_gb300 import build as b
    b.build()
    oracle.build()
    from paper_2310_00889_gb300 import inputs as I
    from paper_2310_00889_gb300 import sbq
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")
    eta = sbq.slender_eta(0.01)
    for panels in [int(x) for x in args.sizes.split(",")]:
        c = I.config3(panels=panels)
        s = c["surf"]
        n = s.size
        op = sbq.StokesOp(t(s.x), t(s.n), t(s.w), eta)
        sig = t(c["sigma"])
        out = {}
        times = {}
        for prec in ("fp32c", "fp32", "df32", "fp64"):
            op.autotune(prec) if prec != "fp64" or n <= 300000 else None
            o = torch.empty_like(sig)
            reps = 1 if prec == "fp64" or (prec == "df32" and n > 300000) else 5
            times[prec] = _cuda_timer(lambda: op.matvec(sig, prec=prec, out=o), reps, stream)
            out[prec] = o
        u64 = out["fp64"]
        rows = c["sub"]
        t0 = time.perf_counter()
        ref = oracle.combined(s.x, s.n, s.w, c["sigma"], s.x[:, rows], eta, 1.0) + 0.5 * c["sigma"][:, rows]
        t_or = time.perf_counter() - t0
        line = {"workload": "precision_sweep_random_loop", "nodes": n, "panels": panels,
                "eta": eta, "pairs": float(n) * n, "oracle_rows": int(len(rows)),
                "oracle_seconds": t_or, "oracle_cores": oracle.num_threads()}
        for prec in ("fp64", "df32", "fp32", "fp32c"):
            u = out[prec]
            e_full = float(((u - u64).abs().max() / u64.abs().max()).item())
            un = u[:, torch.as_tensor(rows, device="cuda")].cpu().numpy()
            e_or = float(np.abs(un - ref).max() / np.abs(ref).max())
            line[prec] = {"ms": times[prec], "pairs_per_s": n * n / (times[prec] * 1e-3),
                          "relerr_vs_fp64_gpu_all_rows": e_full,
                          "relerr_vs_oracle_sampled_rows": e_or,
                          "tune": op.tune(prec) if prec != "fp64" or n <= 300000 else None}
        print(json.dumps(line), flush=True)
        op.close()
        del out, u64, sig
        torch.cuda.empty_cache()
    return 0


def run_batch(args):
    """64 independent capped arcs (angles U[30, 180] degrees, wall node counts log-uniform
    in [2K, 64K], seed 3) as one block-diagonal operator: every apply is one persistent
    launch over the work list of all segments; GMRES-IR over the whole batch."""
    import torch
    from paper_2310_00889_gb300 import build as b
    b.build()
    from paper_2310_00889_gb300 import inputs as I
    from paper_2310_00889_gb300 import sbq
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")
    c = I.config4()
    segs = c["segments"]
    off = np.cumsum([0] + [g["surf"].size for g in segs])
    n = int(off[-1])
    X = np.concatenate([g["surf"].x for g in segs], axis=1)
    Nn = np.concatenate([g["surf"].n for g in segs], axis=1)
    W = np.concatenate([g["surf"].w for g in segs])
    B = np.concatenate([g["rhs"] for g in segs], axis=1)
    eta = sbq.slender_eta(c["slenderness"])
    plan = sbq.BatchPlan(off)
    t0 = time.perf_counter()
    op = sbq.StokesOp(t(X), t(Nn), t(W), eta, plan=plan)
    tune = {p: op.autotune(p) for p in ("fp32c", "fp64")}
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t0) * 1e3
    pairs = float(np.sum(np.diff(off).astype(np.float64) ** 2))
    sig = t(I.density(n, seed=7))
    o = torch.empty_like(sig)
    mv = {p: _cuda_timer(lambda: op.matvec(sig, prec=p, out=o), 5 if p != "fp64" else 1, stream)
          for p in ("fp32c", "fp32", "df32", "fp64")}
    # batched apply == the same segments applied one by one (same tile shape)
    u = op.matvec(sig, prec="fp32c").clone()
    u64 = op.matvec(sig, prec="fp64").clone()
    worst = 0.0
    for i in (0, 17, 63):
        a, b_ = int(off[i]), int(off[i + 1])
        p1 = sbq.BatchPlan([0, b_ - a], tune=op.tune("fp64"))
        o1 = sbq.StokesOp(t(X[:, a:b_]), t(Nn[:, a:b_]), t(W[a:b_]), eta, plan=p1)
        r1 = o1.matvec(sig[:, a:b_].contiguous(), prec="fp64")
        worst = max(worst, float(((r1 - u64[:, a:b_]).abs().max() / r1.abs().max()).item()))
        o1.close()
    rhs = t(B)
    # solves: the same batch with the double-layer singularity subtraction of every
    # segment (each segment is one closed body); without it the punctured sums leave
    # some segments' discrete operators indefinite and restarted GMRES stagnates
    t0 = time.perf_counter()
    corr = None
    if not args.no_correction:
        corr = sbq.dl_gauss_correction(t(X), t(Nn), t(W), off, prec="df32")
    opc = sbq.StokesOp(t(X), t(Nn), t(W), eta, correction=corr, plan=plan)
    torch.cuda.synchronize()
    corr_ms = (time.perf_counter() - t0) * 1e3
    sopt = dict(tol=1e-10, restart=100, inner_prec="fp32c", inner_tol=1e-5,
                resid_prec=args.resid_prec)
    x, rep = opc.solve(rhs, **sopt)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    x, rep = opc.solve(rhs, **sopt)
    torch.cuda.synchronize()
    mixed_ms = (time.perf_counter() - t0) * 1e3
    # residual of every segment (FP64 operator)
    kx = opc.matvec(x, prec="fp64")
    seg_res = []
    for i in range(len(segs)):
        a, b_ = int(off[i]), int(off[i + 1])
        seg_res.append(float(((rhs[:, a:b_] - kx[:, a:b_]).norm() / rhs[:, a:b_].norm()).item()))
    if max(seg_res) > 1e-10:
        raise RuntimeError("batched solve: a segment's FP64 residual is %.3e" % max(seg_res))
    line = {"workload": "batch_64_capped_arcs", "segments": len(segs), "nodes": n,
            "pairs_per_matvec": pairs, "setup_ms": setup_ms, "tune": tune,
            "correction": "none" if args.no_correction else
            "double-layer singularity subtraction per segment, double-float row sums",
            "resid": args.resid_prec,
            "correction_and_operator_ms": corr_ms,
            "matvec_ms": mv, "pairs_per_s": {p: pairs / (v * 1e-3) for p, v in mv.items()},
            "fp32c_relerr_vs_fp64": float(((u - u64).abs().max() / u64.abs().max()).item()),
            "batched_vs_single_segment_fp64_relerr": worst,
            "mixed_solve": {"ms": mixed_ms, "iters": rep["iters"], "refinements": rep["outer_iters"],
                            "matvecs_fp32c": rep["matvecs_low"], "matvecs_fp64": rep["matvecs_fp64"],
                            "rel_res": rep["rel_res"], "graph": rep["graph_used"],
                            "max_segment_rel_res": max(seg_res)}}
    if args.fp64_solve:
        t0 = time.perf_counter()
        x64, rep64 = opc.solve(rhs, tol=1e-10, restart=100, inner_prec="fp64")
        torch.cuda.synchronize()
        line["fp64_solve"] = {"ms": (time.perf_counter() - t0) * 1e3, "iters": rep64["iters"],
                              "rel_res": rep64["rel_res"]}
    else:
        line["fp64_solve_estimate_ms"] = mv["fp64"] * (rep["iters"] + 2)
    print(json.dumps(line), flush=True)
    op.close()
    opc.close()
    return 0


def run_helix(args):
    """Helical pipe (helix radius 3, pitch --helix-pitch (3), 4 turns, tube radius 1, 2048 x 8 x 64
    = 1,048,576 wall nodes, two 16 x 64 caps) with 100 spheres of radius 0.2 (600 nodes
    each) inside: one mixed-precision GMRES-IR solve to 1e-10 (zero wall and sphere data,
    parabolic cap profiles); the plain FP64 solve is estimated from its iteration count and
    the measured FP64 apply time unless --fp64-solve is given."""
    import torch
    import oracle
    from paper_2310_00889_gb300 import build as b
    b.build()
    oracle.build()
    from paper_2310_00889_gb300 import inputs as I
    from paper_2310_00889_gb300 import sbq
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")
    t0 = time.perf_counter()
    c = I.config5(panels=args.helix_panels, pitch=args.helix_pitch)
    s = c["surf"]
    n = s.size
    rhs = np.zeros((3, n))
    a_, b_ = 3.0, args.helix_pitch / (2.0 * np.pi)
    pe = np.array([0.0, 2.0 * np.pi * 4.0])
    cend = np.stack([a_ * np.cos(pe), a_ * np.sin(pe), b_ * pe])
    tend = np.stack([-a_ * np.sin(pe), a_ * np.cos(pe), np.full(2, b_)])
    tend /= np.linalg.norm(tend, axis=0)
    for nm, lo, hi in s.parts:
        if nm in ("cap0", "cap1"):
            k = 0 if nm == "cap0" else 1
            rho2 = np.sum((s.x[:, lo:hi] - cend[:, k:k + 1]) ** 2, axis=0)
            rhs[:, lo:hi] = (1.0 - rho2)[None, :] * tend[:, k:k + 1]
    gen_s = time.perf_counter() - t0
    eta = sbq.slender_eta(c["slenderness"])
    t0 = time.perf_counter()
    op = sbq.StokesOp(t(s.x), t(s.n), t(s.w), eta)
    tune32 = op.autotune("fp32c")
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t0) * 1e3
    sig = t(I.density(n, seed=5))
    o = torch.empty_like(sig)
    ms32 = _cuda_timer(lambda: op.matvec(sig, prec="fp32c", out=o), 2, stream)
    u32 = o.clone()
    # one FP64 apply here takes about a minute: fix the tile shape (the autotuner takes
    # the first shape when one apply is that long), then time one apply
    op.autotune("fp64")
    ms64 = _cuda_timer(lambda: op.matvec(sig, prec="fp64", out=o), 1, stream, warm=False)
    u64 = o.clone()
    op.autotune("df32")
    msdf = _cuda_timer(lambda: op.matvec(sig, prec="df32", out=o), 1, stream, warm=False)
    udf = o.clone()
    rows = np.sort(np.random.default_rng(4).choice(n, 4096, replace=False))
    sg = sig.cpu().numpy()
    ref = oracle.combined(s.x, s.n, s.w, sg, s.x[:, rows], eta, 1.0) + 0.5 * sg[:, rows]
    ri = torch.as_tensor(rows, device="cuda")
    e64 = float(np.abs(u64[:, ri].cpu().numpy() - ref).max() / np.abs(ref).max())
    e32 = float(np.abs(u32[:, ri].cpu().numpy() - ref).max() / np.abs(ref).max())
    edf = float(np.abs(udf[:, ri].cpu().numpy() - ref).max() / np.abs(ref).max())
    # solve with the double-layer singularity subtraction per closed body (the capped
    # pipe, each sphere), its row sums in double-float
    t0 = time.perf_counter()
    corr = None
    if not args.no_correction:
        corr = sbq.dl_gauss_correction(t(s.x), t(s.n), t(s.w), I.body_offsets(s), prec="df32")
    op.close()
    op = sbq.StokesOp(t(s.x), t(s.n), t(s.w), eta, correction=corr)
    torch.cuda.synchronize()
    corr_ms = (time.perf_counter() - t0) * 1e3
    t0 = time.perf_counter()
    x, rep = op.solve(t(rhs), tol=1e-10, restart=100, inner_prec="fp32c", inner_tol=1e-5,
                      max_iter=400, resid_prec=args.resid_prec)
    torch.cuda.synchronize()
    mixed_ms = (time.perf_counter() - t0) * 1e3
    # the returned x, checked with an FP64 residual (one FP64 apply)
    rhs_d = t(rhs)
    x64chk = float((rhs_d - op.matvec(x, prec="fp64")).norm() / rhs_d.norm())
    line = {"workload": "helix_pipe_with_spheres", "nodes": n, "spheres": len(c["centres"]),
            "pitch": args.helix_pitch, "eta": eta, "pairs_per_matvec": float(n) * n,
            "generation_s": gen_s,
            "setup_ms": setup_ms, "tune_fp32c": tune32,
            "matvec_ms": {"fp32c": ms32, "df32": msdf, "fp64": ms64},
            "pairs_per_s": {"fp32c": n * n / (ms32 * 1e-3), "df32": n * n / (msdf * 1e-3),
                            "fp64": n * n / (ms64 * 1e-3)},
            "relerr_vs_oracle_4096_rows": {"fp64": e64, "df32": edf, "fp32c": e32},
            "correction": "none" if args.no_correction else
            "double-layer singularity subtraction per body (pipe, 100 spheres), double-float",
            "resid": args.resid_prec,
            "correction_and_operator_ms": corr_ms,
            "mixed_solve": {"ms": mixed_ms, "iters": rep["iters"], "refinements": rep["outer_iters"],
                            "matvecs_fp32c": rep["matvecs_low"], "matvecs_fp64": rep["matvecs_fp64"],
                            "rel_res": rep["rel_res"], "x_fp64_rel_res": x64chk,
                            "hist": rep["hist"], "graph": rep["graph_used"],
                            "status": rep["status_name"]}}
    if args.fp64_solve:
        t0 = time.perf_counter()
        x64, rep64 = op.solve(t(rhs), tol=1e-10, restart=100, inner_prec="fp64")
        torch.cuda.synchronize()
        line["fp64_solve"] = {"ms": (time.perf_counter() - t0) * 1e3, "iters": rep64["iters"],
                              "rel_res": rep64["rel_res"]}
    else:
        line["fp64_solve_estimate_ms"] = ms64 * (rep["iters"] + 2)
    print(json.dumps(line), flush=True)
    op.close()
    return 0


def run_laplace(args):
    """Laplace combined field (paper Sec. 4.1, eta = 1/(2 eps log(1/eps)), eps = 0.01) on
    random slender loops of 65,536 and 262,144 nodes: time of every precision's apply (CUDA
    events), error against the FP64 oracle on 1024 sampled rows; and the torus
    Green's-identity test (Eq. greens-rep) inside the tube under refinement."""
    import torch
    import oracle
    from paper_2310_00889_gb300 import build as b
    b.build()
    oracle.build()
    from paper_2310_00889_gb300 import inputs as I
    from paper_2310_00889_gb300 import sbq
    torch.cuda.set_device(0)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")
    eta = sbq.slender_eta(0.01)
    flops_lcf = 19
    info = sbq.device_info()
    peak = info["sms"] * info["fp32_lanes_per_sm"] * 2 * 2070.0e6 / 1e12
    for panels in (512, 2048):
        s = I.random_loop(seed=1, panels=panels, ns=8, nth=16)
        n = s.size
        sig = I.density(n, seed=2)[0]
        src, nrm, w, sg = t(s.x), t(s.n), t(s.w), t(sig)
        rows = np.sort(np.random.default_rng(3).choice(n, 1024, replace=False))
        ref = oracle.laplace(s.x, s.n, s.w, sig, s.x[:, rows], eta, 1.0)
        out = torch.empty(n, dtype=torch.float64, device="cuda")
        res = {}
        for prec in ("fp32c", "fp32", "df32", "fp64"):
            sbq.laplace_apply(src, nrm, w, sg, src, eta, 1.0, prec=prec, out=out)
            torch.cuda.synchronize()
            reps = 3 if prec != "fp64" else 1
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                sbq.laplace_apply(src, nrm, w, sg, src, eta, 1.0, prec=prec, out=out)
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1) / reps
            u = out.cpu().numpy()[rows]
            res[prec] = {"ms": ms, "pairs_per_s": n * n / (ms * 1e-3),
                         "relerr_vs_oracle_1024_rows":
                             float(np.abs(u - ref).max() / np.abs(ref).max())}
        res["fp32c"]["tflops"] = flops_lcf * n * n / (res["fp32c"]["ms"] * 1e-3) / 1e12
        res["fp32c"]["frac_of_fp32_peak"] = res["fp32c"]["tflops"] / peak
        print(json.dumps({"workload": "laplace_combined_random_loop", "nodes": n, "eta": eta,
                          "flops_per_pair": flops_lcf, "apply": res,
                          "timing": "CUDA events around the whole apply (pack, kernel, "
                                    "reduction), temporary packs included"}), flush=True)
    green = []
    x0 = np.array([1.0, 0.0, 0.45])
    phi = np.linspace(0, 2 * np.pi, 7)[:-1]
    xin = np.stack([np.cos(phi), np.sin(phi), 0.05 * np.ones_like(phi)])
    g_in = 1.0 / (4 * np.pi * np.linalg.norm(xin - x0[:, None], axis=0))
    for panels, nth in ((8, 16), (16, 32), (32, 64), (64, 128)):
        tor = I.torus(1.0, 0.25, panels, 8, nth)
        r = tor.x - x0[:, None]
        rl = np.linalg.norm(r, axis=0)
        u = 1.0 / (4 * np.pi * rl)
        dudn = -np.sum(r * tor.n, axis=0) / (4 * np.pi * rl ** 3)
        sp = sbq.laplace_apply(t(tor.x), None, t(tor.w), t(dudn), t(xin), 1.0, 0.0, prec="fp64")
        dp = sbq.laplace_apply(t(tor.x), t(tor.n), t(tor.w), t(u), t(xin), 0.0, 1.0, prec="fp64")
        err = float(np.abs(sp.cpu().numpy() - dp.cpu().numpy() - g_in).max() / np.abs(g_in).max())
        green.append({"nodes": tor.size, "interior_relerr": err})
    print(json.dumps({"workload": "laplace_torus_green_identity", "R": 1.0, "radius": 0.25,
                      "charge": x0.tolist(), "refinement": green}), flush=True)
    return 0


def run_mobility(args):
    """Sedimentation of 32 slender rings (tori R = 1, eps = 0.05, 8192 nodes each, random
    orientations, 262,144 nodes): unit force -e_z on every ring, no torque; the slender
    combined-field mobility formulation (Sec. 4.2) with the double-layer correction per ring,
    GMRES-IR (compensated FP32 inner, double-float residuals where their bound certifies the
    tolerance), the rigid velocities V = -L sigma, and the returned sigma checked with an FP64
    apply of the mobility operator."""
    import torch
    from paper_2310_00889_gb300 import build as b
    b.build()
    from paper_2310_00889_gb300 import inputs as I
    from paper_2310_00889_gb300 import sbq
    torch.cuda.set_device(0)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")
    s = I.rings()
    off = I.body_offsets(s)
    nb = len(off) - 1
    eta = sbq.slender_eta(0.05)
    t0 = time.perf_counter()
    corr = sbq.dl_gauss_correction(t(s.x), t(s.n), t(s.w), off, prec="df32")
    op = sbq.StokesOp(t(s.x), t(s.n), t(s.w), eta, correction=corr)
    op.set_mobility(off)
    op.autotune("fp32c")
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t0) * 1e3
    F = np.tile([0.0, 0.0, -1.0], (nb, 1))
    T = np.zeros((nb, 3))
    t0 = time.perf_counter()
    rhs = op.mobility_rhs(F, T, prec="df32")
    x, rep = op.solve(rhs, tol=1e-10, restart=100, inner_prec="fp32c", inner_tol=1e-5,
                      resid_prec=args.resid_prec)
    uw = op.mobility_velocity(x)
    torch.cuda.synchronize()
    solve_ms = (time.perf_counter() - t0) * 1e3
    chk = float((rhs - op.matvec(x, prec="fp64")).norm() / rhs.norm())
    vz = uw[:, 2]
    print(json.dumps({"workload": "mobility_32_rings", "nodes": s.size, "bodies": nb, "eta": eta,
                      "setup_ms": setup_ms, "rhs_and_solve_ms": solve_ms,
                      "iters": rep["iters"], "refinements": rep["outer_iters"],
                      "resid_fallbacks": rep["resid_fallbacks"], "rel_res": rep["rel_res"],
                      "x_fp64_rel_res": chk, "status": rep["status_name"],
                      "sedimentation_speed": {"mean": float(-vz.mean()), "min": float(-vz.max()),
                                              "max": float(-vz.min())},
                      "max_angular_speed": float(np.linalg.norm(uw[:, 3:], axis=1).max())}),
          flush=True)
    op.close()
    return 0


def run_quadrature(args):
    """Quadrature correction E of the tube elements (Sec. 3.2.1-3.2.4).
    (1) The paper's torus test (Sec. 5.1, Table t:conv-biest): on-surface Laplace Green's
        identity at every node for its four discretisations, with the E build time.
    (2) The paper's slender-loop problem (Sec. 5.2): exterior Laplace Dirichlet problem
        u = 1 on a random loop of radius 0.005..0.015, eta = 64; GMRES-IR (compensated FP32
        inner, FP64 residuals) with E at panels x 8 x 16 and at 2 panels x 8 x 24 nodes, and
        with the punctured operator; the field at points at least 0.5 from the surface is
        compared with the finer corrected solution.
    (3) Build time of the Stokes combined-field E on the coarse loop."""
    import torch
    from paper_2310_00889_gb300 import build as b
    b.build()
    from paper_2310_00889_gb300 import inputs as I
    from paper_2310_00889_gb300 import sbq
    torch.cuda.set_device(0)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed_build(*a, **k):
        ms = []
        for _ in range(2):
            e0.record()
            E = sbq.tube_correction(*a, **k)
            e1.record()
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return E, ms[-1]

    def csr_apply(E, v):
        rowptr, col, val = E
        m = torch.sparse_csr_tensor(rowptr, col, val, size=(rowptr.shape[0] - 1, v.shape[0]))
        return (m @ v.unsqueeze(1)).squeeze(1)

    if args.build_only:
        # the Stokes combined-field E of the random loop alone, inside the NVTX range
        # 'kernel_only' (for profilers)
        s = I.random_loop(seed=1, panels=args.quad_panels, ns=8, nth=16)
        args_ = (t(s.x), t(s.n), t(s.w), args.quad_panels, 8, 16)
        sbq.tube_correction(*args_, kind="stokes", alpha=sbq.slender_eta(0.01), beta=1.0,
                            near_factor=args.near_factor)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("kernel_only")
        t0 = time.perf_counter()
        for _ in range(max(1, args.kernel_reps)):
            E = sbq.tube_correction(*args_, kind="stokes", alpha=sbq.slender_eta(0.01), beta=1.0,
                                    near_factor=args.near_factor)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3 / max(1, args.kernel_reps)
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"build_only": "stokes", "nodes": s.size, "build_ms": ms,
                          "nnz": int(E[2].shape[0])}), flush=True)
        return 0

    # (1) the paper's torus table
    printed = {320: (3.3e-3, 0.016), 720: (7.6e-7, 0.055), 1280: (1.1e-9, 0.166), 2000: (2.1e-10, 0.357)}
    table = []
    x0 = np.array([1.0, 2.0, 3.0])
    for ne, nt in ((4, 8), (6, 12), (8, 16), (10, 20)):
        S = I.torus(R0=1.0, eps=0.25, panels=ne, ns=10, nth=nt)
        d = S.x - x0[:, None]
        r = np.linalg.norm(d, axis=0)
        u = 1.0 / (4.0 * np.pi * r)
        dudn = -np.sum(d * S.n, axis=0) / (4.0 * np.pi * r ** 3)
        src, nrm, w = t(S.x), t(S.n), t(S.w)
        ES, ms_s = timed_build(src, nrm, w, ne, 10, nt, kind="laplace", alpha=1.0, beta=0.0,
                               near_factor=args.near_factor)
        ED, ms_d = timed_build(src, nrm, w, ne, 10, nt, kind="laplace", alpha=0.0, beta=1.0,
                               near_factor=args.near_factor)
        Sp = sbq.laplace_apply(src, nrm, w, t(dudn), src, 1.0, 0.0, prec="fp64")
        Dp = sbq.laplace_apply(src, nrm, w, t(u), src, 0.0, 1.0, prec="fp64")
        lhs = (Sp + csr_apply(ES, t(dudn)) - Dp - csr_apply(ED, t(u))).cpu().numpy()
        err = float(np.abs(lhs - 0.5 * u).max() / np.abs(u).max())
        punct = float(np.abs((Sp - Dp).cpu().numpy() - 0.5 * u).max() / np.abs(u).max())
        table.append({"N": S.size, "elements": ne, "ntheta": nt, "relerr_all_nodes": err,
                      "relerr_punctured": punct, "paper_err": printed[S.size][0],
                      "setup_ms_S_and_D": ms_s + ms_d, "paper_setup_s": printed[S.size][1]})
    print(json.dumps({"workload": "quadrature_paper_torus_table", "ns": 10, "charge": x0.tolist(),
                      "rows": table}), flush=True)

    # (2) the slender loop, exterior Laplace Dirichlet u = 1
    eta = 64.0
    P = args.quad_panels
    res = {}
    pts = None
    fields = {}
    for tag, panels, nt, corrected in (("coarse_E", P, 16, True), ("fine_E", 2 * P, 24, True),
                                        ("coarse_punctured", P, 16, False)):
        s = I.random_loop(seed=1, panels=panels, ns=8, nth=nt)
        n = s.size
        if pts is None:
            rng = np.random.default_rng(5)
            lo, hi = s.x.min(axis=1), s.x.max(axis=1)
            cand = lo[:, None] + (hi - lo)[:, None] * rng.random((3, 4096))
            dmin = np.array([np.linalg.norm(s.x - cand[:, k:k + 1], axis=0).min() for k in range(4096)])
            pts = cand[:, dmin > 0.5][:, :512]
        src, nrm, w = t(s.x), t(s.n), t(s.w)
        E, ms = (timed_build(src, nrm, w, panels, 8, nt, kind="laplace", alpha=eta, beta=1.0,
                             near_factor=args.near_factor) if corrected else (None, 0.0))
        op = sbq.LaplaceOp(src, nrm, w, eta, correction=E)
        op.autotune("fp32c")
        rhs = torch.ones(n, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        tt = time.perf_counter()
        x, rep = op.solve(rhs, tol=1e-10, restart=100, inner_prec="fp32c", inner_tol=1e-5,
                          resid_prec="fp64")
        torch.cuda.synchronize()
        solve_ms = (time.perf_counter() - tt) * 1e3
        fields[tag] = sbq.laplace_apply(src, nrm, w, x, t(pts), eta, 1.0, prec="fp64").cpu().numpy()
        res[tag] = {"nodes": n, "panels": panels, "ntheta": nt, "setup_ms": ms,
                    "setup_unknowns_per_s": n / (ms * 1e-3) if ms else None,
                    "nnz": int(E[2].shape[0]) if E is not None else 0,
                    "solve_ms": solve_ms, "iters": rep["iters"], "refinements": rep["outer_iters"],
                    "rel_res": rep["rel_res"], "status": rep["status_name"]}
        if corrected and args.iteration_study:
            # iteration counts of the same system: plain FP64 GMRES(100) (no FP32 inner solve)
            # and both solvers with a longer restart, to separate the operator's conditioning,
            # the restart length and the FP32 inner solves
            study = {}
            for name, kw in (("fp64_restart100", dict(inner_prec="fp64", restart=100)),
                             ("fp64_restart256", dict(inner_prec="fp64", restart=256)),
                             ("fp32c_restart256", dict(inner_prec="fp32c", restart=256,
                                                       inner_tol=1e-5, resid_prec="fp64"))):
                _, r2 = op.solve(rhs, tol=1e-10, max_iter=3000, **kw)
                study[name] = {"iters": r2["iters"], "cycles_or_refinements": r2["outer_iters"],
                               "rel_res": r2["rel_res"], "status": r2["status_name"]}
            res[tag]["iteration_study"] = study
        op.close()
        del E
        torch.cuda.empty_cache()
    ref = fields["fine_E"]
    for tag in ("coarse_E", "coarse_punctured"):
        res[tag]["field_err_vs_fine_E"] = float(np.abs(fields[tag] - ref).max() / np.abs(ref).max())
    print(json.dumps({"workload": "quadrature_slender_loop_laplace_u1", "eta": eta,
                      "check_points": int(pts.shape[1]), "check_min_distance": 0.5,
                      "near_factor": args.near_factor, "solves": res}), flush=True)

    # (3) Stokes combined-field E on the coarse loop
    s = I.random_loop(seed=1, panels=P, ns=8, nth=16)
    E, ms = timed_build(t(s.x), t(s.n), t(s.w), P, 8, 16, kind="stokes", alpha=sbq.slender_eta(0.01),
                        beta=1.0, near_factor=args.near_factor)
    nnz = int(E[2].shape[0])
    items = nnz // (9 * 8 * 16)
    # the oracle building rows of the same E, on a bounded sample of targets (CPU baseline)
    import warnings
    from oracle import tube_quadrature as TQ
    tg = np.random.default_rng(17).choice(s.size, 4, replace=False)
    tt = time.perf_counter()
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        rows = TQ.correction_rows(s.x, s.n, s.w, P, 8, 16, "stokes", sbq.slender_eta(0.01), 1.0,
                                  args.near_factor, tg)
    sec = time.perf_counter() - tt
    o_items = sum(len(v) for v in rows.values())
    print(json.dumps({"workload": "quadrature_stokes_build_random_loop", "nodes": s.size,
                      "build_ms": ms, "nnz": nnz, "csr_bytes": nnz * 16,
                      "target_element_items": items, "us_per_item": ms * 1e3 / items,
                      "items_per_s": items / (ms * 1e-3),
                      "unknowns_per_s": 3 * s.size / (ms * 1e-3),
                      "roofline": {"bound": "fp64", "profile":
                                   "profiles/tube_correction_stokes_random_loop_32768.md"},
                      "cpu_baseline": {"kind": "oracle", "value": o_items / sec,
                                       "unit": "(target, element) items/s", "cores": 1,
                                       "sample": "%d targets, %d items of the same E in %.1f s "
                                                 "(numpy)" % (len(tg), o_items, sec)}}),
          flush=True)
    return 0


def run_peaks(args):
    """Arithmetic peaks measured with FMA chains on every SM (FP32, packed FP32x2, FP64),
    beside the FP32 peak the pair-sum roofline uses (SMs x 128 lanes x 2 x max SM clock) and
    the SM clock sampled while they run."""
    import torch
    from paper_2310_00889_gb300 import build as b
    b.build()
    from paper_2310_00889_gb300 import sbq
    torch.cuda.set_device(0)
    info = sbq.device_info()
    sm_max = 2070.0
    try:
        sm_max = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("sm_max_mhz", sm_max))
    except (OSError, ValueError):
        pass
    model = info["sms"] * info["fp32_lanes_per_sm"] * 2 * sm_max * 1e6 / 1e12
    res = {}
    for kind in ("fp32", "fp32x2", "fp64"):
        tf, ms = sbq.peak_probe(kind)
        tf, ms = sbq.peak_probe(kind)
        res[kind] = {"tflops": tf, "ms": ms}
    print(json.dumps({"workload": "peaks_fma_chains", "sms": info["sms"],
                      "fp32_model_tflops": model, "sm_max_mhz": sm_max, "measured": res,
                      "fp32_measured_over_model": res["fp32"]["tflops"] / model,
                      "fp32x2_measured_over_model": res["fp32x2"]["tflops"] / model}), flush=True)
    return 0


def run_tree(args):
    """Far-field acceleration: the treecode (stokes_tree_*) for the single layer and for the
    operator's combined field on the slender random loop at 1,048,576 and 4,194,304 nodes
    (Sec. 5.2 recipe), against the plain FP32 direct sums: apply times (CUDA events, median
    of the repetitions), kernel evaluations per apply, and the error of each on 2,048 sampled
    rows against the FP64 direct sum."""
    import torch
    import numpy as np
    from paper_2310_00889_gb300 import build as b
    b.build()
    from paper_2310_00889_gb300 import sbq, inputs as I
    torch.cuda.set_device(0)
    rng = np.random.default_rng(7)

    def t(a):
        return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")

    def timed(fn, reps):
        out, ms = None, []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            out = fn()
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return out, float(np.median(ms))

    rows = []
    for panels in [int(v) for v in args.tree_panels.split(",")]:
        s = I.random_loop(seed=1, panels=panels, ns=8, nth=16)
        n = s.size
        src, w = t(s.x), t(s.w)
        sig = t(rng.standard_normal((3, n)))
        sub = np.sort(rng.choice(n, 2048, replace=False))
        ref = sbq.sl_apply(src, w, sig, t(s.x[:, sub]), prec="fp64").cpu().numpy()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tree = sbq.SlTree(src, w, theta=0.5, order=8)
        torch.cuda.synchronize()
        setup_ms = (time.perf_counter() - t0) * 1e3
        u, tree_ms = timed(lambda: tree.apply(sig), 5)
        err_tree = float(np.abs(u.cpu().numpy()[:, sub] - ref).max() / np.abs(ref).max())
        st = tree.stats()
        tree.close()
        ud, direct_ms = timed(lambda: sbq.sl_apply(src, w, sig, src, prec="fp32"), 2 if n <= 2 ** 21 else 1)
        err_direct = float(np.abs(ud.cpu().numpy()[:, sub] - ref).max() / np.abs(ref).max())
        del ud, u
        torch.cuda.empty_cache()
        # the operator's combined field eta S + D with the same tree parameters
        eta = sbq.slender_eta(0.01)
        nrm = t(s.n)
        refc = sbq.combined_apply(src, nrm, w, sig, t(s.x[:, sub]), eta, 1.0, prec="fp64").cpu().numpy()
        ctree = sbq.StokesTree(src, w, nrm=nrm, alpha=eta, beta=1.0, theta=0.5, order=8)
        uc, ctree_ms = timed(lambda: ctree.apply(sig), 5)
        err_c = float(np.abs(uc.cpu().numpy()[:, sub] - refc).max() / np.abs(refc).max())
        ctree.close()
        del uc
        uc, cdirect_ms = timed(lambda: sbq.combined_apply(src, nrm, w, sig, src, eta, 1.0, prec="fp32"), 1)
        err_cd = float(np.abs(uc.cpu().numpy()[:, sub] - refc).max() / np.abs(refc).max())
        del uc
        torch.cuda.empty_cache()
        rows.append({"nodes": n, "theta": 0.5, "order": 8,
                     "combined_field": {"eta": eta, "apply_ms": ctree_ms, "err_vs_fp64": err_c,
                                        "direct_fp32_ms": cdirect_ms,
                                        "direct_fp32_err_vs_fp64": err_cd,
                                        "speedup": cdirect_ms / ctree_ms},
                     "setup_ms": setup_ms, "apply_ms": tree_ms,
                     "kernel_evaluations": st["pairs"], "direct_pairs": float(n) * n,
                     "cells": st["cells"], "proxies": st["proxies"], "list_entries": st["entries"],
                     "err_vs_fp64": err_tree, "direct_fp32_ms": direct_ms,
                     "direct_fp32_err_vs_fp64": err_direct, "speedup": direct_ms / tree_ms})
    # the headline geometry (helix wall, caps, 100 spheres; 1.1M nodes): the operator's
    # combined field by the treecode against the compensated-FP32 direct sum the benchmark
    # line times
    hs, heps, hsig = headline_inputs(args.helix_panels)
    hsrc, hnrm, hw, hs_sig = t(hs.x), t(hs.n), t(hs.w), t(hsig)
    heta = sbq.slender_eta(heps)
    hsub = np.sort(rng.choice(hs.size, 2048, replace=False))
    href = sbq.combined_apply(hsrc, hnrm, hw, hs_sig, t(hs.x[:, hsub]), heta, 1.0, prec="fp64").cpu().numpy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    htree = sbq.StokesTree(hsrc, hw, nrm=hnrm, alpha=heta, beta=1.0, theta=0.5, order=8)
    torch.cuda.synchronize()
    hsetup = (time.perf_counter() - t0) * 1e3
    hu, hms = timed(lambda: htree.apply(hs_sig), 5)
    herr = float(np.abs(hu.cpu().numpy()[:, hsub] - href).max() / np.abs(href).max())
    hst = htree.stats()
    htree.close()
    del hu
    hd, hdms = timed(lambda: sbq.combined_apply(hsrc, hnrm, hw, hs_sig, hsrc, heta, 1.0, prec="fp32c"), 1)
    hderr = float(np.abs(hd.cpu().numpy()[:, hsub] - href).max() / np.abs(href).max())
    del hd
    torch.cuda.empty_cache()
    helix = {"nodes": hs.size, "eta": heta, "setup_ms": hsetup, "apply_ms": hms, "err_vs_fp64": herr,
             "kernel_evaluations": hst["pairs"], "direct_pairs": float(hs.size) ** 2,
             "direct_fp32c_ms": hdms, "direct_fp32c_err_vs_fp64": hderr, "speedup": hdms / hms}
    solve = None
    if args.tree_solve_panels > 0:
        # GMRES-IR for K = I/2 + D + eta S + E (tube correction, near factor 0.5) with FP64
        # residuals: treecode inner solves against compensated-FP32 direct ones
        P = args.tree_solve_panels
        s = I.random_loop(seed=1, panels=P, ns=8, nth=16)
        n = s.size
        src, nrm, w = t(s.x), t(s.n), t(s.w)
        eta = sbq.slender_eta(0.01)
        E = sbq.tube_correction(src, nrm, w, P, 8, 16, kind="stokes", alpha=eta, beta=1.0,
                                near_factor=0.5)
        op = sbq.StokesOp(src, nrm, w, eta, correction=E)
        rhs = t(rng.standard_normal((3, n)))
        res = {}
        for name, inner in (("treecode_inner", "fp32"), ("compensated_fp32_inner", "fp32c")):
            if inner == "fp32":
                op.set_tree(0.5, 8)
            else:
                op.set_tree(0.0)
                op.autotune("fp32c")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            x, rep = op.solve(rhs, tol=1e-10, inner_prec=inner, inner_tol=1e-5, resid_prec="fp64")
            torch.cuda.synchronize()
            res[name] = {"ms": (time.perf_counter() - t0) * 1e3, "iters": rep["iters"],
                         "refinements": rep["outer_iters"], "rel_res": rep["rel_res"],
                         "status": rep["status_name"]}
            res[name + "_x"] = x
        res["solution_rel_diff"] = float((res.pop("treecode_inner_x") - res["compensated_fp32_inner_x"]).abs().max().item()
                                         / res.pop("compensated_fp32_inner_x").abs().max().item())
        op.close()
        solve = {"nodes": n, "eta": eta, "near_factor": 0.5, "tol": 1e-10, **res}
    print(json.dumps({"workload": "treecode_random_loop", "rows": rows, "headline_geometry": helix,
                      "solve": solve}), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "helix":
        return run_helix(args)
    if args.workload == "precision_sweep":
        return run_precision_sweep(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "laplace":
        return run_laplace(args)
    if args.workload == "mobility":
        return run_mobility(args)
    if args.workload == "quadrature":
        return run_quadrature(args)
    if args.workload == "peaks":
        return run_peaks(args)
    if args.workload == "curved_pipe":
        return run_curved_pipe(args)
    if args.workload == "tree":
        return run_tree(args)
    return run_headline(args)


if __name__ == "__main__":
    sys.exit(main())
