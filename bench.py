"""Benchmark: matrix-free CG on the 2D Dirichlet 5-point Laplacian on GB300.

Workload (one "step"): the 4096 x 4096 binary64 grid, b = A u* + 1e-3 xi
(u* = sin(pi x) sin(pi y), xi ~ N(0,1), seed 2), x0 = 0, solved by classic CG
(Algorithm 1) for 500 fixed iterations and then by NewCG (Algorithm 2) for 500
fixed iterations, each in one persistent launch.  Metric: grid points x CG
iterations per second over the whole job.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints ONE JSON line (rank 0).  Under torchrun (N > 1) every rank solves its
own replica of the step on its own GPU (the solver does not shard across GPUs);
value = all ranks' points*iterations / max-over-ranks time.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import lap5_inputs as gen  # noqa: E402

METRIC = "grid-pts·CG-iters/s and HBM GB/s vs peak; time-to-1e-10 mixed vs FP64 CG"
UNIT = "grid-pts*CG-iters/s"
NX = NY = 4096
ITERS = 500
SEED = 2
VARIANTS = ("classic", "newcg")
WORKLOAD = ("4096x4096 interior grid, FP64, b = A u* + 1e-3 N(0,1) (seed 2), x0 = 0; classic CG then NewCG, "
            "500 fixed iterations each, one persistent launch per solve")

# Algorithmic cost per grid point per iteration of each fused kernel (binary64):
# bytes = minimum HBM traffic of the variant (each state vector read/written once),
# ops = FP64-pipe instructions (stencil 4, each axpy 1, each dot 1).
COST = {
    # store-z form with the x update deferred into the next phase P:
    # phase P reads r, p_old, x and writes p, z, x; phase R reads r, z and writes r
    "classic": {"bytes": 72, "fp64_ops": 9, "kernel": "k_classic<double,4>"},  # four columns a lane
    "newcg": {"bytes": 96, "fp64_ops": 12, "kernel": "k_newcg<double,2>"},
}
FP64_PEAK_TFLOPS = 1.25  # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (nominal GB300 FP64)
FP64_PEAK = {"tflops": FP64_PEAK_TFLOPS, "kind": "nominal"}  # replaced by the measured rate at start-up


def measure_fp64_peak(lap5cg, dev):
    """The FP64 roofline denominator measured in this run: the library's FMA
    throughput kernel (lap5cg_fp64_rate), FMA = 2 flop."""
    try:
        r = lap5cg.fp64_rate(dev)
    except Exception as e:
        return {"tflops": FP64_PEAK_TFLOPS, "kind": "nominal (measurement failed: %s)" % str(e)[:100]}
    return {"tflops": 2 * r["fma_per_s"] / 1e12, "kind": "measured", "add_tflops": 2 * r["add_per_s"] / 1e12,
            "nominal_tflops": FP64_PEAK_TFLOPS}


def captured_traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary, or None when the
    kernel sources changed since the capture (stale counters are not reported)."""
    import hashlib
    try:
        d = json.load(open(os.path.join(ROOT, "profiles", "traffic_per_launch.json")))[kernel]
        m = hashlib.sha1()
        for f in d["files"]:  # the kernel sources the counters were taken from
            m.update(open(os.path.join(ROOT, "paper_1803_03797_gb300", "csrc", f), "rb").read())
        return d["bytes_per_launch"] if m.hexdigest() == d["source_sha1"] else None
    except Exception:
        return None


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # the raw samples go to LAP5CG_CLOCKS_DIR when set (kept for inspection), else a temporary folder
        d = os.environ.get("LAP5CG_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, "lap5cg_clocks_rank%d.csv" % index)

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
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
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(ms, device=None):
    """Slowest rank's time (the job finishes when the last replica does)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank_step, steps, world, max_ms):
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return world * units_per_rank_step * steps / (max_ms * 1e-3)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def host_cores():
    """Cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def _oracle_sample(oracle, b, sample_iters):
    t0 = time.perf_counter()
    for v in VARIANTS:
        oracle.cg_solve(b, variant=v, tol=0.0, maxit=sample_iters)
    return time.perf_counter() - t0


def cpu_baseline(sample_iters=4):
    """The oracle (plain C, as it stands) on a bounded sample of the step: both
    variants for sample_iters iterations on the full grid, in its two timing
    modes -- the sequential parity build (one core) and the OpenMP build (its
    row loops and per-thread partial dot products on every core this process
    may use).  value / cores are the OpenMP mode's when that build is
    available, else the sequential one's."""
    import oracle
    b = gen.manufactured_rhs(NX, NY, seed=SEED)
    units = len(VARIANTS) * NX * NY * sample_iters
    dt1 = _oracle_sample(oracle, b, sample_iters)
    out = {"value": units / dt1, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": "%dx%d FP64, classic + NewCG, %d iterations each (incl. setup and final true-residual pass)"
                     % (NX, NY, sample_iters), "seconds": dt1, "value_single_thread": units / dt1,
           "cores_available": host_cores()}
    try:
        with oracle.timing_build() as tb:
            _oracle_sample(oracle, b, 1)  # thread pool start-up outside the timing
            dtn = _oracle_sample(oracle, b, sample_iters)
        out.update({"value": units / dtn, "cores": tb.threads, "seconds": dtn, "mode": "openmp"})
    except Exception as e:  # no OpenMP toolchain: the sequential figure stands
        out["mode"] = "single-thread (OpenMP build unavailable: %s)" % str(e).splitlines()[0][:120]
    return out


def fused_f32_roofline(lap5cg, torch, dev, hbm_peak, n=8192, iters=200, reps=3):
    """Binary32 classic CG (the inner loop of the mixed-precision solve) on the
    n x n uniform right-hand side, fixed iterations: HBM roofline of the fused
    iteration (32 algorithmic bytes per point per iteration, A p recomputed)."""
    b = torch.from_numpy(gen.uniform_rhs(n, n, seed=3).astype(np.float32)).to(dev)
    x = torch.zeros_like(b)
    ws = torch.empty(lap5cg.workspace_size(n, n, n, "classic", "f32"), dtype=torch.uint8, device=dev)
    info = torch.empty(lap5cg.INFO_BYTES, dtype=torch.uint8, device=dev)
    pts_it = n * n * iters

    def timed(lane_vec):
        opts = lap5cg.default_opts(true_residual=0, lane_vec=lane_vec)

        def run():
            lap5cg.cg_solve(b, tol=0.0, maxit=iters, precision="f32", workspace=ws, info=info, out=x, opts=opts)

        run()
        torch.cuda.synchronize(dev)
        ms = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            run()
            e1.record()
            torch.cuda.synchronize(dev)
            ms.append(e0.elapsed_time(e1))
        return float(np.median(ms)) * 1e-3

    t = timed(0)  # the default: eight columns a lane at this width
    t4 = timed(4)
    gbs = 32 * pts_it / t / 1e9
    del b, x, ws
    return {"kernel": "k_classic<float,8>", "workload": "%dx%d binary32 classic CG, U[-1,1) (seed 3), %d fixed "
            "iterations, A p recomputed" % (n, n, iters), "ms_per_launch": t * 1e3, "pts_iters_per_s": pts_it / t,
            "hbm": {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                    "bytes_per_pt_iter": 32},
            "lane_vec_4": {"ms_per_launch": t4 * 1e3, "hbm_frac": 32 * pts_it / t4 / 1e9 / hbm_peak}}


def stencil_roofline(lap5cg, torch, dev, hbm_peak, n=8192, reps=11):
    """lap5_apply (y = A x) on an n x n grid per storage type, timed alone after
    an L2 flush (median of reps): HBM roofline at 2 * element-size algorithmic
    bytes per point (x read once, y written once), and for binary64 the FP64
    pipe at 4 operations per point.  The flush writes a buffer larger than L2
    and then reads another one, so that the flush's own dirty lines are written
    back before the timed launch instead of inside it (a 134 MB bf16 apply
    would otherwise pay for writing back ~100 MB of the flush)."""
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device=dev)  # larger than L2
    evict = torch.ones(256 * 2 ** 20, dtype=torch.uint8, device=dev)
    out = {}
    for name, dt in (("f64", torch.float64), ("f32", torch.float32), ("bf16", torch.bfloat16)):
        x = torch.from_numpy(gen.uniform_rhs(n, n, seed=5)).to(dev).to(dt)
        y = torch.empty_like(x)
        lap5cg.lap5_apply(x, out=y)
        ms = []
        for _ in range(reps):
            flush.zero_()
            evict.max()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            lap5cg.lap5_apply(x, out=y)
            e1.record()
            torch.cuda.synchronize(dev)
            ms.append(e0.elapsed_time(e1))
        t = float(np.median(ms)) * 1e-3
        gbs = 2 * x.element_size() * n * n / t / 1e9
        out[name] = {"ms": t * 1e3, "hbm": {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                                            "bytes_per_pt": 2 * x.element_size()}}
        if name == "f64":
            tfl = 2 * 4 * n * n / t / 1e12
            out[name]["fp64"] = {"achieved": tfl, "peak": FP64_PEAK["tflops"], "unit": "TFLOP/s",
                                 "frac": tfl / FP64_PEAK["tflops"], "peak_kind": FP64_PEAK["kind"], "ops_per_pt": 4}
        del x, y
    out["workload"] = ("%dx%d grid, U[-1,1) (seed 5), one lap5_apply per storage type; L2 flushed by a 256 MiB write, "
                       "its dirty lines then evicted by a 256 MiB read" % (n, n))
    return out


def time_to_solution(lap5cg, torch, dev, n, rhs, tol=1e-10):
    """Wall time on the GPU (CUDA events, one solve after a warm-up) to reach
    relative residual tol: FP64 classic and NewCG vs mixed precision and the
    multigrid-preconditioned CG (binary64 PCG, binary32 / binary64 V-cycle)."""
    b = torch.from_numpy(rhs).to(dev)
    out = {}
    # NewCG to 1e-10 at these condition numbers needs residual replacement
    # (without it Algorithm 2 breaks down in binary64, on the oracle as well)
    # (the stabilised NewCG forms alpha from dot products of the current vectors)
    for name, variant, prec, rr, stab in (("f64_classic", "classic", "f64", 0, 0),
                                          ("f64_newcg_rr100", "newcg", "f64", 100, 0),
                                          ("f64_newcg_stable_rr100", "newcg", "f64", 100, 1),
                                          ("ir_f32", "classic", "ir_f32", 0, 0), ("ir_bf16pr", "classic", "ir_bf16pr", 0, 0),
                                          ("pcg_mg_f32", "classic", "mg_f32", 0, 0), ("pcg_mg_f64", "classic", "mg_f64", 0, 0),
                                          ("pipelined_pcg_mg_f64", "newcg", "mg_f64", 0, 0)):
        opts = lap5cg.default_opts(rr_period=rr, stabilized=stab)
        # buffers allocated before the timed solve (an allocation inside it
        # would leave the GPU idle while the host allocates)
        ws = torch.empty(lap5cg.workspace_size(n, n, n, variant, prec), dtype=torch.uint8, device=dev)
        x = torch.zeros_like(b)
        info = torch.empty(lap5cg.INFO_BYTES, dtype=torch.uint8, device=dev)
        if prec.startswith("mg"):
            # warm-up: the full solve (milliseconds), which also instantiates the
            # multigrid graph for this shape and workspace (cached afterwards)
            lap5cg.cg_solve(b, tol=tol, maxit=10 ** 6, variant=variant, precision=prec, opts=opts, workspace=ws,
                            out=x, info=info)
        else:
            # warm-up (first launch of each kernel) on a 512^2 corner, not the full solve (seconds)
            lap5cg.cg_solve(b[:512, :512].contiguous(), tol=tol, maxit=10 ** 6, variant=variant, precision=prec,
                            opts=opts)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        x, info = lap5cg.cg_solve(b, tol=tol, maxit=10 ** 6, variant=variant, precision=prec, opts=opts, workspace=ws,
                                  out=x, info=info)
        e1.record()
        torch.cuda.synchronize(dev)
        rec = lap5cg.decode_info(info)[0]
        out[name] = {"ms": e0.elapsed_time(e1), "iters": rec["iters"], "outer_iters": rec["outer_iters"],
                     "status": rec["status"], "relres_true": rec["relres_true"]}
        del x
    def speedup(name):  # only between solves that both reached the tolerance
        ok = out["f64_classic"]["status"] == 0 and out[name]["status"] == 0
        return out["f64_classic"]["ms"] / out[name]["ms"] if ok else None

    out["speedup_ir_f32_vs_f64_classic"] = speedup("ir_f32")
    out["speedup_ir_bf16pr_vs_f64_classic"] = speedup("ir_bf16pr")
    out["speedup_pcg_mg_f32_vs_f64_classic"] = speedup("pcg_mg_f32")
    return out


def batched_workload(lap5cg, torch, dev, tune=True):
    """The batched workload: 256 grids with sides ~U{64..1024} (seed 4), each
    its own U[-1,1) right-hand side, mixed precision (binary32 inner CG, FP64
    refinement) to 1e-10 in one persistent launch, optionally autotuned."""
    nxs, nys = gen.batched_shapes(256, 64, 1024, seed=4)
    bs = [torch.from_numpy(b).to(dev) for b in gen.batched_rhs(nxs, nys, seed=4, elem_bytes=8, align_bytes=32)]
    xs = [torch.zeros_like(b) for b in bs]
    lds = [b.shape[1] for b in bs]
    need = lap5cg.batched_workspace_size(nxs, nys, lds, "classic", "ir_f32")
    ws = torch.empty(need, dtype=torch.uint8, device=dev)
    info = torch.empty(256 * lap5cg.INFO_BYTES, dtype=torch.uint8, device=dev)
    def timed(opts):
        # x0 = 0 and the solve, captured once in a CUDA graph; the timed
        # region is one replay
        def run():
            for x in xs:
                x.zero_()
            lap5cg.cg_solve_batched(bs, xs=xs, tol=1e-10, maxit=10 ** 7, precision="ir_f32", nx_list=nxs, opts=opts,
                                    workspace=ws, info=info)

        run()  # warm-up (and the library's one-time setup) outside the capture
        torch.cuda.synchronize(dev)
        g = torch.cuda.CUDAGraph()
        cs = torch.cuda.Stream(dev)
        cs.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.graph(g, stream=cs):
            run()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.replay()
        e1.record()
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1), lap5cg.decode_info(info)

    ms_default, recs_default = timed(lap5cg.default_opts())
    ms, recs, tuned = ms_default, recs_default, None
    if tune:  # trials solve every instance to 1e-4, so the queue's tail weighs as in the real solve
        opts, tms = lap5cg.autotune_batched(bs, precision="ir_f32", iters=0, nx_list=nxs, cache=False)
        tuned = {k: int(getattr(opts, k)) for k in ("team_ctas", "warps_per_cta", "ring_slots", "min_rows")}
        ms, recs = timed(opts)
    pts_it = sum(nx * ny * r["iters"] for nx, ny, r in zip(nxs, nys, recs))
    return {"workload": "256 grids, sides U{64..1024} (seed 4), U[-1,1) RHS, IR: binary32 inner classic CG + FP64 "
                        "refinement to 1e-10, one persistent launch captured in a CUDA graph (timed: one replay)", "ms": ms, "ms_default_opts": ms_default,
            "total_points": int(sum(nx * ny for nx, ny in zip(nxs, nys))),
            "inner_pts_iters_per_s": pts_it / (ms * 1e-3),
            "all_converged": all(r["status"] == 0 for r in recs + recs_default),
            "max_relres_true": max(r["relres_true"] for r in recs + recs_default), "tuned_opts": tuned}


def autograd_workload(lap5cg, torch, dev, n=2048, k=16, tol=1e-10):
    """The differentiable solve: n x n grid, k right-hand sides (U[-1,1), seeds
    5000+s), x_target Gaussian (seeds 6000+s), loss = 0.5 ||x - x_target||^2;
    forward = k solves to tol, backward = the k adjoint solves.  CUDA events
    around forward and backward, per precision."""
    b0 = np.stack([gen.uniform_rhs(n, n, seed=5000 + s) for s in range(k)])
    xt = torch.from_numpy(np.stack([gen.gaussian_field(n, n, seed=6000 + s) for s in range(k)])).to(dev)
    out = {"workload": "%dx%d grid, %d right-hand sides, loss 0.5||x - x_target||^2, tol %g" % (n, n, k, tol)}
    # the loss's elementwise, reduction and gradient kernels run once untimed:
    # their first launch in a process can include seconds of driver-side
    # compilation on the host
    w = torch.zeros(4, dtype=torch.float64, device=dev, requires_grad=True)
    (0.5 * ((w - xt.flatten()[:4]) ** 2).sum()).backward()
    torch.cuda.synchronize(dev)
    for precision in ("f64", "ir_f32", "mg_f32"):
        b = torch.from_numpy(b0).to(dev).requires_grad_(True)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record()
        x, info = lap5cg.CGSolve.apply(b, tol, 10 ** 7, "classic", precision, None)
        loss = 0.5 * ((x - xt) ** 2).sum()
        ev[1].record()
        loss.backward()
        ev[2].record()
        torch.cuda.synchronize(dev)
        recs = lap5cg.decode_info(info)
        out[precision] = {"forward_ms": ev[0].elapsed_time(ev[1]), "backward_ms": ev[1].elapsed_time(ev[2]),
                          "forward_iters": int(sum(r["iters"] for r in recs)),
                          "all_converged": all(r["status"] == 0 for r in recs)}
        del b, x
    return out


def paper_size_workload(lap5cg, torch, dev, reps=20):
    """The paper's largest grid: 100 x 100 FP64, U[-1,1) (seed 1), x0 = 0, to 1e-8;
    latency-bound.  Through cg_solve ("cg_solve": the cluster-resident kernel,
    the grid held in the shared memory of a 16-CTA cluster) and through
    cg_solve_batched with one instance ("batched_1": one cluster team working
    from global memory)."""
    b = torch.from_numpy(gen.uniform_rhs(100, 100, seed=1)).to(dev)
    out = {}
    for variant in ("classic", "newcg"):
        for path in ("cg_solve", "batched_1"):
            def run():
                if path == "cg_solve":
                    return lap5cg.cg_solve(b, tol=1e-8, maxit=10000, variant=variant)[1]
                return lap5cg.cg_solve_batched([b], tol=1e-8, maxit=10000, variant=variant, precision="f64")[1]
            run()
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                info = run()
            e1.record()
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1) / reps
            rec = lap5cg.decode_info(info)[0]
            out["%s_%s" % (variant, path)] = {"ms": ms, "iters": rec["iters"], "status": rec["status"],
                                              "us_per_iter": ms * 1e3 / max(rec["iters"], 1)}
    return out


def reproducible_workload(lap5cg, torch, dev, b, iters=500, reps=2):
    """The benchmark's 4096 x 4096 FP64 step in reproducible mode (exact dot
    products, fused updates): grid-point iterations per second per variant,
    next to the default mode timed the same way."""
    n = b.shape[0]
    out = {}
    for variant in VARIANTS:
        for rep in (0, 1):
            opts = lap5cg.default_opts(reproducible=rep, true_residual=0)

            def run():
                lap5cg.cg_solve(b, tol=0.0, maxit=iters, variant=variant, opts=opts)

            run()
            torch.cuda.synchronize(dev)
            ms = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                run()
                e1.record()
                torch.cuda.synchronize(dev)
                ms.append(e0.elapsed_time(e1))
            t = min(ms) * 1e-3
            out["%s_%s" % (variant, "reproducible" if rep else "default")] = {"ms": t * 1e3,
                                                                              "pts_iters_per_s": n * n * iters / t}
    for variant in VARIANTS:
        out["%s_cost" % variant] = (out["%s_default" % variant]["pts_iters_per_s"] /
                                    out["%s_reproducible" % variant]["pts_iters_per_s"])
    return out


def targets_summary(extras, roofline):
    """The headline targets (HBM fractions, FP64 fraction, times to 1e-10 and their speedups) as flat scalars
    (None where not measured)."""
    def get(*path):
        d = extras
        for k in path:
            if not isinstance(d, dict) or k not in d:
                return None
            d = d[k]
        return d

    t = {"fp64_fma_peak_tflops": FP64_PEAK["tflops"], "fp64_peak_kind": FP64_PEAK["kind"],
         "dominant_kernel_fp64_frac": roofline["frac"], "dominant_kernel_hbm_frac": roofline["hbm_frac"],
         "fused_f32_8192_hbm_frac": get("fused_f32_8192", "hbm", "frac"),
         "lap5_apply_8192_f32_hbm_frac": get("lap5_apply_8192", "f32", "hbm", "frac"),
         "lap5_apply_8192_bf16_hbm_frac": get("lap5_apply_8192", "bf16", "hbm", "frac")}
    for n in (4096, 8192):
        key = "time_to_1e-10_%d" % n
        if key not in extras:
            continue
        for name in ("f64_classic", "f64_newcg_rr100", "f64_newcg_stable_rr100", "ir_f32", "ir_bf16pr", "pcg_mg_f32"):
            t["tts%d_%s_ms" % (n, name)] = get(key, name, "ms")
            t["tts%d_%s_status" % (n, name)] = get(key, name, "status")
        t["tts%d_speedup_ir_f32_vs_f64" % n] = get(key, "speedup_ir_f32_vs_f64_classic")
        t["tts%d_speedup_ir_bf16pr_vs_f64" % n] = get(key, "speedup_ir_bf16pr_vs_f64_classic")
    p = extras.get("paper_100x100_to_1e-8")
    if p:
        t["paper100_us_per_iter_classic"] = p["classic_cg_solve"]["us_per_iter"]
        t["paper100_us_per_iter_newcg"] = p["newcg_cg_solve"]["us_per_iter"]
    t["batched_256_ms"] = get("batched_256_ir_f32", "ms")
    return t


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    b = gen.manufactured_rhs(NX, NY, seed=SEED)
    import oracle
    sample_iters = 3
    cores, mode = 1, "single-thread"
    tb = None
    try:  # the oracle's OpenMP timing build on every core this process may use
        tb = oracle.timing_build()
        tb.__enter__()
        cores, mode = tb.threads, "openmp"
    except Exception as e:
        tb = None
        mode = "single-thread (OpenMP build unavailable: %s)" % str(e).splitlines()[0][:120]

    def step():
        for v in VARIANTS:
            oracle.cg_solve(b, variant=v, tol=0.0, maxit=sample_iters)

    for _ in range(max(0, min(args.warmup, 1))):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    if tb is not None:
        tb.__exit__(None, None, None)
    units = args.steps * len(VARIANTS) * NX * NY * sample_iters
    value = units / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD + " (reference arm: the CPU oracle, %d iterations per variant per step)"
                                   % sample_iters, "nx": NX, "ny": NY},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "mode": mode,
                             "cores_available": host_cores(),
                             "sample": "%d iterations per variant per step on the full grid" % sample_iters},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def _apply_overrides(args):
    global NX, NY, ITERS, VARIANTS, WORKLOAD
    v = tuple(x for x in args.variants.split(",") if x)
    if (args.n, args.iters, v) != (NX, ITERS, VARIANTS):
        NX = NY = args.n
        ITERS = args.iters
        VARIANTS = v
        WORKLOAD = "PROFILING CASE (not the benchmark workload): %dx%d FP64, %s, %d iterations" % (
            NX, NY, "+".join(VARIANTS), ITERS)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the f32 roofline and time-to-solution runs")
    ap.add_argument("--tts", action="store_true", help="also time FP64 vs mixed precision to 1e-10 at 8192^2")
    ap.add_argument("--autograd", action="store_true",
                    help="also time the differentiable solve (2048^2, 16 right-hand sides, forward + adjoint)")
    # profiling-size overrides (the defaults are the benchmark workload)
    ap.add_argument("--n", type=int, default=NX, help="grid side (profiling only)")
    ap.add_argument("--iters", type=int, default=ITERS, help="iterations per solve (profiling only)")
    ap.add_argument("--variants", default=",".join(VARIANTS), help="comma list (profiling only)")
    ap.add_argument("--profile-f32", type=int, default=0,
                    help="profiling only: run the binary32 8192^2 solve for this many iterations and exit")
    ap.add_argument("--profile-apply", type=int, default=0,
                    help="profiling case: lap5_apply on an N x N grid, twice (for ncu)")
    ap.add_argument("--profile-apply-dtype", default="f32", choices=["f32", "bf16", "f64"],
                    help="storage type of the --profile-apply case")
    ap.add_argument("--profile-solve", default="", choices=["", "newcg_stable_4096", "newcg_small_100"],
                    help="profiling case, solved twice: newcg_stable_4096 = the stabilised NewCG on the 4096^2 "
                         "manufactured problem, 20 fixed iterations; newcg_small_100 = NewCG on a 100^2 uniform "
                         "right-hand side to 1e-8 (the cluster-resident kernel)")
    ap.add_argument("--profile-mg", type=int, default=0,
                    help="profiling only: solve the n^2 manufactured problem to 1e-10 twice with the multigrid-"
                         "preconditioned CG (binary32 V-cycle) and exit")
    args = ap.parse_args()
    _apply_overrides(args)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_1803_03797_gb300 as lap5cg

    if args.profile_apply:
        lap5cg.lib()
        n = args.profile_apply
        dt = {"f32": torch.float32, "bf16": torch.bfloat16, "f64": torch.float64}[args.profile_apply_dtype]
        xa = torch.from_numpy(gen.uniform_rhs(n, n, seed=5)).to(torch.device("cuda", 0)).to(dt)
        ya = torch.empty_like(xa)
        for _ in range(2):
            lap5cg.lap5_apply(xa, out=ya)
        torch.cuda.synchronize()
        print(json.dumps({"profiling_case": {"lap5_apply": args.profile_apply_dtype, "n": n,
                                             "checksum": float(ya.double().sum())}}))
        return 0

    if args.profile_solve:
        lap5cg.lib()
        if args.profile_solve == "newcg_stable_4096":
            bp = gen.manufactured_rhs(4096, 4096, seed=SEED)
            kw = dict(tol=0.0, maxit=20, opts=lap5cg.default_opts(stabilized=1, true_residual=0))
        else:
            bp = gen.uniform_rhs(100, 100, seed=1)
            kw = dict(tol=1e-8, maxit=10000)
        bd = torch.from_numpy(bp).to(torch.device("cuda", 0))
        for _ in range(2):
            _, info = lap5cg.cg_solve(bd, variant="newcg", **kw)
        torch.cuda.synchronize()
        print(json.dumps({"profiling_case": dict(lap5cg.decode_info(info)[0], case=args.profile_solve)}))
        return 0

    if args.profile_mg:
        lap5cg.lib()
        n = args.profile_mg
        bm = torch.from_numpy(gen.manufactured_rhs(n, n, seed=SEED)).to(torch.device("cuda", 0))
        for _ in range(2):
            _, info = lap5cg.cg_solve(bm, tol=1e-10, maxit=500, precision="mg_f32",
                                      opts=lap5cg.default_opts(true_residual=0))
        torch.cuda.synchronize()
        print(json.dumps({"profiling_case": lap5cg.decode_info(info)[0]}))
        return 0

    if args.profile_f32:
        lap5cg.lib()
        r = fused_f32_roofline(lap5cg, torch, torch.device("cuda", 0), load_peaks()[0], iters=args.profile_f32,
                               reps=1)
        print(json.dumps({"profiling_case": r}))
        return 0

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    lap5cg.lib()

    b_host = gen.manufactured_rhs(NX, NY, seed=SEED)
    b = torch.from_numpy(b_host).to(dev)
    xs = {v: torch.zeros_like(b) for v in VARIANTS}
    wsz = max(lap5cg.workspace_size(NX, NY, NX, v, "f64") for v in VARIANTS)
    workspace = torch.empty(wsz, dtype=torch.uint8, device=dev)
    info = {v: torch.empty(lap5cg.INFO_BYTES, dtype=torch.uint8, device=dev) for v in VARIANTS}
    stream = torch.cuda.current_stream(dev)
    opts = lap5cg.default_opts()

    def solve(v):
        xs[v].zero_()
        lap5cg.cg_solve(b, tol=0.0, maxit=ITERS, variant=v, workspace=workspace, info=info[v], out=xs[v],
                        opts=opts, stream=stream)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        for v in VARIANTS:
            solve(v)
    barrier()
    for v in VARIANTS:
        rec = lap5cg.decode_info(info[v])[0]
        if rec["iters"] != ITERS or rec["status"] not in (lap5cg.OK, lap5cg.NOT_CONVERGED):
            raise RuntimeError("warm-up solve failed: %s %r" % (v, rec))
    # the FP64 roofline denominator, measured right after the warm-up (clocks up)
    FP64_PEAK.update(measure_fp64_peak(lap5cg, dev))

    ev = {v: [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)] for v in VARIANTS}
    clocks = ClockSampler(dev.index)
    clocks.start()
    barrier()
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for k in range(args.steps):
        for v in VARIANTS:
            ev[v][k][0].record(stream)
            solve(v)
            ev[v][k][1].record(stream)
    stop.record(stream)
    barrier()
    clk = clocks.stop()
    elapsed_ms = max_over_ranks(start.elapsed_time(stop), dev)
    units_per_step = len(VARIANTS) * NX * NY * ITERS
    value = job_value(units_per_step, args.steps, ws, elapsed_ms)

    hbm_peak, peak_kind = load_peaks()
    per_kernel = {}
    for v in VARIANTS:
        ms = float(np.mean([s.elapsed_time(e) for s, e in ev[v]]))
        pts_it = NX * NY * ITERS
        gbs = COST[v]["bytes"] * pts_it / (ms * 1e-3) / 1e9
        tfl = 2 * COST[v]["fp64_ops"] * pts_it / (ms * 1e-3) / 1e12
        fp64_peak = FP64_PEAK["tflops"]
        per_kernel[v] = {"kernel": COST[v]["kernel"], "ms_per_launch": ms, "pts_iters_per_s": pts_it / (ms * 1e-3),
                         "hbm": {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                                 "bytes_per_pt_iter": COST[v]["bytes"]},
                         "fp64": {"achieved": tfl, "peak": fp64_peak, "unit": "TFLOP/s",
                                  "frac": tfl / fp64_peak, "frac_of_nominal": tfl / FP64_PEAK_TFLOPS,
                                  "ops_per_pt_iter": COST[v]["fp64_ops"]}}
    dom = max(VARIANTS, key=lambda v: per_kernel[v]["ms_per_launch"])
    pk = per_kernel[dom]
    traffic = captured_traffic(COST[dom]["kernel"]) if (NX, ITERS) == (4096, 500) else None
    roofline = {"bound": "alu", "achieved": pk["fp64"]["achieved"], "peak": FP64_PEAK["tflops"], "unit": "TFLOP/s",
                "frac": pk["fp64"]["frac"], "traffic": traffic, "kernel": pk["kernel"],
                "peak_kind": FP64_PEAK["kind"] + " FP64 FMA rate (lap5cg_fp64_rate throughput kernel in this run; "
                             "FMA = 2 flop; every FP64 instruction of the solver counted as one FMA)",
                "peak_nominal": FP64_PEAK_TFLOPS, "frac_of_nominal": pk["fp64"]["frac_of_nominal"],
                "peak_fp64_add_tflops": FP64_PEAK.get("add_tflops"),
                "hbm_achieved": pk["hbm"]["achieved"], "hbm_peak": hbm_peak, "hbm_frac": pk["hbm"]["frac"],
                "hbm_view": pk["hbm"], "hbm_peak_kind": peak_kind}

    e2e = None
    if not args.no_e2e:
        # Copies run on two streams of their own and overlap the solves: the
        # next step's b goes into the other of two device buffers while this
        # step solves, and each solution is read back while the next solve runs.
        b_pin = torch.from_numpy(b_host).pin_memory()
        x_pin = {v: torch.empty_like(b_pin).pin_memory() for v in VARIANTS}
        b_dev = [torch.empty_like(b), torch.empty_like(b)]
        xs_dev = {v: torch.empty_like(b) for v in VARIANTS}
        info_pin = torch.empty(lap5cg.INFO_BYTES * 2, dtype=torch.uint8).pin_memory()
        h2d, d2h = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        b_free = [torch.cuda.Event(), torch.cuda.Event()]   # the solves reading b_dev[j] are done
        x_read = {v: torch.cuda.Event() for v in VARIANTS}  # xs_dev[v] has been copied out
        for e in b_free + list(x_read.values()):
            e.record(stream)

        def e2e_step(k):
            bk = b_dev[k % 2]
            h2d.wait_event(b_free[k % 2])
            with torch.cuda.stream(h2d):
                bk.copy_(b_pin, non_blocking=True)
            landed = torch.cuda.Event()
            landed.record(h2d)
            stream.wait_event(landed)
            for i, v in enumerate(VARIANTS):
                stream.wait_event(x_read[v])
                lap5cg.cg_solve(bk, tol=0.0, maxit=ITERS, variant=v, workspace=workspace, info=info[v],
                                out=xs_dev[v], opts=opts, stream=stream)
                solved = torch.cuda.Event()
                solved.record(stream)
                d2h.wait_event(solved)
                with torch.cuda.stream(d2h):
                    x_pin[v].copy_(xs_dev[v], non_blocking=True)
                    info_pin[i * lap5cg.INFO_BYTES:(i + 1) * lap5cg.INFO_BYTES].copy_(info[v], non_blocking=True)
                x_read[v].record(d2h)
            b_free[k % 2].record(stream)

        e2e_step(0)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h2d.wait_event(e0)
        for k in range(args.steps):
            e2e_step(k + 1)
        stream.wait_stream(d2h)  # the last read-back is inside the timed region
        e1.record(stream)
        barrier()
        ems = max_over_ranks(e0.elapsed_time(e1), dev)
        e2e = {"value": job_value(units_per_step, args.steps, ws, ems), "unit": UNIT,
               "h2d_bytes_per_step": int(b_pin.numel() * 8),
               "d2h_bytes_per_step": int(sum(x.numel() * 8 for x in x_pin.values()) + info_pin.numel()),
               "ms_per_step": ems / args.steps}

    extras = {}
    if not args.no_extras and ws == 1 and (NX, ITERS) == (4096, 500):
        extras["fused_f32_8192"] = fused_f32_roofline(lap5cg, torch, dev, hbm_peak)
        extras["lap5_apply_8192"] = stencil_roofline(lap5cg, torch, dev, hbm_peak)
        extras["time_to_1e-10_4096"] = time_to_solution(lap5cg, torch, dev, 4096, b_host)
        extras["batched_256_ir_f32"] = batched_workload(lap5cg, torch, dev)
        extras["paper_100x100_to_1e-8"] = paper_size_workload(lap5cg, torch, dev)
        extras["reproducible_4096"] = reproducible_workload(lap5cg, torch, dev, b)
        if args.tts:
            extras["time_to_1e-10_8192"] = time_to_solution(lap5cg, torch, dev, 8192,
                                                            gen.uniform_rhs(8192, 8192, seed=3))
        if args.autograd:
            extras["autograd_2048x16"] = autograd_workload(lap5cg, torch, dev)

    line = None
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and ws == 1:
            cpu = cpu_baseline()
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "nx": NX, "ny": NY, "iters_per_solve": ITERS,
                           "variants": list(VARIANTS), "parallelism": "replicas" if ws > 1 else "single-gpu",
                           "l2": "inputs larger than L2: each 4096^2 FP64 vector is 134 MB > 126 MB L2, "
                                 "working set ~1 GB"},
                "roofline": roofline, "per_kernel": per_kernel, "cpu_baseline": cpu, "e2e": e2e,
                "clocks": clk, "gpu_launches": len(VARIANTS) * args.steps, "extras": extras}
        line["targets"] = targets_summary(extras, roofline)  # last: compact figures, kept in short tails
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
