#!/usr/bin/env python
"""Benchmark of one adaptive FR cycle on the largest single-GPU vortex workload: four 3D vortex
tubes in the periodic box [0,80]^3, p=3 (64 points per hexahedron), base level 5, max level 10
(about 3M leaves), density-gradient indicator, FP64.

One bench step = one pass of the whole hot path: `adapt_every` (10) SSP-RK3 time steps -- each
stage an interface kernel (Rusanov, mortar projection) and an element kernel (corrected-flux
divergence, RK combination, traces) -- followed by one adaptation (indicator, refine/coarsen edit,
2:1 balance, mapping, transfer, connectivity).  K timed steps after W warm-up steps; the inputs
(~7.7 GB per state copy) are far larger than L2, and L2 is flushed between steps as well (a 512 MB
write outside the timed events).

value  = DOF-updates/s = sum over time steps of M*N*nv / device time of the K cycles
         (point_updates_per_s: the same over M*N, the unit of the paper's throughput figures).
e2e    = the same metric through the public API with host buffers: fr_set_state from pinned host
         arrays, the cycle, fr_get_leaves + fr_get_state back to host, every step.
cpu_baseline and --impl reference time the CPU oracle (single thread) on a bounded sample of the
same configuration (see oracle_sample); with --gpus N > 1 every rank runs an independent replica
(the method does not shard here).
"""
from __future__ import annotations

import argparse
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

METRIC = "adaptive FR DOF-updates/s at fixed vortex L2 error; adaptation % of walltime"
UNIT = "DOF-updates/s"
WORKLOAD = "vortex3d_p3_multi"
REF_BUDGET_S = 120.0  # CPU seconds the reference arm spends at most on its timed steps
# The oracle's bounded sample of a workload whose cycle does not fit a bounded CPU run: the same
# configuration (domain, vortices, p, thresholds, base level) with the maximum depth lowered to
# this value, timed per SSP-RK3 step and per adaptation.  An octree over the cube cannot be cut to
# a z-slab, so lowering the depth is the way to keep every other parameter of the workload.
ORACLE_SAMPLE_DMAX = {"vortex3d_p3_multi": 6, "vortex3d_p2_tube": 6}
FP64_PEAK_TFLOPS = 152 * 2.07e9 * 4 / 1e12  # 2 DFMA/clk/SM x 152 SMs x 2.07 GHz = 1.259 TFLOP/s


def flops_per_point_stage(dim, p):
    """Algorithmic FP64 flops of the element kernel per solution point (sum-factorised form):
    primitives, Euler fluxes, folded derivative+correction, RK combination, traces of the result.
    A divide or square root counts as one flop."""
    n, nv = p + 1, dim + 2
    prim = 3 * dim + 1 + 3
    flux = dim * (dim + 3)
    deriv = dim * nv * (2 * n + 3)
    rk = 6 * nv
    traces = 4 * dim * nv
    return prim + flux + deriv + rk + traces


def bytes_per_point_stage(dim, p):
    """Algorithmic DRAM bytes of the element kernel per solution point: read u_s, read u^n, write
    the result, read the common fluxes and write the traces (2*dim*nv/n values each)."""
    n, nv = p + 1, dim + 2
    return 8 * (3 * nv + 2 * (2 * dim * nv / n))


def _clock_sampler_start(path):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        fh = open(path, "w")
        return subprocess.Popen(["nvidia-smi", "--query-gpu=" + q, "--format=csv,noheader,nounits",
                                 "-lms", "200"], stdout=fh, stderr=subprocess.DEVNULL), fh
    except Exception:
        return None, None


def _clock_sampler_stop(proc, fh, path, device_index):
    if proc is None:
        return None
    proc.terminate()
    try:
        proc.wait(timeout=5)
    except Exception:
        proc.kill()
    fh.close()
    sm, mx, reasons = [], 0.0, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            if int(parts[0]) != device_index:
                continue
            sm.append(float(parts[1]))
            mx = max(mx, float(parts[2]))
        except ValueError:
            continue
        for nm, val in zip(names, parts[5:9]):
            if val.lower() == "active":
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
            "samples": len(sm)}


def host_cpu():
    """CPU model and core count of the host that runs the oracle."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    import platform
    return {"model": model or platform.processor() or platform.machine(), "nproc": os.cpu_count(),
            "machine": platform.machine()}


def oracle_sample(cfg, workload):
    """(configuration the oracle runs, whole_cycles, description) for a bounded CPU sample."""
    if workload in ORACLE_SAMPLE_DMAX:
        d = ORACLE_SAMPLE_DMAX[workload]
        return (dict(cfg, Dmax=d), False,
                "%s with the maximum depth lowered from %d to %d (same domain, vortices, p, "
                "thresholds and base level)" % (workload, cfg["Dmax"], d))
    return cfg, True, workload


class OracleTimer:
    """Times the CPU oracle on the sample of oracle_sample.  Whole cycles (adapt_every SSP-RK3
    steps + one adaptation) where one fits the budget; otherwise single SSP-RK3 steps, with one
    adaptation timed after them and weighted as in the cycle (one per adapt_every steps):
    rate = sum of step DOF-updates / (sum of step times + steps/adapt_every * adaptation time)."""

    def __init__(self, cfg, workload):
        import oracle as O
        self.cfg, self.whole, self.what = oracle_sample(cfg, workload)
        self.ae = cfg["adapt_every"]
        self.N = (cfg["p"] + 1) ** cfg["dim"]
        self.nv = cfg["dim"] + 2
        self.o = O.OracleMesh(self.cfg)
        self.dof = self.t_steps = self.t_adapt = 0.0
        self.steps = 0  # SSP-RK3 steps timed
        self.adapts = 0

    def one(self, timed=True):
        """One bench step of the oracle: a whole cycle, or one SSP-RK3 step."""
        M = self.o.M
        n = self.ae if self.whole else 1
        a = time.perf_counter()
        self.o.step(n)
        b = time.perf_counter()
        if self.whole:
            self.o.adapt()
        c = time.perf_counter()
        if timed:
            self.dof += n * M * self.N * self.nv
            self.t_steps += b - a
            self.steps += n
            if self.whole:
                self.t_adapt += c - b
                self.adapts += 1
        return c - a

    def finish(self):
        """Times one adaptation after single-step samples; returns (value, seconds charged)."""
        if not self.whole and self.steps:
            a = time.perf_counter()
            self.o.adapt()
            ta = time.perf_counter() - a
            self.t_adapt = ta * self.steps / self.ae
            self.adapts = 1
        t = self.t_steps + self.t_adapt
        return self.dof / t, t

    def sample_text(self):
        if self.whole:
            return "%d whole cycles (10 SSP-RK3 steps + 1 adaptation each) of %s, %d leaves at the end" % (
                self.adapts, self.what, self.o.M)
        return ("%d single SSP-RK3 steps of %s (%d leaves), plus one adaptation timed after them and "
                "charged once per %d steps" % (self.steps, self.what, self.o.M, self.ae))


def _cpu_baseline(cfg, budget_s=15.0):
    """The oracle as it stands, single-threaded, on a bounded sample of the workload (about
    budget_s of CPU time)."""
    ot = OracleTimer(cfg, WORKLOAD)
    t0 = time.perf_counter()
    while True:
        ot.one()
        if time.perf_counter() - t0 > budget_s:
            break
    value, t = ot.finish()
    return {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
            "host_cpu": host_cpu(), "threads": 1,
            "sample": "%s, %.1f s charged" % (ot.sample_text(), t)}


def _config_line(cfg):
    from paper_2306_06744_gb300 import workloads as W
    base = W.config(WORKLOAD)
    name = WORKLOAD if cfg["Dmax"] == base["Dmax"] else "%s (Dmax %d)" % (WORKLOAD, cfg["Dmax"])
    return {"workload": name, "dim": cfg["dim"], "p": cfg["p"],
            "domain": "[0,%g]^%d" % (cfg["L"], cfg["dim"]), "Dbase": cfg["Dbase"], "Dmax": cfg["Dmax"],
            "adapt_every": cfg["adapt_every"], "time_steps_per_step": cfg["adapt_every"],
            "indicator": "density gradient %g/%g" % (cfg["th_refine"], cfg["th_coarsen"]),
            # the same keys and values in both arms (the reference arm's sample is in cpu_baseline)
            "l2": "inputs larger than L2; the GPU arm also flushes L2 between steps (512 MB write)",
            "parallelism": "replicas" if int(os.environ.get("WORLD_SIZE", "1")) > 1 else "one device"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2306_06744_gb300 import workloads as W
    cfg = W.config(WORKLOAD)
    ot = OracleTimer(cfg, WORKLOAD)
    for _ in range(args.warmup):
        ot.one(timed=False)
    # each bench step is one bounded sample of the workload (OracleTimer.one); the run stops early
    # once REF_BUDGET_S of CPU time is spent, so it ends within a few minutes, and the rate is
    # that of the samples done
    done = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ot.one()
        done += 1
        if time.perf_counter() - t0 > REF_BUDGET_S:
            break
    value, t = ot.finish()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / done,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": _config_line(cfg),
            "adaptation_pct": 100.0 * ot.t_adapt / t if t else None,
            "point_updates_per_s": value / ot.nv,
            "l2_rho": ot.o.norms()["l2_rho"], "M_final": ot.o.M,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "threads": 1, "kind": "oracle",
                             "host_cpu": host_cpu(),
                             "sample": "%d of %d steps after %d warm-up steps: %s, %.1f s charged" %
                                       (done, args.steps, args.warmup, ot.sample_text(), t)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_tree(args):
    """Tree completion from a point cloud and 2:1 balance (the paper's meshing benchmark, Sec. 5.1;
    a seeded torus surface stands in for its scanned model): wall time of each library call,
    including the host copies of its input and result, best of 3 after a warm-up; the oracle's
    times on the same points are the CPU baseline, and the outputs are compared bit for bit."""
    import numpy as np
    import torch
    import oracle as O
    from paper_2306_06744_gb300 import fr
    from paper_2306_06744_gb300 import workloads as W

    def best(f, reps=3):
        r = f()
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            a = time.perf_counter()
            r = f()
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - a)
        return r, min(ts)

    for Dmin, Dmax, n in ((4, 9, 600_000), (4, 10, 2_000_000)):
        pts = W.torus_points(n, 11)
        keys, t_c = best(lambda: fr.tree_complete(3, Dmin, Dmax, 1.0, pts))
        bal, t_b = best(lambda: fr.tree_balance(3, Dmax, keys))
        line = {"metric": "tree completion + 2:1 balance wall time", "mode": "tree",
                "value": 1e3 * (t_c + t_b), "unit": "ms", "higher_is_better": False,
                "complete_ms": 1e3 * t_c, "balance_ms": 1e3 * t_b,
                "ns_per_balanced_leaf": 1e9 * t_b / len(bal),
                "config": {"workload": "torus surface points, seed 11", "dim": 3, "points": n,
                           "Dmin": Dmin, "Dmax": Dmax, "completed_leaves": int(len(keys)),
                           "balanced_leaves": int(len(bal))}}
        if not args.no_cpu_baseline:
            a = time.perf_counter()
            okeys = O.tree_complete(3, Dmin, Dmax, 1.0, pts)
            b = time.perf_counter()
            obal = O.balance(3, Dmax, okeys)
            c = time.perf_counter()
            line["cpu_baseline"] = {"value": 1e3 * (c - a), "unit": "ms", "cores": 1, "kind": "oracle",
                                    "complete_ms": 1e3 * (b - a), "balance_ms": 1e3 * (c - b),
                                    "sample": "the same points, once"}
            line["bit_exact"] = bool(np.array_equal(keys, okeys) and np.array_equal(bal, obal))
        print(json.dumps(line), flush=True)
    return 0


def aggregate_ranks(units, seconds, device="cuda"):
    """Whole-job throughput inputs over the ranks of a replica run: the units every rank
    processed, summed, and the slowest rank's time (one rank: unchanged)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(units), float(seconds)
    a = torch.tensor([float(units)], dtype=torch.float64, device=device)
    b = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(a, op=dist.ReduceOp.SUM)
    dist.all_reduce(b, op=dist.ReduceOp.MAX)
    return float(a.item()), float(b.item())


def _kernel_source_hash():
    """Hash of the element-stage kernel's source text (the k_stage_t definition)."""
    import hashlib
    src = open(os.path.join(ROOT, "paper_2306_06744_gb300", "csrc", "fr_kernels.cuh")).read()
    a = src.index("k_stage_t(StageArgs")
    b = src.index("// ---- per-precision launch bodies")
    return hashlib.sha256(src[a:b].encode()).hexdigest()[:16]


def _traffic_from_profiles(kernel):
    """Per-launch DRAM bytes of `kernel` recorded in profiles/ (a `bench-key:` line), if the
    recorded source hash still matches the kernel's source (otherwise the counters are stale)."""
    h = _kernel_source_hash()
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return None
    for fn in sorted(os.listdir(pdir)):
        if not fn.endswith(".md"):
            continue
        for line in open(os.path.join(pdir, fn)):
            parts = line.split()
            if len(parts) >= 5 and parts[0] == "bench-key:" and parts[1] == kernel and parts[3] == h:
                try:
                    return {"bytes": float(parts[2]), "points": float(parts[4])}
                except ValueError:
                    return None
    return None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=6)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-forms", action="store_true")
    from paper_2306_06744_gb300 import workloads as W
    ap.add_argument("--tree", action="store_true",
                    help="instead: tree completion + 2:1 balance of a 3D point cloud, with the oracle beside it")
    ap.add_argument("--workload", default=WORKLOAD, choices=list(W.CONFIG_NAMES),
                    help="configuration to measure (default: the four 3D p=3 vortex tubes, the largest "
                         "configuration that fits one GPU)")
    ap.add_argument("--dmax", type=int, default=0,
                    help="override the maximum depth (smaller meshes of the same workload, e.g. for "
                         "profiler captures); the line then names the changed depth")
    args = ap.parse_args()
    globals()["WORKLOAD"] = args.workload
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.tree:
        return run_tree(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2306_06744_gb300 import fr
    from paper_2306_06744_gb300 import workloads as W

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    cfg = W.config(WORKLOAD)
    if args.dmax:
        cfg["Dmax"] = args.dmax
    dim, p = cfg["dim"], cfg["p"]
    N, nv = (p + 1) ** dim, dim + 2
    ae = cfg["adapt_every"]
    stream = torch.cuda.current_stream()
    mesh = fr.Mesh(cfg, stream=stream)
    for _ in range(args.warmup):
        mesh.step(ae)
        mesh.adapt()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
            torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    Ms = []
    clk_path = os.path.join(tempfile.gettempdir(), "fr_bench_clocks_%d.csv" % os.getpid())
    proc, fh = _clock_sampler_start(clk_path)
    time.sleep(0.3)
    # per-kernel CUDA events on every 5th stage of the timed region (a recorded event costs the
    # stream a few microseconds; sampling keeps that under 2% of the step time)
    mesh.profile_enable(True, stride=5)
    launches0 = fr.kernel_launches()
    barrier()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))
        Ms.append(mesh.M)
        e0, e1, e2 = evs[k]
        e0.record(stream)
        mesh.step(ae)
        e1.record(stream)
        mesh.adapt()
        e2.record(stream)
    barrier()
    wall = time.perf_counter() - wall0
    launches = fr.kernel_launches() - launches0
    prof = mesh.profile_read()
    mesh.profile_enable(False)
    clocks = _clock_sampler_stop(proc, fh, clk_path, local)
    t_step = sum(a.elapsed_time(b) for a, b, _ in evs) / 1e3
    t_adapt = sum(b.elapsed_time(c) for _, b, c in evs) / 1e3
    t_tot = t_step + t_adapt
    dof_rank = sum(ae * m * N * nv for m in Ms)
    dof_all, t_tot = aggregate_ranks(dof_rank, t_tot)
    value = dof_all / t_tot
    norms = mesh.norms()  # state, time and leaf count at the end of the timed cycles
    M_final = mesh.M

    # element-kernel roofline (FP64: bound by the FP64 pipe)
    st_s = prof["stage_ms"] / 1e3
    stage_avg_ms = prof["stage_ms"] / max(1, prof["stage_launches"])
    n_stage = 3 * ae * args.steps  # element (and interface) kernel launches in the timed region
    flops = prof["stage_points"] * flops_per_point_stage(dim, p)
    nbytes = prof["stage_points"] * bytes_per_point_stage(dim, p)
    achieved_tflops = flops / st_s / 1e12
    achieved_gbs = nbytes / st_s / 1e9
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    kname = "k_stage<%d,%d>" % (dim, p + 1)
    tr = _traffic_from_profiles(kname)
    # DRAM bytes per launch from the ncu capture of this kernel instance, scaled to this run's
    # mean launch size
    traffic = (tr["bytes"] * (prof["stage_points"] / max(1, prof["stage_launches"])) / tr["points"]
               if tr else None)
    roofline = {"kernel": kname + " (element stage)", "bound": "alu",
                "flop_per_point": flops_per_point_stage(dim, p),
                "bytes_per_point": bytes_per_point_stage(dim, p),
                "points_per_launch": prof["stage_points"] / max(1, prof["stage_launches"]),
                "achieved": achieved_tflops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved_tflops / FP64_PEAK_TFLOPS, "traffic": traffic,
                "peak_source": "FP64 pipe: 152 SMs x 2 DFMA/clk x 2.07 GHz (recipe unit counts "
                               "and clocks)",
                "avg_launch_ms": stage_avg_ms,
                "hbm": {"achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                        "frac": achieved_gbs / hbm_peak, "peak_source": "measured" if peaks else "fallback"},
                "share_of_step_time": stage_avg_ms * n_stage / (1e3 * t_step) if t_step else None,
                "face_kernel_share": (prof["face_ms"] / max(1, prof["face_launches"])) * n_stage /
                                     (1e3 * t_step) if t_step else None,
                "timed_launches_sampled": "every 5th stage"}

    # end-to-end through the public API with host buffers
    e2e = None
    if args.e2e_steps > 0:
        # pinned host buffers for the step's inputs and its result, sized with room for growth
        cap = mesh.M + mesh.M // 4 + 1024
        kin = torch.empty(cap, dtype=torch.int64).pin_memory().numpy().view(np.uint64)
        uin = torch.empty(cap * nv * N, dtype=torch.float64).pin_memory().numpy()
        kout = torch.empty(cap, dtype=torch.int64).pin_memory().numpy().view(np.uint64)
        uout = torch.empty(cap * nv * N, dtype=torch.float64).pin_memory().numpy()
        keys_h = None
        dof_e, t_e, bi, bo = 0, 0.0, 0, 0
        e2e_warm = 2  # untimed passes: the first DMA transfers from fresh pinned buffers can be slow
        for k in range(args.e2e_steps + e2e_warm):
            if mesh.M > cap:  # the inputs must fit the pinned buffers: grow them (untimed)
                cap = mesh.M + mesh.M // 4 + 1024
                kin = torch.empty(cap, dtype=torch.int64).pin_memory().numpy().view(np.uint64)
                uin = torch.empty(cap * nv * N, dtype=torch.float64).pin_memory().numpy()
                kout = torch.empty(cap, dtype=torch.int64).pin_memory().numpy().view(np.uint64)
                uout = torch.empty(cap * nv * N, dtype=torch.float64).pin_memory().numpy()
            kn = mesh.leaves(out=kin)
            un_ = mesh.state(out=uin)
            torch.cuda.synchronize()
            flush.fill_(float(k))
            torch.cuda.synchronize()
            a = time.perf_counter()
            mesh.set_state(kn, un_)
            M0 = mesh.M
            mesh.step(ae)
            mesh.adapt()
            fits = mesh.M <= cap  # else (a mesh grown past the headroom) pageable arrays
            k2 = mesh.leaves(out=kout if fits else None)
            u2 = mesh.state(out=uout if fits else None)
            b = time.perf_counter()
            if k < e2e_warm:
                continue
            dof_e += ae * M0 * N * nv
            t_e += b - a
            bi += kn.nbytes + un_.nbytes
            bo += k2.nbytes + u2.nbytes
        dof_e, t_e = aggregate_ranks(dof_e, t_e)
        e2e = {"value": dof_e / t_e, "unit": UNIT,
               "h2d_bytes_per_step": bi // args.e2e_steps, "d2h_bytes_per_step": bo // args.e2e_steps,
               "steps": args.e2e_steps, "warmup": e2e_warm}
        del keys_h

    # the other arithmetic forms of the time-step kernels on the same workload and cycles:
    # same simulated time, so time_to_solution compares forms at their own vortex L2 error
    forms = {"f64": {"value": value, "l2_rho": norms["l2_rho"], "time_to_solution_s": t_tot,
                     "adaptation_pct": 100.0 * t_adapt / (t_step + t_adapt), "M_final": M_final,
                     "stage_kernel_avg_ms": stage_avg_ms}}
    # the FP64 mesh is not needed any more: its ~67 GB (largest workload) go back to the cache
    mesh.close()
    if not args.no_forms:
        forms_run = [(1, "f32_mixed_f64_rk"), (4, "f64x2f32_double_word")]
        if (dim, p) == (3, 3):  # the tensor-core operator forms are built for 3D p = 3
            forms_run[1:1] = [(2, "tf32_tensor_core_f64_rk"), (3, "bf16x3_tensor_core_f64_rk")]
        for prec, name in forms_run:
            fm = fr.Mesh(dict(cfg, precision=prec), stream=stream)
            for _ in range(args.warmup):
                fm.step(ae)
                fm.adapt()
            fev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
                    torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
            fMs = []
            fm.profile_enable(True, stride=5)
            for k in range(args.steps):
                flush.fill_(float(k))
                fMs.append(fm.M)
                a, b, c = fev[k]
                a.record(stream)
                fm.step(ae)
                b.record(stream)
                fm.adapt()
                c.record(stream)
            torch.cuda.synchronize()
            fp = fm.profile_read()
            fs = sum(a.elapsed_time(b) for a, b, _ in fev) / 1e3
            fa = sum(b.elapsed_time(c) for _, b, c in fev) / 1e3
            fn = fm.norms()
            fM = fm.M
            fdof, ft = aggregate_ranks(sum(ae * m * N * nv for m in fMs), fs + fa)
            dl2 = abs(fn["l2_rho"] - norms["l2_rho"]) / norms["l2_rho"]
            dM = abs(fM - M_final) / M_final
            forms[name] = {"value": fdof / ft,
                           "l2_rho": fn["l2_rho"], "time_to_solution_s": fs + fa,
                           "speedup_vs_f64": t_tot / (fs + fa),
                           "adaptation_pct": 100.0 * fa / (fs + fa), "M_final": fM,
                           "stage_kernel_avg_ms": fp["stage_ms"] / max(1, fp["stage_launches"]),
                           "l2_rel_diff_vs_f64": dl2, "M_rel_diff_vs_f64": dM,
                           # same vortex L2 error (within 5%) on the same mesh (leaf count within
                           # 5%): only then is time_to_solution a like-for-like comparison
                           "same_solution_as_f64": bool(dl2 <= 0.05 and dM <= 0.05)}
            if not forms[name]["same_solution_as_f64"]:
                forms[name]["mesh_diverged"] = True
            fm.close()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = _cpu_baseline(cfg)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": _config_line(cfg),
            "adaptation_pct": 100.0 * t_adapt / (t_step + t_adapt),
            # solution-point updates per second (DOF-updates / conserved variables), the unit of
            # the paper's throughput figures
            "point_updates_per_s": value / nv,
            "l2_rho": norms["l2_rho"], "t_final": norms["t"], "M_final": M_final,
            "M_mean": sum(Ms) / len(Ms), "wall_s": wall,
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "forms": forms,
            "gpu_launches": launches}
    if rank == 0:
        print(json.dumps(line))
    mesh.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
