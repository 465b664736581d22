"""Benchmark of the hot path: composite geometric-multigrid solves of the fourth-order
finite-volume elliptic systems on a two-level 2-D AMR hierarchy.

Workload ``bumps2d``: base 256^2 on the unit square, one ratio-2 box over [0.25,0.75]^2
(256^2 fine cells), right-hand side = exact cell averages of a seeded sum of 8 Gaussian
bumps.  One step = one pass of the whole hot path: the pure-Neumann pressure Poisson
equation (solvability fix, V-cycles to ||r||_inf <= 1e-10 ||f||_inf, mean-zero) and the
viscous Helmholtz system (alpha = 1, beta = -gamma nu k, gamma = 0.25, nu = 1e-3,
k = 1/256, Dirichlet) solved to the same tolerance.  Metric: V-cycle DOF/s = valid cells
x V-cycles / time, summed over both systems and all ranks.

``python bench.py [--gpus N --steps K --warmup W]``        this library (GB300)
``python bench.py --impl reference ...``                    the CPU oracle on host cores
Under torchrun (N > 1) every rank solves its own replica (the solve does not shard:
replicas only) and rank 0 prints one JSON line.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "V-cycle DOF/s & time-to-1e-10 residual; HBM GB/s vs 8 TB/s; mixed vs FP64"
UNIT = "DOF*V-cycles/s"
WORKLOAD = ("bumps2d: 2-D two-level AMR, base 256^2 on [0,1]^2 + ratio-2 box [0.25,0.75]^2 "
            "(256^2 fine cells), RHS = cell averages of 8 seeded Gaussian bumps; per step: pure-Neumann "
            "PPE + Helmholtz (gamma=0.25, nu=1e-3, k=1/256, Dirichlet), each to ||r||_inf <= 1e-10 ||f||_inf")
RTOL = 1e-10


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="host-driven V-cycle loop instead of the captured solve")
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64 comparison and the large-grid roofline")
    ap.add_argument("--no-3d", action="store_true", help="skip the 3-D workload in the extras")
    ap.add_argument("--profile-case", choices=["none", "large", "bench", "single3d", "bumps3d"], default="none",
                    help="large: one mixed-precision solve of the single-level 4096^2 case; bench: one warm-up "
                         "and one timed step of the bench workload and nothing else; single3d: two mixed-precision "
                         "V-cycles of a single-level 256^3 Helmholtz problem; bumps3d: the mixed-precision PPE and "
                         "one Helmholtz solve of the 3-D workload, host-driven loop (all for ncu)")
    return ap.parse_args()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _workload():
    from paper_2506_02663_gb300 import workloads as wl
    dim, n0, boxes, rhs = wl.bumps2d_rhs()
    systems = [("ppe", [1, 1, 1, 1], 0.0, 1.0), ("helmholtz", [0, 0, 0, 0], 1.0, wl.HELMHOLTZ_BETA)]
    return dim, n0, boxes, rhs, systems


def valid_dof(n0, boxes):
    """Valid cells of a two-level hierarchy: level-0 cells minus the coarsened level-1
    boxes, plus every level-1 cell (top level has no invalid region)."""
    D = len(n0)
    n = 1
    for v in n0:
        n *= v
    fine = 0
    cover = 0
    for lo, hi in boxes[1]:
        c = 1
        for d in range(D):
            c *= hi[d] - lo[d] + 1
        fine += c
        cover += c // 2 ** D
    return n - cover + fine


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.device)], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _kernel_source_hash():
    h = hashlib.sha256()
    for f in ("kernels.cuh", "solver.cu"):
        with open(os.path.join(ROOT, "paper_2506_02663_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic(kernel_class_name):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the current
    kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        e = d.get(kernel_class_name)
        if e and e.get("source_hash") == _kernel_source_hash():
            return e.get("dram_bytes_per_launch")
    except Exception:
        pass
    return None


# ============================================================================ oracle arm
def _oracle_vcycles(seconds, max_cycles=None):
    """Time oracle V-cycles (PPE and Helmholtz alternately, setup excluded) on the full
    workload for about ``seconds``; returns (DOF*V-cycles per second, cycles, seconds)."""
    import numpy as np
    from oracle import composite as cp, mg, solve as so
    from oracle.hierarchy import Hierarchy as OH
    dim, n0, boxes, rhs, systems = _workload()
    dof = valid_dof(n0, boxes)
    runs = []
    for name, bc, alpha, beta in systems:
        H = OH(dim, n0, boxes, bc=bc)
        F = cp.new_field(H)
        for l, lev in enumerate(H.levels):
            for k, (lo, hi) in enumerate(lev.boxes):
                F[l][lev.box_slice(lo, hi)] = rhs[l][k]
        if so.is_pure_neumann(H, alpha):
            F, _ = so.solvability_fix(H, F)
        runs.append((H, mg.CompositeMG(H, alpha, beta), F))
    phis = [cp.new_field(H) for H, _, _ in runs]
    cycles = 0
    t0 = time.perf_counter()
    while True:
        for i, (H, m, F) in enumerate(runs):
            phis[i] = m.vcycle(phis[i], F)
            cycles += 1
        el = time.perf_counter() - t0
        if el >= seconds or (max_cycles and cycles >= max_cycles):
            break
    return dof * cycles / el, cycles, el


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    # each step: one oracle V-cycle of each system on the full workload
    vals = []
    for _ in range(args.warmup):
        _oracle_vcycles(0.0, max_cycles=2)
    t_all = 0.0
    dofv = 0.0
    for _ in range(args.steps):
        v, c, el = _oracle_vcycles(0.0, max_cycles=2)
        vals.append(v)
        t_all += el
        dofv += v * el
    value = dofv / t_all
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_all / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "arm": "FP64 numpy oracle, one V-cycle per system per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} steps x (1 PPE + 1 Helmholtz oracle V-cycle) on the full workload, setup excluded"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ============================================================================ our arm
def aggregate(total_ms, dofv_rank, ws, dist=None, device="cpu"):
    """Whole-job figures of a replicas run: the slowest rank's device time (max over ranks)
    and value = ws x this rank's DOF x V-cycles / that time (every rank solves the same
    workload).  ``dist`` is torch.distributed (initialised) or None for one process."""
    import torch
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    tmax = float(t.item())
    return tmax, ws * dofv_rank / (tmax * 1e-3)


def run_ours(args):
    import numpy as np
    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2506_02663_gb300 import amr
    dim, n0, boxes, rhs, systems = _workload()
    dof = valid_dof(n0, boxes)
    gh = amr.Hierarchy(dim, n0, boxes)
    f_host = gh.pack(rhs)
    f = torch.from_numpy(f_host).cuda()
    ops = [amr.Operator(gh, a, b, bc) for _, bc, a, b in systems]
    phis = [torch.zeros_like(f) for _ in systems]
    prec = amr.MIXED if args.precision == "mixed" else amr.FP64
    graph = 0 if args.no_graph else 1
    params = amr.default_params(rtol=RTOL, max_vcycles=100, precision=prec, use_graph=graph)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2
    stream = torch.cuda.current_stream()

    def step(p):
        vc = []
        ps = p if isinstance(p, list) else [p] * len(ops)
        for op, phi, pi in zip(ops, phis, ps):
            st = op.solve(phi, f, params=pi, allow_not_converged=isinstance(p, list))
            vc.append(st["vcycles"])
        return vc

    def timed(p, k):
        ts, vcs = [], []
        for _ in range(k):
            flush.fill_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            vcs.append(step(p))
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return ts, vcs

    for _ in range(args.warmup):
        step(params)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    l0 = amr.kernel_launches()
    ts, vcs = timed(params, args.steps)
    launches = amr.kernel_launches() - l0
    torch.cuda.synchronize()
    clocks = sampler.stop()
    if dist:
        dist.barrier()
    dofv_rank = sum(dof * sum(v) for v in vcs)
    tmax, value = aggregate(sum(ts), dofv_rank, ws, dist, "cuda")
    vc_per_system = [statistics.mean(v[i] for v in vcs) for i in range(len(systems))]

    # ---------------- end to end through the C ABI with host buffers
    import torch as _t
    fh = _t.from_numpy(f_host).pin_memory().numpy()
    ph = _t.zeros(gh.nelems, dtype=_t.float64).pin_memory().numpy()
    e2e_v = 0
    for op in ops:
        op.solve_host(ph, fh, params=params)
    torch.cuda.synchronize()
    te = time.perf_counter()
    for _ in range(args.steps):
        for op in ops:
            st = op.solve_host(ph, fh, params=params)
            e2e_v += st["vcycles"]
    te = time.perf_counter() - te
    e2e = {"value": ws * dof * e2e_v / te if te > 0 else None, "unit": UNIT,
           "h2d_bytes_per_step": len(systems) * gh.nelems * 8, "d2h_bytes_per_step": len(systems) * gh.nelems * 8,
           "ms_per_step": 1e3 * te / args.steps}

    # ---------------- roofline of the dominant kernel (weighted-Jacobi sweeps), live
    peak, peak_kind = _peaks()
    # instrumented pass: the same solves on the host-driven loop with CUDA events around
    # every instrumented launch; the library keeps the GPU busy briefly before each V-cycle
    # so the launches are queued ahead and the event intervals hold kernel time only
    prof_params = amr.default_params(rtol=RTOL, max_vcycles=100, precision=prec, use_graph=0)
    amr.profile_enable(True)
    timed(prof_params, max(1, min(args.steps, 5)))
    amr.profile_enable(False)
    classes = _class_table(amr)
    dom = _dominant(classes)
    roofline = _roofline_entry(classes, dom, peak, peak_kind, "bumps2d")
    others = {k: {"launches": v["launches"], "ms": v["ms"]} for k, v in classes.items() if k != dom}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tmax / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 V-cycles in f64 refinement" if prec == amr.MIXED else "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "dof_per_system": dof, "systems": [s[0] for s in systems],
                   "precision": args.precision, "rtol": RTOL, "vcycles_per_system": vc_per_system,
                   "l2": "flushed (256 MB write) before every timed step; the working set fits in L2",
                   "solve": "one captured CUDA graph per solve (device-side while loop over V-cycles)" if graph
                   else "host-driven V-cycle loop",
                   "parallelism": f"replicas x{ws}"},
        "gpu_launches": launches,
        "clocks": clocks,
        "e2e": e2e,
        "roofline": roofline,
        "kernel_classes_ms": others,
    }

    if not args.no_extras and rank == 0:
        p64 = amr.default_params(rtol=RTOL, max_vcycles=100, precision=amr.FP64 if prec == amr.MIXED else amr.MIXED,
                                 use_graph=graph)
        step(p64)
        ts2, vcs2 = timed(p64, args.steps)
        v2 = dof * sum(sum(v) for v in vcs2) / (sum(ts2) * 1e-3)
        key = "fp64" if prec == amr.MIXED else "mixed"
        line[key] = {"value": v2, "ms_per_step": sum(ts2) / args.steps,
                     "vcycles_per_system": [statistics.mean(v[i] for v in vcs2) for i in range(len(systems))]}
        line["large_grid_roofline"] = _large_grid_roofline(amr, torch, peak, peak_kind)
        line["batch"] = _batch_measure(amr, torch)
        line["adjoint"] = _adjoint_measure(amr, torch)
        if not args.no_3d:
            line["bumps3d"] = _bumps3d_measure(amr, torch, peak, peak_kind)

    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        v, c, el = _oracle_vcycles(12.0)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{c} FP64 numpy-oracle V-cycles (PPE and Helmholtz alternating) on the full "
                                          f"workload in {el:.1f} s, setup excluded; numpy element-wise ops use one core"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


KERNEL_CLASSES = {
    "jacobi": ("KC_JACOBI", "k_level_op2d_tiled<float,JACOBI> / k_level_op<float,*,JACOBI>: one weighted-Jacobi sweep"),
    "residual": ("KC_RESID", "k_level_op*<*,RESID/APPLY>: level residual or operator"),
    "restrict": ("KC_RESTRICT", "k_restrict2d_resid / k_restrict: residual restriction and average-down"),
    "prolong": ("KC_PROLONG", "k_prolong2d / k_prolong: linear prolongation + correction"),
    "down_leg": ("KC_DOWN", "k_mg_down2d<float>: nu1 sweeps + residual + restriction, one launch per grid"),
    "up_leg": ("KC_UP", "k_mg_up2d<float>: prolongation + nu2 sweeps, one launch per grid"),
    "coarse_block": ("KC_COARSE", "k_mg_coarse2d<float>: the V-cycle on the grids <= 64^2, one block"),
}


def _class_table(amr):
    out = {}
    for name, (kc, _) in KERNEL_CLASSES.items():
        r = amr.profile_read(getattr(amr, kc))
        if r["launches"]:
            out[name] = r
    return out


def _dominant(classes):
    return max(classes, key=lambda k: classes[k]["ms"]) if classes else None


def _roofline_entry(classes, dom, peak, peak_kind, workload):
    if dom is None:
        return {"bound": "hbm", "achieved": None, "peak": peak, "unit": "GB/s", "frac": None, "traffic": None}
    c = classes[dom]
    achieved = c["bytes"] / (c["ms"] * 1e-3) / 1e9 if c["ms"] > 0 else None
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak if achieved else None,
            "traffic": _traffic(f"{dom}_{workload}"),
            "kernel": KERNEL_CLASSES[dom][1], "class": dom,
            "launches": c["launches"], "avg_launch_us": 1e3 * c["ms"] / max(c["launches"], 1),
            "bytes_per_launch": c["bytes"] / max(c["launches"], 1), "peak_source": f"{peak_kind} hbm_gbs",
            "share_of_instrumented_ms": c["ms"] / sum(v["ms"] for v in classes.values())}


def _batch_measure(amr, torch, reps=3):
    """The batch workload: 96 independent single-level Helmholtz problems of uneven sizes
    N in {64,...,512} (seeded), mixed precision to 1e-10, all solved by one amr_batch_solve
    call (concurrent captured solves); compared with the same solves one after another and
    with FP64 V-cycles."""
    from paper_2506_02663_gb300 import workloads as wl
    probs = wl.batch2d_problems()
    hs, ops, fs, phis = [], [], [], []
    dof = 0
    for pr in probs:
        n = pr["n"]
        gh = amr.Hierarchy(2, (n, n), [[((0, 0), (n - 1, n - 1))]])
        hs.append(gh)
        ops.append(amr.Operator(gh, pr["alpha"], pr["beta"], [0, 0, 0, 0]))
        fs.append(torch.from_numpy(gh.pack([[pr["rhs"]]])).cuda())
        phis.append(torch.zeros_like(fs[-1]))
        dof += n * n
    out = {"workload": "batch2d: 96 single-level 2-D Helmholtz problems, N in {64,96,128,192,256,384,512} (seeded), "
                       "alpha=1, beta=-0.25*nu/256, nu log-uniform [1e-4,1e-2], Fourier RHS |k|<=16",
           "dof": dof}
    stream = torch.cuda.current_stream()
    for name, prec in (("mixed", amr.MIXED), ("fp64", amr.FP64)):
        p = amr.default_params(rtol=RTOL, max_vcycles=100, precision=prec, use_graph=1)
        amr.batch_solve(ops, phis, fs, params=p)  # warm-up: captures every graph
        ts, vcs = [], []
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            st, status = amr.batch_solve(ops, phis, fs, params=p)
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
            vcs.append(sum(pr["n"] ** 2 * s["vcycles"] for pr, s in zip(probs, st)))
        out[name] = {"ms_per_batch": statistics.median(ts), "value": statistics.mean(vcs) / (statistics.median(ts) * 1e-3),
                     "unit": UNIT, "all_converged": all(x == 0 for x in status)}
    # one after another on one stream
    p = amr.default_params(rtol=RTOL, max_vcycles=100, precision=amr.MIXED, use_graph=1)
    for op, x, f in zip(ops, phis, fs):
        op.solve(x, f, params=p)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for op, x, f in zip(ops, phis, fs):
        op.solve(x, f, params=p)
    b.record(stream)
    b.synchronize()
    out["sequential_mixed_ms"] = a.elapsed_time(b)
    for op in ops:
        op.close()
    for gh in hs:
        gh.close()
    return out


def _large_grid_roofline(amr, torch, peak, peak_kind, n=4096):
    """The same kernels on a single-level n^2 Helmholtz solve (fields >> L2): the HBM
    efficiency of the smoothing kernels when they are not launch-bound."""
    from paper_2506_02663_gb300 import workloads as wl
    gh = amr.Hierarchy(2, (n, n), [[((0, 0), (n - 1, n - 1))]])
    op = amr.Operator(gh, 1.0, wl.HELMHOLTZ_BETA * 16.0, [0, 0, 0, 0])
    g = torch.Generator(device="cuda")
    g.manual_seed(1)
    f = torch.randn(gh.nelems, dtype=torch.float64, device="cuda", generator=g)
    phi = torch.zeros_like(f)
    p = amr.default_params(rtol=1e-10, max_vcycles=40, precision=amr.MIXED, use_graph=0)
    op.solve(phi, f, params=p)
    amr.profile_enable(True)
    st = op.solve(phi, f, params=p)
    amr.profile_enable(False)
    classes = _class_table(amr)
    dom = _dominant(classes)
    out = _roofline_entry(classes, dom, peak, peak_kind, f"single{n}")
    out["workload"] = f"single-level {n}^2 Helmholtz, mixed precision, {st['vcycles']} V-cycles"
    out["classes"] = {k: {"launches": v["launches"], "ms": v["ms"], "GB/s": v["bytes"] / (v["ms"] * 1e-3) / 1e9}
                      for k, v in classes.items()}
    op.close()
    gh.close()
    return out


def _bumps3d_measure(amr, torch, peak, peak_kind, reps=2):
    """The 3-D workload: base 256^3 on [0,1]^3 plus a ratio-2 box over [0.375,0.625]^3
    (128^3 fine cells); RHS = cell averages of seeded Gaussian bumps; one pure-Neumann PPE and
    three Helmholtz solves (gamma=0.25, nu=1e-3, k=1/256, Dirichlet) per step, mixed
    precision to 1e-10.  The three velocity components are one amr_batch_solve call (one
    hierarchy object per component, so that their captured graphs run concurrently); the same
    step with the components solved one after another is timed beside it.  The backward pass
    is the four adjoint solves (amr_solve_transpose, mixed precision, same tolerance).  The
    fields (about 150 MB each in FP64) are larger than L2."""
    from paper_2506_02663_gb300 import workloads as wl
    dim, n0, boxes, rhs = wl.bumps3d_rhs()
    gh = amr.Hierarchy(dim, n0, boxes)
    dof = valid_dof(n0, boxes)
    f = torch.from_numpy(gh.pack(rhs)).cuda()
    ppe = amr.Operator(gh, 0.0, 1.0, [1] * 6)
    ghc = [amr.Hierarchy(dim, n0, boxes) for _ in range(3)]
    helms = [amr.Operator(g, 1.0, wl.HELMHOLTZ_BETA, [0] * 6) for g in ghc]
    phis = [torch.zeros_like(f) for _ in range(4)]
    stream = torch.cuda.current_stream()
    out = {"workload": "bumps3d: 3-D two-level AMR, base 256^3 + ratio-2 box [0.375,0.625]^3 (128^3 fine cells), "
                       "Gaussian-bump RHS; per step: pure-Neumann PPE + 3 Helmholtz (gamma=0.25, nu=1e-3, k=1/256) "
                       "batched in one amr_batch_solve call, each to ||r||_inf <= 1e-10 ||f||_inf",
           "dof_per_system": dof}

    def time_step(fn):
        fn()
        ts, vcs = [], []
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            vcs.append(fn())
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts), vcs[-1]

    for name, prec in (("mixed", amr.MIXED), ("fp64", amr.FP64)):
        p = amr.default_params(rtol=RTOL, max_vcycles=100, precision=prec, use_graph=1)

        def step():
            vc = [ppe.solve(phis[0], f, params=p)["vcycles"]]
            st, status = amr.batch_solve(helms, phis[1:], [f] * 3, params=p)
            if any(status):
                raise RuntimeError(f"batched Helmholtz solves: statuses {status}")
            return vc + [s["vcycles"] for s in st]

        def step_sequential():
            vc = [ppe.solve(phis[0], f, params=p)["vcycles"]]
            for c in range(3):
                vc.append(helms[c].solve(phis[1 + c], f, params=p)["vcycles"])
            return vc
        ms, vc = time_step(step)
        out[name] = {"ms_per_step": ms, "vcycles_per_system": vc,
                     "value": dof * sum(vc) / (ms * 1e-3), "unit": UNIT}
        if name == "mixed":
            ms_seq, vc_seq = time_step(step_sequential)
            out[name]["components_one_after_another"] = {"ms_per_step": ms_seq, "vcycles_per_system": vc_seq}
    # backward: the adjoint solves of the step (host-driven refinement loop)
    pa = amr.default_params(rtol=RTOL, max_vcycles=100, precision=amr.MIXED, use_graph=0)
    lam = [torch.zeros_like(f) for _ in range(4)]

    def backward():
        vc = [ppe.solve_transpose(lam[0], f, params=pa)["vcycles"]]
        for c in range(3):
            vc.append(helms[c].solve_transpose(lam[1 + c], f, params=pa)["vcycles"])
        return vc
    try:
        ms_b, vc_b = time_step(backward)
        out["adjoint_mixed"] = {"ms_per_step": ms_b, "vcycles_per_system": vc_b,
                                "what": "A^T solves of the PPE (solvability-corrected solve map) and the three "
                                        "Helmholtz operators, right-hand side f, mixed precision to 1e-10"}
    except Exception as exc:  # reported, not fatal: the forward numbers stand on their own
        out["adjoint_mixed"] = {"error": str(exc)[:200]}
    helm = helms[0]
    # kernel classes of one instrumented mixed step (host-driven loop)
    pp = amr.default_params(rtol=RTOL, max_vcycles=100, precision=amr.MIXED, use_graph=0)
    amr.profile_enable(True)
    ppe.solve(phis[0], f, params=pp)
    helm.solve(phis[1], f, params=pp)
    amr.profile_enable(False)
    classes = _class_table(amr)
    dom = _dominant(classes)
    out["roofline"] = _roofline_entry(classes, dom, peak, peak_kind, "bumps3d")
    out["classes"] = {k: {"launches": v["launches"], "ms": v["ms"], "GB/s": v["bytes"] / (v["ms"] * 1e-3) / 1e9}
                      for k, v in classes.items()}
    ppe.close()
    for op in helms:
        op.close()
    for g in ghc:
        g.close()
    gh.close()
    return out


def _adjoint_measure(amr, torch, reps=3):
    """The adjoint2d workload (base 256^2, boxes [0.2,0.8]^2 -> 308^2 and [0.35,0.65]^2 ->
    308^2 fine cells, two smoothed N(0,1) forcing components): forward = two Helmholtz solves
    and the composite projection; backward = the projection's adjoint and two adjoint
    Helmholtz solves, FP64 to 1e-12 (the accuracy the finite-difference check needs)."""
    from paper_2506_02663_gb300 import workloads as wl
    dim, n0, boxes, comps = wl.adjoint2d_forcing()
    gh = amr.Hierarchy(dim, n0, boxes, h0=1.0 / n0[0])
    helm = amr.Operator(gh, 1.0, wl.HELMHOLTZ_BETA, [0] * 4)
    ppe = amr.Operator(gh, 0.0, 1.0, [1] * 4)
    p = amr.default_params(rtol=1e-12, max_vcycles=200, precision=amr.FP64, use_graph=1)
    g = [torch.from_numpy(gh.pack(comps[d])).cuda() for d in range(dim)]
    w = [torch.zeros_like(g[0]) for _ in range(dim)]
    u = [torch.zeros_like(g[0]) for _ in range(dim)]
    v = [torch.zeros_like(g[0]) for _ in range(dim)]
    lam = [torch.zeros_like(g[0]) for _ in range(dim)]
    phi = torch.zeros_like(g[0])
    psi = torch.zeros_like(g[0])
    stream = torch.cuda.current_stream()

    def forward():
        vc = 0
        for d in range(dim):
            vc += helm.solve(w[d], g[d], params=p)["vcycles"]
        vc += amr.project(ppe, [0] * 4, w, u, phi, params=p)["vcycles"]
        return vc

    def backward():
        vc = amr.project_transpose(ppe, [0] * 4, u, v, psi, params=p)["vcycles"]
        for d in range(dim):
            vc += helm.solve_transpose(lam[d], v[d], params=p)["vcycles"]
        return vc

    def timeit(fn):
        fn()
        ts, vcs = [], []
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            vcs.append(fn())
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts), vcs[-1]
    tf, vf = timeit(forward)
    tb, vb = timeit(backward)
    ppe.close()
    helm.close()
    gh.close()
    return {"workload": "adjoint2d: three-level 2-D AMR (256^2 base, 308^2 + 308^2 fine), two components; "
                        "forward = 2 Helmholtz solves + composite projection, backward = adjoint projection + "
                        "2 adjoint Helmholtz solves, FP64 to 1e-12",
            "forward_ms": tf, "backward_ms": tb, "backward_over_forward": tb / tf,
            "vcycles_forward": vf, "vcycles_backward": vb}


def _profile_case():
    import torch
    from paper_2506_02663_gb300 import amr
    from paper_2506_02663_gb300 import workloads as wl
    n = 4096
    gh = amr.Hierarchy(2, (n, n), [[((0, 0), (n - 1, n - 1))]])
    op = amr.Operator(gh, 1.0, wl.HELMHOLTZ_BETA * 16.0, [0, 0, 0, 0])
    f = torch.ones(gh.nelems, dtype=torch.float64, device="cuda")
    phi = torch.zeros_like(f)
    # host-driven loop: kernels inside a graph's conditional body cannot be profiled; the
    # second solve inside the "measured" range
    p = amr.default_params(rtol=1e-10, max_vcycles=40, precision=amr.MIXED, use_graph=0)
    op.solve(phi, f, params=p)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("measured")
    st = op.solve(torch.zeros_like(f), f, params=p)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"profile_case": "large", "vcycles": st["vcycles"], "final_res": st["final_res"]}))
    return 0


def _profile_single3d(n=256):
    """Two mixed-precision V-cycles (host-driven loop) of a single-level n^3 Helmholtz problem
    with homogeneous Dirichlet data: the 3-D level-operator kernels on a grid whose fields
    exceed L2 (67 MB per FP32 field at 256^3)."""
    import torch
    from paper_2506_02663_gb300 import amr
    from paper_2506_02663_gb300 import workloads as wl
    gh = amr.Hierarchy(3, (n, n, n), [[((0, 0, 0), (n - 1, n - 1, n - 1))]])
    op = amr.Operator(gh, 1.0, wl.HELMHOLTZ_BETA, [0] * 6)
    f = torch.ones(gh.nelems, dtype=torch.float64, device="cuda")
    phi = torch.zeros_like(f)
    st = op.solve(phi, f, params=amr.default_params(rtol=1e-30, max_vcycles=2, precision=amr.MIXED, use_graph=0),
                  allow_not_converged=True)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": "single3d", "vcycles": st["vcycles"], "final_res": st["final_res"]}))
    return 0


def _profile_bumps3d():
    """The 3-D workload's instrumented pass (PPE + one Helmholtz solve, mixed precision, host-
    driven loop), for per-launch DRAM traffic of its kernel classes."""
    import torch
    from paper_2506_02663_gb300 import amr
    from paper_2506_02663_gb300 import workloads as wl
    dim, n0, boxes, rhs = wl.bumps3d_rhs()
    gh = amr.Hierarchy(dim, n0, boxes)
    f = torch.from_numpy(gh.pack(rhs)).cuda()
    pp = amr.default_params(rtol=RTOL, max_vcycles=100, precision=amr.MIXED, use_graph=0)
    ops = [amr.Operator(gh, a, b, bc) for bc, a, b in (([1] * 6, 0.0, 1.0), ([0] * 6, 1.0, wl.HELMHOLTZ_BETA))]
    for op in ops:  # warm-up: scratch set-up and tile autotuning stay outside the measured range
        op.solve(torch.zeros_like(f), f, params=pp)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("measured")
    vc = [op.solve(torch.zeros_like(f), f, params=pp)["vcycles"] for op in ops]
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"profile_case": "bumps3d", "vcycles": vc}))
    return 0


def _profile_bench(args):
    """One warm-up step and one step of the bench workload (graph mode), for launch lists."""
    import torch
    from paper_2506_02663_gb300 import amr
    dim, n0, boxes, rhs, systems = _workload()
    gh = amr.Hierarchy(dim, n0, boxes)
    f = torch.from_numpy(gh.pack(rhs)).cuda()
    ops = [amr.Operator(gh, a, b, bc) for _, bc, a, b in systems]
    prec = amr.MIXED if args.precision == "mixed" else amr.FP64
    p = amr.default_params(rtol=RTOL, max_vcycles=100, precision=prec, use_graph=0 if args.no_graph else 1)
    for it in range(2):  # the second step inside the "measured" range
        if it == 1:
            torch.cuda.nvtx.range_push("measured")
        l0 = amr.kernel_launches()
        vc = [op.solve(torch.zeros_like(f), f, params=p)["vcycles"] for op in ops]
        torch.cuda.synchronize()
        if it == 1:
            torch.cuda.nvtx.range_pop()
        print(json.dumps({"profile_case": "bench", "vcycles": vc, "launches": amr.kernel_launches() - l0}))
    return 0


def main():
    args = _args()
    if args.profile_case == "large":
        return _profile_case()
    if args.profile_case == "bench":
        return _profile_bench(args)
    if args.profile_case == "single3d":
        return _profile_single3d()
    if args.profile_case == "bumps3d":
        return _profile_bumps3d()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
