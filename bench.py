"""Benchmark of the hot path: composite geometric-multigrid solves of the fourth-order
finite-volume elliptic systems on a two-level 3-D AMR hierarchy.

Workload ``bumps3d``: base 256^3 on the unit cube, one ratio-2 box over [0.375,0.625]^3
(128^3 fine cells); right-hand sides = exact cell averages of seeded sums of 8 Gaussian
bumps, one independent set per system.  One step = one pass of the whole hot path: the
pure-Neumann pressure Poisson equation (solvability fix, V-cycles to ||r||_inf <= 1e-10
||f||_inf, mean-zero) and the viscous Helmholtz systems of the three velocity components
(alpha = 1, beta = -gamma nu k, gamma = 0.25, nu = 1e-3, k = 1/256, Dirichlet), the three
batched in one amr_batch_solve call, each to the same tolerance; FP32 V-cycles inside FP64
iterative refinement.  Metric: V-cycle DOF/s = valid cells x V-cycles / time, summed over
the four systems and all ranks; ms_per_step is the time to the 1e-10 residual of all four.

Besides the line's headline keys, rank 0 reports (unless --no-extras) the step in the other
precision, the mixed-against-FP64 and stored-oracle errors, the adjoint of the 3-D step,
the interface conditions of a subcycled level solve on the 3-D workload's refined level
(``cic3d``: CF ghosts at t* from four coarse times and the corrected interface face
averages, against the FP64 rate), the regridding clustering on the host (``regrid3d``) and
the 2-D workloads.

``python bench.py [--gpus N --steps K --warmup W]``        this library (GB300)
``python bench.py --impl reference ...``                    the CPU oracle on the host cores
Under torchrun (N > 1) every rank solves its own replica (the solve does not shard:
replicas only) and rank 0 prints one JSON line.
"""
import argparse
import hashlib
import json
import math
import multiprocessing as mp
import os
import platform
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
WORKLOAD = ("bumps3d: 3-D two-level AMR, base 256^3 on [0,1]^3 + ratio-2 box [0.375,0.625]^3 (128^3 fine "
            "cells); per step: pure-Neumann PPE + Helmholtz systems of 3 velocity components (gamma=0.25, "
            "nu=1e-3, k=1/256, Dirichlet) batched in one call, RHS = cell averages of seeded Gaussian-bump "
            "sums (one set per system), each to ||r||_inf <= 1e-10 ||f||_inf")
RTOL = 1e-10
# FP32 correction cycles per FP64 residual in the mixed-precision solves of the 3-D workload
# (amr_solver_params.cycles_per_refinement; the iterate equals that of one cycle per step, so
# the V-cycle counts stay those of one cycle per step when they divide: PPE 18, Helmholtz 8, 6)
CPR_PPE = 3
CPR_HELM = 2


def _params3d(amr, prec, use_graph):
    """Solver parameters of the 3-D step: (PPE, Helmholtz systems)."""
    return tuple(amr.default_params(rtol=RTOL, max_vcycles=100, precision=prec, use_graph=use_graph,
                                    cycles_per_refinement=c) for c in (CPR_PPE, CPR_HELM))


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the other workloads and the FP64 arm")
    ap.add_argument("--profile-case", choices=["none", "large", "bench", "single3d", "resid64", "bumps3d", "bumps2d",
                                               "cic3d"],
                    default="none",
                    help="large: one mixed-precision solve of the single-level 4096^2 case; bench: one warm-up "
                         "and one timed step of the bench workload; bumps2d: the same for the 2-D two-level "
                         "workload; single3d: one mixed-precision V-cycle of a single-level 256^3 Helmholtz "
                         "problem; resid64: three FP64 level residuals of a single-level 256^3 Helmholtz problem; "
                         "bumps3d: the mixed-precision PPE and one Helmholtz solve of the 3-D workload, "
                         "host-driven loop; cic3d: the interface-condition calls on the 3-D workload's refined "
                         "level (all for ncu)")
    return ap.parse_args()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


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


def _host_info():
    model = platform.processor() or platform.machine()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model, "machine": platform.machine()}


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


def _kernel_source_hash(files=("kernels.cuh", "sweep3d.cuh", "solver.cu")):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2506_02663_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic(key):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the current
    sources of that kernel (the entry's ``sources``); else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        e = d.get(key)
        if e and e.get("source_hash") == _kernel_source_hash(tuple(e.get("sources", ("kernels.cuh", "sweep3d.cuh",
                                                                                       "solver.cu")))):
            return e.get("dram_bytes_per_launch")
    except Exception:
        pass
    return None


# ============================================================================ oracle (CPU)
def _oracle_worker(args):
    """One process: the oracle's V-cycles of one system of the 3-D workload at quarter size
    (64^3 base + 32^3 fine box), setup excluded.  mode "rate": V-cycles for ``seconds``;
    mode "steps": ``warmup`` untimed then ``steps`` timed V-cycles (one per step)."""
    comp, mode, seconds, warmup, steps = args
    sys.path.insert(0, ROOT)
    from oracle import composite as cp, mg, solve as so
    from oracle.hierarchy import Hierarchy as OH
    from paper_2506_02663_gb300 import workloads as wl
    dim, n0, boxes, rhs = wl.bumps3d_rhs(scale=4, component=comp)
    bc, alpha, beta = ([1] * 6, 0.0, 1.0) if comp == 0 else ([0] * 6, 1.0, wl.HELMHOLTZ_BETA)
    H = OH(dim, n0, boxes, bc=bc)
    F = cp.new_field(H)
    for l, lev in enumerate(H.levels):
        for k, (lo, hi) in enumerate(lev.boxes):
            F[l][lev.box_slice(lo, hi)] = rhs[l][k]
    if so.is_pure_neumann(H, alpha):
        F, _ = so.solvability_fix(H, F)
    M = mg.CompositeMG(H, alpha, beta)
    phi = cp.new_field(H)
    dof = valid_dof(n0, boxes)
    if mode == "rate":
        cycles = 0
        t0 = time.perf_counter()
        while True:
            phi = M.vcycle(phi, F)
            cycles += 1
            el = time.perf_counter() - t0
            if el >= seconds:
                return dof, cycles, el, []
    for _ in range(warmup):
        phi = M.vcycle(phi, F)
    ts = []
    for _ in range(steps):
        t0 = time.perf_counter()
        phi = M.vcycle(phi, F)
        ts.append(time.perf_counter() - t0)
    return dof, steps, sum(ts), ts


def _oracle_pool(nproc, mode, seconds=0.0, warmup=0, steps=0):
    ctx = mp.get_context("spawn")  # a pool forked after CUDA initialisation hangs
    jobs = [(c % 4, mode, seconds, warmup, steps) for c in range(nproc)]
    with ctx.Pool(nproc) as pool:
        return pool.map(_oracle_worker, jobs)


def _cpu_baseline():
    """The oracle (plain FP64 numpy, as it stands) on the host: one process alone, then one
    process per host core at once, each running V-cycles of one of the workload's four
    systems (PPE, three Helmholtz) on the workload at quarter size."""
    info = _host_info()
    ncores = max(1, int(info["nproc"] or 1))
    one = _oracle_pool(1, "rate", seconds=10.0)
    d1, c1, e1, _ = one[0]
    allc = _oracle_pool(ncores, "rate", seconds=12.0)
    v_all = sum(d * c / e for d, c, e, _ in allc)
    return {"value": v_all, "unit": UNIT, "cores": ncores, "kind": "oracle",
            "sample": (f"FP64 numpy-oracle V-cycles of the workload at quarter size (base 64^3 + 32^3 fine box, "
                       f"{d1} DOF per system), one process per core, the four systems round-robin, about 12 s each "
                       f"after setup; rate summed over processes"),
            "single_core": {"value": d1 * c1 / e1, "vcycles": c1, "seconds": e1},
            "host": info}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    info = _host_info()
    ncores = max(1, int(info["nproc"] or 1))
    res = _oracle_pool(ncores, "steps", warmup=args.warmup, steps=args.steps)
    step_s = [max(r[3][i] for r in res) for i in range(args.steps)]  # processes run side by side
    dofv = sum(r[0] * r[1] for r in res)
    value = dofv / sum(step_s)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(step_s),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "arm": "FP64 numpy oracle on the host cores; each step = one V-cycle of "
                                                 "one system per process at quarter size, all processes at once"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": ncores, "kind": "oracle",
                         "sample": (f"{args.steps} steps x {ncores} processes x one oracle V-cycle of one system "
                                    f"(PPE / Helmholtz round-robin) of the workload at quarter size (64^3 base + "
                                    f"32^3 fine box), setup and {args.warmup} warm-up cycles excluded"),
                         "host": info},
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


def _valid_mask(gh, torch):
    """1 on the valid cells (Eq. validRegion) of every patch, 0 elsewhere (invalid, ghost and
    padding cells), from the library's index maps, as a device field in the composite layout."""
    import numpy as np
    vm = gh.index_maps()["valid"].astype(np.float64)
    off = 0
    per = []
    for bl in gh.boxes:
        lev = []
        for lo, hi in bl:
            shape = tuple(hi[e] - lo[e] + 1 for e in range(gh.dim))
            n = int(np.prod(shape))
            lev.append(vm[off:off + n].reshape(shape[::-1]).transpose())
            off += n
        per.append(lev)
    return torch.from_numpy(gh.pack(per)).cuda()


def _bumps3d(amr, torch, scale=1):
    """Hierarchies, operators and right-hand sides of the 3-D workload: one hierarchy object
    per system, so that the three Helmholtz solves' captured graphs run concurrently."""
    from paper_2506_02663_gb300 import workloads as wl
    dim, n0, boxes, _ = wl.bumps3d_rhs(scale, 0)
    ghs = [amr.Hierarchy(dim, n0, boxes) for _ in range(4)]
    f_host = [ghs[0].pack(wl.bumps3d_rhs(scale, c)[3]) for c in range(4)]
    ops = [amr.Operator(ghs[0], 0.0, 1.0, [1] * 6)]
    ops += [amr.Operator(g, 1.0, wl.HELMHOLTZ_BETA, [0] * 6) for g in ghs[1:]]
    fs = [torch.from_numpy(a).cuda() for a in f_host]
    return {"dim": dim, "n0": n0, "boxes": boxes, "dof": valid_dof(n0, boxes), "ghs": ghs, "ops": ops,
            "f_host": f_host, "fs": fs, "phis": [torch.zeros_like(fs[0]) for _ in range(4)]}


def _close(w):
    for op in w["ops"]:
        op.close()
    for g in w["ghs"]:
        g.close()


def _step3d(amr, w, pp):
    """One step: the PPE, then the three Helmholtz components in one batched call; pp = the
    parameters of the PPE and of the Helmholtz systems."""
    ops, phis, fs = w["ops"], w["phis"], w["fs"]
    vc = [ops[0].solve(phis[0], fs[0], params=pp[0])["vcycles"]]
    st, status = amr.batch_solve(ops[1:], phis[1:], fs[1:], params=pp[1])
    if any(status):
        raise RuntimeError(f"batched Helmholtz solves: statuses {status}")
    return vc + [s["vcycles"] for s in st]


def _timed(torch, fn, k, flush=None):
    stream = torch.cuda.current_stream()
    ts, out = [], []
    for _ in range(k):
        if flush is not None:
            flush.fill_(1.0)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        out.append(fn())
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return ts, out


KERNEL_CLASSES = {
    "jacobi": ("KC_JACOBI", "weighted-Jacobi sweep (k_sweep3d / k_level_op3d_zc / k_level_op3d_march / k_level_op2d_tiled)"),
    "residual": ("KC_RESID", "FP32 level residual or operator application (k_sweep3d / k_level_op3d_zc / k_level_op*)"),
    "residual64": ("KC_RESID64", "FP64 level residual of the refinement loop (3-D: k_absmax_patch + k_resid3d_fx, "
                                 "fixed-point stencil sums)"),
    "restrict": ("KC_RESTRICT", "residual restriction and average-down (k_restrict*)"),
    "prolong": ("KC_PROLONG", "linear prolongation + correction (k_prolong*)"),
    "down_leg": ("KC_DOWN", "k_mg_down2d<float>: nu1 sweeps + residual + restriction, one launch per grid"),
    "up_leg": ("KC_UP", "k_mg_up2d<float>: prolongation + nu2 sweeps, one launch per grid"),
    "coarse_block": ("KC_COARSE", "k_mg_coarse2d<float>: the V-cycle on the grids <= 64^2, one block"),
}
# grid-size buckets (cells) of the 3-D workload's grids: the 256^3 base, the 128^3 grids (fine
# box, second multigrid grid), 64^3, and the coarse end
SIZE_BUCKETS = (("256^3", 1e7, 1e9), ("128^3", 1e6, 1e7), ("64^3", 1e5, 1e6), ("<=32^3", 0.0, 1e5))


def _class_table(amr, buckets=None):
    out = {}
    for name, (kc, _) in KERNEL_CLASSES.items():
        if buckets is None:
            r = amr.profile_read(getattr(amr, kc))
            if r["launches"]:
                out[name] = r
        else:
            for bname, lo, hi in buckets:
                r = amr.profile_read_range(getattr(amr, kc), lo, hi)
                if r["launches"]:
                    out[f"{name}@{bname}"] = r
    return out


def _roofline_entry(classes, peak, peak_kind, workload):
    """The dominant kernel (by summed launch time) of an instrumented pass: algorithmic bytes
    per launch over the average CUDA-event launch duration, against the measured copy
    bandwidth; traffic = ncu DRAM bytes per launch of the same kernel on the same grid."""
    if not classes:
        return {"bound": "hbm", "achieved": None, "peak": peak, "unit": "GB/s", "frac": None, "traffic": None}
    dom = max(classes, key=lambda k: classes[k]["ms"])
    c = classes[dom]
    achieved = c["bytes"] / (c["ms"] * 1e-3) / 1e9 if c["ms"] > 0 else None
    base = dom.split("@")[0]
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak if achieved else None,
            "traffic": _traffic(f"{dom}_{workload}"),
            "kernel": KERNEL_CLASSES[base][1], "class": dom,
            "launches": c["launches"], "avg_launch_us": 1e3 * c["ms"] / max(c["launches"], 1),
            "bytes_per_launch": c["bytes"] / max(c["launches"], 1), "peak_source": f"{peak_kind} hbm_gbs",
            "share_of_instrumented_ms": c["ms"] / sum(v["ms"] for v in classes.values())}


def _classes_summary(classes):
    return {k: {"launches": v["launches"], "ms": v["ms"], "GB/s": v["bytes"] / (v["ms"] * 1e-3) / 1e9}
            for k, v in classes.items()}


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
    w = _bumps3d(amr, torch)
    dof = w["dof"]
    prec = amr.MIXED if args.precision == "mixed" else amr.FP64
    params = _params3d(amr, prec, 1)

    for _ in range(args.warmup):
        _step3d(amr, w, params)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    l0 = amr.kernel_launches()
    ts, vcs = _timed(torch, lambda: _step3d(amr, w, params), args.steps)
    launches = amr.kernel_launches() - l0
    torch.cuda.synchronize()
    clocks = sampler.stop()
    if dist:
        dist.barrier()
    dofv_rank = sum(dof * sum(v) for v in vcs)
    tmax, value = aggregate(sum(ts), dofv_rank, ws, dist, "cuda")
    vc_per_system = [statistics.mean(v[i] for v in vcs) for i in range(4)]
    phi_main = [p.clone() for p in w["phis"]] if rank == 0 else None

    # ---------------- end to end through the C ABI with host buffers: amr_solve_host for the
    # PPE, amr_batch_solve_host for the three components (H2D of every f, D2H of every phi
    # inside the timed region)
    fh = [torch.from_numpy(a).pin_memory().numpy() for a in w["f_host"]]
    ph = [torch.zeros(w["ghs"][0].nelems, dtype=torch.float64).pin_memory().numpy() for _ in range(4)]
    ops = w["ops"]

    def e2e_step():
        vc = [ops[0].solve_host(ph[0], fh[0], params=params[0])["vcycles"]]
        st, _ = amr.batch_solve_host(ops[1:], ph[1:], fh[1:], params=params[1])
        return vc + [s["vcycles"] for s in st]
    e2e_step()
    torch.cuda.synchronize()
    te = time.perf_counter()
    e2e_v = 0
    for _ in range(args.steps):
        e2e_v += sum(e2e_step())
    te = time.perf_counter() - te
    nbytes = 4 * w["ghs"][0].nelems * 8
    e2e = {"value": ws * dof * e2e_v / te if te > 0 else None, "unit": UNIT, "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": nbytes, "ms_per_step": 1e3 * te / args.steps,
           "how": "amr_solve_host (PPE) + amr_batch_solve_host (3 components) from pinned host buffers, "
                  "host wall clock"}

    # ---------------- roofline of the dominant kernel, live (instrumented host-driven loop)
    peak, peak_kind = _peaks()
    prof = _params3d(amr, prec, 0)
    amr.profile_enable(True)
    for k, (op, phi, f) in enumerate(zip(ops, w["phis"], w["fs"])):
        op.solve(phi, f, params=prof[0 if k == 0 else 1])
    amr.profile_enable(False)
    classes = _class_table(amr, SIZE_BUCKETS)
    roofline = _roofline_entry(classes, peak, peak_kind, "bumps3d")

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tmax / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 V-cycles in f64 refinement" if prec == amr.MIXED else "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "dof_per_system": dof, "systems": ["ppe", "helmholtz_u", "helmholtz_v",
                                                                             "helmholtz_w"],
                   "precision": args.precision, "rtol": RTOL,
                   "cycles_per_refinement": {"ppe": CPR_PPE, "helmholtz": CPR_HELM},
                   "vcycles_per_system": vc_per_system,
                   "l2": "no flush: every input and solution field (about 160 MB in FP64) is larger than the "
                         "129 MB L2",
                   "solve": "one captured CUDA graph per solve (device-side while loop over V-cycles); the three "
                            "Helmholtz graphs run concurrently",
                   "parallelism": f"replicas x{ws}"},
        "gpu_launches": launches,
        "clocks": clocks,
        "e2e": e2e,
        "roofline": roofline,
        "kernel_classes": _classes_summary(classes),
    }

    if not args.no_extras and rank == 0:
        other = amr.FP64 if prec == amr.MIXED else amr.MIXED
        p2 = _params3d(amr, other, 1)
        _step3d(amr, w, p2)
        ts2, vcs2 = _timed(torch, lambda: _step3d(amr, w, p2), min(args.steps, 3))
        key = "fp64" if prec == amr.MIXED else "mixed"
        line[key] = {"value": dof * sum(sum(v) for v in vcs2) / (sum(ts2) * 1e-3),
                     "ms_per_step": sum(ts2) / len(ts2),
                     "vcycles_per_system": [statistics.mean(v[i] for v in vcs2) for i in range(4)]}
        # mixed against FP64 at full size (both refined to the same residual), valid cells
        vmask = _valid_mask(w["ghs"][0], torch)
        diffs = []
        for a, b in zip(phi_main, w["phis"]):
            diffs.append(float(torch.max(torch.abs(a - b) * vmask) / torch.max(torch.abs(b) * vmask)))
        line["precision"] = {
            "bumps3d_full_size_mixed_vs_fp64_rel_maxdiff_valid_cells": diffs,
            "stored_oracle_solutions": _golden_errors(amr, torch),
        }
        line["bumps3d_adjoint"] = _bumps3d_adjoint(amr, torch, w)
        line["cic3d"] = _cic3d_measure(amr, torch, w, peak, peak_kind)
        try:
            line["regrid3d"] = _regrid_measure(amr)
        except Exception as ex:  # the main line must not depend on this extra
            line["regrid3d"] = {"error": f"{type(ex).__name__}: {ex}"}
        _close(w)
        del w
        torch.cuda.empty_cache()
        line["bumps2d"] = _bumps2d_measure(amr, torch, peak, peak_kind, args.steps)
        line["ms2d"] = _ms2d_measure(amr, torch)
        line["batch2d"] = _batch_measure(amr, torch)
        line["adjoint2d"] = _adjoint_measure(amr, torch)
        line["large_grid_roofline"] = _large_grid_roofline(amr, torch, peak, peak_kind)

    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = _cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


# FP64 rate of the GB300 (nominal 1.25 TFLOP/s: 2 FP64 multiply-adds per clock per SM, 152 SMs,
# 2070 MHz): the bound of the interface-ghost kernels, which are FP64-ALU-bound
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def _cic3d_measure(amr, torch, w, peak, peak_kind, reps=20):
    """Interface conditions of the 3-D workload's refined level (the 128^3 box): per velocity
    component the CF ghosts at t* from four coarse times (value and time derivative), then
    the corrected interface face averages of the three components (Sec. 6.3-6.4).  CUDA events
    around `reps` calls, and around `reps` single ghost calls for the roofline.  Bytes =
    the coarse cells inside the union of the AMRCFI windows read once per coarse time and
    component, the ghost values and derivatives written, four cells read and one value
    written per interface face.  Flops of one ghost call = the two time combinations of every
    window cell (8 multiply-adds) + AMRCFI of the two combinations per coarse parent (2 x
    (2 x 125 + 4 x 25 + 8 x 5) multiply-adds), 2 flops per multiply-add."""
    try:
        return _cic3d_run(amr, torch, w, peak, peak_kind, reps)
    except Exception as ex:  # the main line must not depend on this extra
        return {"error": f"{type(ex).__name__}: {ex}"}


def _cic3d_run(amr, torch, w, peak, peak_kind, reps):
    import numpy as np
    gh, op = w["ghs"][0], w["ops"][0]
    n = gh.nelems
    g = torch.Generator(device="cuda").manual_seed(9)
    coarse = [torch.randn(n, dtype=torch.float64, device="cuda", generator=g) for _ in range(4)]
    vel = [torch.randn(n, dtype=torch.float64, device="cuda", generator=g) for _ in range(3)]
    rate = [torch.empty_like(vel[0]) for _ in range(3)]
    for x in coarse + vel:
        op.fill_ghosts(x)
    info = amr.cic_faces(gh, 1)
    nf, nc = len(info["face"]), info["ncomponents"]
    faces = torch.empty(nf, dtype=torch.float64, device="cuda")
    delta = torch.empty(nc, dtype=torch.float64, device="cuda")
    k, eta = 1.0 / 256.0, 0.5 / 256.0

    def ghosts(d=0):
        amr.cic_ghosts(gh, 1, coarse, k, eta, vel[d], rate[d])

    def call():
        for d in range(3):
            ghosts(d)
        amr.cic_face_averages(gh, 1, vel, faces, delta=delta)
    for _ in range(3):
        call()
    torch.cuda.synchronize()
    l0 = amr.kernel_launches()
    ts, _ = _timed(torch, call, reps)
    launches = (amr.kernel_launches() - l0) // reps
    tg, _ = _timed(torch, ghosts, reps)
    maps = gh.index_maps()
    starts = maps["cfi_start"]
    ncfi = len(starts)
    band = np.zeros(gh.n0, bool)
    for o in np.ndindex(5, 5, 5):
        band[starts[:, 0] + o[0], starts[:, 1] + o[1], starts[:, 2] + o[2]] = True
    nband = int(band.sum())
    nbytes = 3 * (4 * nband * 8 + 2 * ncfi * 8) + nf * (4 * 8 + 8)
    ngroups = ncfi // 8
    flops = 2.0 * (8 * nband + ngroups * 2 * (2 * 125 + 4 * 25 + 8 * 5))
    ms, msg = statistics.median(ts), statistics.median(tg)
    gbs = nbytes / (ms * 1e-3) / 1e9
    tf = flops / (msg * 1e-3) / 1e12
    tot = float(faces.sum()) if nf else 0.0
    return {"ms_per_call": ms, "kernel_launches_per_call": launches, "cf_ghosts_per_component": ncfi,
            "coarse_window_cells": nband, "interface_faces": nf, "components": nc,
            "bytes_per_call": nbytes, "gbs_per_call": gbs,
            "ghost_call_ms": msg,
            "roofline": {"bound": "alu", "kernels": "k_cic_combine + k_cic_grp3 (one amr_cic_ghosts call)",
                         "achieved": tf, "peak": FP64_PEAK_TFLOPS, "unit": "FP64 TFLOP/s", "frac": tf / FP64_PEAK_TFLOPS,
                         "flops_per_call": flops, "peak_kind": "nominal (2 FP64 FMA/clk/SM x 152 SMs x 2070 MHz)"},
            "corrected_face_sum": tot,
            "how": "3 x amr_cic_ghosts (value + rate) + amr_cic_face_averages on level 1 of bumps3d, median of "
                   "CUDA-event times; the ghost kernels are FP64-rate-bound"}


def _regrid_tags(dim, n0, nlevels, ratio, seed=7):
    """Tagged cells per level for the regridding entry: cells within a spherical shell around
    three random vortex centres (the stand-in for |curl u| >= eps), thinner on finer levels."""
    import numpy as np
    rng = np.random.default_rng(seed)
    tags = []
    for l in range(nlevels - 1):
        nd = [v * ratio ** l for v in n0]
        g = np.stack(np.meshgrid(*[np.arange(v) for v in nd], indexing="ij"), axis=-1).reshape(-1, dim)
        x = (g + 0.5) / np.asarray(nd)
        c = rng.random((3, dim)) * 0.5 + 0.25
        d = np.min([np.sqrt(np.sum((x - ci) ** 2, axis=1)) for ci in c], axis=0)
        tags.append(g[(d < 0.15 / (l + 1)) & (d > 0.08 / (l + 1))].astype(np.int32))
    return tags


def _regrid_measure(amr, reps=5):
    """Regridding (RDM-2/3, host): amr_regrid on a three-level 3-D hierarchy (64^3 base), host
    wall clock; the result is checked by the library's own hierarchy validation (the box lists
    are compared with the oracle's in the tests)."""
    dim, n0, nl, r = 3, (64, 64, 64), 3, 2
    tags = _regrid_tags(dim, n0, nl, r)
    got = amr.regrid(dim, n0, nl, tags, 0.75, 2, r)
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        amr.regrid(dim, n0, nl, tags, 0.75, 2, r)
        ts.append(time.perf_counter() - t0)
    amr.Hierarchy(dim, n0, got).close()  # proper nesting, refinement and box sizes hold
    return {"ms": 1e3 * statistics.median(ts), "tags_per_level": [len(t) for t in tags],
            "boxes_per_level": [len(b) for b in got],
            "how": "amr_regrid (Berger-Rigoutsos clustering, RDM-2/3) on the host, efficiency 0.75, min width 2; "
                   "the new hierarchy passes amr_hierarchy_create"}


def _golden_errors(amr, torch):
    """Error of the GPU solutions against the oracle's stored direct solutions (tests/golden,
    written by a script that calls only the oracle): the 2-D and 3-D workloads at 1/8 size,
    pure-Neumann PPE and Helmholtz, both precisions, max over the stored samples relative to
    max|phi|."""
    import numpy as np
    from paper_2506_02663_gb300 import workloads as wl
    out = {}
    for name, fname in (("bumps2d_1/8", "amr2d.json"), ("bumps3d_1/8", "amr3d.json")):
        with open(os.path.join(ROOT, "tests", "golden", fname)) as fh:
            gold = json.load(fh)
        for sysname in ("ppe", "helmholtz"):
            if name.startswith("bumps2d"):
                dim, n0, boxes, rhs = wl.bumps2d_rhs(scale=8)
                bc, alpha, beta = ([1] * 4, 0.0, 1.0) if sysname == "ppe" else ([0] * 4, 1.0, wl.HELMHOLTZ_BETA)
            else:
                dim, n0, boxes, rhs = wl.bumps3d_rhs(scale=8, component=0 if sysname == "ppe" else 1)
                bc, alpha, beta = ([1] * 6, 0.0, 1.0) if sysname == "ppe" else ([0] * 6, 1.0, wl.HELMHOLTZ_BETA)
            gh = amr.Hierarchy(dim, n0, boxes)
            op = amr.Operator(gh, alpha, beta, bc)
            f = torch.from_numpy(gh.pack(rhs)).cuda()
            for pname, prec in (("fp64", amr.FP64), ("mixed", amr.MIXED)):
                x = torch.zeros_like(f)
                op.solve(x, f, params=amr.default_params(rtol=1e-12, max_vcycles=100, precision=prec))
                per = gh.unpack(x.cpu().numpy())
                err = 0.0
                for s in gold[sysname]["samples_level_index_value"]:
                    l, idx, v = s[0], s[1:1 + dim], s[1 + dim]
                    # stored indices are into the oracle's level array (bounding box + 2 ghosts)
                    lo = [min(b[0][d] for b in boxes[l]) - 2 for d in range(dim)]
                    g = [idx[d] + lo[d] for d in range(dim)]
                    for k, (blo, bhi) in enumerate(boxes[l]):
                        if all(blo[d] <= g[d] <= bhi[d] for d in range(dim)):
                            err = max(err, abs(float(per[l][k][tuple(g[d] - blo[d] for d in range(dim))]) - v))
                out[f"{name}/{sysname}/{pname}"] = err / gold[sysname]["max_abs"]
            op.close()
            gh.close()
    return out


def _bumps3d_adjoint(amr, torch, w, reps=2):
    """The backward pass of the 3-D step: the four adjoint solves (amr_solve_transpose, mixed
    precision, same tolerance; host-driven refinement loop)."""
    pa = amr.default_params(rtol=RTOL, max_vcycles=100, precision=amr.MIXED, use_graph=0)
    lam = [torch.zeros_like(w["fs"][0]) for _ in range(4)]

    def backward():
        return [op.solve_transpose(l, f, params=pa)["vcycles"] for op, l, f in zip(w["ops"], lam, w["fs"])]
    try:
        backward()
        ts, vcs = _timed(torch, backward, reps)
        return {"ms_per_step": statistics.median(ts), "vcycles_per_system": vcs[-1],
                "what": "A^T solves of the PPE (solvability-corrected solve map) and the three Helmholtz operators, "
                        "right-hand side f, mixed precision to 1e-10"}
    except Exception as exc:  # reported, not fatal: the forward numbers stand on their own
        return {"error": str(exc)[:200]}


def _bumps2d_measure(amr, torch, peak, peak_kind, steps):
    """The 2-D two-level workload (base 256^2 + ratio-2 box [0.25,0.75]^2, 256^2 fine cells):
    PPE + Helmholtz to 1e-10, both precisions; its working set fits in L2, so L2 is flushed
    (256 MB write) before every timed step; e2e through amr_solve_host; roofline of its
    dominant kernel (launch-latency-bound: its fraction measures launch latency, not HBM)."""
    from paper_2506_02663_gb300 import workloads as wl
    dim, n0, boxes, rhs = wl.bumps2d_rhs()
    dof = valid_dof(n0, boxes)
    gh = amr.Hierarchy(dim, n0, boxes)
    f_host = gh.pack(rhs)
    f = torch.from_numpy(f_host).cuda()
    systems = [([1] * 4, 0.0, 1.0), ([0] * 4, 1.0, wl.HELMHOLTZ_BETA)]
    ops = [amr.Operator(gh, a, b, bc) for bc, a, b in systems]
    phis = [torch.zeros_like(f) for _ in systems]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    out = {"workload": "bumps2d: 2-D two-level AMR, base 256^2 + ratio-2 box [0.25,0.75]^2 (256^2 fine cells), "
                       "8 Gaussian bumps; PPE + Helmholtz to 1e-10", "dof_per_system": dof,
           "l2": "flushed (256 MB write) before every timed step"}
    for name, prec in (("mixed", amr.MIXED), ("fp64", amr.FP64)):
        p = amr.default_params(rtol=RTOL, max_vcycles=100, precision=prec, use_graph=1)

        def step():
            return [op.solve(x, f, params=p)["vcycles"] for op, x in zip(ops, phis)]
        step()
        ts, vcs = _timed(torch, step, steps, flush)
        out[name] = {"value": dof * sum(sum(v) for v in vcs) / (sum(ts) * 1e-3), "ms_per_step": sum(ts) / len(ts),
                     "vcycles_per_system": vcs[-1]}
    p = amr.default_params(rtol=RTOL, max_vcycles=100, precision=amr.MIXED, use_graph=1)
    fh = torch.from_numpy(f_host).pin_memory().numpy()
    ph = torch.zeros(gh.nelems, dtype=torch.float64).pin_memory().numpy()
    for op in ops:
        op.solve_host(ph, fh, params=p)
    te = time.perf_counter()
    v = 0
    for _ in range(steps):
        for op in ops:
            v += op.solve_host(ph, fh, params=p)["vcycles"]
    te = time.perf_counter() - te
    out["e2e"] = {"value": dof * v / te, "unit": UNIT, "ms_per_step": 1e3 * te / steps}
    amr.profile_enable(True)
    pp = amr.default_params(rtol=RTOL, max_vcycles=100, precision=amr.MIXED, use_graph=0)
    for op, x in zip(ops, phis):
        op.solve(x, f, params=pp)
    amr.profile_enable(False)
    classes = _class_table(amr)
    out["roofline"] = _roofline_entry(classes, peak, peak_kind, "bumps2d")
    out["classes"] = _classes_summary(classes)
    for op in ops:
        op.close()
    gh.close()
    return out


def _ms2d_measure(amr, torch, reps=5):
    """The 64^2 manufactured-solution Poisson problem (Dirichlet face averages of
    phi = sin 2 pi x sin 3 pi y + x^2 y): FP64 to 1e-12, time to tolerance, V-cycles, the error
    against the exact cell averages and the observed order from 32^2, 64^2, 128^2."""
    import numpy as np
    from paper_2506_02663_gb300 import workloads as wl
    out = {"workload": "ms2d: single-level 2-D Poisson, 64^2 cells, manufactured solution, FP64 to 1e-12"}
    errs = {}
    for n in (32, 64, 128):
        rhs, bcd, exact = wl.ms2d(n)
        gh = amr.Hierarchy(2, (n, n), [[((0, 0), (n - 1, n - 1))]])
        op = amr.Operator(gh, 0.0, 1.0, [0, 0, 0, 0])
        f = torch.from_numpy(gh.pack([[rhs]])).cuda()
        bc = torch.from_numpy(gh.pack_bc([bcd])).cuda()
        x = torch.zeros_like(f)
        p = amr.default_params(rtol=1e-12, max_vcycles=100, precision=amr.FP64, use_graph=1)
        st = op.solve(x, f, bc=bc, params=p)
        got = gh.unpack(x.cpu().numpy())[0][0]
        e = got - exact
        errs[n] = (float(np.sum(np.abs(e))) / n ** 2, float(np.max(np.abs(e))))
        if n == 64:
            ts, _ = _timed(torch, lambda: op.solve(x, f, bc=bc, params=p), reps)
            out.update({"ms_to_1e-12": statistics.median(ts), "vcycles": st["vcycles"],
                        "final_rel_res": st["final_res"] / st["rhs_norm"], "err_l1": errs[n][0],
                        "err_linf": errs[n][1]})
        op.close()
        gh.close()
    out["observed_order_l1"] = [math.log2(errs[32][0] / errs[64][0]), math.log2(errs[64][0] / errs[128][0])]
    out["observed_order_linf"] = [math.log2(errs[32][1] / errs[64][1]), math.log2(errs[64][1] / errs[128][1])]
    return out


def _batch_golden_errors(hs, phis):
    """Error of batch solutions against the oracle's stored direct solutions of four problems
    (tests/golden/batch2d.json): max over the samples relative to max|phi|, worst problem."""
    with open(os.path.join(ROOT, "tests", "golden", "batch2d.json")) as fh:
        gold = json.load(fh)
    worst = 0.0
    for k, e in gold["problems"].items():
        per = hs[int(k)].unpack(phis[int(k)].cpu().numpy())[0][0]
        for i, j, v in e["samples_index_value"]:
            worst = max(worst, abs(float(per[i - 2, j - 2]) - v) / e["max_abs"])  # oracle arrays carry 2 ghosts
    return worst


def _batch_measure(amr, torch, reps=3):
    """The batch workload: 96 independent single-level Helmholtz problems of uneven sizes
    N in {64,...,512} (seeded), mixed precision to 1e-10, all solved by one amr_batch_solve
    call (work-list graph); compared with the same solves one after another and with FP64."""
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
    for name, prec in (("mixed", amr.MIXED), ("fp64", amr.FP64)):
        p = amr.default_params(rtol=RTOL, max_vcycles=100, precision=prec, use_graph=1)
        amr.batch_solve(ops, phis, fs, params=p)  # warm-up: captures every graph
        res = []
        ts, _ = _timed(torch, lambda: res.append(amr.batch_solve(ops, phis, fs, params=p)), reps)
        st, status = res[-1]
        vc = sum(pr["n"] ** 2 * s["vcycles"] for pr, s in zip(probs, st))
        out[name] = {"ms_per_batch": statistics.median(ts), "value": vc / (statistics.median(ts) * 1e-3),
                     "unit": UNIT, "all_converged": all(x == 0 for x in status),
                     "error_vs_stored_oracle": _batch_golden_errors(hs, phis)}
    p = amr.default_params(rtol=RTOL, max_vcycles=100, precision=amr.MIXED, use_graph=1)

    def seq():
        for op, x, f in zip(ops, phis, fs):
            op.solve(x, f, params=p)
    seq()
    ts, _ = _timed(torch, seq, 1)
    out["sequential_mixed_ms"] = ts[0]
    for op in ops:
        op.close()
    for gh in hs:
        gh.close()
    return out


def _adjoint_measure(amr, torch, reps=3, ndir=64):
    """The adjoint2d workload (base 256^2, boxes [0.2,0.8]^2 -> 308^2 and [0.35,0.65]^2 ->
    308^2 fine cells, two smoothed N(0,1) forcing components): forward = two Helmholtz solves
    and the composite projection, J = 1/2 sum over valid cells of u^2; backward = the
    projection's adjoint and two adjoint Helmholtz solves, FP64 to 1e-12.  The gradient's
    directional derivatives are checked against central differences (eps = 1e-3) along 64
    seeded random unit directions: J is quadratic, so the difference is exact up to rounding
    and the solve tolerance."""
    import numpy as np
    from paper_2506_02663_gb300 import workloads as wl
    dim, n0, boxes, comps = wl.adjoint2d_forcing()
    gh = amr.Hierarchy(dim, n0, boxes, h0=1.0 / n0[0])
    helm = amr.Operator(gh, 1.0, wl.HELMHOLTZ_BETA, [0] * 4)
    ppe = amr.Operator(gh, 0.0, 1.0, [1] * 4)
    p = amr.default_params(rtol=1e-12, max_vcycles=200, precision=amr.FP64, use_graph=1)
    g = [torch.from_numpy(gh.pack(comps[d])).cuda() for d in range(dim)]
    valid = _valid_mask(gh, torch)
    w = [torch.zeros_like(g[0]) for _ in range(dim)]
    u = [torch.zeros_like(g[0]) for _ in range(dim)]
    v = [torch.zeros_like(g[0]) for _ in range(dim)]
    lam = [torch.zeros_like(g[0]) for _ in range(dim)]
    phi = torch.zeros_like(g[0])
    psi = torch.zeros_like(g[0])

    def forward(gg=g):
        vc = 0
        for d in range(dim):
            vc += helm.solve(w[d], gg[d], params=p)["vcycles"]
        vc += amr.project(ppe, [0] * 4, w, u, phi, params=p)["vcycles"]
        return vc

    def J(gg):
        forward(gg)
        return 0.5 * float(sum(torch.sum(valid * ud * ud) for ud in u))

    def backward():
        uv = [valid * ud for ud in u]
        vc = amr.project_transpose(ppe, [0] * 4, uv, v, psi, params=p)["vcycles"]
        for d in range(dim):
            vc += helm.solve_transpose(lam[d], v[d], params=p)["vcycles"]
        return vc

    forward()
    tf, vf = _timed(torch, forward, reps)
    tb, vb = _timed(torch, backward, reps)
    forward()
    backward()
    grad = [valid * x.clone() for x in lam]
    rng = np.random.default_rng(229)
    eps = 1e-3
    errs = []
    for _ in range(ndir):
        dv = [valid * torch.from_numpy(rng.standard_normal(gh.nelems)).cuda() for _ in range(dim)]
        nrm = float(torch.sqrt(sum(torch.sum(x * x) for x in dv)))
        dv = [x / nrm for x in dv]
        jp = J([a + eps * b for a, b in zip(g, dv)])
        jm = J([a - eps * b for a, b in zip(g, dv)])
        fd = (jp - jm) / (2 * eps)
        adj = float(sum(torch.sum(a * b) for a, b in zip(grad, dv)))
        errs.append(abs(fd - adj) / abs(fd))
    ppe.close()
    helm.close()
    gh.close()
    return {"workload": "adjoint2d: three-level 2-D AMR (256^2 base, 308^2 + 308^2 fine), two components; "
                        "forward = 2 Helmholtz solves + composite projection, backward = adjoint projection + "
                        "2 adjoint Helmholtz solves, FP64 to 1e-12",
            "forward_ms": statistics.median(tf), "backward_ms": statistics.median(tb),
            "backward_over_forward": statistics.median(tb) / statistics.median(tf),
            "vcycles_forward": vf[-1], "vcycles_backward": vb[-1],
            "fd_directions": ndir, "max_rel_fd_error": max(errs), "median_rel_fd_error": statistics.median(errs)}


def _large_grid_roofline(amr, torch, peak, peak_kind, n=4096):
    """The 2-D kernels on a single-level n^2 Helmholtz solve (fields >> L2): the HBM
    efficiency of the temporally blocked legs when they are not launch-bound."""
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
    out = _roofline_entry(classes, peak, peak_kind, f"single{n}")
    out["workload"] = f"single-level {n}^2 Helmholtz, mixed precision, {st['vcycles']} V-cycles"
    out["classes"] = _classes_summary(classes)
    op.close()
    gh.close()
    return out


# ============================================================================ ncu cases
def _profile_case():
    import torch
    from paper_2506_02663_gb300 import amr
    from paper_2506_02663_gb300 import workloads as wl
    n = 4096
    gh = amr.Hierarchy(2, (n, n), [[((0, 0), (n - 1, n - 1))]])
    op = amr.Operator(gh, 1.0, wl.HELMHOLTZ_BETA * 16.0, [0, 0, 0, 0])
    f = torch.ones(gh.nelems, dtype=torch.float64, device="cuda")
    phi = torch.zeros_like(f)
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
    """One mixed-precision V-cycle (host-driven loop) of a single-level n^3 Helmholtz problem
    with homogeneous Dirichlet data: the 3-D level-operator kernels on a grid whose fields
    exceed L2 (67 MB per FP32 field at 256^3; about 1 GB on the device in all)."""
    import torch
    from paper_2506_02663_gb300 import amr
    from paper_2506_02663_gb300 import workloads as wl
    gh = amr.Hierarchy(3, (n, n, n), [[((0, 0, 0), (n - 1, n - 1, n - 1))]])
    op = amr.Operator(gh, 1.0, wl.HELMHOLTZ_BETA, [0] * 6)
    f = torch.ones(gh.nelems, dtype=torch.float64, device="cuda")
    phi = torch.zeros_like(f)
    st = op.solve(phi, f, params=amr.default_params(rtol=1e-30, max_vcycles=1, precision=amr.MIXED, use_graph=0),
                  allow_not_converged=True)
    torch.cuda.synchronize()
    amr.check_kernel_flags()
    print(json.dumps({"profile_case": "single3d", "vcycles": st["vcycles"], "final_res": st["final_res"]}))
    return 0


def _profile_resid64(n=256):
    """Three FP64 level residuals (amr_residual) of a single-level n^3 Helmholtz problem with
    homogeneous Dirichlet data and seeded random x and f: the fixed-point FP64 residual and its
    frame pass on a grid whose fields exceed L2 (134 MB per FP64 field; about 1 GB on the
    device in all)."""
    import torch
    from paper_2506_02663_gb300 import amr
    from paper_2506_02663_gb300 import workloads as wl
    gh = amr.Hierarchy(3, (n, n, n), [[((0, 0, 0), (n - 1, n - 1, n - 1))]], h0=1.0 / n)
    op = amr.Operator(gh, 1.0, wl.HELMHOLTZ_BETA, [0] * 6)
    g = torch.Generator(device="cuda").manual_seed(5)
    x = torch.randn(gh.nelems, dtype=torch.float64, device="cuda", generator=g)
    f = torch.randn(gh.nelems, dtype=torch.float64, device="cuda", generator=g)
    r = torch.zeros_like(x)
    for _ in range(3):
        op.residual(x, f, r)
    torch.cuda.synchronize()
    amr.check_kernel_flags()
    print(json.dumps({"profile_case": "resid64", "max_abs_residual": float(r.abs().max())}))
    return 0


def _profile_bumps3d():
    """The 3-D workload's PPE and one Helmholtz solve, mixed precision, host-driven loop."""
    import torch
    from paper_2506_02663_gb300 import amr
    w = _bumps3d(amr, torch)
    pp = amr.default_params(rtol=RTOL, max_vcycles=100, precision=amr.MIXED, use_graph=0)
    for op, f in zip(w["ops"][:2], w["fs"][:2]):  # warm-up: scratch set-up and tile autotuning
        op.solve(torch.zeros_like(f), f, params=pp)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("measured")
    vc = [op.solve(torch.zeros_like(f), f, params=pp)["vcycles"] for op, f in zip(w["ops"][:2], w["fs"][:2])]
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"profile_case": "bumps3d", "vcycles": vc}))
    return 0


def _profile_bench(args):
    """One warm-up step and one step of the bench workload (graph mode), for launch lists."""
    import torch
    from paper_2506_02663_gb300 import amr
    w = _bumps3d(amr, torch)
    prec = amr.MIXED if args.precision == "mixed" else amr.FP64
    p = _params3d(amr, prec, 1)
    for it in range(2):  # the second step inside the "measured" range
        if it == 1:
            torch.cuda.nvtx.range_push("measured")
        l0 = amr.kernel_launches()
        vc = _step3d(amr, w, p)
        torch.cuda.synchronize()
        if it == 1:
            torch.cuda.nvtx.range_pop()
        print(json.dumps({"profile_case": "bench", "vcycles": vc, "launches": amr.kernel_launches() - l0}))
    return 0


def _profile_bumps2d():
    """One warm-up step and one step of the 2-D two-level workload (graph mode)."""
    import torch
    from paper_2506_02663_gb300 import amr
    from paper_2506_02663_gb300 import workloads as wl
    dim, n0, boxes, rhs = wl.bumps2d_rhs()
    gh = amr.Hierarchy(dim, n0, boxes)
    f = torch.from_numpy(gh.pack(rhs)).cuda()
    ops = [amr.Operator(gh, a, b, bc) for bc, a, b in (([1] * 4, 0.0, 1.0), ([0] * 4, 1.0, wl.HELMHOLTZ_BETA))]
    p = amr.default_params(rtol=RTOL, max_vcycles=100, precision=amr.MIXED, use_graph=1)
    for it in range(2):
        if it == 1:
            torch.cuda.nvtx.range_push("measured")
        vc = [op.solve(torch.zeros_like(f), f, params=p)["vcycles"] for op in ops]
        torch.cuda.synchronize()
        if it == 1:
            torch.cuda.nvtx.range_pop()
        print(json.dumps({"profile_case": "bumps2d", "vcycles": vc}))
    return 0


def _profile_cic3d():
    """The interface-condition calls alone on the 3-D workload's geometry (timed as in the
    bench's cic3d entry)."""
    import torch
    from paper_2506_02663_gb300 import amr
    from paper_2506_02663_gb300 import workloads as wl
    dim, n0, boxes = wl.hierarchy_boxes("bumps3d", 1)
    gh = amr.Hierarchy(dim, n0, boxes)
    w = {"ghs": [gh], "ops": [amr.Operator(gh, 0.0, 1.0, [1] * 6)]}
    peak, peak_kind = _peaks()
    print(json.dumps({"profile_case": "cic3d", **_cic3d_measure(amr, torch, w, peak, peak_kind)}))
    return 0


def main():
    args = _args()
    if args.profile_case == "cic3d":
        return _profile_cic3d()
    if args.profile_case == "large":
        return _profile_case()
    if args.profile_case == "bench":
        return _profile_bench(args)
    if args.profile_case == "bumps2d":
        return _profile_bumps2d()
    if args.profile_case == "single3d":
        return _profile_single3d()
    if args.profile_case == "resid64":
        return _profile_resid64()
    if args.profile_case == "bumps3d":
        return _profile_bumps3d()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
