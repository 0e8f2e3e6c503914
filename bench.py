#!/usr/bin/env python
"""Benchmark of the LOR-preconditioned matrix-free Q_p Poisson solver on GB300.

Workload: 3D variable-coefficient Poisson, continuous Q_8 on a 32^3 hex mesh of
the unit cube, interior vertices perturbed by U(-0.15h, 0.15h), kappa = exp(Z),
Z ~ N(0,1) per element, f = 1, homogeneous Dirichlet (16,581,375 unknowns).
One step = one solve to ||r|| <= 1e-8 ||b|| with the chosen form (mixed
precision: FP32 operator/preconditioner with bf16 ILU factors inside FP64
iterative refinement), inputs resident in HBM.  The JSON line also carries the
plain FP64 solve time, per-apply MDOF/s of apply_A and apply_P in FP64 and FP32,
the roofline of the dominant kernel, the end-to-end number through the host-
buffer C-ABI call, and the CPU oracle timed on a bounded sample.

N > 1 GPUs (torchrun): independent replicas, one problem per rank (seed = rank);
no data-path collective.  `--impl reference` times the CPU oracle instead.
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
sys.path.insert(0, ROOT)

METRIC = "3D Q_p PCG time-to-1e-8 and MDOF/s per apply: plain FP64 vs chosen form"
REF_ITERS = 152   # FP64 PCG iterations to 1e-8 on the Q8 32^3 workload (measured on GB300)
# DRAM bytes (read + written) of one patch-kernel launch on Q8 32^3, mixed bf16: the ncu
# capture of one launch on Q8 12^3 scaled by the factor rows (profiles/patch_warp_q8_dram.md);
# measured on the kernel as built (two warps per patch)
PATCH_TRAFFIC_Q8N32 = 23.3e9
WORKLOAD = "3D CG Q8, 32^3 perturbed hex mesh (+-0.15h), log-normal kappa (sigma 1), f=1, rtol 1e-8"


def max_over_ranks(seconds: float, world: int, device=None) -> float:
    """The slowest rank's time: every rank calls this; identity for one rank."""
    if world <= 1:
        return seconds
    import torch
    import torch.distributed as dist
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(seconds_max: float, steps: int, world: int) -> float:
    """Whole-job solves/s: each of `world` replicas solved `steps` problems, and the
    job took as long as its slowest rank."""
    return world * steps / seconds_max


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--p", type=int, default=8)
    ap.add_argument("--n", type=int, default=32)
    ap.add_argument("--form", default="mixed-bf16", choices=["mixed-bf16", "mixed-fp32", "fp64"])
    ap.add_argument("--no-extras", action="store_true", help="skip FP64 solve, per-apply and CPU legs")
    ap.add_argument("--no-batch", action="store_true", help="skip the 256-solve batched leg")
    ap.add_argument("--no-dg", action="store_true", help="skip the DG penalty-sweep leg")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-correction leg (Q6 32^3)")
    ap.add_argument("--no-schwarz", action="store_true", help="skip the B(1) / B(V) / hybrid comparison leg")
    ap.add_argument("--batch-n", type=int, default=256)
    ap.add_argument("--cpu-sample-s", type=float, default=15.0)
    ap.add_argument("--weighting", type=int, default=0, choices=[0, 1, 2],
                    help="patch-sum weighting of the timed form: 0 unit (the paper's method), 1 counting matrix, "
                         "2 partition of unity")
    ap.add_argument("--leg", choices=["learned", "schwarz", "batch"],
                    help="run only this leg at --p/--n (learned: trained on an n/2 mesh for --learned-steps "
                         "steps) and print its JSON; a profiling entry point, not the bench line")
    ap.add_argument("--learned-steps", type=int, default=300)
    ap.add_argument("--summarize-ncu", metavar="CSV",
                    help="print per-kernel launches, total time and share of an ncu launch list "
                         "(--metrics gpu__time_duration.sum --csv) and exit")
    return ap.parse_args()


def summarize_ncu_launches(path: str) -> str:
    """Per kernel of an ncu launch list: launches, total device time (ms) and share."""
    import csv
    import re
    from collections import defaultdict
    rows = list(csv.reader(open(path)))
    hdr = None
    for i, r in enumerate(rows):
        if "Kernel Name" in r and "Metric Name" in r:
            hdr, rows = r, rows[i + 1:]
            break
    if hdr is None:
        raise ValueError(f"{path}: no ncu CSV header (Kernel Name, Metric Name)")
    k_name, k_metric, k_val, k_unit = (hdr.index(x) for x in ("Kernel Name", "Metric Name", "Metric Value",
                                                             "Metric Unit"))
    to_ms = {"ns": 1e-6, "nsecond": 1e-6, "us": 1e-3, "usecond": 1e-3, "ms": 1.0, "msecond": 1.0}
    tot, cnt = defaultdict(float), defaultdict(int)
    for r in rows:
        if len(r) <= k_val or r[k_metric] != "gpu__time_duration.sum":
            continue
        name = re.sub(r"<unnamed>::|\(anonymous namespace\)::", "", r[k_name])   # before the argument list goes
        name = re.sub(r"\(.*", "", name).replace("void ", "").strip()
        tot[name] += float(r[k_val].replace(",", "")) * to_ms.get(r[k_unit], 1.0)
        cnt[name] += 1
    all_ms = sum(tot.values())
    out = [f"{'kernel':70s} {'launches':>9s} {'total ms':>11s} {'share':>7s}"]
    for name in sorted(tot, key=lambda n: -tot[n]):
        out.append(f"{name[:70]:70s} {cnt[name]:9d} {tot[name]:11.3f} {100 * tot[name] / all_ms:6.2f}%")
    out.append(f"{'all':70s} {sum(cnt.values()):9d} {all_ms:11.3f}")
    return "\n".join(out)


# --------------------------------------------------------------------- CPU leg
def cpu_sample_worker(p: int, n: int, seed: int, budget_s: float, iters: int) -> dict:
    """Times the CPU oracle as it stands on a bounded sample of the workload and
    extrapolates one solve: per iteration nel element applies (dense element
    matrix times element vector, the oracle's assembled-operator cost), J patch
    V-cycles (ILU(0) V(1,1) on a 2x2x2-element patch), the coarse-space
    correction and the PCG vector updates, times `iters`."""
    import numpy as np
    from oracle import cg as ocg
    from oracle import lor as olor
    from oracle.mesh import Mesh
    from paper_1908_07071_gb300.synthetic import make_mesh

    t_start = time.perf_counter()
    verts, kappa = make_mesh(3, n, seed=seed, perturb=0.15)
    m = Mesh(verts, kappa)
    rng = np.random.default_rng(0)
    t_el, n_el = 0.0, 0
    t_pa, n_pa = 0.0, 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < 0.4 * budget_s or n_el < 2:
        e = tuple(int(v) for v in rng.integers(0, n, 3))
        Ke = ocg.element_stiffness(m.corners(e), m.kappa_of(e), p)
        xe = rng.standard_normal(Ke.shape[0])
        ts = time.perf_counter()
        for _ in range(5):
            Ke @ xe
        t_el += (time.perf_counter() - ts) / 5
        n_el += 1
    t1 = time.perf_counter()
    while time.perf_counter() - t1 < 0.6 * budget_s or n_pa < 1:
        v = [int(x) for x in rng.integers(1, n, 3)]
        sub_v = verts[:, v[2] - 1:v[2] + 2, v[1] - 1:v[1] + 2, v[0] - 1:v[0] + 2].copy()
        sub_k = kappa[v[2] - 1:v[2] + 1, v[1] - 1:v[1] + 1, v[0] - 1:v[0] + 1].copy()
        B = olor.LORPreconditioner(Mesh(sub_v, sub_k), p, patch_subset=[(1, 1, 1)], coarse=False)
        pt = B.patches[0]
        r = rng.standard_normal(len(pt["levels"][0]["idx"]))
        ts = time.perf_counter()
        B.vcycle(pt["levels"], 0, r)
        t_pa += time.perf_counter() - ts
        n_pa += 1
    nel = n ** 3
    J = (n + 1) ** 3
    ndof = (n * p + 1) ** 3
    # the coarse-space correction (P_0^T r, the vertex-grid solve, P_0 e) on a Q_p mesh
    # of 4^3 elements, and two inner products plus three vector updates of 2^22
    # entries, each scaled to the workload by its unknowns (both are linear in them,
    # Section 3.6 Table 1)
    vc, kc = make_mesh(3, 4, seed=seed, perturb=0.15)
    Bc = olor.LORPreconditioner(Mesh(vc, kc), p, patch_subset=[], coarse=True)
    rc0 = rng.standard_normal(Bc.P0.shape[0])
    ts = time.perf_counter()
    for _ in range(3):
        ec = np.zeros(Bc.P0.shape[1])
        ec[Bc.vmask] = Bc.coarse_solve((Bc.P0.T @ rc0)[Bc.vmask])
        Bc.P0 @ ec
    t_co = (time.perf_counter() - ts) / 3 * ndof / Bc.P0.shape[0]
    mv = 1 << 22
    xv, yv = rng.standard_normal(mv), rng.standard_normal(mv)
    ts = time.perf_counter()
    for _ in range(3):
        xv @ yv
        xv @ yv
        for _ in range(3):
            yv += 0.5 * xv
    t_vec = (time.perf_counter() - ts) / 3 * ndof / mv
    per_it = nel * t_el / n_el + J * t_pa / n_pa + t_co + t_vec
    solve_s = iters * per_it
    return {"solve_s": solve_s, "wall_s": time.perf_counter() - t_start, "sample": f"{n_el} element applies (Q{p}, dense element matrix) and {n_pa} "
            f"interior patch V-cycles timed, extrapolated to {nel} elements + {J} patches per iteration; "
            f"the coarse-space correction (timed on Q{p} 4^3) and 2 inner products + 3 vector updates "
            f"(timed at 2^22 entries) scaled to {ndof} unknowns; x {iters} iterations", "cores": 1}


def run_cpu_leg(p, n, seed, budget_s, iters):
    """Runs the oracle sample in a single-threaded subprocess (BLAS pinned to 1 thread)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = (f"import json,sys; sys.path.insert(0, {ROOT!r}); import bench; "
            f"print(json.dumps(bench.cpu_sample_worker({p},{n},{seed},{budget_s},{iters})))")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def run_cpu_leg_all_cores(p, n, budget_s, iters, cores):
    """The same sample on every host core at once: one single-threaded process per core
    (BLAS pinned to 1 thread, seed = process index), started together; the whole-host
    throughput of independent solves is the sum of the per-process rates."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    procs = []
    for i in range(cores):
        code = (f"import json,sys; sys.path.insert(0, {ROOT!r}); import bench; "
                f"print(json.dumps(bench.cpu_sample_worker({p},{n},{i},{budget_s},{iters})))")
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    rates = []
    for pr in procs:
        out, err = pr.communicate(timeout=900)
        if pr.returncode != 0:
            raise RuntimeError(err[-2000:])
        rates.append(1.0 / json.loads(out.strip().splitlines()[-1])["solve_s"])
    return {"value": sum(rates), "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": f"{cores} concurrent single-threaded processes, each timing the single-core sample "
                      f"(seeds 0..{cores - 1}); sum of their rates"}


# ------------------------------------------------------------------- clocks
class Clocks:
    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self, dev_index=0):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9 or not f[0].isdigit() or int(f[0]) != dev_index:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------- reference arm
def reference_arm(args, rank):
    if rank != 0:
        return
    steps, walls = [], []
    res = None
    for k in range(args.warmup + args.steps):
        res = run_cpu_leg(args.p, args.n, 0, args.cpu_sample_s, REF_ITERS)
        if k >= args.warmup:
            steps.append(res["solve_s"])
            walls.append(res["wall_s"])
    # a step is one bounded sample of the workload (its wall time is ms_per_step); the
    # solves/s value extrapolates the sample to whole solves
    solve_s = statistics.mean(steps)
    value = 1.0 / solve_s
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(walls) * 1e3,
            "extrapolated_solve_s": solve_s, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "p": args.p, "n": args.n},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": res["cores"], "kind": "oracle",
                             "sample": res["sample"] + f" ({REF_ITERS} iterations per solve: the FP64 PCG count on this workload)"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ batched leg
def leg_batch(nsolves, rank):
    """256 independent CG solves (n ~ U{4..16} per axis, p ~ U{2..7}, perturbed mesh,
    log-normal kappa, seed = solve index): batched flexible CG, FP32 preconditioner,
    FP64 residual, one CUDA graph per iteration."""
    import numpy as np
    import torch
    from paper_1908_07071_gb300 import lor
    from paper_1908_07071_gb300.synthetic import batch_plan, make_mesh
    plan = batch_plan(nsolves, seed=rank, nmin=4, nmax=16, pmin=2, pmax=7)
    t0 = time.perf_counter()
    solvers, bs, xs = [], [], []
    for i, (n, p) in enumerate(plan):
        v, k = make_mesh(3, n, seed=1000 * rank + i, perturb=0.15)
        s = lor.Solver(v, k, p, rtol=1e-8, factor_bf16=True)
        b = torch.empty(s.nvec, dtype=torch.float64, device="cuda")
        s.rhs(b, 0)
        solvers.append(s)
        bs.append(b)
        xs.append(torch.zeros_like(b))
    batch = lor.Batch(solvers)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    batch.solve(bs, xs)                      # warm-up (captures the graph)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    its, rels = batch.solve(bs, xs)
    e1.record()
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    ndofs = [s.info.ndof for s in solvers]
    _, nodes = batch.stats()
    out = {"workload": f"{nsolves} solves, n~U{{4..16}}^3, p~U{{2..7}}, perturbed, log-normal kappa, rtol 1e-8",
           "time_s": t, "solves_per_s": nsolves / t,
           "dof_iterations_per_s": float(sum(d * i for d, i in zip(ndofs, its))) / t,
           "total_dofs": int(sum(ndofs)), "iterations_mean": float(np.mean(its)), "iterations_max": int(max(its)),
           "max_rel_res": float(max(rels)), "graph_nodes": nodes, "setup_s": setup_s,
           "form": "flexible CG, FP64 vectors/dots, FP32 preconditioner with bf16 ILU factors"}
    batch.close()
    for s in solvers:
        s.close()
    return out


# ----------------------------------------------------------------- DG leg
def leg_dg():
    """3D SIPG and BR2 on a 24^3 perturbed mesh, p=4, log-normal kappa: iterations of
    B_DG-preconditioned CG for eta in {1,10,100,1000} x eta_min (FP64, mixed, and mixed with
    the counting-matrix weighted patch sum), and DG per-apply throughput."""
    import torch
    from paper_1908_07071_gb300 import lor
    from paper_1908_07071_gb300.synthetic import make_mesh
    v, k = make_mesh(3, 24, seed=0, perturb=0.15)
    # eta_min: smallest eta on the grid 2^(k/4), from the probe start (SIPG: 2^(1/4),
    # coercive on the 3^3 member; BR2: the literature bound 2d = 6), for which FP64
    # PCG on this mesh does not break down (p.Ap > 0 throughout)
    start = {"ip": 2.0 ** 0.25, "br2": 6.0}
    out = {"workload": "3D DG p=4, 24^3 perturbed hex mesh, log-normal kappa, f=1, rtol 1e-8"}
    eta_min = {}
    for form, disc in (("ip", lor.LOR_DG_IP), ("br2", lor.LOR_DG_BR2)):
        rows = []
        eta0 = start[form]
        for mult in (1.0, 10.0, 100.0, 1000.0):
            while True:
                s = lor.Solver(v, k, 4, disc=disc, eta=eta0 * mult, rtol=1e-8, factor_bf16=True)
                b = torch.empty(s.nvec, dtype=torch.float64, device="cuda")
                s.rhs(b, 0)
                x = torch.zeros_like(b)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                try:
                    e0.record()
                    it, rel = s.solve(b, x)
                    e1.record()
                    torch.cuda.synchronize()
                    break
                except lor.LorError as exc:
                    s.close()
                    if mult != 1.0 or eta0 > 64 * start[form]:
                        raise exc
                    eta0 *= 2.0 ** 0.25       # not coercive yet on this mesh: next grid value
            row = {"eta": eta0 * mult, "eta_mult": mult, "iterations_fp64": it, "time_ms_fp64": e0.elapsed_time(e1)}
            s.set_prec(lor.LOR_MIXED)
            x2 = torch.zeros_like(b)
            e0.record()
            it2, rel2 = s.solve(b, x2)
            e1.record()
            torch.cuda.synchronize()
            row.update({"iterations_mixed": it2, "time_ms_mixed": e0.elapsed_time(e1), "rel_res_mixed": rel2})
            # the same mixed solve with weighted patch sums (options beyond the paper)
            for wmode, tag in ((1, "count_weighted"), (2, "pou_weighted")):
                try:
                    s.set_weighting(wmode)
                    x3 = torch.zeros_like(b)
                    e0.record()
                    it3, rel3 = s.solve(b, x3)
                    e1.record()
                    torch.cuda.synchronize()
                    row.update({f"iterations_mixed_{tag}": it3, f"time_ms_mixed_{tag}": e0.elapsed_time(e1),
                                f"rel_res_mixed_{tag}": rel3})
                except lor.LorError as exc:
                    row[f"{tag}_error"] = str(exc)
                finally:
                    s.set_weighting(0)
            if mult == 10.0:
                xa = torch.randn(s.nvec, dtype=torch.float64, device="cuda")
                ya = torch.empty_like(xa)
                per = {}
                for name, fn in (("apply_A_fp64", lambda: s.apply_A(xa, ya)),
                                 ("apply_P_fp64", lambda: s.apply_P(xa, ya))):
                    fn()
                    e0.record()
                    for _ in range(5):
                        fn()
                    e1.record()
                    torch.cuda.synchronize()
                    ms = e0.elapsed_time(e1) / 5
                    per[name] = {"ms": ms, "MDOF/s": s.nvec / (ms * 1e-3) / 1e6}
                # DG apply_A FP64 against the FP64 peak: volume sum factorization plus the
                # sum-factorized face terms, 17 contractions of (p+1)^3 multiply-adds per face
                # side (normal derivative, interpolation to and from the face points, node
                # updates) and ~10 operations per face point
                Qd, nel_dg = 5, 24 ** 3
                nface = 3 * 25 * 24 * 24
                fl = nel_dg * (24 * Qd ** 4 + 18 * Qd ** 3) + nface * (2 * 2 * 17 * Qd ** 3 + 10 * Qd ** 2)
                ach = fl / (per["apply_A_fp64"]["ms"] * 1e-3) / 1e12
                pk64 = lor.measure_fp64_peak()
                per["apply_A_fp64"]["roofline"] = {"bound": "alu", "achieved": ach, "peak": pk64, "unit": "TFLOP/s",
                                                   "frac": ach / pk64, "peak_kind": "measured (project FP64 FMA probe)",
                                                   "work": f"{fl:.4g} flop per apply"}
                row["per_apply"] = per
            rows.append(row)
            s.close()
        eta_min[form] = eta0
        out[form] = rows
    out["eta_min"] = eta_min
    return out


def leg_schwarz(n: int = 12, degrees=(2, 4, 6, 8)):
    """B(1) (the whole domain as one patch) against B(V) (one patch per vertex, additive
    coarse space) and the hybrid form (coarse space multiplicative), the comparison of
    Section 4.1 / Table 2 on the GPU: 3D CG on a 12^3 perturbed hex mesh, log-normal
    kappa, f=1, FP64 PCG to 1e-8, p in {2,4,6,8}; and DG BR2 (eta 10) at p=4 with the
    three forms inside the DG preconditioner.  Reports iterations, time to tolerance and
    milliseconds per preconditioner apply (CUDA events, 5 applies after a warm-up)."""
    import torch
    from paper_1908_07071_gb300 import lor
    from paper_1908_07071_gb300.synthetic import make_mesh
    v, k = make_mesh(3, n, seed=0, perturb=0.15)
    forms = (("B(V)", 0), ("hybrid", 1), ("B(1)", 2))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def run(s):
        b = torch.empty(s.nvec, dtype=torch.float64, device="cuda")
        s.rhs(b, 0)
        row = {}
        for name, mode in forms:
            s.set_schwarz(mode)
            x = torch.zeros_like(b)
            e0.record()
            it, rel = s.solve(b, x)
            e1.record()
            torch.cuda.synchronize()
            z = torch.empty_like(b)
            s.apply_P(b, z)
            e0.record()
            for _ in range(5):
                s.apply_P(b, z)
            e1.record()
            torch.cuda.synchronize()
            row[name] = {"iterations": it, "rel_res": rel, "time_to_tol_ms": None, "ms_per_apply": e0.elapsed_time(e1) / 5}
            x.zero_()
            e0.record()
            it, rel = s.solve(b, x)
            e1.record()
            torch.cuda.synchronize()
            row[name]["time_to_tol_ms"] = e0.elapsed_time(e1)
        s.set_schwarz(0)
        return row

    out = {"workload": f"3D CG on a {n}^3 perturbed hex mesh, log-normal kappa, f=1, FP64 PCG to 1e-8; "
                       f"DG BR2 eta=10 p=4 on the same mesh", "cg": [], "dg_br2": None}
    for p in degrees:
        s = lor.Solver(v, k, p, rtol=1e-8)
        row = {"p": p, "ndof": s.info.ndof}
        row.update(run(s))
        out["cg"].append(row)
        s.close()
    s = lor.Solver(v, k, 4, disc=lor.LOR_DG_BR2, eta=10.0, rtol=1e-8)
    out["dg_br2"] = {"p": 4, "ndof": s.info.ndof}
    out["dg_br2"].update(run(s))
    s.close()
    return out


def leg_learned(n: int = 32, p: int = 6, train_n: int = 16, steps: int = 300):
    """The learned form (configuration 5): 3D CG Q6 on a 32^3 perturbed mesh, log-normal
    kappa.  The per-patch network is trained on the GPU on a mesh of the same family
    (16^3, seed 100) by the library's own tensor-core forward/backward kernels and Adam,
    then loaded into the 32^3 context; both forms solve to 1e-8 in mixed precision (the
    learned one by flexible CG), and their time to tolerance, iterations and FP64-checked
    residuals are reported."""
    import numpy as np
    import torch
    from paper_1908_07071_gb300 import lor
    from paper_1908_07071_gb300.synthetic import learned_init_params, make_mesh
    vt, kt = make_mesh(3, train_n, seed=100, perturb=0.15)
    tr = lor.Solver(vt, kt, p, prec=lor.LOR_MIXED, rtol=1e-8, factor_bf16=True)
    tr.learned_params(learned_init_params(seed=1))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    hist = tr.learned_train(steps, batch=256, lr=2e-3, seed=5)
    e1.record()
    torch.cuda.synchronize()
    train_ms = e0.elapsed_time(e1)
    params = tr.learned_params()
    tr.close()
    v, k = make_mesh(3, n, seed=0, perturb=0.15)
    s = lor.Solver(v, k, p, prec=lor.LOR_MIXED, rtol=1e-8, factor_bf16=True)
    s.learned_params(params)
    b = torch.empty(s.nvec, dtype=torch.float64, device="cuda")
    s.rhs(b, 0)
    out = {"workload": f"3D CG Q{p}, {n}^3 perturbed hex mesh, log-normal kappa, f=1, rtol 1e-8, mixed precision",
           "ndof": s.info.ndof, "train": {"mesh": f"{train_n}^3, seed 100", "steps": steps, "batch": 256,
                                          "ms": train_ms, "loss_first5": float(np.mean(hist[:5])),
                                          "loss_last20": float(np.mean(hist[-20:]))}}
    def timed(key):
        x = torch.zeros_like(b)
        s.solve(b, x)
        x.zero_()
        e0.record()
        it, rel = s.solve(b, x)
        e1.record()
        torch.cuda.synchronize()
        out[key] = {"time_to_tol_ms": e0.elapsed_time(e1), "iterations": it, "rel_res_fp64": rel}

    for on, key in ((False, "plain"), (True, "learned")):
        s.learned_enable(on)
        timed(key)
    out["speedup_learned_vs_plain"] = out["plain"]["time_to_tol_ms"] / out["learned"]["time_to_tol_ms"]
    # replace variant: the correction takes the place of the level-0 post-smoothing;
    # trained on the same family with that cycle's pairs
    tr = lor.Solver(vt, kt, p, prec=lor.LOR_MIXED, rtol=1e-8, factor_bf16=True)
    tr.learned_variant(1)
    tr.learned_params(learned_init_params(seed=1))
    hist_r = tr.learned_train(steps, batch=256, lr=2e-3, seed=5)
    params_r = tr.learned_params()
    tr.close()
    s.learned_variant(1)
    s.learned_params(learned_init_params(seed=1))     # zero output layer: the cut cycle alone
    s.learned_enable(True)
    timed("cycle_without_level0_post_smoothing")
    s.learned_params(params_r)
    timed("replace_variant")
    out["replace_variant"]["loss_first5"] = float(np.mean(hist_r[:5]))
    out["replace_variant"]["loss_last20"] = float(np.mean(hist_r[-20:]))
    s.close()
    return out


# ----------------------------------------------------------------- our arm
def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def main():
    args = parse()
    if args.summarize_ncu:
        print(summarize_ncu_launches(args.summarize_ncu))
        return
    if args.leg:
        if args.leg == "learned":
            out = leg_learned(n=args.n, p=args.p, train_n=max(2, args.n // 2), steps=args.learned_steps)
        elif args.leg == "schwarz":
            out = leg_schwarz(n=args.n, degrees=(args.p,))
        else:
            out = leg_batch(args.batch_n, 0)
        print(json.dumps(out), flush=True)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1908_07071_gb300 import lor
    from paper_1908_07071_gb300.build import build_library
    from paper_1908_07071_gb300.synthetic import make_mesh
    if rank == 0:
        build_library()
    if world > 1:
        dist.barrier()

    p, n = args.p, args.n
    verts, kappa = make_mesh(3, n, seed=rank, perturb=0.15)
    bf16 = args.form == "mixed-bf16"
    form = lor.LOR_FP64 if args.form == "fp64" else lor.LOR_MIXED
    t_setup = time.perf_counter()
    s = lor.Solver(verts, kappa, p, prec=form, rtol=1e-8, factor_bf16=bf16, weighting=args.weighting)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup
    ndof = s.info.ndof
    b = torch.empty(s.nvec, dtype=torch.float64, device="cuda")
    s.rhs(b, 0)
    x = torch.zeros_like(b)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        s.solve(b, x)
    barrier()
    clocks = Clocks()
    clocks.start()
    l0 = s.launches()
    s.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    its, rels = [], []
    e0.record(stream)
    for _ in range(args.steps):
        it, rel = s.solve(b, x)
        its.append(it)
        rels.append(rel)
    e1.record(stream)
    barrier()
    elapsed = e0.elapsed_time(e1) / 1e3
    s.profile(False)
    launches = s.launches() - l0
    prof = {k: s.profile_read(k) for k in range(6)}
    clk = clocks.stop(local)
    elapsed = max_over_ranks(elapsed, world, device="cuda")
    ms_per_step = elapsed / args.steps * 1e3
    value = replica_throughput(elapsed, args.steps, world)

    extras = {}
    if not args.no_extras:
        # end to end through the host-buffer call (copies inside the timed region)
        hb = torch.empty(s.nvec, dtype=torch.float64).pin_memory()
        hb.copy_(b)
        hx = torch.empty_like(hb).pin_memory()
        hbn, hxn = hb.numpy(), hx.numpy()
        s.solve_host(hbn, hxn)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            s.solve_host(hbn, hxn)
        barrier()
        e2e = replica_throughput(max_over_ranks(time.perf_counter() - t0, world, device="cuda"), args.steps, world)
        extras["e2e"] = {"value": e2e, "unit": "solves/s", "h2d_bytes_per_step": int(s.nvec * 8),
                         "d2h_bytes_per_step": int(s.nvec * 8)}
        # per-apply throughput
        xa = torch.randn(s.nvec, dtype=torch.float64, device="cuda")
        ya = torch.empty_like(xa)
        xf, yf = xa.float(), torch.empty(s.nvec, dtype=torch.float32, device="cuda")
        mdofs = {}
        for name, fn in (("apply_A_fp64", lambda: s.apply_A(xa, ya)),
                         ("apply_A_fp32", lambda: s.apply_A(xf, yf, lor.LOR_FP32)),
                         ("apply_P_fp64", lambda: s.apply_P(xa, ya)),
                         ("apply_P_fp32", lambda: s.apply_P(xf, yf, lor.LOR_FP32))):
            for _ in range(2):
                fn()
            reps = 10
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            for _ in range(reps):
                fn()
            a1.record(stream)
            torch.cuda.synchronize()
            ms = a0.elapsed_time(a1) / reps
            mdofs[name] = {"ms": ms, "MDOF/s": ndof / (ms * 1e-3) / 1e6}
        extras["per_apply"] = mdofs
        # plain FP64 solve for comparison (the paper's method: unit weights)
        if form != lor.LOR_FP64 or args.weighting:
            s.set_prec(lor.LOR_FP64)
            s.set_weighting(0)
            x64 = torch.zeros_like(b)
            s.solve(b, x64)
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            it64, rel64 = s.solve(b, x64)
            f1.record(stream)
            torch.cuda.synchronize()
            s.set_prec(form)
            s.set_weighting(args.weighting)
            dx = float(torch.linalg.norm(x - x64) / torch.linalg.norm(x64))
            extras["fp64_plain"] = {"time_to_tol_ms": f0.elapsed_time(f1), "iterations": it64,
                                    "rel_res": rel64, "chosen_vs_fp64_x_rel_diff": dx,
                                    "speedup_chosen_vs_fp64": f0.elapsed_time(f1) / ms_per_step}
        # the chosen form with a weighted patch sum (options beyond the paper's unit
        # weights; context only, the headline keeps unit weights): 1 counting matrix,
        # 2 partition of unity
        for wmode, key in ((1, "count_weighted"), (2, "pou_weighted")) if args.weighting == 0 else ():
            try:
                s.set_weighting(wmode)
                xw = torch.zeros_like(b)
                s.solve(b, xw)
                w0, w1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                xw.zero_()
                w0.record(stream)
                itw, relw = s.solve(b, xw)
                w1.record(stream)
                torch.cuda.synchronize()
                extras[key] = {"time_to_tol_ms": w0.elapsed_time(w1), "iterations": itw, "rel_res": relw,
                               "speedup_vs_unit_weights": ms_per_step / w0.elapsed_time(w1)}
            except Exception as exc:   # an optional leg must not hide the main result
                extras[key] = {"error": f"{type(exc).__name__}: {exc}"}
            finally:
                try:
                    s.set_weighting(0)
                except Exception:
                    pass

    # roofline of the dominant kernel class inside the timed region
    pk = peaks()
    hbm = pk.get("hbm_gbs", 6800.0)
    fp64_peak = lor.measure_fp64_peak()   # TFLOP/s, the project's FP64 FMA probe on this GPU
    names = {0: "patch_vcycle_fp64", 1: "patch_vcycle_fp32", 2: "apply_A_fp64", 3: "apply_A_fp32",
             4: "coarse_fp64", 5: "coarse_fp32"}
    dom = max(prof, key=lambda k: prof[k][0])
    tot_ms, nl = prof[dom]
    per_launch_s = tot_ms / max(nl, 1) / 1e3
    Q = p + 1
    nel = n ** 3
    info = s.info
    rows = info.factor_rows
    if dom in (0, 1):
        fb = 8 if dom == 0 else (2 if bf16 else 4)
        vb = 8 if dom == 0 else 4
        lev_nodes = sum(((n * m + 1) ** 3) for m in level_intervals(p))
        # per factor row: L and U parts of 14 values each (13 couplings + diagonal; the stored records
        # carry 16 slots); level stencils 27 values per node; r read, z RMW
        alg = rows * 2 * 14 * fb + lev_nodes * 27 * vb + 3 * s.nvec * vb
        roof = {"bound": "hbm", "achieved": alg / per_launch_s / 1e9, "peak": hbm, "unit": "GB/s",
                "peak_kind": "measured" if "hbm_gbs" in pk else "fallback"}
    elif dom == 2:
        flops = nel * (24 * Q ** 4 + 18 * Q ** 3)
        roof = {"bound": "alu", "achieved": flops / per_launch_s / 1e12, "peak": fp64_peak, "unit": "TFLOP/s",
                "peak_kind": "measured (project FP64 FMA probe)"}
    else:
        bts = nel * 6 * Q ** 3 * (8 if dom == 4 else 4) + 3 * s.nvec * 4
        roof = {"bound": "hbm", "achieved": bts / per_launch_s / 1e9, "peak": hbm, "unit": "GB/s",
                "peak_kind": "measured" if "hbm_gbs" in pk else "fallback"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    # DRAM bytes per launch from the ncu capture of this kernel as it is built now
    # (profiles/patch_warp_q8_dram.md: one launch on Q8 12^3, scaled to 32^3 by the factor rows)
    roof["traffic"] = None
    if (names[dom], p, n, args.form, args.weighting) == ("patch_vcycle_fp32", 8, 32, "mixed-bf16", 0):
        roof["traffic"] = PATCH_TRAFFIC_Q8N32
    roof["kernel"] = names[dom]
    roof["launch_ms"] = per_launch_s * 1e3
    roof["launches_in_timed_region"] = nl
    roof["kernel_time_share"] = {names[k]: round(prof[k][0] / max(elapsed * 1e3, 1e-9), 4) for k in prof if prof[k][1]}
    # the other hot kernels against their own bounds (per-apply timings above)
    others = {}
    pa = extras.get("per_apply", {})
    if "apply_A_fp64" in pa:
        fl = nel * (24 * Q ** 4 + 18 * Q ** 3)
        ach = fl / (pa["apply_A_fp64"]["ms"] * 1e-3) / 1e12
        others["apply_A_fp64"] = {"bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                                  "frac": ach / fp64_peak, "peak_kind": "measured (project FP64 FMA probe)",
                                  "work": f"{fl:.4g} flop per apply (24 Q^4 + 18 Q^3 per element)"}
    if "apply_A_fp32" in pa:
        bts = nel * 6 * Q ** 3 * 4 + 3 * s.nvec * 4
        ach = bts / (pa["apply_A_fp32"]["ms"] * 1e-3) / 1e9
        others["apply_A_fp32"] = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                                  "peak_kind": "measured" if "hbm_gbs" in pk else "fallback",
                                  "work": f"{bts:.4g} B per apply (6 geometric factors per Gauss point, x read, y RMW)"}
    roof["others"] = others

    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+bf16/f64" if bf16 else ("f32/f64" if form != lor.LOR_FP64 else "f64"),
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "p": p, "n": n, "ndof": ndof, "form": args.form,
                       "weighting": ["unit", "counting matrix", "partition of unity"][args.weighting],
                       "l2": "working set (ILU factors, stencils) >> 129 MB L2; no flush needed",
                       "parallelism": f"replicas x{world}"},
            "iterations": its[-1], "rel_res": rels[-1], "setup_s": t_setup, "gpu_launches": launches,
            "roofline": roof, "clocks": clk}
    line.update(extras)
    if not args.no_batch:
        try:
            line["batch"] = leg_batch(args.batch_n, rank)
        except Exception as exc:   # a failing leg is reported, it does not hide the main result
            line["batch"] = {"error": f"{type(exc).__name__}: {exc}"}
    if not args.no_dg:
        try:
            line["dg"] = leg_dg()
        except Exception as exc:
            line["dg"] = {"error": f"{type(exc).__name__}: {exc}"}
    if not args.no_learned:
        try:
            line["learned"] = leg_learned()
        except Exception as exc:
            line["learned"] = {"error": f"{type(exc).__name__}: {exc}"}
    if not args.no_schwarz:
        try:
            line["schwarz"] = leg_schwarz()
        except Exception as exc:
            line["schwarz"] = {"error": f"{type(exc).__name__}: {exc}"}
    if rank == 0 and not args.no_extras:
        its64 = extras.get("fp64_plain", {}).get("iterations", 60)
        try:
            cb = run_cpu_leg(p, n, 0, args.cpu_sample_s, its64)
            line["cpu_baseline"] = {"value": 1.0 / cb["solve_s"], "unit": "solves/s", "cores": cb["cores"],
                                    "kind": "oracle", "sample": cb["sample"]}
        except Exception as exc:   # the CPU leg must not hide the GPU result
            line["cpu_baseline"] = {"value": None, "unit": "solves/s", "cores": 1, "kind": "oracle",
                                    "sample": f"failed: {exc}"}
        try:
            cores = max(1, min(os.cpu_count() or 1, 64))
            line["cpu_baseline_all_cores"] = run_cpu_leg_all_cores(p, n, args.cpu_sample_s, its64, cores)
        except Exception as exc:
            line["cpu_baseline_all_cores"] = {"error": f"{type(exc).__name__}: {exc}"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    s.close()
    if world > 1:
        dist.destroy_process_group()


def level_intervals(p):
    sels = [list(range(p + 1))]
    while len(sels[-1]) > 2:
        c = sels[-1][0::2]
        if c[-1] != sels[-1][-1]:
            c.append(sels[-1][-1])
        sels.append(c)
    return [len(s) - 1 for s in sels]


if __name__ == "__main__":
    main()
