#!/usr/bin/env python
"""Benchmark: solve time to 1e-8 relative residual, s-step vs plain, on one GB300.

Workload: the 3-D convection-diffusion system on a 128^3 interior grid
(n = 2,097,152), beta = (30, 20, 10), 7-point centred stencil, FP64,
x_true ~ U[-1, 1] from SplitMix64 seed (rank), f = A x_true, x0 = 0.
One step = one complete solve to ||f - A x|| / ||f|| <= 1e-8 with s-step GMRES
(m = 40), every kernel of the hot path included. The working set (a 42-column
basis of 16.8 MB columns) is larger than L2, so no flush is needed.

With N GPUs (torchrun) every rank solves its own system (replicas, weak
scaling); the step time is the maximum over ranks.

--impl reference times the CPU oracle (numpy FP64, one thread) on the same
system: each step is one restart cycle of its own s-step GMRES solve, and the
value is the mean cycle time times the number of cycles the oracle's solve took
(run in the same call).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "solve time to 1e-8 rel. residual & HBM GB/s vs peak; s-step vs plain, 1 GB300"
N_GRID = 128
BETA = (30.0, 20.0, 10.0)
M = 40
TOL = 1e-8


def workload(N):
    return f"3-D convection-diffusion {N}^3 (n={N ** 3:,}), beta=(30,20,10), 7-point, FP64, x0=0, tol 1e-8"


WORKLOAD = workload(N_GRID)
FP64_PEAK_TFLOPS = 2 * 152 * 2 * 2.07e9 / 1e12   # 2 DFMA/clk/SM x 152 SMs x 2.07 GHz, FMA = 2 flops


def _hbm_peak_gbs():
    """The measured copy bandwidth of this machine's GPUs (MEASURED_PEAKS.json), else the
    6800 GB/s of an earlier GB300 measurement."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6800.0


HBM_PEAK_GBS = _hbm_peak_gbs()   # the algorithmic GB/s of the dominant kernel are reported against it

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the dominant
# kernel kind, averaged over the launches of one solve, from an ncu capture of this bench
# (the profiles directory has the command and the per-kernel table). Keyed by precision
# mode ("fp64_tc": the tensor-core Gram and block-update passes; "fp64": the FP64-pipe
# kernels, SSTEP_TC_GRAM=0), with a hash of the kernel sources it was taken on: once the
# sources change, the figure no longer describes the kernel and the bench reports null.
# A "launch" is one block of the cycle, as in sstep_gmres_work: for the tensor-core path
# the projection (blocks k > 0) and the Gram pass of the s + 1 new columns together,
# (10 full cycles + the 2 blocks of the last) / 52 blocks of the 128^3 solve.
TRAFFIC = {
    "fp64": {"kernel": "block_update", "bytes_per_launch": 471.3e6,
             "sources": ("common.cuh", "kernels.cuh", "epilogue.cuh", "kernels.cu"),
             "sha256": "42dddf2a1f6c61fa"},
    "fp64_tc": {"kernel": "block_update", "bytes_per_launch": 690.7e6,
                "sources": ("ozaki.cu", "ozaki.cuh"),
                "sha256": "d9ce67d97ba559a1"},
}


def sources_sha(names):
    import hashlib

    h = hashlib.sha256()
    for nm in names:
        with open(os.path.join(ROOT, "paper_2001_04886_gb300", "csrc", nm), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(precision, kernel, tc=True):
    t = TRAFFIC.get(precision if not (precision == "fp64" and tc) else "fp64_tc")
    if not t or t["kernel"] != kernel or sources_sha(t["sources"]) != t["sha256"]:
        return None
    return t["bytes_per_launch"]


def env_ranks():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def reduce_max(value, dist, device=None):
    """Maximum of a per-rank float over all ranks (the replicas' step time); identity without dist."""
    if dist is None:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--s", type=int, default=8, help="block size of the headline s-step GMRES")
    ap.add_argument("--grid", type=int, default=N_GRID, help="side of the 3-D grid (the workload is 128)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "df64", "fp32"],
                    help="basis precision of the headline solve")
    ap.add_argument("--no-variants", action="store_true", help="the headline solve only")
    ap.add_argument("--variants", default="small,solvers,precision,batched,paper",
                    help="comma list of the extra measurements: small (the 2-D 64^2 system, s = 4, m = 20, "
                         "against GMRES(20); multi-kernel and one persistent launch), solvers (s = 2/4/8, GMRES, Orthomin, "
                         "mixed-precision bases, Newton basis, red-black ILU(0)), precision (the 256^3 "
                         "FP32-refinement form), batched (512 systems), paper (the paper's test problem, "
                         "Sec. 5), learned (the learned initial guess; minutes)")
    ap.add_argument("--learned", action="store_true", help="add 'learned' to --variants")
    ap.add_argument("--learned-train", type=int, default=20000)
    ap.add_argument("--learned-test", type=int, default=1000)
    ap.add_argument("--learned-epochs", type=int, default=24)
    ap.add_argument("--no-cpu", action="store_true")
    a = ap.parse_args()
    a.groups = set() if a.no_variants else {g.strip() for g in a.variants.split(",") if g.strip()}
    if a.learned:
        a.groups.add("learned")
    return a


# ------------------------------------------------------------------ clocks
class Clocks:
    """nvidia-smi samples of this GPU's clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_id), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
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
        os.unlink(self.path)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ algorithmic work
def cycle_steps(history, s, m, tol):
    """Krylov steps of each cycle, read off a GMRES-type history.

    The history holds, per cycle, the explicit restart residual and then one
    least-squares estimate per step, in blocks of s; a cycle stops after m steps
    or after a block whose last estimate is <= tol. The final entry is the
    restart residual that met tol.
    """
    steps, i = [], 1
    while i < len(history):
        k = 0
        while k < m and i + s <= len(history):
            i += s
            k += s
            if history[i - 1] <= tol:
                break
        steps.append(k)
        i += 1   # the next restart entry
    return steps


def sstep_gmres_work(n, dim, s, m, history, tol):
    """Algorithmic FP64 flops, bytes and launches per kernel kind of one s-step GMRES solve.

    Per kernel: the FMAs of the definition (FMA = 2 flops), the compulsory
    traffic (every array read or written once, halo re-reads excluded) and the
    launches that did work (a cycle that converges early skips the rest of its
    blocks: those launches return at once and are not counted). Block k of a
    cycle (o = k s earlier columns) costs: powers s sweeps of (2(2d+1)) flops and
    16 B per point plus the 8 B scaled start vector; Gram 2 o s flops and (o + s)
    columns; update 2 o s + (s+1)(s+2) flops, (o+s+1) columns read and s written
    (none when o = 0); next vector 2s+2 flops, s+1 columns read, 1 written.
    """
    pts = 2 * (2 * dim + 1)
    W = {k: [0.0, 0.0, 0] for k in ("stencil_powers", "gram", "block_update", "next_vector", "residual", "basis_axpy")}
    cycles = cycle_steps(history, s, m, tol)
    for steps in cycles:
        nblk = steps // s
        for k in range(nblk):
            o = k * s
            W["stencil_powers"][0] += s * pts * n
            W["stencil_powers"][1] += (s * 16 + 8) * n
            W["stencil_powers"][2] += s
            if k > 0:
                W["gram"][0] += 2 * o * s * n
                W["gram"][1] += (o + s) * 8 * n
                W["gram"][2] += 1
            W["block_update"][0] += (2 * o * s + (s + 1) * (s + 2)) * n
            W["block_update"][1] += ((o + s + 1) + (s if o > 0 else 0)) * 8 * n
            W["block_update"][2] += 1
            W["next_vector"][0] += (2 * s + 2) * n
            W["next_vector"][1] += (s + 2) * 8 * n
            W["next_vector"][2] += 1
        W["basis_axpy"][0] += 2 * nblk * s * n
        W["basis_axpy"][1] += (nblk * s + 2) * 8 * n
        W["basis_axpy"][2] += 1
    # the norm of f, one explicit residual per restart and the final check
    W["residual"][0] += (len(cycles) + 3) * (pts + 2) * n
    W["residual"][1] += (len(cycles) + 3) * 24 * n
    W["residual"][2] += len(cycles) + 2
    return W


# ------------------------------------------------------------------ oracle baseline
ORACLE_SNIPPET = r"""
import os, sys, time, json
sys.path.insert(0, {root!r})
import numpy as np
from oracle import stencil, sstep
from paper_2001_04886_gb300 import inputs
A = stencil.convdiff(({n}, {n}, {n}), {beta!r})
f = A.apply(inputs.x_true({seed}, A.n))
sigma = 1.0 / A.norm_inf()
times = []
for _ in range({reps}):
    t = time.perf_counter()
    sstep.sstep_gmres(A, f, np.zeros(A.n), {s}, {m}, {tol}, sigma, max_cycles=1)
    times.append(time.perf_counter() - t)
print(json.dumps(times))
"""


def oracle_cycle_seconds(s, reps, seed=0, threads=1, grid=N_GRID):
    """Seconds per restart cycle of the oracle's s-step GMRES in a fresh process, with its
    BLAS (the dense products of the Gram pass and the updates) on `threads` threads."""
    t = str(threads)
    env = dict(os.environ, OPENBLAS_NUM_THREADS=t, OMP_NUM_THREADS=t, MKL_NUM_THREADS=t)
    code = ORACLE_SNIPPET.format(root=ROOT, n=grid, beta=BETA, seed=seed, reps=reps, s=s, m=M, tol=TOL)
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=1800)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


# ------------------------------------------------------------------ reference arm
REFERENCE_SNIPPET = r"""
import sys, time, json
sys.path.insert(0, {root!r})
import numpy as np
from oracle import stencil, sstep
from paper_2001_04886_gb300 import inputs
A = stencil.convdiff(({n}, {n}, {n}), {beta!r})
f = A.apply(inputs.x_true({seed}, A.n))
sigma = 1.0 / A.norm_inf()
x = np.zeros(A.n)
times, solves, cyc, tsol = [], [], 0, 0.0
while len(times) < {reps} or not solves:
    t = time.perf_counter()
    r = sstep.sstep_gmres(A, f, x, {s}, {m}, {tol}, sigma, max_cycles=1)
    dt = time.perf_counter() - t
    times.append(dt)
    cyc, tsol, x = cyc + 1, tsol + dt, r["x"]
    if r["status"] == 0:
        solves.append([cyc, tsol])
        x, cyc, tsol = np.zeros(A.n), 0, 0.0
print(json.dumps({{"times": times, "solves": solves}}))
"""


def reference_arm(args):
    """The oracle's restarted s-step GMRES on the same system, run cycle by cycle.

    Each step is one restart cycle of the oracle's own solve (a restart cycle starts from
    the iterate the previous one left, so the steps in a row are the solve itself; after
    the solve converges the next step starts a new solve from x0 = 0). The run continues
    past the timed steps until one whole solve has finished. value = the mean measured
    cycle time x the number of cycles the oracle's own solve took; the first whole solve's
    measured time is reported beside it."""
    rank, world, _ = env_ranks()
    if rank != 0:
        return 0
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = REFERENCE_SNIPPET.format(root=ROOT, n=args.grid, beta=BETA, seed=0, reps=args.warmup + args.steps,
                                    s=args.s, m=M, tol=TOL)
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=3600)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    rec = json.loads(out.stdout.strip().splitlines()[-1])
    t = rec["times"][args.warmup: args.warmup + args.steps]
    cycles, solve_s = rec["solves"][0]
    ms = 1e3 * sum(t) / len(t) * cycles
    sample = (f"each step = 1 restart cycle of the numpy oracle's s-step GMRES (s={args.s}, m={M}, 1 thread), "
              f"consecutive cycles of its own solve; value = mean measured cycle time x the {cycles} cycles "
              f"the oracle's solve took; its first whole solve measured {1e3 * solve_s:.0f} ms")
    line = {
        "impl": "reference", "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * sum(t) / len(t), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload(args.grid), "method": f"oracle s-step GMRES s={args.s} m={M}", "cores": 1,
                   "step": "one restart cycle of the oracle's solve (ms_per_step); value = solve time",
                   "cycles_per_solve": cycles, "whole_solve_ms": 1e3 * solve_s},
        "cpu_baseline": {"value": ms, "unit": "ms", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ our arm
def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    rank, world, local = env_ranks()
    import numpy as np
    import torch

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    import __graft_entry__ as entry

    if rank == 0:
        entry.build()
    if dist:
        dist.barrier()
    import paper_2001_04886_gb300 as pkg
    from paper_2001_04886_gb300 import inputs

    pkg.lib()
    shape = (args.grid,) * 3
    A = pkg.StencilMatrix(3, shape, beta=BETA)
    n = A.n
    xt = torch.tensor(inputs.x_true(rank, n), dtype=torch.float64, device=dev)
    f = torch.empty_like(xt)
    A.apply(xt, f)
    x = torch.zeros_like(f)
    s = args.s

    def solve(xv, method="sstep", **kw):
        prec = kw.get("precision", "fp64")
        if method == "sstep":
            return pkg.sstep_gmres_solve(A, f, xv, kw.get("s", s), M, TOL, max_cycles=200, history_cap=8192,
                                         precision=kw.get("precision", args.precision),
                                         basis=kw.get("basis", "monomial"), precond=kw.get("precond"))
        if method == "gmres":
            return pkg.gmres_solve(A, f, xv, M, TOL, max_cycles=200, history_cap=8192, precision=prec)
        return pkg.sstep_omin_solve(A, f, xv, kw["s"], kw["k"], TOL, max_iters=20000, history_cap=8192,
                                    basis=kw.get("basis", "monomial"))

    nw = max(args.warmup, 3)
    for i in range(nw):
        if i == nw - 1:
            # the last warm-up solve is traced launch by launch: the per-kind breakdown and
            # the dominant kind, which alone is bracketed with events in the timed region
            pkg.trace_select(None)
            pkg.trace_enable(True)
        x.zero_()
        res = solve(x)
    assert res["status"] == 0, res
    breakdown = pkg.trace_read()
    pkg.trace_enable(False)
    work = sstep_gmres_work(n, 3, s, M, res["history"], TOL)
    dom = max((k for k in breakdown if k in work and breakdown[k][1] > 0), key=lambda k: breakdown[k][0])
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        gpu_id = str(local)
    clocks = Clocks(gpu_id)
    pkg.trace_select([dom])
    pkg.trace_enable(True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        x.zero_()
        res = solve(x)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1) / args.steps
    trace = pkg.trace_read()
    pkg.trace_enable(False)
    clk = clocks.stop()
    ms = reduce_max(ms, dist, dev)
    relres = res["relres"]
    err = float((x - xt).norm() / xt.norm())

    pkg.trace_select(None)
    # roofline of the dominant kernel kind (largest share of the traced warm-up solve),
    # timed by its own event pairs inside the timed region
    work = sstep_gmres_work(n, 3, s, M, res["history"], TOL)
    kinds = {k: v for k, v in trace.items() if v[1] > 0}
    t_dom = kinds[dom][0] / args.steps / 1e3             # seconds per solve
    flops, bytes_, launches_dom = work[dom]
    achieved = flops / t_dom / 1e12
    issued_dom = kinds[dom][1] / args.steps   # includes launches a converged cycle skips at once
    tc = args.precision == "fp64" and os.environ.get("SSTEP_TC_GRAM", "1") != "0"
    gbs = bytes_ / t_dom / 1e9
    common = {"kernel": dom, "launches_per_solve": launches_dom, "launches_issued_per_solve": issued_dom,
              "algorithmic_bytes_per_launch": bytes_ / launches_dom,
              "traffic": measured_traffic(args.precision, dom, tc),
              "fp64_equivalent_tflops": achieved, "fp64_peak_tflops": FP64_PEAK_TFLOPS,
              "share_of_step": kinds[dom][0] / args.steps / ms}
    if tc:
        # the Gram and block-update contractions run on the tensor cores in exact fixed point,
        # off the FP64 pipe: the roof of these streaming kernels is HBM bandwidth
        roofline = {"bound": "hbm", "achieved": gbs, "peak": HBM_PEAK_GBS, "unit": "GB/s",
                    "frac": gbs / HBM_PEAK_GBS,
                    "peak_source": "measured HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs), burst", **common}
    else:
        roofline = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP64_PEAK_TFLOPS,
                    "peak_source": "FP64: 2 DFMA/clk/SM x 152 SMs x 2070 MHz (nominal 1.25 TFLOP/s)",
                    "hbm_gbs": gbs, "hbm_peak_gbs": HBM_PEAK_GBS, "hbm_frac": gbs / HBM_PEAK_GBS, **common}

    # the comparison the metric names: standard GMRES(m) (classical Gram-Schmidt, Alg. 2.2)
    # on the same system and GPU, timed the same way
    x.zero_()
    solve(x, method="gmres")
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(3):
        x.zero_()
        rp = solve(x, method="gmres")
    e1.record(stream)
    torch.cuda.synchronize()
    plain = {"method": f"GMRES({M}), classical Gram-Schmidt", "ms": e0.elapsed_time(e1) / 3, "timed_solves": 3,
             "status": rp["status"], "cycles": rp["cycles"], "matvecs": rp["matvecs"], "relres": rp["relres"]}
    plain["ms"] = reduce_max(plain["ms"], dist, dev)

    # end to end through the public API: inputs from pinned host memory, x back to the host
    f_h = f.cpu().pin_memory()
    x_h = torch.zeros(n, dtype=torch.float64).pin_memory()
    out_h = torch.empty(n, dtype=torch.float64).pin_memory()
    f_d = torch.empty_like(f)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        f_d.copy_(f_h, non_blocking=True)
        x.copy_(x_h, non_blocking=True)
        r2 = pkg.sstep_gmres_solve(A, f_d, x, s, M, TOL, max_cycles=200, history_cap=0, precision=args.precision)
        out_h.copy_(x, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / args.steps
    assert r2["status"] == 0

    variants = {}
    if "solvers" in args.groups:
        for name, kw in [("sstep_gmres_s2", dict(method="sstep", s=2)), ("sstep_gmres_s4", dict(method="sstep", s=4)),
                         ("sstep_gmres_s8", dict(method="sstep", s=8)),
                         ("sstep_gmres_s8_newton", dict(method="sstep", s=8, basis="newton")),
                         ("sstep_gmres_s4_rbilu0", dict(method="sstep", s=4, precond="rbilu0")),
                         ("sstep_gmres_s8_rbilu0", dict(method="sstep", s=8, precond="rbilu0")),
                         ("gmres", dict(method="gmres")),
                         ("sstep_omin_s4_k1", dict(method="omin", s=4, k=1)),
                         ("sstep_omin_s4_k1_ortho", dict(method="omin", s=4, k=1, basis="ortho")),
                         ("sstep_omin_s8_k1", dict(method="omin", s=8, k=1)),
                         ("sstep_omin_s8_k1_ortho", dict(method="omin", s=8, k=1, basis="ortho")),
                         ("omin_k1", dict(method="omin", s=1, k=1)), ("omin_k7", dict(method="omin", s=1, k=7)),
                         ("df64_sstep_gmres_s4", dict(method="sstep", s=4, precision="df64")),
                         ("df64_sstep_gmres_s8", dict(method="sstep", s=8, precision="df64")),
                         ("df64_gmres", dict(method="gmres", precision="df64")),
                         ("fp32ir_sstep_gmres_s8", dict(method="sstep", s=8, precision="fp32")),
                         ("fp32ir_sstep_gmres_s8_newton", dict(method="sstep", s=8, precision="fp32",
                                                               basis="newton"))]:
            x.zero_()
            solve(x, **kw)                                  # warm the workspace
            torch.cuda.synchronize()
            e0.record(stream)
            reps = 3
            for _ in range(reps):
                x.zero_()
                rv = solve(x, **kw)
            e1.record(stream)
            torch.cuda.synchronize()
            variants[name] = {"ms": e0.elapsed_time(e1) / reps, "status": rv["status"], "cycles": rv["cycles"],
                              "iters": rv["iters"], "matvecs": rv["matvecs"], "relres": rv["relres"]}

    if "small" in args.groups:
        # the 2-D workload: 64^2 interior grid (n = 4096), beta = (20, 20), s-step GMRES with
        # s = 4, m = 20 against GMRES(20) on the same system. Its 32 KB columns sit in L2, so
        # every solve is bound by launch latency and the per-cycle host read; besides the
        # multi-kernel solvers, the batched solver runs the same system as one persistent
        # launch (one thread-block cluster, no host round trip per cycle)
        A2 = pkg.StencilMatrix(2, (64, 64), beta=(20.0, 20.0))
        xt2 = torch.tensor(inputs.x_true(rank, A2.n), dtype=torch.float64, device=dev)
        f2 = torch.empty_like(xt2)
        A2.apply(xt2, f2)
        x2 = torch.zeros_like(f2)
        small = {"workload": "2-D convection-diffusion 64^2 (n=4,096), beta=(20,20), 5-point, FP64, x0=0, tol 1e-8"}
        reps = 10
        for name, fn in (("sstep_gmres_s4_m20", lambda xv: pkg.sstep_gmres_solve(A2, f2, xv, 4, 20, TOL, max_cycles=2000,
                                                                                 history_cap=0)),
                         ("gmres_m20", lambda xv: pkg.gmres_solve(A2, f2, xv, 20, TOL, max_cycles=2000, history_cap=0))):
            x2.zero_()
            fn(x2)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(reps):
                x2.zero_()
                r2s = fn(x2)
            e1.record(stream)
            torch.cuda.synchronize()
            small[name] = {"ms": e0.elapsed_time(e1) / reps, "status": r2s["status"], "cycles": r2s["cycles"],
                           "matvecs": r2s["matvecs"], "relres": r2s["relres"]}
        for s_, name, prec in ((4, "persistent_sstep_gmres_s4_m20", "fp64"), (1, "persistent_gmres_m20_s1", "fp64"),
                               (4, "persistent_sstep_gmres_s4_m20_fp32_basis", "fp32")):
            Bs = pkg.BatchSolver([A2], s_, 20, TOL, max_cycles=2000, precision=prec)
            x2.zero_()   # tuned on the solve it will time (tune() restores this guess)
            cfg = Bs.tune([f2], [x2])
            x2.zero_()
            Bs.solve([f2], [x2])
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(reps):
                x2.zero_()
                rb = Bs.solve([f2], [x2])
            e1.record(stream)
            torch.cuda.synchronize()
            small[name] = {"ms": e0.elapsed_time(e1) / reps, "status": rb[0]["status"], "cycles": rb[0]["cycles"],
                           "matvecs": rb[0]["matvecs"], "relres": rb[0]["relres"], "tuned": cfg}
            Bs.close()
        variants["small_2d_64_s4_m20"] = small
        del A2, xt2, f2, x2

    if "precision" in args.groups:
        # the precision form: 3-D 256^3, beta = (50, 0, 0), s = 8, m = 32, to 1e-10; FP32
        # iterative refinement against the all-FP64 s-step solve
        A3 = pkg.StencilMatrix(3, (256, 256, 256), beta=(50.0, 0.0, 0.0))
        xt3 = torch.tensor(inputs.x_true(rank, A3.n), dtype=torch.float64, device=dev)
        f3 = torch.empty_like(xt3)
        A3.apply(xt3, f3)
        x3 = torch.zeros_like(f3)
        form = {}
        for prec in ("fp32", "df64", "fp64"):
            x3.zero_()
            pkg.sstep_gmres_solve(A3, f3, x3, 8, 32, 1e-10, max_cycles=400, history_cap=0, precision=prec)
            x3.zero_()
            torch.cuda.synchronize()
            e0.record(stream)
            r3 = pkg.sstep_gmres_solve(A3, f3, x3, 8, 32, 1e-10, max_cycles=400, history_cap=0, precision=prec)
            e1.record(stream)
            torch.cuda.synchronize()
            form[prec] = {"ms": e0.elapsed_time(e1), "status": r3["status"], "cycles": r3["cycles"],
                          "matvecs": r3["matvecs"], "relres": r3["relres"],
                          "x_err_vs_x_true": float((x3 - xt3).norm() / xt3.norm())}
        variants["precision_form_256cube_s8_m32_tol1e-10"] = form
        del A3, xt3, f3, x3

    if "batched" in args.groups:
        # the batched form: 512 systems, sides L ~ U{32..256}, beta ~ U[0, 50], s = 4, m = 20, tol 1e-8
        systems = inputs.batched_systems(rank, 512)
        mats, fs, xs, xts = [], [], [], []
        for sy in systems:
            Ab = pkg.StencilMatrix(2, (sy["L"], sy["L"]), beta=(sy["beta"], sy["beta"]))
            xb = torch.tensor(inputs.x_true(sy["xseed"], Ab.n), dtype=torch.float64, device=dev)
            fb = torch.empty_like(xb)
            Ab.apply(xb, fb)
            mats.append(Ab)
            fs.append(fb)
            xs.append(torch.zeros_like(fb))
            xts.append(xb)
        Bs = pkg.BatchSolver(mats, 4, 20, TOL, max_cycles=2000)
        t0 = time.perf_counter()
        cfg = Bs.tune(fs, xs)
        tune_s = time.perf_counter() - t0
        out = {"systems": 512, "unknowns": int(sum(A_.n for A_ in mats)), "tuned": cfg, "tune_s": tune_s}
        for mode, name in ((Bs.PERSISTENT, "persistent_graph"), (Bs.PER_SYSTEM, "per_system_launches")):
            for x_ in xs:
                x_.zero_()
            torch.cuda.synchronize()
            e0.record(stream)
            rb = Bs.solve(fs, xs, mode=mode)
            e1.record(stream)
            torch.cuda.synchronize()
            out[name] = {"ms": e0.elapsed_time(e1), "all_converged": all(r["status"] == 0 for r in rb),
                         "cycles_total": int(sum(r["cycles"] for r in rb)),
                         "max_relres": float(max(r["relres"] for r in rb))}
        Bs.close()
        # the same batch with the FP32 basis (FP64 residual, x and scalar work), tuned apart
        Bf = pkg.BatchSolver(mats, 4, 20, TOL, max_cycles=2000, precision="fp32")
        for x_ in xs:
            x_.zero_()   # tuned on the solve it will time (tune() restores these guesses)
        out["fp32_basis_tuned"] = Bf.tune(fs, xs)
        for x_ in xs:
            x_.zero_()
        torch.cuda.synchronize()
        e0.record(stream)
        rb = Bf.solve(fs, xs, mode=Bf.PERSISTENT)
        e1.record(stream)
        torch.cuda.synchronize()
        out["fp32_basis_persistent_graph"] = {
            "ms": e0.elapsed_time(e1), "all_converged": all(r["status"] == 0 for r in rb),
            "cycles_total": int(sum(r["cycles"] for r in rb)), "max_relres": float(max(r["relres"] for r in rb)),
            "max_x_err_vs_x_true": float(max(float((x_ - xt_).norm() / xt_.norm()) for x_, xt_ in zip(xs, xts)))}
        variants["batched_512_s4_m20"] = out
        Bf.close()
        del mats, fs, xs

    if "paper" in args.groups:
        # the paper's test problem (Sec. 5): variable coefficients, gamma = 50, beta = 1,
        # the paper's initial guess, to 1e-8 relative; Table 6.1's settings: GMRES(10),
        # 2-step GMRES(10) (the paper's 2-GMRES(5): m = 10 Krylov vectors per cycle), Omin(4)
        # and 2-step Omin(2); unpreconditioned, with the paper's ILU(0) (natural ordering,
        # hyperplane sweeps) and with the red-black ILU(0)
        paper = {}
        for Np in (64, 128, 192, 256):
            Pp = inputs.paper_problem(Np)
            Ap = pkg.StencilMatrix(2, (Np, Np), fields=[torch.tensor(c, device=dev) for c in Pp["coef"]])
            gp = torch.tensor(Pp["g"], device=dev)
            row = {}
            for name, kw in (("gmres10_rbilu0", dict(s=1, m=10, precond="rbilu0")),
                             ("sstep2_gmres10_rbilu0", dict(s=2, m=10, precond="rbilu0")),
                             ("sstep2_gmres10", dict(s=2, m=10)),
                             ("omin4", dict(omin=True, s=1, k=4)), ("sstep2_omin2", dict(omin=True, s=2, k=2)),
                             ("omin4_rbilu0", dict(omin=True, s=1, k=4, precond="rbilu0")),
                             ("sstep2_omin2_rbilu0", dict(omin=True, s=2, k=2, precond="rbilu0")),
                             ("gmres10_ilu0", dict(s=1, m=10, precond="ilu0")),
                             ("sstep2_gmres10_ilu0", dict(s=2, m=10, precond="ilu0")),
                             ("omin4_ilu0", dict(omin=True, s=1, k=4, precond="ilu0")),
                             ("sstep2_omin2_ilu0", dict(omin=True, s=2, k=2, precond="ilu0"))):
                xp = torch.tensor(Pp["x0"], device=dev)
                for rep in range(2):
                    xp.copy_(torch.tensor(Pp["x0"], device=dev))
                    torch.cuda.synchronize()
                    e0.record(stream)
                    if kw.get("omin"):
                        rp = pkg.sstep_omin_solve(Ap, gp, xp, kw["s"], kw["k"], TOL, max_iters=100000, history_cap=0,
                                                  precond=kw.get("precond"))
                    else:
                        rp = pkg.sstep_gmres_solve(Ap, gp, xp, kw["s"], kw["m"], TOL, max_cycles=20000, history_cap=0,
                                                   precond=kw.get("precond"))
                    e1.record(stream)
                    torch.cuda.synchronize()
                row[name] = {"ms": e0.elapsed_time(e1), "status": rp["status"], "cycles": rp["cycles"],
                             "iters": rp["iters"], "matvecs": rp["matvecs"],
                             "max_err_vs_analytic_u": float((xp - torch.tensor(Pp["u"], device=dev)).abs().max())}
            paper[str(Np)] = row
        variants["paper_problem_sec5"] = paper

    if "learned" in args.groups:
        from paper_2001_04886_gb300 import learned

        t0 = time.perf_counter()
        ev = learned.run(N=128, train_seeds=range(args.learned_train),
                         test_seeds=range(20000, 20000 + args.learned_test),
                         epochs=args.learned_epochs, batch=32, lr=1e-3, log=lambda m: print(m, file=sys.stderr))
        ev["total_s"] = time.perf_counter() - t0
        variants["learned_x0_128"] = ev

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        try:
            ts = oracle_cycle_seconds(s, 2, grid=args.grid)
            cycles = res["cycles"]
            cpu = {"value": 1e3 * min(ts) * cycles, "unit": "ms", "cores": 1, "kind": "oracle",
                   "sample": f"1 restart cycle of the numpy oracle's s-step GMRES (s={s}, m={M}) on the same "
                             f"system, best of 2, x {cycles} cycles of the full solve"}
            ncpu = os.cpu_count() or 1
            ta = oracle_cycle_seconds(s, 2, threads=ncpu, grid=args.grid)
            cpu["all_cores"] = {"value": 1e3 * min(ta) * cycles, "unit": "ms", "cores": ncpu,
                                "sample": "the same, with the oracle's BLAS on every host core"}
        except Exception as ex:   # the baseline is reported, never required
            cpu = {"value": None, "unit": "ms", "cores": 1, "kind": "oracle", "sample": f"failed: {ex}"[:200]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload(args.grid), "method": f"s-step GMRES s={s} m={M}, sigma=1/||A||_inf",
                       "l2": "inputs larger than L2 (basis 42 x 16.8 MB), no flush", "parallelism": f"replicas{world}",
                       "cycles": res["cycles"], "matvecs": res["matvecs"], "relres": relres,
                       "x_err_vs_x_true": err},
            "roofline": roofline,
            "plain_gmres_ms": plain["ms"],
            "speedup_vs_plain": plain["ms"] / ms,
            "plain_gmres": plain,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": 2 * 8 * n, "d2h_bytes_per_step": 8 * n},
            # every kernel of a solve is traced in the last warm-up solve; the timed solves
            # repeat the same launch sequence (the dominant kind alone is traced there)
            "gpu_launches": int(args.steps * sum(v[1] for v in breakdown.values())),
            "clocks": clk,
            "kernel_ms_per_solve": {k: v[0] for k, v in breakdown.items() if v[1] > 0},
            "kernel_algorithmic_gbs": {k: work[k][1] / (v[0] / 1e3) / 1e9 for k, v in breakdown.items()
                                       if v[1] > 0 and k in work and v[0] > 0},
            "variants": variants,
        }
        if "small_2d_64_s4_m20" in variants:   # the 2-D 64^2 workload, compact, ahead of the variants
            sm = variants["small_2d_64_s4_m20"]
            line = {**{k: v for k, v in line.items() if k != "variants"},
                    "small_2d_64_ms": {k: round(v["ms"], 3) for k, v in sm.items() if isinstance(v, dict)},
                    "variants": variants}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
