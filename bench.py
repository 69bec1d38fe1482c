#!/usr/bin/env python
"""Benchmark of the primal hybrid FEM hot path on one GB300.

Workload: the L-shaped domain [-1,1]^2 minus (0,1]^2, 32 x 32 squares per unit
square with seeded vertex jitter (0.2 h), red-refined 5 times (6,291,456
triangles, 9,441,280 edges); a = 1 + 0.5 sin(2 pi x) sin(2 pi y) averaged per
triangle at the edge midpoints, delta = 1, f = 1, u = 0 on the outer boundary,
zero flux on the two re-entrant sides.

One step = the whole path from the raw mesh to the paper's unknowns:
phfem_mesh_build (edge tables, CSR pattern) -> phfem_assemble -> phfem_solve
to a relative FP64 residual of 1e-10 (FP32 inner iterations with FP64
refinement) -> recovery of U (3 nT) and Lambda (L).  Inputs are resident in HBM
when the timed region starts; the working set (~1.5 GB) is larger than L2.
`value` = triangles / s of that step.  The FP64 path, the end-to-end variant
with host buffers, the kernel roofline and the CPU oracle are reported beside.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
With --gpus N > 1 (torchrun) every rank solves its own replica of the workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "triangles/s & solves/s, FP32+refine vs FP64 at 1e-10 rel. residual; p50/p99 ms"
UNIT = "triangles/s"
LEVELS = 5
CPU_SAMPLE_LEVEL = 2
# The dominant kernel of the FP32 iteration is the operator product with the
# direction update folded in (k_fcg_spmv_staged).  Per edge row it must
# move the values of the row (four l_es and the reaction part: 20 B), the
# preconditioned residual u and the previous direction p_old it forms p from
# (8 B), and write p and q = S p (8 B): 36 B.  The plain product y = S x needs
# values + x + y = 28 B (x read once); the four 16-bit neighbour differences
# (8 B) are index data and are reported apart.
SPMV_ALG_BYTES_PER_ROW = 20 + 4 + 4 + 4 + 4
SPMV_PLAIN_BYTES_PER_ROW = 20 + 4 + 4
SPMV_INDEX_BYTES_PER_ROW = 8


def assembly_bytes(nT, nE, nV, nD, nN, fp32=True):
    """Algorithmic bytes of the assembly (elliptic trace form with a_T, f and
    the boundary data), every array touched once:
      triangle pass: tri 12 + a_T 8 per triangle, xy 16 per vertex;
      edge pass: the edge's tables ed2el 16, lk 1, class 1, f 8 per edge, the
      boundary datum 8 on boundary edges and the length 8 on Neumann edges;
      writes the FP64 row (5 x 8), the inner row (4 l, r, 1/d in the inner
      precision) and the rhs 8 per edge.
    The 32-byte element record the triangle pass writes and the edge pass reads
    back is an intermediate of the two-pass design, not counted."""
    isz = 4 if fp32 else 8
    tri = (12 + 8) * nT + 16 * nV
    rows = (16 + 1 + 1 + 8 + 40 + 6 * isz + 8) * nE + 8 * (nD + nN) + 8 * nN
    return tri, rows


def _json_default(o):
    """NumPy scalars and arrays in the printed line."""
    import numpy as np
    if isinstance(o, np.generic):
        return o.item()
    if isinstance(o, np.ndarray):
        return o.tolist()
    raise TypeError(f"not serialisable: {type(o).__name__}")


def hbm_peak():
    """(GB/s, source) of the measured copy bandwidth, else the fallback figure."""
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        if peaks.get("hbm_gbs"):
            return float(peaks["hbm_gbs"]), "measured"
    except Exception:
        pass
    return 6800.0, "fallback"
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the product kernel at the full workload, from one ncu capture; valid only for
# the kernel source whose hash is recorded with it.
# Kernel timing inside the timed region brackets every 17th launch of each
# kernel with CUDA events (an event between two launches keeps the second from
# overlapping the first's drain, so timing every launch would slow the step).
PROFILE_EVERY = 17  # not a multiple of 4: the update kernel adds y every fourth launch
SPMV_TRAFFIC = 401.9e6
SPMV_TRAFFIC_SRC_SHA = "3db2b061050bf045"
# Warp instructions per triangle of the compensated FP32 triangle pass
# (k_asm_tri<1>), smsp__inst_executed.sum / nT from one ncu capture of the
# level-5 assembly (137,634,987 / 6,291,456); valid only for the sources whose
# hash is recorded with it.  The pass is bound by the issue rate: each SM's
# four schedulers issue one warp instruction per clock.
ASM_TRI_WARP_INST_PER_TRI = 137634987 / 6291456
ASM_TRI_SRC_SHA = "ef8c13adb824adfa"


def _function_src(path, signature):
    """Source text of one function: from its signature to the closing brace at
    column 0."""
    src = open(path).read()
    i = src.index(signature)
    j = src.index("\n}\n", i)
    return src[i:j + 3]


def _sha_spmv_src():
    """Hash of the product kernel's own source (k_fcg_spmv_staged and its
    shared-memory stage), so that the captured traffic stays valid while
    unrelated code changes."""
    cg = os.path.join(ROOT, "paper_2401_15557_gb300", "csrc", "cg.cu")
    text = (_function_src(cg, "__global__ void __launch_bounds__(kBlock) k_fcg_spmv_staged(")
            + _function_src(cg, "struct __align__(16) FStage {"))
    return hashlib.sha256(text.encode()).hexdigest()[:16]


def _sha_asm_tri_src():
    """Hash of the compensated triangle pass's source: the kernel, the record
    functions it calls and the compensated arithmetic."""
    csrc = os.path.join(ROOT, "paper_2401_15557_gb300", "csrc")
    text = (_function_src(os.path.join(csrc, "assemble.cu"), "__global__ void k_asm_tri(")
            + _function_src(os.path.join(csrc, "kernels.cuh"), "__device__ __forceinline__ void tri_record32_store(")
            + open(os.path.join(csrc, "c32.cuh")).read())
    return hashlib.sha256(text.encode()).hexdigest()[:16]


def sm_max_mhz():
    """The SM clock the GPU runs at without a throttle reason (nvidia-smi), or None."""
    import torch
    try:
        out = subprocess.run(["nvidia-smi", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits", "-i",
                              str(torch.cuda.current_device())], capture_output=True, text=True, timeout=20)
        return float(out.stdout.strip().splitlines()[0])
    except Exception:
        return None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--levels", type=int, default=LEVELS)
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--refine-steps", type=int, default=3, help="timed device refinements of the mesh (0: skip)")
    ap.add_argument("--mg-steps", type=int, default=3, help="timed steps of the multigrid variant (0: skip)")
    ap.add_argument("--asm-runs", type=int, default=20, help="event-timed assembly runs (0: skip)")
    ap.add_argument("--mg-fp64", type=int, default=1, help="also time the FP64 multigrid variant")
    ap.add_argument("--mg-nu", type=int, default=0, help="multigrid smoothing degree (0: library default)")
    ap.add_argument("--mg-ratio", type=float, default=0.0, help="multigrid smoothing interval ratio (0: default)")
    ap.add_argument("--mg-eps", type=float, default=0.0, help="multigrid coarsest reduction (0: default)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--workload", default="lshape", choices=["lshape", "batched", "heat", "serve"],
                    help="lshape: the L-shaped 6.3M-triangle solve (default); batched: 4096 meshes in one "
                         "launch; heat: Crank-Nicolson on 512 x 512 squares, 512 steps")
    ap.add_argument("--heat-n", type=int, default=512)
    ap.add_argument("--heat-mg", type=int, default=1, help="heat: also run under the multigrid preconditioner")
    ap.add_argument("--requests", type=int, default=120, help="serve: measured requests")
    ap.add_argument("--serve-modes", default="jacobi,multigrid", help="serve: request streams (jacobi, multigrid)")
    ap.add_argument("--serve-precisions", default="fp32_refined,fp64", help="serve: precisions served")
    ap.add_argument("--rates", default="", help="serve: comma-separated arrival rates of a sweep (requests/s)")
    ap.add_argument("--rate", type=float, default=200.0, help="serve: Poisson arrival rate (requests/s)")
    ap.add_argument("--slots", type=int, default=8, help="serve: worker slots")
    ap.add_argument("--batch-count", type=int, default=4096)
    ap.add_argument("--no-clocks", action="store_true",
                    help="do not sample nvidia-smi clocks (profiling runs under ncu)")
    ap.add_argument("--max-iter", type=int, default=0,
                    help="cap the CG iterations (short runs for profiling only; not a benchmark)")
    ap.add_argument("--batch-sample", type=int, default=512,
                    help="main line: meshes of the batched workload measured beside the step (0: skip)")
    ap.add_argument("--cn-steps", type=int, default=64,
                    help="main line: Crank-Nicolson steps on 512 x 512 measured beside the step (0: skip)")
    ap.add_argument("--serve-requests", type=int, default=100,
                    help="main line: measured requests of the served stream beside the step (0: skip)")
    ap.add_argument("--serve-warmup", type=int, default=20)
    ap.add_argument("--cpu-procs", type=int, default=0, help="oracle processes of the all-core CPU leg (0: nproc)")
    return ap.parse_args()


def workload(levels):
    from paper_2401_15557_gb300 import inputs as I
    mesh = I.lshape_mesh(n=32, jitter=0.2, seed=I.seed_for(1, 0), levels=levels)
    aT = I.element_mean_at_midpoints(mesh.xy, mesh.tri, I.coeff_lshape)
    return mesh, aT


def problem():
    from paper_2401_15557_gb300 import inputs as I
    return I.Problem(f=lambda x, y: 1.0 + 0 * x, g=lambda x, y, nx, ny: 0 * x, uD=lambda x, y: 0 * x, delta=1.0)


# ---------------------------------------------------------------------------
# CPU oracle (reported baseline, and the reference arm)
# ---------------------------------------------------------------------------

def oracle_step(mesh, aT, keep=None):
    from oracle import phfem_oracle as O
    t = time.perf_counter()
    r = O.solve_saddle(mesh, problem(), aT=aT)
    el = time.perf_counter() - t
    if keep is not None:
        keep["U"], keep["Lambda"] = r["U"], r["Lambda"]
    return el


def cpu_sample():
    mesh, aT = workload(CPU_SAMPLE_LEVEL)
    return mesh, aT, (f"L-shaped workload at refinement level {CPU_SAMPLE_LEVEL} ({mesh.nT} triangles): "
                      "oracle topology + saddle-point assembly + sparse direct solve (scipy SuperLU)")


def cpu_info():
    """nproc and the CPU model of this host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "hardware", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return {"nproc": os.cpu_count(), "cpu_model": model}


def _oracle_job(job):
    """One timed oracle run in a worker process (one thread): ("direct", level)
    = topology + saddle-point assembly + SuperLU; ("pcg", level) = the condensed
    edge system + plain Jacobi-PCG to 1e-10 + recovery."""
    kind, level = job
    sys.path.insert(0, ROOT)
    from oracle import phfem_oracle as O
    mesh, aT = workload(level)
    t = time.perf_counter()
    if kind == "direct":
        O.solve_saddle(mesh, problem(), aT=aT)
        info = {}
    else:
        r = O.solve_condensed(mesh, problem(), aT=aT, method="pcg", rtol=1e-10)
        info = {"iterations": int(r["info"]["iterations"]), "rel_residual": float(r["info"]["rel_residual"])}
    return time.perf_counter() - t, mesh.nT, info


def cpu_baseline_legs(procs=0):
    """The oracle on the host cores, each process single-threaded: the direct
    solve at 1 core on the level-1 and level-2 samples, the condensed
    Jacobi-PCG oracle at 1 core on level 2, and `procs` (default nproc)
    concurrent direct solves of the level-2 sample (all-core throughput).
    Processes are spawned, not forked, and start with one BLAS/OpenMP thread."""
    import concurrent.futures as cf
    import multiprocessing as mp
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    info = cpu_info()
    procs = procs or info["nproc"] or 1
    ctx = mp.get_context("spawn")
    legs = {}
    with cf.ProcessPoolExecutor(max_workers=1, mp_context=ctx) as ex:
        ex.submit(_oracle_job, ("direct", 0)).result()  # imports and first-touch outside the timing
        for lev in (1, CPU_SAMPLE_LEVEL):
            el, nT, _ = ex.submit(_oracle_job, ("direct", lev)).result()
            legs[f"direct_level{lev}_1core"] = {"triangles": nT, "s": el, "triangles_per_s": nT / el}
        el, nT, inf = ex.submit(_oracle_job, ("pcg", CPU_SAMPLE_LEVEL)).result()
        legs[f"condensed_pcg_level{CPU_SAMPLE_LEVEL}_1core"] = {"triangles": nT, "s": el, "triangles_per_s": nT / el,
                                                               **inf}
    with cf.ProcessPoolExecutor(max_workers=procs, mp_context=ctx) as ex:
        list(ex.map(_oracle_job, [("direct", 0)] * procs))  # warm every worker
        t = time.perf_counter()
        res = list(ex.map(_oracle_job, [("direct", CPU_SAMPLE_LEVEL)] * procs))
        wall = time.perf_counter() - t
    nT = res[0][1]
    legs[f"direct_level{CPU_SAMPLE_LEVEL}_all_cores"] = {"processes": procs, "triangles": nT * procs, "wall_s": wall,
                                                          "triangles_per_s": nT * procs / wall}
    return info, legs


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    mesh, aT, sample = cpu_sample()
    for _ in range(args.warmup):
        oracle_step(mesh, aT)
    times = [oracle_step(mesh, aT) for _ in range(args.steps)]
    tot = sum(times)
    v = mesh.nT * len(times) / tot
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"lshape-jitter-level{args.levels}", "sampled_level": CPU_SAMPLE_LEVEL,
                       "sampled_triangles": mesh.nT, "rtol": 1e-10,
                       "step": "oracle topology + saddle-point assembly + direct solve"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample, **cpu_info()},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line, default=_json_default), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.p = None
        self.path = os.path.join("/tmp", f"phfem_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.fh.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _gpu_setup():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    return torch.device("cuda", torch.cuda.current_device())


def batched_measure(count, steps=2, warmup=1, single_sample=32, parity=True, no_clocks=True):
    """Meshes 0..count-1 of the batched workload (unit squares with sides
    log-uniform in [8, 256], a = exp(0.5 z) from a seeded Fourier field,
    delta ~ U[0, 2], f = 1, u = 0 on x = 0, 1, zero flux on y = 0, 1):
    assembly + solve + recovery of every mesh in one persistent launch, FP32 +
    refinement and FP64 (block size from the autotuner), against the plain
    single-mesh FP64 path (assemble + solve per mesh) on the first meshes."""
    import numpy as np
    import torch
    from paper_2401_15557_gb300 import inputs as I
    from paper_2401_15557_gb300 import phfem as P
    dev = _gpu_setup()
    t0 = time.perf_counter()
    sides = I.batch_sides(4096)[:count]
    members = [I.batch_member(i, n) for i, n in enumerate(sides)]
    t_gen = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    ctx = P.phfem_ctx_create(stream)
    d = lambda a, t: torch.as_tensor(np.ascontiguousarray(a), dtype=t, device=dev)
    t0 = time.perf_counter()
    meshes = [P.phfem_mesh_build(ctx, d(m.xy, torch.float64), d(m.tri, torch.int32), d(m.dirichlet, torch.int32),
                                 d(m.neumann, torch.int32)) for m, _, _ in members]
    batch = P.phfem_batch_create(ctx, meshes)
    torch.cuda.synchronize()
    t_tables = time.perf_counter() - t0
    keep = min(single_sample, count)
    infos = [P.phfem_mesh_info_get(h) for h in meshes[:keep]]
    for h in meshes[keep:]:
        P.phfem_mesh_destroy(h)
    toff, eoff, loff = P.phfem_batch_offsets(batch, count)
    nT, nE = int(toff[-1]), int(eoff[-1])
    aT = d(np.concatenate([a for _, a, _ in members]), torch.float64)
    delta = d(np.array([dl for _, _, dl in members]), torch.float64)
    f = torch.ones(nE, dtype=torch.float64, device=dev)
    U = torch.empty(3 * nT, dtype=torch.float64, device=dev)
    L = torch.empty(int(loff[-1]), dtype=torch.float64, device=dev)
    opts = P.solve_opts(rtol=1e-10)
    out = {"meshes": count, "triangles": nT, "edges": nE, "sides": [int(sides.min()), int(sides.max())],
           "setup_s": {"host_generation": t_gen, "tables": t_tables}}
    clocks = None if no_clocks else ClockSampler(torch.cuda.current_device())
    # the launch shape is tuned for each precision (each is compared at its best shape)
    for prec, name in ((P.PHFEM_FP32_IR, "fp32_refined"), (P.PHFEM_FP64, "fp64")):
        chosen, tune_ms = P.phfem_batch_tune(batch, delta, a_T=aT, f_mid=f, precision=prec, opts=opts)
        shape = dict(block=chosen[0], cluster=chosen[1])
        res = None
        for _ in range(warmup):
            res = P.phfem_batch_solve(batch, count, delta, a_T=aT, f_mid=f, precision=prec, opts=opts, U=U, Lambda=L,
                                      **shape)
        if clocks and name == "fp32_refined":
            clocks.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            res = P.phfem_batch_solve(batch, count, delta, a_T=aT, f_mid=f, precision=prec, opts=opts, U=U, Lambda=L,
                                      **shape)
        e1.record(stream)
        torch.cuda.synchronize()
        if clocks and name == "fp32_refined":
            out["clocks"] = clocks.stop()
        ms = e0.elapsed_time(e1) / steps
        out[name] = {"ms_per_launch": ms, "solves_per_s": count * 1e3 / ms, "triangles_per_s": nT * 1e3 / ms,
                     "shape": {"block": chosen[0], "cluster": chosen[1]}, "tune_ms_per_shape": tune_ms,
                     "iterations": {"median": float(np.median(res["iterations"])), "max": int(res["iterations"].max())},
                     "converged": {"rtol": int((res["converged"] == 1).sum()), "floor": int((res["converged"] == 2).sum()),
                                   "not": int((res["converged"] == 0).sum())},
                     "rel_residual_max": float(res["rel_residual"].max())}
    # the plain FP64 single-mesh path (assemble + solve per mesh) on the first meshes
    t0 = time.perf_counter()
    tri_sample = 0
    for i in range(keep):
        m, a, dl = members[i]
        fm = torch.ones(infos[i]["nE"], dtype=torch.float64, device=dev)
        sh = P.phfem_assemble(meshes[i], fm, None, a_T=d(a, torch.float64), delta=dl, precision=P.PHFEM_FP64)
        P.phfem_solve(sh, opts)
        P.phfem_sys_destroy(sh)
        tri_sample += m.nT
    torch.cuda.synchronize()
    t_single = time.perf_counter() - t0
    out["single_mesh_fp64"] = {"meshes": keep, "triangles_per_s": tri_sample / t_single, "solves_per_s": keep / t_single}
    if parity:
        # FP32 + refinement U of the four smallest meshes against the oracle's direct saddle-point solve
        from oracle import phfem_oracle as O
        P.phfem_batch_solve(batch, count, delta, a_T=aT, f_mid=f, precision=P.PHFEM_FP32_IR, opts=opts, U=U)
        Uh = U.cpu().numpy()
        worst = 0.0
        picks = np.argsort(sides, kind="stable")[:4]
        for i in picks:
            m, a, dl = members[i]
            pb = I.Problem(f=lambda x, y: 1.0 + 0 * x, g=lambda x, y, nx, ny: 0 * x, uD=lambda x, y: 0 * x, delta=dl)
            ref = O.solve_saddle(m, pb, aT=a)
            got = Uh[3 * int(toff[i]):3 * int(toff[i + 1])]
            worst = max(worst, float(np.max(np.abs(got - ref["U"])) / np.max(np.abs(ref["U"]))))
        out["oracle_parity"] = {"meshes": [int(i) for i in picks], "U_max_rel_error": worst}
    for h in meshes[:keep]:
        P.phfem_mesh_destroy(h)
    P.phfem_batch_destroy(batch)
    P.phfem_ctx_destroy(ctx)
    return out


def run_batched(args):
    """All 4096 meshes of the batched workload (separate line)."""
    b = batched_measure(args.batch_count, steps=args.steps, warmup=args.warmup, single_sample=128,
                        parity=not args.no_cpu, no_clocks=args.no_clocks)
    g = b["fp32_refined"]
    line = {"metric": METRIC, "value": g["triangles_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": g["ms_per_launch"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"batched-{b['meshes']}-unit-squares", "meshes": b["meshes"],
                       "triangles": b["triangles"], "edges": b["edges"], "sides": b["sides"],
                       "step": "assemble+solve+recover of every mesh, one launch"},
            "solves_per_s": g["solves_per_s"], "batched": b, "clocks": b.get("clocks")}
    print(json.dumps(line, default=_json_default), flush=True)
    return 0


def heat_measure(n, steps, host=False, mg=True):
    """Crank-Nicolson for u_t - Lap u = f on the unit square, n x n squares,
    dt = 1/n: u = e^-t sin(pi x) sin(pi y), u = 0 on x = 0, 1 and the exact flux
    on y = 0, 1.  One step = right-hand side, solve to 1e-10 (warm start) and
    multiplier recovery, replayed from the captured CUDA graph (and, with
    host=True, host-driven), FP32 + refinement and FP64, Jacobi and (mg=True)
    the multigrid preconditioner over the n = n0 2^k hierarchy.  `steps` steps
    are timed after two warm-up steps; the vertex error is taken after them."""
    import numpy as np
    import torch
    from paper_2401_15557_gb300 import inputs as I
    from paper_2401_15557_gb300 import phfem as P
    dev = _gpu_setup()
    mesh = I.square_mesh(n)
    pi = np.pi
    sfun = lambda x, y: np.sin(pi * x) * np.sin(pi * y)
    ctx = P.phfem_ctx_create(torch.cuda.current_stream())
    d = lambda a, t: torch.as_tensor(np.ascontiguousarray(a), dtype=t, device=dev)
    dt = 1.0 / n
    nt = steps + 2
    phi = np.exp(-dt * np.arange(nt + 1))[None]
    t_end = dt * nt
    fsrc = lambda x, y: (2 * pi * pi - 1.0) * sfun(x, y)
    gsrc = lambda x, y, nx, ny: pi * (np.cos(pi * x) * np.sin(pi * y) * nx + np.sin(pi * x) * np.cos(pi * y) * ny)

    def data(xy, tabs):
        f0, g0 = I.edge_data(xy, tabs["ed2el"], tabs["eclass"], fsrc, gsrc, lambda x, y: 0 * x)
        w0, _ = I.edge_data(xy, tabs["ed2el"], tabs["eclass"], sfun)
        return d(f0[None], torch.float64), d(g0[None], torch.float64), d(w0, torch.float64)

    def run(sysh, F, G, W, mode, xy, tri):
        cn = P.phfem_cn_create(sysh, F, G, phi, W)
        stepf = P.phfem_cn_step_graph if mode == "graph" else P.phfem_cn_step
        stepf(cn, 2, P.solve_opts(rtol=1e-10))  # capture (graph) and warm up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = stepf(cn, steps, P.solve_opts(rtol=1e-10))
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        U = torch.empty(3 * tri.shape[0], dtype=torch.float64, device=dev)
        P.phfem_cn_read(cn, U=U)
        P.phfem_cn_destroy(cn)
        P_ = xy[tri]
        ue = np.exp(-t_end) * sfun(P_[..., 0], P_[..., 1]).ravel()
        return {"steps_per_s": steps / el, "ms_per_step": 1e3 * el / steps, "triangles_per_s": steps * tri.shape[0] / el,
                "iterations_per_step": st["iterations"] / max(1, steps), "converged": st["converged"],
                "rel_residual_max": st["rel_residual"], "max_vertex_error": float(np.max(np.abs(U.cpu().numpy() - ue)))}

    out = {"n": n, "triangles": mesh.nT, "dt": dt, "steps": steps, "t_end": t_end}
    mh = P.phfem_mesh_build(ctx, d(mesh.xy, torch.float64), d(mesh.tri, torch.int32),
                            d(mesh.dirichlet, torch.int32), d(mesh.neumann, torch.int32))
    out["edges"] = P.phfem_mesh_info_get(mh)["nE"]
    T_ = {k: v.cpu().numpy() for k, v in P.phfem_mesh_tables(mh).items()}
    F, G, W = data(mesh.xy, T_)
    for prec, name in ((P.PHFEM_FP32_IR, "fp32_refined"), (P.PHFEM_FP64, "fp64")):
        sysh = P.phfem_assemble(mh, None, None, delta=0.0, dt=dt, precision=prec)
        for mode in ("graph", "host") if host else ("graph",):
            out[f"jacobi_{name}_{mode}"] = run(sysh, F, G, W, mode, mesh.xy, mesh.tri)
        P.phfem_sys_destroy(sysh)
    P.phfem_mesh_destroy(mh)
    k = 0
    while n % (2 ** (k + 1)) == 0:
        k += 1
    if mg and k >= 1:  # the n x n square as the k-fold device refinement of an (n / 2^k)-square mesh
        m0 = I.square_mesh(n >> k)
        hs = [P.phfem_mesh_build(ctx, d(m0.xy, torch.float64), d(m0.tri, torch.int32),
                                 d(m0.dirichlet, torch.int32), d(m0.neumann, torch.int32))]
        for _ in range(k - 1):
            hs.append(P.phfem_mesh_refine(hs[-1]))
        hf, arr = P.phfem_mesh_refine(hs[-1], build=True, arrays=True)
        hs.append(hf)
        xyf, trif = arr["xy"].cpu().numpy(), arr["tri"].cpu().numpy()
        Tf = {kk: v.cpu().numpy() for kk, v in P.phfem_mesh_tables(hf).items()}
        F1, G1, W1 = data(xyf, Tf)
        for prec, name in ((P.PHFEM_FP32_IR, "fp32_refined"), (P.PHFEM_FP64, "fp64")):
            sysh = P.phfem_assemble(hf, None, None, delta=0.0, dt=dt, precision=prec)
            mgh = P.phfem_mg_create(sysh, hs)
            out["mg_levels"] = P.phfem_mg_info(mgh)["levels"]
            P.phfem_sys_set_mg(sysh, mgh)
            out[f"multigrid_{name}_graph"] = run(sysh, F1, G1, W1, "graph", xyf, trif)
            P.phfem_mg_destroy(mgh)
            P.phfem_sys_destroy(sysh)
        for h in reversed(hs):
            P.phfem_mesh_destroy(h)
    P.phfem_ctx_destroy(ctx)
    return out


def run_heat(args):
    """Crank-Nicolson on 512 x 512 squares, 512 steps (separate line)."""
    h = heat_measure(args.heat_n, args.heat_n - 2, host=True, mg=bool(args.heat_mg))
    g = h["jacobi_fp32_refined_graph"]
    line = {"metric": METRIC, "value": g["triangles_per_s"], "unit": UNIT + " (per CN step)", "n_gpus": 1,
            "steps": h["steps"], "warmup": 2, "ms_per_step": g["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"heat-cn-{h['n']}x{h['n']}", "triangles": h["triangles"], "edges": h["edges"],
                       "dt": h["dt"], "steps": h["steps"] + 2}, "cn": h}
    print(json.dumps(line, default=_json_default), flush=True)
    return 0


def serve_measure(requests, warmup, rate, slots, modes=("jacobi", "multigrid"), precisions=("fp32_refined",),
                  no_clocks=True):
    """Poisson arrivals (seeded; mean rate 200/s) of 70 % elliptic and 30 %
    Crank-Nicolson requests (16..128 steps, dt = 1/n), meshes with triangle
    counts log-uniform in [1e3, 4e6] (n x n unit squares, n = round(sqrt(nT/2))),
    a = exp(0.5 z) and delta ~ U[0, 2] as in the batched workload, f = 1,
    homogeneous boundary data, FP32 + FP64 refinement; the server admits by a
    120 GB HBM budget.  Inputs are uploaded before the arrival clock starts;
    latency = finish - submit.  The same arrival stream is served twice: with
    the meshes as given (Jacobi-PCG), and as refinement requests (the side n
    realised as n0 2^k, n0 in [4, 8), the coarse n0-square refined k times by
    the server, which then solves with the multigrid preconditioner).  Each
    stream is served in every precision of `precisions` (FP32 + refinement
    and/or FP64).  Saturated, the completion rate is the server's capacity:
    the highest arrival rate it sustains."""
    import numpy as np
    import torch
    from paper_2401_15557_gb300 import inputs as I
    from paper_2401_15557_gb300 import phfem as P
    dev = _gpu_setup()
    R = requests + warmup
    seed = I.seed_for(4, 0)
    u = I.uniform(seed ^ 0x5E5E, 4 * R)
    nT_target = np.exp(np.log(1e3) + u[0::4] * (np.log(4e6) - np.log(1e3)))
    n_target = np.sqrt(nT_target / 2)
    sides = np.maximum(2, np.rint(n_target)).astype(int)
    kinds = (u[1::4] < 0.3).astype(int)
    steps = 16 + np.floor(u[2::4] * 113).astype(int)
    arrivals = I.poisson_arrivals(R, rate, seed)
    d = lambda a, t: torch.as_tensor(np.ascontiguousarray(a), dtype=t, device=dev)
    ctx = P.phfem_ctx_create(torch.cuda.current_stream())

    def member(i):
        s_ = I.seed_for(4, i + 1)
        return I.fourier_field(s_), 2.0 * float(I.uniform(s_ ^ 0xDE17A, 1)[0])

    def a_T_device(fld, xy, tri):
        """a_T = mean of a = exp(0.5 z) at the three edge midpoints, on the device."""
        P_ = xy[tri.long()]
        mids = [0.5 * (P_[:, 1] + P_[:, 2]), 0.5 * (P_[:, 0] + P_[:, 2]), 0.5 * (P_[:, 0] + P_[:, 1])]
        acc = torch.zeros(tri.shape[0], dtype=torch.float64, device=dev)
        for mxy in mids:
            z = torch.zeros_like(acc)
            for al, (kx, ky), ph in zip(fld.alpha, fld.k, fld.phi):
                z += float(al) * torch.cos(2 * np.pi * (float(kx) * mxy[:, 0] + float(ky) * mxy[:, 1]) + float(ph))
            acc += torch.exp(0.5 * z)
        return acc / 3.0

    def build(mode):
        reqs, keep = [], []
        for i in range(R):
            fld, delta = member(i)
            if mode == "jacobi":
                m = I.square_mesh(int(sides[i]))
                levels, n_real = 0, int(sides[i])
            else:
                k = max(0, int(np.floor(np.log2(n_target[i] / 4.0)))) if n_target[i] >= 8 else 0
                n0 = max(2, int(np.rint(n_target[i] / 2 ** k)))
                m = I.square_mesh(n0)
                levels, n_real = k, n0 * 2 ** k
            t = dict(xy=d(m.xy, torch.float64), tri=d(m.tri, torch.int32), dd=d(m.dirichlet, torch.int32),
                     nn=d(m.neumann, torch.int32))
            if levels == 0:
                t["aT"] = d(I.element_mean_at_midpoints(m.xy, m.tri, fld.a), torch.float64)
                nT_fine = m.nT
            else:  # the coefficient on the refined mesh (the server refines the same way)
                h = P.phfem_mesh_build(ctx, t["xy"], t["tri"], t["dd"], t["nn"])
                hs = [h]
                for _ in range(levels - 1):
                    hs.append(P.phfem_mesh_refine(hs[-1]))
                arr = P.phfem_mesh_refine(hs[-1], build=False, arrays=True)
                for hh in reversed(hs):
                    P.phfem_mesh_destroy(hh)
                t["aT"] = a_T_device(fld, arr["xy"], arr["tri"])
                nT_fine = arr["tri"].shape[0]
                del arr
            t["U"] = torch.empty(3 * nT_fine, dtype=torch.float64, device=dev)
            rq = P.make_request(t["xy"], t["tri"], t["dd"], t["nn"], kind=int(kinds[i]), a_T=t["aT"], delta=delta,
                                f=1.0, dt=1.0 / n_real, steps=int(steps[i]), precision=P.PHFEM_FP32_IR,
                                U_out=t["U"], levels=levels)
            reqs.append((rq, nT_fine))
            keep.append(t)
        torch.cuda.synchronize()
        return reqs, keep

    def serve(reqs):
        srv = P.phfem_server_create(slots, 120e9, P.solve_opts(rtol=1e-10))
        clocks = ClockSampler(torch.cuda.current_device()) if not no_clocks else None
        if clocks:
            clocks.start()
        start = time.perf_counter()
        ids = []
        for (rq, _), ta in zip(reqs, arrivals):
            delay = ta - (time.perf_counter() - start)
            if delay > 0:
                time.sleep(delay)
            ids.append(P.phfem_server_submit(srv, rq))
        P.phfem_server_drain(srv)
        clk = clocks.stop() if clocks else None
        res = [P.phfem_server_poll(srv, i, wait=False) for i in ids]
        P.phfem_server_destroy(srv)
        meas = res[warmup:]
        lat = np.array([r["t_finish"] - r["t_submit"] for r in meas]) * 1e3
        wait = np.array([r["t_admit"] - r["t_submit"] for r in meas]) * 1e3
        span = max(r["t_finish"] for r in meas) - min(r["t_submit"] for r in meas)
        tri = sum(nt for (_, nt) in reqs[warmup:])
        ok = sum(1 for r in meas if r["status"] == 0)
        return {"solves_per_s": ok / span, "span_s": span, "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "mean_queue_wait_ms": float(wait.mean()),
                "triangles_per_s": tri / span, "ok": ok, "failed": len(meas) - ok,
                "offered_triangles_per_s": tri / (arrivals[-1] - arrivals[warmup]) if len(meas) > 1 else None,
                "offered_requests_per_s": (len(meas) - 1) / (arrivals[-1] - arrivals[warmup]) if len(meas) > 1 else None,
                "iterations_median": float(np.median([r["iterations"] for r in meas])), "clocks": clk}

    out = {"requests": requests, "warmup": warmup, "rate_per_s": rate, "slots": slots, "hbm_budget_gb": 120,
           "mix": "70% elliptic / 30% Crank-Nicolson 16-128 steps", "triangles": "log-uniform 1e3..4e6"}
    pmap = {"fp32_refined": P.PHFEM_FP32_IR, "fp64": P.PHFEM_FP64}
    for mode in modes:
        t0 = time.perf_counter()
        reqs, keep = build(mode)
        t_setup = time.perf_counter() - t0
        for pname in precisions:
            for rq, _ in reqs:
                rq.precision = pmap[pname]
            r = serve(reqs)
            r["setup_s"] = t_setup
            r["saturated"] = bool(r["offered_requests_per_s"] is not None
                                  and r["solves_per_s"] < 0.9 * r["offered_requests_per_s"])
            out[f"{mode}_{pname}"] = r
        del keep
        torch.cuda.empty_cache()
    P.phfem_ctx_destroy(ctx)
    return out


def run_serve(args):
    """The request stream of the serving workload (separate line); with --rates
    a sweep of arrival rates, whose knee is the highest rate the server keeps
    up with."""
    modes = tuple(m for m in args.serve_modes.split(",") if m)
    precs = tuple(p for p in args.serve_precisions.split(",") if p)
    sv = serve_measure(args.requests, args.warmup, args.rate, args.slots, modes=modes, precisions=precs,
                       no_clocks=args.no_clocks)
    sweep = []
    for r in [float(x) for x in args.rates.split(",") if x]:
        one = serve_measure(args.requests, args.warmup, r, args.slots, modes=modes[-1:], precisions=precs[:1],
                            no_clocks=True)
        key = f"{modes[-1]}_{precs[0]}"
        res = one[key]
        sweep.append({"rate_per_s": r, "mode": key, "solves_per_s": res["solves_per_s"], "p50_ms": res["p50_ms"],
                      "p99_ms": res["p99_ms"], "saturated": res["saturated"],
                      "offered_requests_per_s": res["offered_requests_per_s"]})
    head = sv[f"{modes[0]}_{precs[0]}"]
    line = {"metric": METRIC, "value": head["solves_per_s"], "unit": "solves/s", "n_gpus": 1, "steps": args.requests,
            "warmup": args.warmup, "ms_per_step": 1e3 * head["span_s"] / args.requests, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "serve-poisson", "rate_per_s": args.rate, "requests": args.requests,
                       "slots": args.slots, "hbm_budget_gb": 120, "modes": list(modes), "precisions": list(precs)},
            "p50_ms": head["p50_ms"], "p99_ms": head["p99_ms"], "serve": sv, "rate_sweep": sweep,
            "clocks": head["clocks"]}
    if sweep:
        ok = [x["rate_per_s"] for x in sweep if not x["saturated"]]
        line["knee_requests_per_s"] = max(ok) if ok else None
    print(json.dumps(line, default=_json_default), flush=True)
    return 0


class Ranks:
    """The processes of one launch: one per GPU under torchrun (RANK, WORLD_SIZE,
    LOCAL_RANK, MASTER_ADDR/PORT from the environment), or a single process.
    Replicas run the same workload with no collective on the data path; the
    launch only synchronises and takes the slowest rank's time."""

    def __init__(self, backend="nccl"):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.backend = backend
        self.dist = None
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend)
            self.dist = dist

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def max(self, v, device=None):
        """The largest v over the ranks (every rank gets it)."""
        if self.dist is None:
            return v
        import torch
        t = torch.tensor([float(v)], dtype=torch.float64, device=device if self.backend == "nccl" else "cpu")
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()
            self.dist = None


def weak_throughput(world, units_per_rank, ms_slowest):
    """Whole-job throughput of `world` replicas that each processed
    units_per_rank units, over the slowest rank's time."""
    return world * units_per_rank * 1e3 / ms_slowest


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "heat":
        return run_heat(args)
    if args.workload == "serve":
        return run_serve(args)

    import numpy as np
    import torch

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    ranks = Ranks("nccl")
    world, rank = ranks.world, ranks.rank

    import __graft_entry__
    __graft_entry__.build()
    from paper_2401_15557_gb300 import phfem as P

    dev = torch.device("cuda", torch.cuda.current_device())
    mesh, aT = workload(args.levels)
    d = lambda a, t: torch.as_tensor(np.ascontiguousarray(a), dtype=t, device=dev)
    xy, tri = d(mesh.xy, torch.float64), d(mesh.tri, torch.int32)
    dd, nn, a = d(mesh.dirichlet, torch.int32), d(mesh.neumann, torch.int32), d(aT, torch.float64)
    stream = torch.cuda.current_stream()
    ctx = P.phfem_ctx_create(stream)
    m0 = P.phfem_mesh_build(ctx, xy, tri, dd, nn)
    info = P.phfem_mesh_info_get(m0)
    P.phfem_mesh_destroy(m0)
    nT, nE, nL = info["nT"], info["nE"], info["nL"]
    f_mid = torch.ones(nE, dtype=torch.float64, device=dev)   # f = 1 at every midpoint
    bc_mid = torch.zeros(nE, dtype=torch.float64, device=dev)  # u_D = 0, g = 0
    U = torch.empty(3 * nT, dtype=torch.float64, device=dev)
    Lam = torch.empty(nL, dtype=torch.float64, device=dev)
    opts = P.solve_opts(rtol=1e-10, max_iter=args.max_iter)

    def ev():
        return torch.cuda.Event(enable_timing=True)

    def step(prec, phases=None, inputs=None):
        X, T_, D_, N_, A_, F_, B_ = inputs or (xy, tri, dd, nn, a, f_mid, bc_mid)
        e0, e1, e2, e3 = ev(), ev(), ev(), ev()
        e0.record(stream)
        m = P.phfem_mesh_build(ctx, X, T_, D_, N_)
        e1.record(stream)
        s = P.phfem_assemble(m, F_, B_, a_T=A_, delta=1.0, precision=prec)
        e2.record(stream)
        st = P.phfem_solve(s, opts, U=U, Lambda=Lam, raise_on_noconv=args.max_iter == 0)
        e3.record(stream)
        P.phfem_sys_destroy(s)
        P.phfem_mesh_destroy(m)
        if phases is not None:
            phases.append((e0, e1, e2, e3, st))
        return st

    barrier = ranks.barrier

    def max_over_ranks(v):
        return ranks.max(v, device=dev)

    # ---- main timed region: FP32 inner + FP64 refinement ------------------
    for _ in range(args.warmup):
        step(P.PHFEM_FP32_IR)
    torch.cuda.synchronize()
    for k in ("cg_spmv", "cg_update", "cg_dir", "residual", "asm_tri", "asm_rows", "recover"):
        P.phfem_ctx_kernel_time(ctx, k, reset=True)
    P.phfem_ctx_profile(ctx, PROFILE_EVERY)
    launches0 = P.phfem_ctx_launches(ctx)
    clocks = ClockSampler(torch.cuda.current_device()) if not args.no_clocks else None
    phases = []
    barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    t_start, t_stop = ev(), ev()
    t_start.record(stream)
    for _ in range(args.steps):
        step(P.PHFEM_FP32_IR, phases)
    t_stop.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop() if clocks else None
    P.phfem_ctx_profile(ctx, False)
    launches = P.phfem_ctx_launches(ctx) - launches0
    ms_total = max_over_ranks(t_start.elapsed_time(t_stop))
    ms_step = ms_total / args.steps
    ktimes = {k: P.phfem_ctx_kernel_time(ctx, k, reset=True)
              for k in ("cg_spmv", "cg_update", "cg_dir", "residual", "asm_tri", "asm_rows", "recover")}
    ph = {"mesh_build": [], "assemble": [], "solve_recover": []}
    iters, refs, rel, conv = [], [], [], []
    for e0, e1, e2, e3, st in phases:
        ph["mesh_build"].append(e0.elapsed_time(e1))
        ph["assemble"].append(e1.elapsed_time(e2))
        ph["solve_recover"].append(e2.elapsed_time(e3))
        iters.append(st["iterations"])
        refs.append(st["refinements"])
        rel.append(st["rel_residual"])
        conv.append(st["converged"])
    value = weak_throughput(world, nT, ms_step)

    # ---- FP64 path ----------------------------------------------------------
    fp64 = None
    if args.fp64_steps > 0:
        step(P.PHFEM_FP64)
        torch.cuda.synchronize()
        a0, a1 = ev(), ev()
        ph64 = []
        a0.record(stream)
        for _ in range(args.fp64_steps):
            step(P.PHFEM_FP64, ph64)
        a1.record(stream)
        torch.cuda.synchronize()
        ms64 = max_over_ranks(a0.elapsed_time(a1)) / args.fp64_steps
        fp64 = {"value": weak_throughput(world, nT, ms64), "unit": UNIT, "ms_per_step": ms64,
                "solves_per_s": world * 1e3 / ms64, "iterations": ph64[-1][4]["iterations"],
                "rel_residual": ph64[-1][4]["rel_residual"], "converged": ph64[-1][4]["converged"]}

    # ---- end to end from pinned host buffers ---------------------------------
    e2e = None
    if args.e2e_steps > 0:
        pin = lambda t: t.cpu().pin_memory()
        host_in = [pin(t) for t in (xy, tri, dd, nn, a, f_mid, bc_mid)]
        host_U = torch.empty(3 * nT, dtype=torch.float64).pin_memory()
        host_L = torch.empty(nL, dtype=torch.float64).pin_memory()
        dev_in = [torch.empty_like(t, device=dev) for t in host_in]
        h2d = sum(t.numel() * t.element_size() for t in host_in)
        d2h = host_U.numel() * 8 + host_L.numel() * 8

        def e2e_step():
            for dt_, ht in zip(dev_in, host_in):
                dt_.copy_(ht, non_blocking=True)
            step(P.PHFEM_FP32_IR, inputs=dev_in)
            host_U.copy_(U, non_blocking=True)
            host_L.copy_(Lam, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            e2e_step()
        torch.cuda.synchronize()
        barrier()
        ms_e2e = max_over_ranks(1e3 * (time.perf_counter() - t0)) / args.e2e_steps
        e2e = {"value": weak_throughput(world, nT, ms_e2e), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": ms_e2e}

    # ---- assembly alone: median of 20 event-timed runs after warm-up ------------
    asm20 = None
    if args.asm_runs > 0:
        mA = P.phfem_mesh_build(ctx, xy, tri, dd, nn)
        res = {}
        for prec, name in ((P.PHFEM_FP32_IR, "fp32_refined"), (P.PHFEM_FP64, "fp64")):
            for _ in range(3):
                P.phfem_sys_destroy(P.phfem_assemble(mA, f_mid, bc_mid, a_T=a, delta=1.0, precision=prec))
            times = []
            for _ in range(args.asm_runs):
                e0, e1 = ev(), ev()
                e0.record(stream)
                sA = P.phfem_assemble(mA, f_mid, bc_mid, a_T=a, delta=1.0, precision=prec)
                e1.record(stream)
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
                P.phfem_sys_destroy(sA)
            mt = statistics.median(times)
            # the same runs again with every launch of the two kernels event-timed
            for k in ("asm_tri", "asm_rows"):
                P.phfem_ctx_kernel_time(ctx, k, reset=True)
            P.phfem_ctx_profile(ctx, True)
            for _ in range(args.asm_runs):
                P.phfem_sys_destroy(P.phfem_assemble(mA, f_mid, bc_mid, a_T=a, delta=1.0, precision=prec))
            torch.cuda.synchronize()
            P.phfem_ctx_profile(ctx, False)
            bt, br = assembly_bytes(nT, nE, xy.shape[0], info["nD"], info["nN"], fp32=prec == P.PHFEM_FP32_IR)
            kern = {}
            for k, nb in (("asm_tri", bt), ("asm_rows", br)):
                kms, kn = P.phfem_ctx_kernel_time(ctx, k, reset=True)
                avg = kms / max(kn, 1)
                kern[k] = {"ms": avg, "bytes": nb, "achieved_gbs": nb / (avg * 1e-3) / 1e9}
            t2 = kern["asm_tri"]["ms"] + kern["asm_rows"]["ms"]
            pk, pk_src = hbm_peak()
            kern["asm_rows"]["roofline"] = {"bound": "hbm", "achieved": kern["asm_rows"]["achieved_gbs"], "peak": pk,
                                            "unit": "GB/s", "frac": kern["asm_rows"]["achieved_gbs"] / pk}
            mhz = sm_max_mhz()
            if prec == P.PHFEM_FP32_IR and mhz and ASM_TRI_SRC_SHA == _sha_asm_tri_src():
                sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
                inst = ASM_TRI_WARP_INST_PER_TRI * nT / (kern["asm_tri"]["ms"] * 1e-3) / 1e9
                peak_i = 4 * sms * mhz * 1e-3
                kern["asm_tri"]["roofline"] = {"bound": "alu", "achieved": inst, "peak": peak_i,
                                               "unit": "G warp instructions/s", "frac": inst / peak_i,
                                               "warp_instructions_per_triangle": ASM_TRI_WARP_INST_PER_TRI,
                                               "peak_source": f"{sms} SMs x 4 schedulers x 1 warp instruction "
                                                              f"per clock at {mhz:.0f} MHz"}
            ach = (bt + br) / (t2 * 1e-3) / 1e9
            res[name] = {"ms": mt, "triangles_per_s": nT * 1e3 / mt, "kernels": kern,
                         "roofline": {"bound": "hbm", "achieved": ach, "peak": pk, "unit": "GB/s",
                                      "frac": ach / pk, "peak_source": pk_src,
                                      "algorithmic_bytes": bt + br, "kernels_ms": t2}}
        P.phfem_mesh_destroy(mA)
        asm20 = {"runs": args.asm_runs, **res,
                 "note": "phfem_assemble alone (allocation, a3-a6 kernels, coefficient check); "
                         "kernels: mean of event-timed launches; roofline: algorithmic bytes of the two "
                         "kernels (without the element record written and read back) over their summed time"}

    # ---- multigrid-preconditioned variant of the same step ----------------------
    # The level-0 mesh is refined on the device (the paper's refinement gives
    # the generator's triangles in the same order, so a_T carries over); the
    # step adds the refinements and the multigrid setup to the Jacobi step.
    mgres = None
    if args.mg_steps > 0:
        from paper_2401_15557_gb300 import inputs as I
        m0 = I.lshape_mesh(n=32, jitter=0.2, seed=I.seed_for(1, 0), levels=0)
        X0, T0 = d(m0.xy, torch.float64), d(m0.tri, torch.int32)
        D0, N0 = d(m0.dirichlet, torch.int32), d(m0.neumann, torch.int32)
        U_mg = torch.empty_like(U)
        opts_mg = P.solve_opts(rtol=1e-10)
        Lam_mg = torch.empty_like(Lam)

        def mg_step(prec, phases=None):
            e0, e1, e2, e3 = ev(), ev(), ev(), ev()
            e0.record(stream)
            hs = [P.phfem_mesh_build(ctx, X0, T0, D0, N0)]
            for _ in range(args.levels):
                hs.append(P.phfem_mesh_refine(hs[-1]))
            e1.record(stream)
            s_ = P.phfem_assemble(hs[-1], f_mid, bc_mid, a_T=a, delta=1.0, precision=prec)
            mg = P.phfem_mg_create(s_, hs, a_T=a, nu=args.mg_nu, smooth_ratio=args.mg_ratio, coarse_eps=args.mg_eps)
            P.phfem_sys_set_mg(s_, mg)
            e2.record(stream)
            st_ = P.phfem_solve(s_, opts_mg, U=U_mg, Lambda=Lam_mg)
            e3.record(stream)
            info_mg = P.phfem_mg_info(mg)
            P.phfem_mg_destroy(mg)
            P.phfem_sys_destroy(s_)
            for h in reversed(hs):
                P.phfem_mesh_destroy(h)
            if phases is not None:
                phases.append((e0, e1, e2, e3, st_, info_mg))
            return st_

        # the device-refined triangles are the generator's, in the same order
        hs = [P.phfem_mesh_build(ctx, X0, T0, D0, N0)]
        for _ in range(args.levels - 1):
            hs.append(P.phfem_mesh_refine(hs[-1]))
        _, arr = P.phfem_mesh_refine(hs[-1], build=True, arrays=True)
        P.phfem_mesh_destroy(_)
        same = bool(torch.equal(arr["xy"][arr["tri"].long()], xy[tri.long()]))
        for h in reversed(hs):
            P.phfem_mesh_destroy(h)
        del arr
        mg_out = {}
        precs = ((P.PHFEM_FP32_IR, "fp32_refined"), (P.PHFEM_FP64, "fp64"))[:2 if args.mg_fp64 else 1]
        for prec, name in precs:
            for _ in range(args.warmup):
                mg_step(prec)
            torch.cuda.synchronize()
            phm = []
            g0, g1 = ev(), ev()
            g0.record(stream)
            for _ in range(args.mg_steps):
                mg_step(prec, phm)
            g1.record(stream)
            torch.cuda.synchronize()
            msm = max_over_ranks(g0.elapsed_time(g1)) / args.mg_steps
            last = phm[-1]
            mg_out[name] = {
                "value": weak_throughput(world, nT, msm), "unit": UNIT, "ms_per_step": msm, "solves_per_s": world * 1e3 / msm,
                "iterations": last[4]["iterations"], "refinements": last[4]["refinements"],
                "rel_residual": last[4]["rel_residual"], "converged": last[4]["converged"],
                "phases_ms_median": {
                    "mesh_build_and_refine": statistics.median(p_[0].elapsed_time(p_[1]) for p_ in phm),
                    "assemble_and_mg_setup": statistics.median(p_[1].elapsed_time(p_[2]) for p_ in phm),
                    "solve_recover": statistics.median(p_[2].elapsed_time(p_[3]) for p_ in phm)},
                "mg": last[5]}
        torch.cuda.synchronize()
        du = float((U_mg - U).abs().max() / U.abs().max())
        mgres = {"workload": f"lshape-jitter-level{args.levels} from level 0 refined on the device",
                 "same_triangles_as_main": same, "max_rel_diff_U_vs_jacobi": du, **mg_out,
                 "step": "mesh_build(level 0)+refine x5+assemble+multigrid setup+solve+recover"}

    # ---- device red refinement of the level-L mesh (Section 2.3) --------------
    refine = None
    if args.refine_steps > 0:
        mL = P.phfem_mesh_build(ctx, xy, tri, dd, nn)
        fine = P.phfem_mesh_refine(mL)  # warm-up (allocations)
        P.phfem_mesh_destroy(fine)
        torch.cuda.synchronize()
        r0, r1 = ev(), ev()
        r0.record(stream)
        for _ in range(args.refine_steps):
            fine = P.phfem_mesh_refine(mL)
            P.phfem_mesh_destroy(fine)
        r1.record(stream)
        torch.cuda.synchronize()
        ms_ref = r0.elapsed_time(r1) / args.refine_steps
        refine = {"from_triangles": nT, "to_triangles": 4 * nT, "ms": ms_ref,
                  "refined_triangles_per_s": 4 * nT * 1e3 / ms_ref,
                  "step": "phfem_mesh_refine: refined arrays and their tables in closed form"}
        P.phfem_mesh_destroy(mL)

    # ---- roofline of the dominant kernel (the product kernel) -----------------
    spmv_ms, spmv_n = ktimes["cg_spmv"]
    peak, peak_src = hbm_peak()
    roof = None
    if spmv_n:
        avg = spmv_ms / spmv_n * 1e-3
        alg = SPMV_ALG_BYTES_PER_ROW * nE
        achieved = alg / avg / 1e9
        traffic = SPMV_TRAFFIC if SPMV_TRAFFIC_SRC_SHA == _sha_spmv_src() else None
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": "k_fcg_spmv_staged (fused FP32 product)", "peak_source": peak_src,
                "algorithmic_bytes_per_launch": alg, "algorithmic_bytes_per_row": SPMV_ALG_BYTES_PER_ROW,
                "index_bytes_per_row": SPMV_INDEX_BYTES_PER_ROW, "avg_launch_ms": avg * 1e3,
                "plain_product_bytes_per_row": SPMV_PLAIN_BYTES_PER_ROW,
                "frac_plain_product_bytes": SPMV_PLAIN_BYTES_PER_ROW * nE / avg / 1e9 / peak,
                "note": "algorithmic bytes: values 20 + u 4 + p_old 4 + p 4 + q 4 per row (the direction update is "
                        "folded into the product); frac_plain_product_bytes counts values + x + y = 28 B only"}
        if traffic:
            roof["traffic_over_algorithmic"] = traffic / alg

    tot_k = sum(v[0] for v in ktimes.values())
    kernel_share = {k: {"ms_timed": v[0], "timed_launches": v[1], "share": v[0] / tot_k if tot_k else None}
                    for k, v in ktimes.items()}
    kernel_share["timed"] = f"every {PROFILE_EVERY}th launch of each kernel"

    # ---- CPU oracle on bounded samples ----------------------------------------
    cpu = None
    parity = None
    if rank == 0 and not args.no_cpu:
        cm, caT, sample = cpu_sample()
        ref = {}
        oracle_step(cm, caT, keep=ref)  # the solution the parity check below compares with
        hinfo, legs = cpu_baseline_legs(args.cpu_procs)
        one = legs[f"direct_level{CPU_SAMPLE_LEVEL}_1core"]
        cpu = {"value": one["triangles_per_s"], "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
               **hinfo, "legs": legs,
               "size_trend": "the direct solve's fill grows like n^1.5 and the PCG iterations like n^0.5, "
                             "so the oracle's triangles/s falls with mesh size (level 1 vs level 2 above)"}
        # the same sample through the CUDA path: forward errors against the oracle's
        # solution and the CSR pattern against the oracle's condensed system
        from oracle import phfem_oracle as O
        cs = O.condensed_system(cm, problem(), aT=caT)
        mh = P.phfem_mesh_build(ctx, d(cm.xy, torch.float64), d(cm.tri, torch.int32),
                                d(cm.dirichlet, torch.int32), d(cm.neumann, torch.int32))
        ci = P.phfem_mesh_info_get(mh)
        tabs = P.phfem_mesh_tables(mh)
        pattern = bool(np.array_equal(tabs["row_ptr"].cpu().numpy(), cs["S"].indptr)
                       and np.array_equal(tabs["col"].cpu().numpy(), cs["S"].indices))
        parity = {"sample": f"level {CPU_SAMPLE_LEVEL} ({cm.nT} triangles)", "csr_pattern_bit_exact": pattern}
        for prec, name in ((P.PHFEM_FP32_IR, "fp32_refined"), (P.PHFEM_FP64, "fp64")):
            sh = P.phfem_assemble(mh, torch.ones(ci["nE"], dtype=torch.float64, device=dev),
                                  torch.zeros(ci["nE"], dtype=torch.float64, device=dev),
                                  a_T=d(caT, torch.float64), delta=1.0, precision=prec)
            Uc = torch.empty(3 * ci["nT"], dtype=torch.float64, device=dev)
            Lc = torch.empty(ci["nL"], dtype=torch.float64, device=dev)
            stc = P.phfem_solve(sh, P.solve_opts(rtol=1e-10), U=Uc, Lambda=Lc)
            P.phfem_sys_destroy(sh)
            eu = float(np.max(np.abs(Uc.cpu().numpy() - ref["U"])) / np.max(np.abs(ref["U"])))
            el = float(np.max(np.abs(Lc.cpu().numpy() - ref["Lambda"])) / np.max(np.abs(ref["Lambda"])))
            parity[name] = {"U_max_rel_error": eu, "Lambda_max_rel_error": el, "rel_residual": stc["rel_residual"]}
        P.phfem_mesh_destroy(mh)

    # ---- the batched, Crank-Nicolson and served forms (compact samples) -----------
    forms = {}
    if rank == 0:
        if args.batch_sample > 0:
            forms["batched"] = batched_measure(args.batch_sample, steps=2, warmup=1, single_sample=16,
                                               parity=not args.no_cpu)
            forms["batched"]["sample"] = (f"meshes 0..{args.batch_sample - 1} of the 4096-mesh batched workload; "
                                          "FP32 + refinement and FP64 in one persistent launch each, the launch "
                                          "shape tuned for each, the plain single-mesh FP64 path on the first 16")
        if args.cn_steps > 0:
            forms["heat_cn"] = heat_measure(args.heat_n, args.cn_steps, host=False, mg=True)
            forms["heat_cn"]["sample"] = (f"{args.cn_steps} of the 512 Crank-Nicolson steps on 512 x 512 squares, "
                                          "graph-captured, FP32 + refinement and FP64, Jacobi and multigrid")
        if args.serve_requests > 0:
            forms["serve"] = serve_measure(args.serve_requests, args.serve_warmup, args.rate, args.slots,
                                           modes=("multigrid",), precisions=("fp32_refined", "fp64"))
            forms["serve"]["sample"] = (f"{args.serve_requests} measured requests after {args.serve_warmup} of the "
                                        "Poisson stream (200/s), served as refinement requests with the multigrid "
                                        "preconditioner; completion rate = capacity when saturated")

    if rank == 0:
        med = lambda v: statistics.median(v) if v else None
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"lshape-jitter-level{args.levels}", "triangles": nT, "edges": nE,
                       "free_edges": info["nF"], "nnz": info["nnz"], "precision": "FP32 inner, FP64 refinement",
                       "rtol": 1e-10, "step": "mesh_build+assemble+solve+recover",
                       "l2": "inputs larger than L2 (system ~1.5 GB)", "parallelism": "replicas" if world > 1 else "1 GPU"},
            "solves_per_s": world * 1e3 / ms_step,
            "phases_ms_median": {k: med(v) for k, v in ph.items()},
            "assembly_triangles_per_s": nT * 1e3 / med(ph["assemble"]) if ph["assemble"] else None,
            "mesh_build_triangles_per_s": nT * 1e3 / med(ph["mesh_build"]) if ph["mesh_build"] else None,
            "solve": {"iterations": med(iters), "refinements": med(refs), "rel_residual_max": max(rel) if rel else None,
                      "converged": sorted(set(conv)), "order": "locality (Morton) order, solution as FP64 pair"},
            "fp64": fp64, "e2e": e2e, "multigrid": mgres, "refine": refine, "roofline": roof,
            "kernels": kernel_share,
            "gpu_launches": launches, "clocks": clk, "cpu_baseline": cpu, "oracle_parity": parity,
            "assembly_median_of_20": asm20,
            **forms,
        }
        if "serve" in forms:
            sv = forms["serve"]["multigrid_fp32_refined"]
            line["p50_ms"], line["p99_ms"] = sv["p50_ms"], sv["p99_ms"]
        print(json.dumps(line, default=_json_default), flush=True)
    P.phfem_ctx_destroy(ctx)
    ranks.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
