"""Benchmark: MDOF/s to a 1e-8 relative residual for FGMRES preconditioned by the monolithic
multigrid V-cycle on the reduced-quadrature Biot system, FP64 V-cycle vs FP32 V-cycle.

Workload (one step): the 512 x 512 triangulated unit square (2,619,394 free DoFs), the
parameter sweep lambda in {1, 1e4, 1e6} x K in {1, 1e-6} with mu = tau = alpha = 1, 1/M = 1,
right-hand side uniform in [-1, 1] on the free DoFs (seeds 0..5, one per parameter pair),
each solved with a Vanka V(1,1) and an inexact Braess-Sarazin V(1,1) preconditioner:
12 plain FP64 solves.  A second arm ("fp32_mg") times the 8 solves with lambda <= 1e4 with
FP32 V-cycles inside FP64 FGMRES against the same 8 solves with FP64 V-cycles (at
lambda/mu = 1e6 an FP32 V-cycle cannot converge: FP32 rounding of a nearly divergence-free
displacement, times lambda, is a 6% error in the grad-div term).  The solves of a step are
independent: they run on --streams concurrent CUDA streams (default 6; one host thread each,
longest solves first), so the latency-bound phases of one solve (small grids, the host read
of each Arnoldi column) overlap the full-GPU kernels of another.  Setup (assembly,
hierarchy, factorisations) is outside the timed region; every input is resident in HBM when
it starts.  L2 (129 MB) is flushed by a 256 MB write before every step (between solves with
--streams 1).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU (torchrun): replicas only -- every rank runs the whole workload on its own GPU.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

LAMBDAS = (1.0, 1e4, 1e6)
KS = (1.0, 1e-6)
INV_M = 1.0
INV_M_PAPER = 1e-2
N_GRID = 512
RTOL = 1e-8
RESTART = 50
MAXIT = 1000
MAXIT_ARM = 300
# roofline denominators: FP64 FMA pipe (nominal 1.25 TFLOP/s for the GB300; measured
# 1.20 TFLOP/s with a register FMA loop), HBM from the measured-peaks file of this GPU model
FP64_PEAK_TFLOPS = 1.25
# DRAM bytes (read + write) per fine-level launch of the FP64 operator inside the sweep, from
# one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum, the fine-level launches of a
# single-stream step): the FGMRES matvec y = A z reads x and K^{-1} (25.60 MB, its output
# stays in L2), the true residual r = b - A x also reads b (47.43 MB); with the SHA-256 prefix
# of the operator source they were taken with: the bench reports the figure only while that
# source is unchanged (else null, until the counters are taken again)
APPLY_TRAFFIC = {"matvec": 25.60e6, "residual": 47.43e6, "digest": "2f675d8d9b2fbe6c"}
# algorithmic work per grid cell of the fine-level kernels: the operator counts the nonzero
# products of the element matrices (156 flops per triangle, two triangles per cell, plus 26
# for the gather and the residual); Vanka: the 20 x 20 inverse (400 FMAs) plus the weighted
# gather; BSR's displacement sweep: the 8 x 8 inverse plus the gather
FLOPS_PER_CELL = {"vanka": 2 * 400 + 10, "apply": 2 * 156 + 26, "vanka_u": 2 * 64 + 10,
                  "restrict": 0, "prolong": 0}
BYTES_PER_CELL_F64 = {"vanka": 240, "apply": 256, "vanka_u": 208, "restrict": 100, "prolong": 180}


def vcycle_bytes_per_cell(fam, precision="fp64", per_patch=False, factors_fp64=None):
    """Algorithmic HBM bytes per grid cell of one fine-level launch: the vectors in the
    V-cycle's precision, plus, with per-patch factors (varying K), one patch inverse per vertex
    read once: 210 packed entries (20-DoF Vanka) or 64 (8-DoF displacement Vanka of BSR), in
    FP64 when ``factors_fp64`` (default: FP64 V-cycles) else FP32."""
    vec = BYTES_PER_CELL_F64[fam] * (0.5 if precision == "fp32" else 1.0)
    if not per_patch or fam not in ("vanka", "vanka_u"):
        return vec
    f64 = (precision == "fp64") if factors_fp64 is None else factors_fp64
    return vec + {"vanka": 210, "vanka_u": 64}[fam] * (8 if f64 else 4)


def apply_traffic(n_matvec, n_residual):
    """Mean recorded DRAM bytes per operator launch over n_matvec FGMRES matvecs and
    n_residual true residuals, if the operator source still matches."""
    import hashlib
    path = os.path.join(ROOT, "paper_2107_04060_gb300", "csrc", "operator.cu")
    try:
        with open(path, "rb") as f:
            digest = hashlib.sha256(f.read()).hexdigest()[:16]
    except OSError:
        return None
    if digest != APPLY_TRAFFIC["digest"] or n_matvec + n_residual <= 0:
        return None
    return (n_matvec * APPLY_TRAFFIC["matvec"] + n_residual * APPLY_TRAFFIC["residual"]) / (n_matvec + n_residual)


# Damping of the V(1,1) cycles at each (lambda, K, 1/M) point of the sweep: the minimisers of
# the two-grid LFA factor (Sec. 4.3 procedure: brute force in steps of 0.02) on the sweep's
# fine grid, h = 1/512.  Vanka: omega; BSR: (omega_J, omega).
OMEGA_LFA = {
    (1.0, 1.0, 1.0): (0.80, 1.08, 0.74), (1.0, 1e-6, 1.0): (0.78, 1.00, 0.82),
    (1e4, 1.0, 1.0): (0.68, 1.00, 0.68), (1e4, 1e-6, 1.0): (0.68, 1.00, 0.68),
    (1e6, 1.0, 1.0): (0.68, 1.00, 0.68), (1e6, 1e-6, 1.0): (0.68, 1.00, 0.68),
    (1.0, 1.0, 1e-2): (0.84, 1.08, 0.74), (1.0, 1e-6, 1e-2): (0.78, 1.00, 0.84),
    (1e4, 1.0, 1e-2): (0.68, 1.00, 0.68), (1e4, 1e-6, 1e-2): (0.68, 1.00, 0.68),
    (1e6, 1.0, 1e-2): (0.68, 1.00, 0.68), (1e6, 1e-6, 1e-2): (0.68, 1.00, 0.68),
}


def smoother_cases(inv_M: float = INV_M):
    """The 12 solves of a sweep step: (lambda, K) pairs with a Vanka and a BSR solve each,
    damped as OMEGA_LFA gives."""
    cases = []
    for li, lam in enumerate(LAMBDAS):
        for ki, K in enumerate(KS):
            seed = li * len(KS) + ki
            om_v, om_j, om_b = OMEGA_LFA[(lam, K, inv_M)]
            cases.append(dict(lam=lam, K=K, seed=seed, smoother="vanka", omega=om_v, omega_J=1.0))
            cases.append(dict(lam=lam, K=K, seed=seed, smoother="bsr", omega=om_b, omega_J=om_j))
    return cases


# ----------------------------------------------------------------------------------------
def measured_hbm_gbs():
    """(GB/s, source): the measured copy bandwidth of this GPU model, else the
    earlier single measurement used as the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured copy bandwidth"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback (no measured peaks file)"


def clocks_sampler(stop_evt, out):
    cmd = ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,"
           "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
           "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
           "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits"]
    while not stop_evt.is_set():
        try:
            line = subprocess.run(cmd, capture_output=True, text=True, timeout=5).stdout.strip()
            if line:
                out.append(line.splitlines()[0])
        except Exception:
            pass
        stop_evt.wait(0.2)


def summarize_clocks(lines):
    import statistics
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in lines:
        p = [x.strip() for x in ln.split(",")]
        try:
            sm.append(float(p[1]))
            mx.append(float(p[2]))
        except (ValueError, IndexError):
            continue
        for nm, v in zip(names, p[5:9]):
            if v.lower().startswith("active"):
                reasons.add(nm)
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
            "samples": len(sm)}


# ----------------------------------------------------------------------------------------
def oracle_sample(n: int, cases) -> dict:
    """Time the CPU oracle (as it stands) on the same 12 solves on an n x n grid; runs in a
    child process with one BLAS / OpenMP thread."""
    code = r"""
import json, sys, time
sys.path.insert(0, %r)
import numpy as np
import synthetic
from oracle import fem, mg, krylov
n = %d
cases = json.loads(%r)
tot, dofs, its = 0.0, 0, []
for c in cases:
    prm = fem.Params(lam=c["lam"], mu=1.0, tau=1.0, alpha=1.0, inv_M=%r)
    kL, kU = synthetic.constant_k(n, c["K"])
    H = mg.Hierarchy(n, prm, 1 / kL, 1 / kU, smoother=c["smoother"], omega=c["omega"],
                     omega_J=c.get("omega_J", 1.0))
    L = H.levels[0]
    b = L.mesh.pack(synthetic.rhs(n, c["seed"]))
    t = time.perf_counter()
    x, info = krylov.fgmres(L.A, b, H.vcycle, rtol=%r, restart=%d, maxit=%d)
    tot += time.perf_counter() - t
    dofs += len(L.mesh.free_idx)
    its.append(info["iters"])
print(json.dumps(dict(seconds=tot, dofs=dofs, iters=its)))
""" % (ROOT, n, json.dumps(cases), INV_M, RTOL, RESTART, MAXIT)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               PYTHONPATH=ROOT)
    p = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=1800)
    if p.returncode != 0:
        raise RuntimeError("oracle sample failed:\n" + p.stderr[-2000:])
    r = json.loads(p.stdout.strip().splitlines()[-1])
    r["mdofs"] = r["dofs"] / r["seconds"] / 1e6
    return r


def oracle_sample_parallel(n: int, cases, inv_M: float = None, reps: int = 1) -> dict:
    """Time the CPU oracle (as it stands) on the same solves on an n x n grid, one solve per
    host core: worker processes (spawned, one BLAS / OpenMP thread each) set up their solve
    once, then `reps` times meet at a barrier, solve and report wall-clock start and end.
    Per repetition, throughput = all solves' free DoFs / (last end - first start)."""
    code = r"""
import json, os, sys, time
import multiprocessing as mp
sys.path.insert(0, %r)

def work(c, n, inv_M, rtol, restart, maxit, reps, barrier, q):
    import numpy as np
    import synthetic
    from oracle import fem, mg, krylov
    prm = fem.Params(lam=c["lam"], mu=1.0, tau=1.0, alpha=1.0, inv_M=inv_M)
    kL, kU = synthetic.constant_k(n, c["K"])
    H = mg.Hierarchy(n, prm, 1 / kL, 1 / kU, smoother=c["smoother"], omega=c["omega"],
                     omega_J=c.get("omega_J", 1.0))
    L = H.levels[0]
    b = L.mesh.pack(synthetic.rhs(n, c["seed"]))
    for rep in range(reps):
        barrier.wait()
        t0 = time.time()
        x, info = krylov.fgmres(L.A, b, H.vcycle, rtol=rtol, restart=restart, maxit=maxit)
        t1 = time.time()
        q.put(dict(rep=rep, t0=t0, t1=t1, dofs=len(L.mesh.free_idx), iters=info["iters"],
                   key=(c["seed"], c["smoother"] != "vanka")))

if __name__ == "__main__":
    n, reps = %d, %d
    cases = json.loads(%r)
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(len(cases))
    q = ctx.Queue()
    ps = [ctx.Process(target=work, args=(c, n, %r, %r, %d, %d, reps, barrier, q)) for c in cases]
    for p in ps:
        p.start()
    res = []
    while len(res) < len(ps) * reps:
        try:
            res.append(q.get(timeout=5))
        except Exception:
            if any(p.exitcode not in (None, 0) for p in ps):
                for p in ps:
                    p.kill()
                raise SystemExit("an oracle worker failed")
    for p in ps:
        p.join()
    walls = []
    for rep in range(reps):
        rr = [r for r in res if r["rep"] == rep]
        walls.append(max(r["t1"] for r in rr) - min(r["t0"] for r in rr))
    last = sorted([r for r in res if r["rep"] == reps - 1], key=lambda r: r["key"])
    print(json.dumps(dict(seconds=walls[-1], walls=walls, dofs=sum(r["dofs"] for r in last),
                          procs=len(ps), cpu_seconds=sum(r["t1"] - r["t0"] for r in last),
                          iters=[r["iters"] for r in last])))
""" % (ROOT, n, reps, json.dumps(cases), INV_M if inv_M is None else inv_M, RTOL, RESTART, MAXIT)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               PYTHONPATH=ROOT)
    import tempfile
    with tempfile.TemporaryDirectory() as tmp:      # spawned workers re-import the script
        script = os.path.join(tmp, "oracle_parallel.py")
        with open(script, "w") as f:
            f.write(code)
        p = subprocess.run([sys.executable, script], capture_output=True, text=True, env=env,
                           timeout=3600)
    if p.returncode != 0:
        raise RuntimeError("parallel oracle sample failed:\n" + p.stderr[-2000:])
    r = json.loads(p.stdout.strip().splitlines()[-1])
    r["mdofs"] = r["dofs"] / r["seconds"] / 1e6
    return r


def run_reference(args, rank, world):
    """--impl reference: the CPU oracle timed on this host's cores (rank 0 only): the 12
    solves of the workload on a 64 x 64 grid, one solve per core, every step a barrier-started
    round of all 12."""
    if rank != 0:
        return
    n = 64
    cases = smoother_cases()
    r = oracle_sample_parallel(n, cases, reps=args.warmup + args.steps)
    walls = r["walls"][args.warmup:]
    sec = sum(walls) / len(walls)
    value = r["dofs"] / sec / 1e6
    sample = (f"the 12 solves of the workload (same parameters, smoothers, seeds, tolerance) on a "
              f"{n}x{n} grid ({r['dofs'] // 12} free DoFs each) instead of 512x512, one solve per "
              f"host core ({r['procs']} processes, one thread each, nproc = {os.cpu_count()}); solve "
              "time only")
    out = {"metric": "MDOF/s to 1e-8 rel. residual (FGMRES + monolithic MG V(1,1))", "value": value,
           "unit": "MDOF/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": f"biot-rq 512x512 sweep (sampled on {n}x{n})", "n": n,
                      "solves_per_step": 12, "iters": r["iters"]},
           "cpu_baseline": {"value": value, "unit": "MDOF/s", "cores": r["procs"], "kind": "oracle",
                            "nproc": os.cpu_count(), "sample": sample},
           "e2e": {"value": value, "unit": "MDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------------------------------
def run_micro(args):
    """One fine-level kernel family on an n x n grid with a lognormal permeability (the
    mixed-precision workload's coefficients), timed with the library's CUDA-event timer."""
    import torch
    import paper_2107_04060_gb300 as bmg
    import synthetic
    n = args.n
    torch.cuda.set_device(0)
    bmg.use_graphs(False)               # every kernel launched (and timed) individually
    if args.uniform_k:
        s = bmg.assemble(n, 1e4, 1.0, None, 1.0, 1.0, 1.0, INV_M)
    else:
        kL, kU = synthetic.lognormal_k(n, 2.0, 0)
        K = torch.from_numpy(bmg.pack_k(n, kL, kU)).cuda()
        s = bmg.assemble(n, 1e4, 1.0, K, 0.0, 1.0, 1.0, INV_M)
    x = torch.from_numpy(bmg.pack(n, synthetic.uniform_field(n, 1))).cuda()
    y = torch.empty_like(x)
    h = None
    if args.micro != "apply":
        h = bmg.setup_hierarchy(s, args.smoother, 1, 1, omega=0.7, precision=args.precision)
    fam = {"apply": "apply", "vanka": "vanka", "vcycle": args.family or "vanka"}[args.micro]
    b = torch.from_numpy(bmg.pack(n, synthetic.rhs(n, 2))).cuda()

    def run():
        if args.micro == "apply" and args.residual:
            s.residual(b, x, y)
        elif args.micro == "apply":
            s.apply(x, y)
        else:
            h.vcycle(x, y)
    for _ in range(3):
        run()
    torch.cuda.synchronize()
    bmg.profile_start(fam, n)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")           # ncu --nvtx-include timed/ selects these launches
    ev0.record()
    for _ in range(args.reps):
        run()
    ev1.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    prof = bmg.profile_stop()
    avg = prof["ms"] / max(prof["launches"], 1)
    cells = prof["cells"] / max(prof["launches"], 1)
    bpc = vcycle_bytes_per_cell(fam, args.precision, per_patch=not args.uniform_k)
    tiles = None
    if h is not None:
        tiles = {str(n >> l): [h.tile(l, "apply"), h.tile(l, "vanka"), h.tile(l, "vanka_u")]
                 for l in range(h.levels - 1)}
    print(json.dumps({"micro": args.micro, "n": n, "precision": args.precision, "uniform_k": args.uniform_k,
                      "residual": args.residual, "tiles_apply_vanka_vankau": tiles,
                      "gbs_algorithmic_this_precision": bpc * cells / (avg * 1e-3) / 1e9,
                      "bytes_per_cell": bpc,
                      "call_ms": ev0.elapsed_time(ev1) / args.reps, "kernel": fam,
                      "kernel_avg_ms": avg, "launches": prof["launches"],
                      "gflops_fp64": FLOPS_PER_CELL[fam] * cells / (avg * 1e-3) / 1e9,
                      "gbs_algorithmic": BYTES_PER_CELL_F64[fam] * cells / (avg * 1e-3) / 1e9}))


def batched_instances(count: int, seed: int = 2026):
    """The batched workload: `count` independent instances with n uniform in {32, 64, 128,
    256}, lambda log-uniform in [1, 1e6], per-triangle lognormal K (sigma = 1), mu = tau =
    alpha = 1/M = 1, right-hand side uniform in [-1, 1]; seeds fixed per instance."""
    import numpy as np
    rng = np.random.default_rng(seed)
    out = []
    for q in range(count):
        n = int(rng.choice([32, 64, 128, 256]))
        lam = float(10.0 ** rng.uniform(0.0, 6.0))
        out.append(dict(n=n, lam=lam, k_seed=1000 + q, b_seed=2000 + q,
                        omega=0.8 if lam < 10.0 else 0.7))
    return out


def shard_instances(count: int, rank: int, world: int):
    """Instances of the batched workload solved by `rank` of `world` (round robin: every
    instance on exactly one rank, sizes spread evenly); no data crosses ranks."""
    return [q for q in range(count) if q % world == rank]


def max_over_ranks(value: float, world: int, device=None) -> float:
    """The largest of the ranks' values (the job's time is its slowest rank's)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_batched(args):
    res = batched_workload(args.batch_count, args.steps, args.warmup, not args.no_autotune,
                           not args.no_sequential)
    if res is not None:
        print(json.dumps(res))


def batched_workload(count, steps, warmup, autotune=True, sequential=True):
    """Batched workload: every instance solved to 1e-8 by one graph launch of the batched
    FGMRES, timed against the same instances solved one after the other with the
    single-instance FGMRES (both with FP64 Vanka V(1,1) preconditioning).  Under torchrun
    the instances are split round robin over the ranks; rank 0 returns the record."""
    import numpy as np
    import torch
    import paper_2107_04060_gb300 as bmg
    import synthetic
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    all_inst = batched_instances(count)
    inst = [all_inst[q] for q in shard_instances(len(all_inst), rank, world)]
    ndof_all = sum(bmg.free_dofs(c["n"]) for c in all_inst)
    t0 = time.perf_counter()
    systems, hs, bs = [], [], []
    for c in inst:
        n = c["n"]
        kL, kU = synthetic.lognormal_k(n, 1.0, c["k_seed"])
        K = torch.from_numpy(bmg.pack_k(n, kL, kU)).to(dev)
        s = bmg.assemble(n, c["lam"], 1.0, K, 0.0, 1.0, 1.0, INV_M)
        systems.append(s)
        hs.append(bmg.setup_hierarchy(s, "vanka", 1, 1, omega=c["omega"]))
        bs.append(torch.from_numpy(bmg.pack(n, synthetic.rhs(n, c["b_seed"]))).to(dev))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    t1 = time.perf_counter()
    batch = bmg.Batch(hs, rtol=RTOL, restart=RESTART, maxit=MAXIT, autotune=autotune)
    create_s = time.perf_counter() - t1
    xs = [torch.zeros_like(b) for b in bs]
    ndof = sum(bmg.free_dofs(c["n"]) for c in inst)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(warmup):
        infos = batch.solve(bs, xs)
    times = []
    for _ in range(steps):
        flush.fill_(1.0)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        l0 = bmg.launch_count()
        ev0.record()
        infos = batch.solve(bs, xs)
        ev1.record()
        torch.cuda.synchronize()
        launches = bmg.launch_count() - l0
        times.append(max_over_ranks(ev0.elapsed_time(ev1), world, dev))
    bad = [i for i in infos if i["status"] != "converged"]
    if bad:
        raise RuntimeError(f"batched solve: {len(bad)} instances did not converge")
    # the same instances one after the other (single-instance FGMRES, host-driven)
    seq_ms = None
    seq_iters = []
    if sequential and world == 1:
        x = [torch.zeros_like(b) for b in bs]
        for q in range(min(3, len(hs))):
            hs[q].fgmres_solve(bs[q], x[q], rtol=RTOL, restart=RESTART, maxit=MAXIT)
        flush.fill_(2.0)
        torch.cuda.synchronize()
        ev0.record()
        for q in range(len(hs)):
            i = hs[q].fgmres_solve(bs[q], x[q], rtol=RTOL, restart=RESTART, maxit=MAXIT)
            seq_iters.append(i["iters"])
        ev1.record()
        torch.cuda.synchronize()
        seq_ms = ev0.elapsed_time(ev1)
    ms = float(np.median(times))
    iters = [i["iters"] for i in infos]
    sizes = sorted({c["n"] for c in inst})
    if rank != 0:
        return None
    res = ({
        "workload": f"batched {len(inst)} instances, n in {{32,64,128,256}}, lambda log-uniform [1,1e6], "
                    "lognormal K sigma 1, FP64 Vanka V(1,1) FGMRES(50) to 1e-8",
        "metric": "MDOF/s to 1e-8 rel. residual (batched)", "unit": "MDOF/s",
        "value": ndof_all / (ms * 1e-3) / 1e6, "ms_per_solve": ms, "steps": steps,
        "warmup": warmup, "free_dofs": ndof_all, "n_gpus": world,
        "scaling": "strong (instances split round robin across ranks, no data-path collective)",
        "sequential_ms": seq_ms,
        "sequential_mdofs": (ndof / (seq_ms * 1e-3) / 1e6) if seq_ms else None,
        "speedup_vs_sequential": (seq_ms / ms) if seq_ms else None,
        "iters_min_median_max": [min(iters), float(np.median(iters)), max(iters)],
        "iters_sum": sum(iters), "sequential_iters_sum": sum(seq_iters) if seq_iters else None,
        "trips": batch.trips, "kernels_per_trip": batch.kernels_per_trip, "gpu_launches": launches,
        "tiles": {str(n): [batch.tile("apply", n), batch.tile("vanka", n)] for n in sizes + [16]},
        "setup_s": setup_s, "batch_create_s": create_s,
        "autotune": autotune})
    batch.close()
    del hs, systems
    return res


def run_mixed(args):
    import torch
    torch.cuda.set_device(0)
    print(json.dumps(mixed_workload(args.mixed_n, args.steps, args.warmup)))


def mixed_workload(n, steps, warmup):
    """Mixed-precision workload: the n x n grid (2048), lambda = 1e4, mu = 1, per-triangle
    lognormal K (sigma = 2, seed 0), right-hand side seed 0; FGMRES(50) to 1e-8 with FP32
    V-cycles (FP32 accumulation, FP64 patch factors rounded to FP32; and with the FP64
    factors and FP64 patch solves) against the same solve with FP64 V-cycles.  Reports per
    solve the time, iterations and FP64 true residual, the error of the FP32-MG solution
    against the FP64 one (2-norm and max-norm, relative), and the HBM rate of the FP32
    V-cycle's fine-level operator and Vanka launches (algorithmic bytes, per-patch factors
    included, over CUDA-event time, the kernels alone on the GPU)."""
    import numpy as np
    import torch
    import paper_2107_04060_gb300 as bmg
    import synthetic
    dev = torch.device("cuda", torch.cuda.current_device())
    kL, kU = synthetic.lognormal_k(n, 2.0, 0)
    K = torch.from_numpy(bmg.pack_k(n, kL, kU)).to(dev)
    t0 = time.perf_counter()
    s = bmg.assemble(n, 1e4, 1.0, K, 0.0, 1.0, 1.0, INV_M)
    h = {p: bmg.setup_hierarchy(s, "vanka", 1, 1, omega=0.7, precision=p) for p in ("fp32", "fp64")}
    h["fp32_patch_fp64"] = bmg.setup_hierarchy(s, "vanka", 1, 1, omega=0.7, precision="fp32",
                                               patch_solve="fp64")
    b = torch.from_numpy(bmg.pack(n, synthetic.rhs(n, 0))).to(dev)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    runs = ("fp32", "fp64", "fp32_mixed_arnoldi", "fp32_patch_fp64")
    x = {p: torch.zeros_like(b) for p in runs}
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {}
    for p in runs:
        hp = h["fp32" if p == "fp32_mixed_arnoldi" else p]
        arn = "mixed" if p == "fp32_mixed_arnoldi" else "fp64"
        for _ in range(warmup):
            hp.fgmres_solve(b, x[p], rtol=RTOL, restart=RESTART, maxit=MAXIT, arnoldi=arn)
        ms = []
        for _ in range(steps):
            torch.cuda.synchronize()
            ev0.record()
            info = hp.fgmres_solve(b, x[p], rtol=RTOL, restart=RESTART, maxit=MAXIT, arnoldi=arn)
            ev1.record()
            torch.cuda.synchronize()
            ms.append(ev0.elapsed_time(ev1))
        r = torch.empty_like(b)
        s.residual(b, x[p], r)
        out[p] = dict(ms=float(np.median(ms)), iters=info["iters"], status=info["status"],
                      true_relres=(torch.linalg.norm(r) / torch.linalg.norm(b)).item(),
                      mdofs=bmg.free_dofs(n) / (float(np.median(ms)) * 1e-3) / 1e6)
    diff = (torch.linalg.norm(x["fp32"] - x["fp64"]) / torch.linalg.norm(x["fp64"])).item()
    dmax = ((x["fp32"] - x["fp64"]).abs().max() / x["fp64"].abs().max()).item()
    # HBM rate of the FP32 V-cycle's fine-level kernels (V-cycle calls only, graphs off)
    peak_gbs, peak_src = measured_hbm_gbs()
    prev = bmg.use_graphs(False)
    hbm = {"unit": "GB/s algorithmic (vectors in FP32, per-patch factors read once), fine level",
           "peak_gbs": peak_gbs, "peak_source": peak_src}
    vin, vout = b.clone(), torch.empty_like(b)
    for key, hp, fam, f64 in (("apply", h["fp32"], "apply", False), ("vanka", h["fp32"], "vanka", False),
                              ("restrict", h["fp32"], "restrict", False), ("prolong", h["fp32"], "prolong", False),
                              ("vanka_fp64_factors", h["fp32_patch_fp64"], "vanka", True)):
        hp.vcycle(vin, vout)
        torch.cuda.synchronize()
        bmg.profile_start(fam, n)
        for _ in range(3):
            hp.vcycle(vin, vout)
        torch.cuda.synchronize()
        r_ = bmg.profile_stop()
        if r_["launches"]:
            avg = r_["ms"] / r_["launches"]
            bpc = vcycle_bytes_per_cell(fam, "fp32", per_patch=True, factors_fp64=f64)
            gbs = bpc * (r_["cells"] / r_["launches"]) / (avg * 1e-3) / 1e9
            hbm[key] = {"gbs": round(gbs, 1), "frac": round(gbs / peak_gbs, 3), "bytes_per_cell": bpc,
                        "avg_launch_ms": round(avg, 4), "launches": r_["launches"],
                        "tile": hp.tile(0, fam)}
    bmg.use_graphs(prev)
    res = {"workload": f"mixed precision {n}x{n}, lambda 1e4, lognormal K sigma 2, "
                       "Vanka V(1,1) FGMRES(50) to 1e-8",
           "free_dofs": bmg.free_dofs(n), "fp32_mg": out["fp32"], "fp64": out["fp64"],
           "fp32_mg_mixed_arnoldi": out["fp32_mixed_arnoldi"],
           "fp32_mg_patch_fp64": out["fp32_patch_fp64"],
           "vcycle_hbm": hbm,
           "speedup_fp32_vs_fp64": out["fp64"]["ms"] / out["fp32"]["ms"],
           "speedup_fp32_mixed_arnoldi_vs_fp64": out["fp64"]["ms"] / out["fp32_mixed_arnoldi"]["ms"],
           "error_fp32_mg_vs_fp64": {"rel_2norm": diff, "rel_maxnorm": dmax,
                                     "reference": "the FP64 GPU solution of the same system (parity-tested "
                                                  "against the CPU oracle on smaller grids; the oracle does "
                                                  "not solve 42M DoFs within the bench)"},
           "setup_s": setup_s, "steps": steps, "warmup": warmup}
    del h, s
    return res


def time_dependent_workload(n, steps, lam=1e4, K=1.0, omega=0.68):
    """Backward-Euler time stepping (Sec. 2.1, Eqs. discrete1-3), the analogue of Sec. 5.2's
    runs (average FGMRES iterations per time step): ``steps`` steps of tau = 1/128 on the
    n x n grid, lambda = 1e4, mu = alpha = 1/M = 1, uniform K, Vanka V(1,1); the loads of step
    m are exp(-t_m) times a seeded field uniform in [-1, 1], each step's right-hand side is
    formed on the device (bmg_backward_euler_rhs: loads plus the pressure-row history term)
    and solved to 1e-8 from the previous step's solution."""
    import numpy as np
    import torch
    import paper_2107_04060_gb300 as bmg
    import synthetic
    dev = torch.device("cuda", torch.cuda.current_device())
    tau = 1.0 / 128
    s = bmg.assemble(n, lam, 1.0, None, K, tau, 1.0, INV_M)
    h = bmg.setup_hierarchy(s, "vanka", 1, 1, omega=omega)
    f0 = torch.from_numpy(bmg.pack(n, synthetic.rhs(n, 7))).to(dev)
    st = torch.cuda.Stream(device=dev)
    x = torch.zeros_like(f0)
    b, ld = torch.empty_like(f0), torch.empty_like(f0)
    iters = []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(st):
        torch.cuda.synchronize()
        ev0.record(st)
        for m in range(1, steps + 1):
            torch.mul(f0, float(np.exp(-m * tau)), out=ld)
            s.backward_euler_rhs(x, ld, b, stream=st)
            info = h.fgmres_solve(b, x, rtol=RTOL, restart=RESTART, maxit=MAXIT, x0_is_zero=False,
                                  stream=st)
            if info["status"] != "converged":
                raise RuntimeError(f"time step {m} did not converge: {info}")
            iters.append(info["iters"])
        ev1.record(st)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    return {"workload": f"backward Euler {n}x{n}, {steps} steps of tau = 1/128, lambda {lam:g}, K {K:g}, "
                        "Vanka V(1,1), seeded loads exp(-t) F, each step to 1e-8 from the previous one",
            "free_dofs": bmg.free_dofs(n), "steps": steps, "ms_per_step": ms / steps,
            "value": bmg.free_dofs(n) * steps / (ms * 1e-3) / 1e6, "unit": "MDOF/s (per time step)",
            "iters_per_step_mean": float(np.mean(iters)), "iters": iters}


def bsr_exact_workload(n, lams=(1.0, 1e4, 1e6), Ks=(1.0, 1e-6)):
    """Exact against inexact Braess-Sarazin (Sec. 3.2.2): the BSR solves of the sweep's
    (lambda, K) points on the n x n grid, V(1,1) with the sweep's LFA damping, once with the
    pressure step relaxed by one Jacobi sweep (inexact, the paper's) and once solved by CG on
    the fixed-stress Schur complement (exact); FGMRES(50) to 1e-8, one solve after the other."""
    import torch
    import paper_2107_04060_gb300 as bmg
    import synthetic
    dev = torch.device("cuda", torch.cuda.current_device())
    st = torch.cuda.Stream(device=dev)
    cases = [c for c in smoother_cases(INV_M) if c["smoother"] == "bsr"]
    rows = []
    with torch.cuda.stream(st):
        for c in cases:
            s = bmg.assemble(n, c["lam"], 1.0, None, c["K"], 1.0, 1.0, INV_M)
            b = torch.from_numpy(bmg.pack(n, synthetic.rhs(n, c["seed"]))).to(dev)
            row = {"lam": c["lam"], "K": c["K"]}
            for sm in ("bsr", "bsr_exact"):
                h = bmg.setup_hierarchy(s, sm, 1, 1, omega=c["omega"], omega_J=c["omega_J"], n_coarse=8)
                x = torch.zeros_like(b)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                info = h.fgmres_solve(b, x, rtol=RTOL, restart=RESTART, maxit=MAXIT, stream=st)
                torch.cuda.synchronize()
                row[sm] = {"iters": info["iters"], "status": info["status"],
                           "s": round(time.perf_counter() - t0, 3)}
                if sm == "bsr_exact":
                    row[sm]["cg_iters_max"] = h.schur_iters()
                del h
            rows.append(row)
            del s
    return {"workload": f"exact vs inexact BSR V(1,1), {n}x{n}, the sweep's BSR points (lambda x K), "
                        "FGMRES(50) to 1e-8; exact: CG on the fixed-stress S to 1e-11, multigrid-preconditioned",
            "free_dofs": bmg.free_dofs(n), "solves": rows}


def run_adjoint(args):
    import torch
    torch.cuda.set_device(0)
    print(json.dumps(adjoint_workload(args.adjoint_n, args.steps, args.warmup, args.fd_dirs)))


def adjoint_workload(n, steps, warmup, fd_dirs):
    """Adjoint workload: J = ||p - p_obs||^2 on the n x n grid (default 1024), p_obs the
    pressure of the FP64 solve with a reference lognormal log-K field (seed 1), theta the
    per-triangle log-permeability (FP32, lognormal sigma 1, seed 2), lambda = 10, mu = 1.3;
    one gradient = forward solve + adjoint solve (MG-FGMRES to 1e-10) + gradient kernel.
    Checked against central differences of J on --fd-dirs seeded random directions."""
    import numpy as np
    import torch
    import paper_2107_04060_gb300 as bmg
    from paper_2107_04060_gb300.differentiable import pressure_solve
    import synthetic
    dev = torch.device("cuda", torch.cuda.current_device())
    cfg = dict(rtol=1e-10, maxit=4000, omega=0.8)
    lam = torch.tensor(10.0, dtype=torch.float64, device=dev, requires_grad=True)
    mu = torch.tensor(1.3, dtype=torch.float64, device=dev, requires_grad=True)
    b = torch.from_numpy(bmg.pack(n, synthetic.rhs(n, 0))).to(dev)
    rL, rU = synthetic.lognormal_k(n, 1.0, 1)
    ref = torch.from_numpy(np.stack([np.log(rL), np.log(rU)]).astype(np.float32)).to(dev)
    with torch.no_grad():
        p_obs = pressure_solve(ref, lam.detach(), mu.detach(), b, **cfg)
    kL, kU = synthetic.lognormal_k(n, 1.0, 2)
    theta0 = torch.from_numpy(np.stack([np.log(kL), np.log(kU)]).astype(np.float32)).to(dev)

    def J(theta, lam_, mu_):
        p = pressure_solve(theta, lam_, mu_, b, **cfg)
        return ((p - p_obs) ** 2).sum()

    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = []
    for it in range(warmup + steps):
        theta = theta0.clone().requires_grad_(True)
        lam.grad = None
        mu.grad = None
        torch.cuda.synchronize()
        ev0.record()
        loss = J(theta, lam, mu)
        loss.backward()
        ev1.record()
        torch.cuda.synchronize()
        if it >= warmup:
            times.append(ev0.elapsed_time(ev1))
    g = theta.grad.double()
    Jv = loss.item()
    rng = np.random.default_rng(5)
    h = 1e-3
    errs = []
    th64 = theta0.double()
    with torch.no_grad():
        for _ in range(fd_dirs):
            d = torch.from_numpy(rng.standard_normal((2, n, n))).to(dev)
            # theta is FP32: perturb in FP64, round, and use the realised step
            tp, tm = (th64 + h * d).float(), (th64 - h * d).float()
            jp = J(tp, lam.detach(), mu.detach()).item()
            jm = J(tm, lam.detach(), mu.detach()).item()
            fd = (jp - jm) / 2.0
            an = float((g * (tp.double() - tm.double()) / 2.0).sum().item())
            errs.append(abs(an - fd) / max(abs(fd), 1e-300))
    return {"workload": f"adjoint gradient {n}x{n}, J = ||p - p_obs||^2, lambda 10, mu 1.3",
            "free_dofs": bmg.free_dofs(n), "ms_per_gradient": float(np.median(times)),
            "J": Jv, "dJ_dlambda": lam.grad.item(), "dJ_dmu": mu.grad.item(),
            "fd_dirs": fd_dirs, "fd_step": h,
            "fd_rel_err_max": max(errs) if errs else None,
            "fd_rel_err_median": float(np.median(errs)) if errs else None,
            "steps": steps, "warmup": warmup}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_GRID)
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--verbose", action="store_true")
    ap.add_argument("--micro", choices=["apply", "vanka", "vcycle"], default=None,
                    help="time one kernel family (fine level) on --n instead of the workload")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--uniform-k", action="store_true", help="--micro: constant K instead of lognormal")
    ap.add_argument("--residual", action="store_true", help="--micro apply: r = b - A x instead of y = A x")
    ap.add_argument("--smoother", default="vanka", choices=["vanka", "bsr"], help="--micro vcycle: smoother")
    ap.add_argument("--family", default=None, choices=["apply", "vanka", "vanka_u", "restrict", "prolong"],
                    help="--micro vcycle: kernel family to time (default vanka)")
    ap.add_argument("--workload", default="sweep", choices=["sweep", "batched", "mixed", "adjoint", "timedep", "bsr_exact"],
                    help="sweep: the 512^2 parameter sweep (default); batched / mixed / adjoint: "
                         "the batched, 2048^2 mixed-precision and 1024^2 adjoint workloads, each "
                         "printed as its own line")
    ap.add_argument("--mixed-n", type=int, default=2048)
    ap.add_argument("--adjoint-n", type=int, default=1024)
    ap.add_argument("--fd-dirs", type=int, default=32)
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-sequential", action="store_true")
    ap.add_argument("--streams", type=int, default=6,
                    help="solves of a step run concurrently on this many CUDA streams")
    ap.add_argument("--no-arms", action="store_true",
                    help="skip the mixed-Arnoldi and 1/M = 1e-2 arms of the sweep")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the mixed-precision, batched and adjoint workloads of the default run")
    ap.add_argument("--breakdown", action="store_true",
                    help="print the device time per kernel family of one step and exit")
    ap.add_argument("--breakdown-precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--breakdown-levels", action="store_true",
                    help="with --breakdown: also per grid level (one step per family and level)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.micro:
        run_micro(args)
        return
    if args.workload == "batched":
        run_batched(args)
        return
    if args.workload == "mixed":
        run_mixed(args)
        return
    if args.workload == "adjoint":
        run_adjoint(args)
        return
    if args.workload == "timedep":
        import torch
        torch.cuda.set_device(0)
        print(json.dumps(time_dependent_workload(args.n, max(1, args.steps))))
        return
    if args.workload == "bsr_exact":
        import torch
        torch.cuda.set_device(0)
        print(json.dumps(bsr_exact_workload(args.n)))
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2107_04060_gb300 as bmg
    import synthetic

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    st = torch.cuda.current_stream()
    n = args.n
    nfree = bmg.free_dofs(n)
    cases = smoother_cases()

    # ---- setup (outside the timed region)
    systems, work = {}, []
    for c in cases:
        key = (c["lam"], c["K"])
        if key not in systems:
            systems[key] = bmg.assemble(n, c["lam"], 1.0, None, c["K"], 1.0, 1.0, INV_M)
    rhs = {}
    for c in cases:
        if c["seed"] not in rhs:
            rhs[c["seed"]] = torch.from_numpy(bmg.pack(n, synthetic.rhs(n, c["seed"]))).to(dev)
    precisions = ["fp64"] + ([] if args.no_fp32 else ["fp32"])
    fp32_cases = [ci for ci, c in enumerate(cases) if c["lam"] <= 1e4]
    hier = {}
    t0 = time.perf_counter()
    for prec in precisions:
        for ci, c in enumerate(cases):
            if prec == "fp32" and ci not in fp32_cases:
                continue
            hier[prec, ci] = bmg.setup_hierarchy(systems[c["lam"], c["K"]], c["smoother"], 1, 1,
                                                 omega=c["omega"], omega_J=c["omega_J"], n_coarse=8,
                                                 precision=prec)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    x = torch.zeros(bmg.vector_len(n), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    nstreams = max(1, args.streams)
    streams = [torch.cuda.Stream(device=dev) for _ in range(nstreams)]
    xs = [torch.zeros(bmg.vector_len(n), dtype=torch.float64, device=dev) for _ in range(nstreams)]
    cost = {}                       # iterations seen per case: longest solves start first

    def one_step(prec, record=None, subset=None, nstreams=nstreams, solve=None, arnoldi="fp64",
                 hset=None, allow_fail=False, maxit=MAXIT):
        """One step: the solves of `cases` (or `subset`), on nstreams concurrent streams, with
        the hierarchies of `hset` (default: the main ones) and the given Arnoldi arithmetic.
        solve(ci, k, stream) -> info overrides the device-buffer solve (used by e2e)."""
        hs_ = hier if hset is None else hset
        todo = [ci for ci in range(len(cases)) if subset is None or ci in subset]
        if nstreams == 1 and solve is None:
            cur = torch.cuda.current_stream()
            streams[0].wait_stream(cur)
            for ci in todo:
                c = cases[ci]
                with torch.cuda.stream(streams[0]):
                    flush.fill_(float(ci))
                    info = hs_[prec, ci].fgmres_solve(rhs[c["seed"]], x, rtol=RTOL, restart=RESTART,
                                                      maxit=maxit, x0_is_zero=True, arnoldi=arnoldi,
                                                      stream=streams[0])
                if info["status"] != "converged" and not allow_fail:
                    raise RuntimeError(f"solve did not converge: {c} {info}")
                cost[ci] = info["iters"]
                if record is not None:
                    record.append((c, info))
            cur.wait_stream(streams[0])
            return
        # independent solves on nstreams streams, one host thread each (the library calls
        # release the interpreter lock); L2 flushed once before the step
        flush.fill_(1.0)
        cur = torch.cuda.current_stream()
        for st_ in streams:
            st_.wait_stream(cur)
        todo.sort(key=lambda ci: -cost.get(ci, 0))
        lock, errors, done = threading.Lock(), [], []

        def worker(k):
            try:
                while True:
                    with lock:
                        if not todo:
                            return
                        ci = todo.pop(0)
                    c = cases[ci]
                    info = solve(ci, k, streams[k])
                    if info["status"] != "converged" and not allow_fail:
                        raise RuntimeError(f"solve did not converge: {c} {info}")
                    with lock:
                        cost[ci] = info["iters"]
                        done.append((ci, c, info))
            except Exception as e:          # reported by the caller
                errors.append(e)

        if solve is None:
            def solve(ci, k, stream):
                c = cases[ci]
                return hs_[prec, ci].fgmres_solve(rhs[c["seed"]], xs[k], rtol=RTOL, restart=RESTART,
                                                  maxit=maxit, x0_is_zero=True, stream=stream,
                                                  arnoldi=arnoldi)
        threads = [threading.Thread(target=worker, args=(k,)) for k in range(nstreams)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        for st_ in streams:
            cur.wait_stream(st_)
        if errors:
            raise errors[0]
        if record is not None:
            record.extend((c, info) for _, c, info in sorted(done, key=lambda d: d[0]))

    def timed(prec, steps, profile=None, subset=None, ns=None, arnoldi="fp64", hset=None,
              allow_fail=False, maxit=MAXIT):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        recs = []
        barrier()
        l0 = bmg.launch_count()
        if profile:
            bmg.profile_start(profile, n)
        torch.cuda.nvtx.range_push("timed")
        ev0.record(st)
        for _ in range(steps):
            one_step(prec, recs, subset, nstreams=ns or nstreams, arnoldi=arnoldi, hset=hset,
                     allow_fail=allow_fail, maxit=maxit)
        ev1.record(st)
        torch.cuda.nvtx.range_pop()
        barrier()
        prof = bmg.profile_stop() if profile else None
        launches = bmg.launch_count() - l0
        ms = ev0.elapsed_time(ev1) / steps
        if world > 1:
            t = torch.tensor([ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        return ms, recs, prof, launches

    # ---- warm-up; the warm-up also decides which kernel family dominates (fine level)
    for prec in precisions:
        for _ in range(args.warmup):
            one_step(prec, subset=None if prec == "fp64" else fp32_cases)
    # kernel-family shares of one step, every kernel launched individually (V-cycle graphs
    # off, so that the V-cycle's launches are timed too)
    shares = {}
    bmg.use_graphs(False)
    for fam in ("vanka", "apply", "vanka_u"):
        bmg.profile_start(fam, n)
        one_step("fp64")
        torch.cuda.synchronize()
        shares[fam] = bmg.profile_stop()
    dominant = max(shares, key=lambda k: shares[k]["ms"])
    # the timed region replays V-cycles from CUDA graphs; the operator's roofline is then
    # timed on its launches outside the V-cycle (FGMRES matvec and true residual: the same
    # kernel on the same fine grid), a V-cycle-only family with the graphs off
    graphs_in_timed = dominant == "apply"
    bmg.use_graphs(graphs_in_timed)
    if args.breakdown:
        # device time per kernel family over all levels, one step each (FP64: the whole
        # sweep; FP32: the FP32-MG arm's solves), every kernel launched individually
        bmg.use_graphs(False)
        bp = args.breakdown_precision
        bsub = None if bp == "fp64" else fp32_cases
        out = {}
        for fam in ("apply", "vanka", "vanka_u", "restrict", "prolong", "coarse", "krylov"):
            bmg.profile_start(fam, 0)
            one_step(bp, subset=bsub)
            torch.cuda.synchronize()
            out[fam] = bmg.profile_stop()
        levels = {}
        if args.breakdown_levels:
            m = n
            while m >= 16:
                for fam in ("apply", "vanka", "vanka_u", "restrict", "prolong"):
                    bmg.profile_start(fam, m)
                    one_step(bp, subset=bsub)
                    torch.cuda.synchronize()
                    r = bmg.profile_stop()
                    levels.setdefault(str(m), {})[fam] = [round(r["ms"], 3), r["launches"]]
                m //= 2
        ms_step, _, _, _ = timed(bp, 1, subset=bsub)
        print(json.dumps({"breakdown_ms": {k: round(v["ms"], 3) for k, v in out.items()},
                          "launches": {k: v["launches"] for k, v in out.items()},
                          "per_level_ms_launches": levels, "step_ms": ms_step}))
        return

    # ---- timed region (FP64 V-cycle), clocks sampled meanwhile
    samples, stop = [], threading.Event()
    th = threading.Thread(target=clocks_sampler, args=(stop, samples), daemon=True)
    th.start()
    ms64, recs64, prof, launches = timed("fp64", args.steps, profile=dominant)
    # the same kernel family timed on one step with the solves run one after the other (each
    # launch then has the GPU to itself; in the timed region launches of concurrent solves
    # share it, which lengthens every launch)
    prof_iso = None
    if nstreams > 1:
        _, _, prof_iso, _ = timed("fp64", 1, profile=dominant, ns=1)
    ms32 = None
    if "fp32" in precisions:
        ms32, recs32, _, _ = timed("fp32", args.steps, subset=fp32_cases)
        ms64s, _, _, _ = timed("fp64", args.steps, subset=fp32_cases)
    # lambda / mu = 1e6 with FP32 V-cycles: FP32 patch solves, FP64 patch solves, and the FP64
    # V-cycle, Vanka, both K (the FP32 arm above stops at lambda = 1e4)
    probe64 = None
    if "fp32" in precisions and not args.no_arms:
        probe64 = []
        for ci in [ci for ci, c in enumerate(cases) if c["lam"] == 1e6 and c["smoother"] == "vanka"]:
            c = cases[ci]
            row = {"lam": c["lam"], "K": c["K"]}
            for label, kw in (("fp32", dict(precision="fp32")),
                              ("fp32_patch_fp64", dict(precision="fp32", patch_solve="fp64")),
                              ("fp64", dict(precision="fp64"))):
                hp = bmg.setup_hierarchy(systems[c["lam"], c["K"]], "vanka", 1, 1, omega=c["omega"],
                                         n_coarse=8, **kw)
                xp = torch.zeros_like(rhs[c["seed"]])
                t0 = time.perf_counter()
                ip = hp.fgmres_solve(rhs[c["seed"]], xp, rtol=RTOL, restart=RESTART, maxit=MAXIT_ARM,
                                     stream=streams[0])
                row[label] = {"iters": ip["iters"], "status": ip["status"],
                              "relres": float(f"{ip['relres']:.3g}"),
                              "s": round(time.perf_counter() - t0, 3)}
                del hp
            probe64.append(row)
    # per solve of the FP32-MG arm: the FP32-MG solution against the FP64-V-cycle solution of
    # the same system (relative 2-norm), and the FP64 true residual of the FP32-MG solution
    err32 = None
    if "fp32" in precisions and not args.no_arms:
        err32 = []
        for ci in fp32_cases:
            c = cases[ci]
            xa, xb = torch.zeros_like(rhs[c["seed"]]), torch.zeros_like(rhs[c["seed"]])
            with torch.cuda.stream(streams[0]):
                hier["fp32", ci].fgmres_solve(rhs[c["seed"]], xa, rtol=RTOL, restart=RESTART, maxit=MAXIT,
                                              stream=streams[0])
                hier["fp64", ci].fgmres_solve(rhs[c["seed"]], xb, rtol=RTOL, restart=RESTART, maxit=MAXIT,
                                              stream=streams[0])
                rr = torch.empty_like(xa)
                systems[c["lam"], c["K"]].residual(rhs[c["seed"]], xa, rr, stream=streams[0])
            torch.cuda.synchronize()
            err32.append({"lam": c["lam"], "K": c["K"], "smoother": c["smoother"],
                          "rel_err_vs_fp64": float(f"{(torch.linalg.norm(xa - xb) / torch.linalg.norm(xb)).item():.3g}"),
                          "true_relres": float(f"{(torch.linalg.norm(rr) / torch.linalg.norm(rhs[c['seed']])).item():.3g}")})
    # the same 12 FP64 solves with the mixed-precision Arnoldi (FP32 first Gram-Schmidt pass,
    # double-float second pass and correction)
    arm_steps = max(1, min(args.steps, 5))
    msA = msW = None
    if not args.no_arms:
        one_step("fp64", arnoldi="mixed")
        msA, recsA, _, _ = timed("fp64", arm_steps, arnoldi="mixed")
        # the 6 BSR solves with W(1,1) cycles against the same 6 with V(1,1) cycles
        bcases = [ci for ci, c in enumerate(cases) if c["smoother"] == "bsr"]
        hierW = {("fp64", ci): bmg.setup_hierarchy(systems[cases[ci]["lam"], cases[ci]["K"]], "bsr", 1, 1,
                                                   omega=cases[ci]["omega"], omega_J=cases[ci]["omega_J"],
                                                   n_coarse=8, cycle="W") for ci in bcases}
        one_step("fp64", subset=bcases, hset=hierW)
        msW, recsW, _, _ = timed("fp64", arm_steps, subset=bcases, hset=hierW)
        msV, recsV, _, _ = timed("fp64", arm_steps, subset=bcases)
        del hierW
    stop.set()
    th.join(timeout=5)
    clocks = summarize_clocks(samples)
    # HBM share of the FP32 V-cycle's fine-level kernels (one profiled FP32 step, outside the
    # timed region): algorithmic bytes per launch / CUDA-event duration, against the
    # measured copy bandwidth
    hbm32 = {}
    if "fp32" in precisions:
        # V-cycle calls only (the FGMRES matvec of an FP32-MG solve is the FP64 operator, which
        # would otherwise share the profiled family), the kernels alone on the GPU
        peak_gbs, _ = measured_hbm_gbs()
        prev_graphs = bmg.use_graphs(False)
        vin = rhs[cases[fp32_cases[0]]["seed"]]
        vout = torch.empty_like(vin)
        for fam in ("apply", "vanka", "vanka_u"):
            bmg.profile_start(fam, n)
            for ci in fp32_cases:
                for _ in range(3):
                    hier["fp32", ci].vcycle(vin, vout)
            torch.cuda.synchronize()
            r = bmg.profile_stop()
            if r["launches"]:
                gbs = BYTES_PER_CELL_F64[fam] * 0.5 * r["cells"] / (r["ms"] * 1e-3) / 1e9
                hbm32[fam] = {"gbs": round(gbs, 1), "frac": round(gbs / peak_gbs, 3),
                              "avg_launch_ms": round(r["ms"] / r["launches"], 4), "launches": r["launches"]}
        bmg.use_graphs(prev_graphs)

    # ---- end to end through the host-buffer entry point (FP64 arm)
    # (the same concurrent step; every solve copies its right-hand side in from pinned host
    # memory and its solution out inside the timed region)
    hb = {s: torch.empty(bmg.vector_len(n), dtype=torch.float64).pin_memory() for s in rhs}
    for s in rhs:
        hb[s].copy_(rhs[s].cpu())
    hxs = [torch.empty(bmg.vector_len(n), dtype=torch.float64).pin_memory() for _ in range(nstreams)]

    def solve_host(ci, k, stream):
        c = cases[ci]
        return hier["fp64", ci].fgmres_solve_host(hb[c["seed"]].numpy(), hxs[k].numpy(), rtol=RTOL,
                                                  restart=RESTART, maxit=MAXIT, stream=stream)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one_step("fp64", solve=solve_host)
    barrier()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps
    vec_bytes = bmg.vector_len(n) * 8

    work_dofs = len(cases) * nfree * world
    value = work_dofs / (ms64 * 1e-3) / 1e6
    out = {
        "metric": "MDOF/s to 1e-8 rel. residual (FGMRES + monolithic MG V(1,1))",
        "value": value, "unit": "MDOF/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms64, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"biot-rq {n}x{n} sweep: lambda {list(LAMBDAS)} x K {list(KS)}, "
                               f"Vanka + BSR V(1,1), 12 FP64 solves to 1e-8",
                   "n": n, "free_dofs": nfree, "solves_per_step": len(cases), "inv_M": INV_M,
                   "parallelism": f"replicas x{world}, {nstreams} concurrent solves per GPU",
                   "vcycle_graphs": graphs_in_timed,
                   "l2": ("flushed (256 MB write) before every step" if nstreams > 1
                          else "flushed (256 MB write) between solves"),
                   "iters": [r[1]["iters"] for r in recs64[:len(cases)]],
                   "setup_s": round(setup_s, 3)},
        "gpu_launches": launches,
        "e2e": {"value": work_dofs / (e2e_ms * 1e-3) / 1e6, "unit": "MDOF/s",
                "h2d_bytes_per_step": len(cases) * vec_bytes, "d2h_bytes_per_step": len(cases) * vec_bytes},
        "clocks": clocks,
    }
    if ms32 is not None:
        sub_dofs = len(fp32_cases) * nfree * world
        out["fp32_mg"] = {"workload": "the 8 solves with lambda <= 1e4", "value": sub_dofs / (ms32 * 1e-3) / 1e6,
                          "unit": "MDOF/s", "ms_per_step": ms32,
                          "fp64_same_solves": {"value": sub_dofs / (ms64s * 1e-3) / 1e6, "ms_per_step": ms64s},
                          "speedup_vs_fp64": ms64s / ms32,
                          "iters": [r[1]["iters"] for r in recs32[:len(fp32_cases)]],
                          "per_solve_vs_fp64": err32,
                          "lambda_1e6_probe": probe64,
                          "vcycle_hbm": {"unit": "GB/s algorithmic, fine level, FP32 V-cycles of the 8 "
                                                 "hierarchies (3 each) alone on the GPU",
                                         "peak_gbs": measured_hbm_gbs()[0],
                                         "peak_source": measured_hbm_gbs()[1], **hbm32}}
    def roofline_of(p):
        avg_ms = p["ms"] / p["launches"]
        cells = p["cells"] / p["launches"]
        achieved = FLOPS_PER_CELL[dominant] * cells / (avg_ms * 1e-3) / 1e12
        return achieved, avg_ms
    if prof and prof["launches"]:
        achieved, avg_ms = roofline_of(prof)
        n_mv = sum(r[1]["iters"] for r in recs64)     # one matvec per FGMRES iteration
        out["roofline"] = {"kernel": dominant + "<double> (fine level)", "bound": "alu",
                           "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                           "frac": achieved / FP64_PEAK_TFLOPS,
                           "traffic": (apply_traffic(n_mv, prof["launches"] - n_mv)
                                       if dominant == "apply" and graphs_in_timed else None),
                           "avg_launch_ms": avg_ms, "launches": prof["launches"],
                           "peak_source": "nominal FP64 rate of the GB300 (1.25 TFLOP/s; a register-FMA loop measured 1.20)",
                           "timed_region": f"{nstreams} concurrent solves: launches share the GPU",
                           "launches_timed": ("the operator's launches outside the V-cycle (FGMRES matvec "
                                              "and true residual), the V-cycles replaying as CUDA graphs"
                                              if graphs_in_timed else "every launch (V-cycle graphs off)"),
                           "shares_ms": {k: round(v["ms"], 3) for k, v in shares.items()}}
        if prof_iso and prof_iso["launches"]:
            a_iso, ms_iso = roofline_of(prof_iso)
            out["roofline_isolated"] = {"kernel": dominant + "<double> (fine level)", "bound": "alu",
                                        "achieved": a_iso, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                                        "frac": a_iso / FP64_PEAK_TFLOPS, "avg_launch_ms": ms_iso,
                                        "launches": prof_iso["launches"],
                                        "how": "one extra step, solves one after the other"}
    if msA is not None:
        iA = [r[1]["iters"] for r in recsA[:len(cases)]]
        i64 = out["config"]["iters"]
        out["arnoldi_mixed"] = {
            "workload": "the same 12 FP64-V-cycle solves; Arnoldi with an FP32 first Gram-Schmidt pass and "
                        "a double-float second pass and correction",
            "value": work_dofs / (msA * 1e-3) / 1e6, "unit": "MDOF/s", "ms_per_step": msA, "steps": arm_steps,
            "iters": iA, "iter_delta_vs_fp64": [a - b for a, b in zip(iA, i64)]}
    if msW is not None:
        bdofs = len(bcases) * nfree * world
        out["bsr_w_cycle"] = {
            "workload": "the 6 BSR solves of the sweep with W(1,1) cycles (the remedy for multilevel inexact "
                        "BSR that the discussion of Table 4 suggests) against the same 6 with V(1,1)",
            "value": bdofs / (msW * 1e-3) / 1e6, "unit": "MDOF/s", "ms_per_step": msW, "steps": arm_steps,
            "iters": [r[1]["iters"] for r in recsW[:len(bcases)]],
            "v_cycle": {"value": bdofs / (msV * 1e-3) / 1e6, "ms_per_step": msV,
                        "iters": [r[1]["iters"] for r in recsV[:len(bcases)]]}}
    # the sweep at the paper's compressibility group: (1/M) mu / alpha^2 = 1e-2, with the
    # paper's rediscretised coarse operators and with Galerkin ones
    if not args.no_arms:
        for key in [k for k in hier if k[0] == "fp32"]:
            del hier[key]
        cases2 = smoother_cases(INV_M_PAPER)
        sys2 = {}
        for c in cases2:
            key = (c["lam"], c["K"])
            if key not in sys2:
                sys2[key] = bmg.assemble(n, c["lam"], 1.0, None, c["K"], 1.0, 1.0, INV_M_PAPER)
        arm = {"workload": f"the 12 FP64 solves of the sweep with 1/M = {INV_M_PAPER} (the paper's "
                           "(1/M) mu / alpha^2 group: M = 1e6 with mu ~ 1e4), FGMRES(50) capped at "
                           f"{MAXIT_ARM} iterations"}
        for co in ("galerkin", "redisc"):
            hier2 = {("fp64", ci): bmg.setup_hierarchy(sys2[c["lam"], c["K"]], c["smoother"], 1, 1,
                                                       omega=c["omega"], omega_J=c["omega_J"], n_coarse=8,
                                                       coarse_op=co)
                     for ci, c in enumerate(cases2)}
            try:
                one_step("fp64", hset=hier2, allow_fail=True, maxit=MAXIT_ARM)
                steps_co = arm_steps if co == "galerkin" else 1
                msM, recsM, _, _ = timed("fp64", steps_co, hset=hier2, allow_fail=True, maxit=MAXIT_ARM)
                infos = [r[1] for r in recsM[:len(cases2)]]
                conv = [i["status"] == "converged" for i in infos]
                arm[co] = {"value": sum(conv) * nfree * world / (msM * 1e-3) / 1e6, "unit": "MDOF/s",
                           "value_counts": "free DoFs of the converged solves only",
                           "ms_per_step": msM, "steps": steps_co, "iters": [i["iters"] for i in infos],
                           "converged": conv, "relres": [float(f"{i['relres']:.3g}") for i in infos]}
            except Exception as e:      # reported, never silently replaced
                arm[co] = {"value": None, "error": str(e)[-300:]}
            del hier2
        arm["omega"] = [[c["smoother"], c["omega"], c["omega_J"]] for c in cases2]
        out["inv_M_1e-2"] = arm
        del sys2
    if rank == 0 and not args.no_cpu_baseline:
        try:
            r = oracle_sample_parallel(64, cases)
            r1 = oracle_sample(64, cases)
            out["cpu_baseline"] = {"value": r["mdofs"], "unit": "MDOF/s", "cores": r["procs"], "kind": "oracle",
                                   "nproc": os.cpu_count(),
                                   "sample": "the 12 solves of this workload on a 64x64 grid "
                                             f"({r['dofs'] // 12} free DoFs each), one solve per host core "
                                             f"({r['procs']} processes, one thread each), solve time only, "
                                             f"{r['seconds']:.1f} s wall, {r['cpu_seconds']:.1f} s CPU",
                                   "one_core": {"value": r1["mdofs"], "unit": "MDOF/s", "cores": 1,
                                                "seconds": r1["seconds"]}}
        except Exception as e:  # reported, never silently replaced
            out["cpu_baseline"] = {"value": None, "error": str(e)[-300:]}
    # the mixed-precision, batched and adjoint workloads (one GPU only: replicas of the sweep
    # keep these out of multi-GPU runs)
    if world == 1 and not args.no_workloads:
        import gc
        hier.clear()
        systems.clear()
        gc.collect()
        torch.cuda.empty_cache()
        wl = {}
        for name, fn in (("mixed_2048", lambda: mixed_workload(args.mixed_n, 1, 1)),
                         ("batched_256", lambda: batched_workload(args.batch_count, 1, 1, True, True)),
                         ("adjoint_1024", lambda: adjoint_workload(args.adjoint_n, 1, 1, args.fd_dirs)),
                         ("time_dependent_512", lambda: time_dependent_workload(n, 16)),
                         ("bsr_exact_256", lambda: bsr_exact_workload(256))):
            try:
                t0 = time.perf_counter()
                wl[name] = fn()
                wl[name]["wall_s"] = round(time.perf_counter() - t0, 1)
            except Exception as e:  # reported, never silently replaced
                wl[name] = {"value": None, "error": str(e)[-300:]}
            gc.collect()
            torch.cuda.empty_cache()
        out["workloads"] = wl
    if args.verbose:
        for c, info in recs64[:len(cases)]:
            print("fp64", c, info, file=sys.stderr)
        if ms32 is not None:
            for c, info in recs32[:len(fp32_cases)]:
                print("fp32", c, info, file=sys.stderr)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
