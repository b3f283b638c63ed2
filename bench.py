"""Benchmark: ICCG time to 1e-8 relative residual on the 3D 7-point Poisson
problem (128^3, n = 2,097,152, 14.58M nonzeros, b ~ U[-1,1] from seed 0) with
Leiden CPM blocking (resolution 0.5) and greedy block coloring: the fastest
blocking on a GB300 of the swept set (ABMC block sizes 8..128, Leiden
modularity, CPM resolutions 0.01..0.5); `--blocking abmc --block-size S`
selects another.
`--workload diffusion96 --fp32` runs the 27-point variable-coefficient
diffusion problem (96^3, ABMC 32) with the FP32 preconditioner (extension 1).
`--workload batch64` runs the batched extension: 64 shifted 7-point systems
(sides U{16..64}), 16 right-hand sides each, ABMC 32, FP32 preconditioner,
all in one launch; a step is the whole batch solved to 1e-8.
`--workload learned` trains the learned-blocking MLP on the GPU (library
kernels) from the committed label sweep and solves the held-out matrices
with the predicted ABMC block size and with the fixed block size 32; a step
is the held-out set solved once with the predicted settings.

A step is one pass of the device hot path on inputs resident in HBM:
iccg_factor (IC(0), FP64) followed by iccg_solve (PCG with block-multicolor
substitutions) from x0 = 0 to ||r||/||b|| <= 1e-8.  Blocking and setup are
excluded (the paper times blocking separately, Sec. 6.6) and reported.
`value` is milliseconds per step (lower is better).  `e2e` times the same
step through the C ABI with host (pinned) b and x, so the host<->device
copies are inside the timed region.

Multi-GPU: one system does not shard (every color needs the previous
colors' results), so N > 1 runs N independent replicas, one per rank.

--impl reference times the CPU oracle (single-threaded FP64) on the same
workload: each step is IC(0) plus a bounded number of PCG iterations, scaled
to the full solve's iteration count.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import gen  # noqa: E402

CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    """Samples nvidia-smi clocks / throttle reasons while the timed region runs."""

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={CLOCK_QUERY}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([s.strip() for s in line.split(",")])

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for k, nm in enumerate(names):
                if len(s) > 5 + k and s[5 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


def max_over_ranks(value, device):
    """The largest `value` of all ranks (every rank gets it), then a barrier:
    the replicas' time is the slowest replica's."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


WORKLOADS = {
    "poisson128": "3D 7-point Poisson {nx}^3",
    "diffusion96": "3D 27-point variable-coefficient diffusion {nx}^3 (contrast 1e3, shift 1e-6 max diag)",
    "batch64": "batch of 64 shifted 3D 7-point systems (sides U{{16..64}}, shift U[1e-4,1e-1]) x 16 right-hand sides",
    "learned": "40 held-out generated SPD matrices (5/7/27-point anisotropic stencils, random geometric graph "
               "Laplacians, 3-dof spring networks; n 2e4-2e5), ABMC block size predicted by the learned-blocking MLP",
}


def workload(args):
    if args.workload == "diffusion96":
        a = gen.diffusion3d_27pt(args.nx, seed=args.seed)
        return a, gen.rhs_uniform(a.n, args.seed)
    a, b, _ = gen.config2(nx=args.nx, seed=args.seed)
    return a, b


# DRAM bytes (read + write) of the substitution sweep per PCG iteration,
# from the ncu launch list of `bench.py --steps 1 --warmup 1 --no-cpu-baseline`
# (profiles/launches_iccg_fp64_poisson128_cpm05.md), keyed by workload and
# blocking; None where no capture of the current kernels exists.
SUBST_TRAFFIC = {("poisson128", 128, "leiden_cpm", 0.5, False): 433152384}


def make_blocking(mod, a, args):
    """The configured blocking by `mod` (the library, or the oracle for the
    reference arm; both give the same permutation)."""
    if args.blocking == "abmc":
        return mod.blocking(a, "abmc", args.block_size)
    return mod.blocking(a, args.blocking, gamma=args.gamma)


def blocking_name(args):
    if args.blocking == "abmc":
        return f"ABMC s={args.block_size}"
    if args.blocking == "leiden_cpm":
        return f"Leiden CPM resolution {args.gamma:g}"
    return "Leiden modularity"


def bytes_model(n, nnz, nL, fp32):
    """Algorithmic bytes per PCG iteration (each array counted once, gathered
    vector reads assumed to hit cache), by kernel family:
      SpMV + <p,q>   sliced-ELL off-diagonal values and columns 12 (nnz - n), the
                     diagonal 8n, slice pointers n/8, p in 8n, q out 8n
      p update       z, p in, p out: 24n (FP32 z: 20n)
      forward sweep  L entries (value + column) per strictly-lower entry, row
                     pointers 4n, 1/L_ii, the fused x/r update (r, q, x, p in,
                     r, x out: 48n), y out
      backward sweep U entries, row pointers 4n, 1/L_ii, y in, z out, r in (dot)
    The substitution roofline uses forward + backward."""
    pe = 4 if fp32 else 8
    spmv = 12 * (nnz - n) + 8 * n + n // 8 + 16 * n
    pupd = (16 + pe) * n
    fwd = (pe + 4) * nL + 4 * n + pe * n + 48 * n + pe * n
    bwd = (pe + 4) * nL + 4 * n + pe * n + pe * n + pe * n + 8 * n
    return {"spmv": spmv, "pupdate": pupd, "subst": fwd + bwd, "total": spmv + pupd + fwd + bwd}


def run_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_2609_00561_gb300 import build as libbuild
    from paper_2609_00561_gb300 import iccg

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    libbuild.build()
    dev = torch.device("cuda", local)

    t0 = time.perf_counter()
    a, b = workload(args)
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    bl = make_blocking(iccg, a, args)
    t_block = time.perf_counter() - t0
    stream = torch.cuda.current_stream(dev)
    t0 = time.perf_counter()
    S = iccg.Solver(a, bl, precond_fp32=args.fp32, warps_per_cta=args.warps, rows_per_thread=args.rows,
                    stream=stream.cuda_stream, factor=False)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    info = S.info()

    bd = torch.tensor(b, device=dev)
    xd = torch.zeros_like(bd)

    def step():
        iccg.iccg_factor(S.ctx)
        xd.zero_()
        return iccg.iccg_solve(S.ctx, bd, xd, args.tol, args.maxit, want_hist=False)

    for _ in range(args.warmup):
        st, iters, _ = step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            st, iters, _ = step()
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    if world > 1:
        ms = max_over_ranks(ms, dev)

    # solve alone and factor alone (same inputs, device events)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(max(1, args.steps)):
        iccg.iccg_factor(S.ctx)
    e1.record(stream)
    torch.cuda.synchronize()
    factor_ms = e0.elapsed_time(e1) / max(1, args.steps)
    xd.zero_()
    e0.record(stream)
    st, iters, hist = iccg.iccg_solve(S.ctx, bd, xd, args.tol, args.maxit)
    e1.record(stream)
    torch.cuda.synchronize()
    solve_ms = e0.elapsed_time(e1)
    x = xd.cpu().numpy()
    true_rel = float(np.linalg.norm(b - a.to_scipy() @ x) / np.linalg.norm(b))

    # per-kernel-family device time of one solve (event pair around every launch)
    xd.zero_()
    _, it_p, phase_ms, phase_ln = iccg.iccg_profile_solve(S.ctx, bd, xd, args.tol, args.maxit)
    bm = bytes_model(info["n"], info["nnz"], info["nL"], args.fp32)
    sub_ms = phase_ms["fwd"] + phase_ms["fused"] + phase_ms["bwd"]
    sub_launch = phase_ln["fwd"] + phase_ln["fused"] + phase_ln["bwd"]
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    achieved = bm["subst"] * it_p / (sub_ms * 1e-3) / 1e9 if sub_ms > 0 else 0.0

    # end-to-end through the C ABI with pinned host buffers
    bh = torch.tensor(b).pin_memory().numpy()
    xh = torch.zeros(a.n, dtype=torch.float64).pin_memory().numpy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        iccg.iccg_factor(S.ctx)
        xh[:] = 0.0
        iccg.iccg_solve(S.ctx, bh, xh, args.tol, args.maxit, want_hist=False)
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps

    n_c = info["n_c"]
    # iccg_factor: one launch per color + finish; iccg_solve: perm_in, the
    # residual SpMV, the 2 n_c - 1 color launches of z0, then per iteration
    # p update + SpMV + 2 n_c - 1 color launches, and perm_out
    launches_per_step = (n_c + 1) + (2 + 2 * n_c - 1) + iters * (2 + 2 * n_c - 1) + 1
    result = {
        "metric": "ICCG time to 1e-8 rel. residual",
        "value": round(ms, 4),
        "unit": "ms",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms, 4),
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64" if args.fp32 else "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload].format(nx=args.nx) +
                               f" (n={a.n}, nnz={a.nnz}), b~U[-1,1] seed {args.seed}, "
                               f"{blocking_name(args)} + greedy coloring (n_b={bl['n_b']}, n_c={n_c}), "
                               f"IC(0) + PCG to {args.tol:g}" + (", FP32 preconditioner" if args.fp32 else ""),
                   "step": "iccg_factor + iccg_solve, inputs resident",
                   "l2": "inputs larger than L2 (matrix + factors > 129 MB)",
                   "parallelism": "replicas only" if world > 1 else "1 GPU",
                   "layout": f"{info['tile_colors']} of {n_c} colors as lane tiles ({info['tiles']} tiles), "
                             f"{info['groups']} CTA groups"},
        "iterations": iters,
        "status": iccg.STATUS.get(st, st),
        "true_relres": true_rel,
        "solve_ms": round(solve_ms, 4),
        "factor_ms": round(factor_ms, 4),
        "us_per_iteration": round(solve_ms * 1e3 / max(iters, 1), 2),
        "setup": {"gen_s": round(t_gen, 3), "blocking_s": round(t_block, 3), "setup_s": round(t_setup, 3)},
        "phase_ms": {k: round(v, 4) for k, v in phase_ms.items()},
        "phase_launches": phase_ln,
        "roofline": {"bound": "hbm", "kernel": "block-multicolor substitution sweep (forward, fused and backward "
                                               "color launches of one PCG iteration)",
                     "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
                     "frac": round(achieved / hbm_peak, 4), "peak_source": peak_src,
                     "bytes_per_iteration": bm["subst"], "launches_per_iteration": sub_launch / max(it_p, 1),
                     "traffic": SUBST_TRAFFIC.get((args.workload, args.nx, args.blocking,
                                                   args.gamma if args.blocking == "leiden_cpm" else args.block_size,
                                                   bool(args.fp32))),
                     "traffic_unit": "bytes per PCG iteration (ncu launch list, cold cache)"},
        "e2e": {"value": round(e2e_ms, 4), "unit": "ms", "h2d_bytes_per_step": 2 * 8 * a.n,
                "d2h_bytes_per_step": 8 * a.n},
        "gpu_launches": int(launches_per_step * args.steps),
        "clocks": clk.summary(),
    }
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        result["cpu_baseline"] = cpu_baseline(a, b, bl, iters, args)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    S.close()
    if rank == 0:
        print(json.dumps(result))


def run_batch(args):
    """Extension 2: the whole batch (every system, every right-hand side) to
    tol in one launch per step; inputs resident.  The plain FP64 GPU solver
    is timed on the first right-hand side of every system (scaled by the
    right-hand-side count) for the comparison."""
    import torch
    from paper_2609_00561_gb300 import build as libbuild
    from paper_2609_00561_gb300 import iccg

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    libbuild.build()
    dev = torch.device("cuda", local)
    t0 = time.perf_counter()
    systems, opt = gen.config4(seed=args.seed, nsys=args.nsys, nrhs=args.nrhs)
    t_gen = time.perf_counter() - t0
    stream = torch.cuda.current_stream(dev)
    t0 = time.perf_counter()
    blocks = [iccg.blocking(a, "abmc", args.block_size) for a, _ in systems]
    t_block = time.perf_counter() - t0
    t0 = time.perf_counter()
    solvers = [iccg.Solver(a, bl, precond_fp32=not args.fp64_batch, lane_block_max=-1, stream=stream.cuda_stream)
               for (a, _), bl in zip(systems, blocks)]
    bs = iccg.BatchSolver(solvers, args.nrhs)
    B = [torch.tensor(b, device=dev) for _, b in systems]
    # shape search on this batch (setup, untimed); --no-tune keeps the default shape
    tune_ms = None if args.no_tune else bs.tune(B, args.tol, args.maxit)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    shape = bs.info()
    X = [torch.zeros_like(b) for b in B]

    def step():
        for x in X:
            x.zero_()
        return bs.solve(B, X, args.tol, args.maxit)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            st, its, stv, _ = step()
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    # accuracy: true residual of every right-hand side; FP64 oracle on a sample
    worst_res = 0.0
    for (a, b), x in zip(systems, X):
        m = a.to_scipy()
        xh = x.cpu().numpy()
        for j in range(b.shape[0]):
            worst_res = max(worst_res, float(np.linalg.norm(b[j] - m @ xh[j]) / np.linalg.norm(b[j])))
    # bytes per right-hand-side iteration (matrix + factors shared, vectors per RHS)
    pe = 8 if args.fp64_batch else 4
    tot_bytes = 0.0
    for (a, b), S, it_s in zip(systems, solvers, its):
        info = S.info()
        mat = 12 * info["nnz"] + (pe + 4) * 2 * info["nL"] + (4 * 3 + pe) * info["n"]
        vec = (8 * 12 + pe * 6) * info["n"]      # x, r, p, q, y, z traffic of one iteration per RHS
        tot_bytes += float(int(it_s.max())) * mat + float(it_s.sum()) * vec
    achieved = tot_bytes / (ms * 1e-3) / 1e9
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    # plain FP64 single-system GPU solve of the first right-hand side of each system
    single_ms = 0.0
    for (a, b), bl in zip(systems, blocks):
        S1 = iccg.Solver(a, bl, stream=stream.cuda_stream)
        bd = torch.tensor(b[0], device=dev)
        xd = torch.zeros_like(bd)
        iccg.iccg_solve(S1.ctx, bd, xd, args.tol, args.maxit, want_hist=False)
        xd.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        iccg.iccg_solve(S1.ctx, bd, xd, args.tol, args.maxit, want_hist=False)
        e1.record(stream)
        torch.cuda.synchronize()
        single_ms += e0.elapsed_time(e1)
        S1.close()
    single_ms *= args.nrhs
    # e2e: host (pinned) right-hand sides and solutions through the C ABI
    Bh = [torch.tensor(b).pin_memory().numpy() for _, b in systems]
    Xh = [torch.zeros(b.shape, dtype=torch.float64).pin_memory().numpy() for _, b in systems]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for x in Xh:
            x[:] = 0.0
        bs.solve(Bh, Xh, args.tol, args.maxit)
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps
    nrhs_total = args.nsys * args.nrhs
    ntot = sum(a.n for a, _ in systems)
    result = {
        "metric": "ICCG time to 1e-8 rel. residual", "value": round(ms, 4), "unit": "ms",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.fp64_batch else "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOADS["batch64"].format(nx=0) + f": n total {ntot}, ABMC s={args.block_size}, "
                               f"{'FP64' if args.fp64_batch else 'FP32'} preconditioner, FP64 CG, tol {args.tol:g}",
                   "step": "iccg_batch_solve of the whole batch, inputs resident",
                   "l2": "inputs larger than L2", "parallelism": "1 GPU", "shape": shape,
                   "autotune": "warps/CTA x CTAs/SM, each candidate timed on this batch's full solve"},
        "rhs_solves_per_s": round(nrhs_total / (ms * 1e-3), 1),
        "iterations": {"min": int(its.min()), "max": int(its.max()), "mean": round(float(its.mean()), 1)},
        "status": iccg.STATUS.get(st, st), "worst_true_relres": worst_res,
        "plain_fp64_single_solves_ms": round(single_ms, 2),
        "speedup_vs_plain_fp64": round(single_ms / ms, 2),
        "setup": {"gen_s": round(t_gen, 3), "blocking_s": round(t_block, 3), "setup_s": round(t_setup, 3)},
        "roofline": {"bound": "hbm", "kernel": "batched persistent ICCG (whole solve)", "achieved": round(achieved, 1),
                     "peak": hbm_peak, "unit": "GB/s", "frac": round(achieved / hbm_peak, 4),
                     "peak_source": "measured" if "hbm_gbs" in peaks else "fallback", "traffic": None},
        "e2e": {"value": round(e2e_ms, 4), "unit": "ms",
                "h2d_bytes_per_step": 2 * 8 * ntot * args.nrhs, "d2h_bytes_per_step": 8 * ntot * args.nrhs},
        "gpu_launches": args.steps,
        "clocks": clk.summary(),
    }
    bs.close()
    for S in solvers:
        S.close()
    if rank == 0:
        print(json.dumps(result))


def run_learned(args):
    import torch
    from paper_2609_00561_gb300 import build as libbuild
    from paper_2609_00561_gb300 import iccg
    from paper_2609_00561_gb300.learn import model as lm

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    libbuild.build()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    data = lm.load_sweep(os.path.join(ROOT, "paper_2609_00561_gb300", "learn", "blocking_sweep.json"))
    X, yc, yr, ta, tc = lm.labels(data)
    tr, te = lm.split(len(yc))
    bs_list, gammas = data["meta"]["block_sizes"], data["meta"]["gammas"]
    m = lm.Model(X.shape[1], len(bs_list), seed=args.seed)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    hist = m.fit(X[tr], yc[tr], yr[tr], epochs=3000)
    e1.record(stream)
    torch.cuda.synchronize()
    train_ms = e0.elapsed_time(e1)
    ev_sweep = lm.evaluate(m, X[te], ta[te], tc[te], gammas, bs_list)
    cls, _ = m.predict(X[te])
    # live: each held-out matrix solved with the predicted and with the fixed block size
    import gen
    solvers = []
    for k, idx in enumerate(te):
        spec = data["records"][idx]["spec"]
        a = gen.config5_matrix(spec)
        b = np.random.default_rng(spec["seed"] + 7).uniform(-1.0, 1.0, a.n)
        pair = []
        for s_blk in (bs_list[int(cls[k])], lm.BASE_BLOCK):
            S = iccg.Solver(a, iccg.blocking(a, "abmc", s_blk), stream=stream.cuda_stream)
            pair.append(S)
        solvers.append((pair, torch.tensor(b, device=dev)))

    def step(which):
        tot = 0.0
        for pair, bd in solvers:
            xd = torch.zeros_like(bd)
            e0.record(stream)
            iccg.iccg_solve(pair[which].ctx, bd, xd, args.tol, args.maxit, want_hist=False)
            e1.record(stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        return tot

    for _ in range(args.warmup):
        step(0)
        step(1)
    with ClockSampler(local) as clk:
        pred_ms = statistics.mean(step(0) for _ in range(args.steps))
    fixed_ms = statistics.mean(step(1) for _ in range(args.steps))
    for pair, _ in solvers:
        for S in pair:
            S.close()
    result = {
        "metric": "ICCG time to 1e-8 rel. residual", "value": round(pred_ms, 3), "unit": "ms",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(pred_ms, 3),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS["learned"], "step": "the 40 held-out systems solved once each, "
                   "inputs resident, blocking and setup excluded", "l2": "mixed (systems 0.5-30 MB)",
                   "parallelism": "1 GPU"},
        "fixed_block32_ms": round(fixed_ms, 3),
        "gain_vs_fixed_block32": round(fixed_ms / pred_ms, 3),
        "train_ms": round(train_ms, 1), "train_loss": [round(v, 4) for v in hist[::6]],
        "held_out_vs_sweep": ev_sweep,
        "roofline": None,
        "e2e": None,
        "gpu_launches": None,
        "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(result))


def oracle_sample(a, b, perm, sample_iters):
    """IC(0) + `sample_iters` PCG iterations of the oracle; returns seconds."""
    import oracle
    t0 = time.perf_counter()
    ah = oracle.permute(a, perm)
    lptr, lcol, aval = oracle.tril_csr(ah)
    t_perm = time.perf_counter() - t0
    t0 = time.perf_counter()
    lval, _ = oracle.ic0(lptr, lcol, aval)
    t_ic = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.pcg(ah, lptr, lcol, lval, b[perm], tol=0.0, maxit=sample_iters)
    t_pcg = time.perf_counter() - t0
    return t_perm, t_ic, t_pcg


def cpu_baseline(a, b, bl, iters_full, args):
    tp, tic, tpcg = oracle_sample(a, b, bl["perm"], args.cpu_sample_iters)
    per_it = tpcg / args.cpu_sample_iters
    value_ms = (tic + per_it * iters_full) * 1e3
    return {"value": round(value_ms, 1), "unit": "ms", "cores": 1, "kind": "oracle",
            "sample": f"IC(0) + {args.cpu_sample_iters} PCG iterations of the FP64 oracle on the same permuted "
                      f"matrix, scaled to the {iters_full} iterations of the full solve "
                      f"({per_it * 1e3:.1f} ms/iteration, IC(0) {tic * 1e3:.0f} ms)"}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    # the reference arm never touches the GPU; blocking comes from the oracle
    import oracle
    a, b = workload(args)
    bl = make_blocking(oracle, a, args)
    iters_full = args.ref_iters
    times = []
    for k in range(args.warmup + args.steps):
        tp, tic, tpcg = oracle_sample(a, b, bl["perm"], args.cpu_sample_iters)
        t = tic + tpcg / args.cpu_sample_iters * iters_full
        if k >= args.warmup:
            times.append(t)
    ms = statistics.mean(times) * 1e3
    result = {"impl": "reference", "metric": "ICCG time to 1e-8 rel. residual", "value": round(ms, 1), "unit": "ms",
              "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 1),
              "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
              "data": "synthetic",
              "config": {"workload": WORKLOADS[args.workload].format(nx=args.nx) +
                                     f", {blocking_name(args)} + greedy coloring, IC(0) + PCG to {args.tol:g} "
                                     f"(CPU oracle)"},
              "cpu_baseline": {"value": round(ms, 1), "unit": "ms", "cores": 1, "kind": "oracle",
                               "sample": f"each step: IC(0) + {args.cpu_sample_iters} PCG iterations, scaled to "
                                         f"{iters_full} iterations"},
              "e2e": {"value": round(ms, 1), "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(result))


def main():
    p = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--workload", default="poisson128", choices=sorted(WORKLOADS))
    p.add_argument("--nx", type=int, default=None, help="grid side (default 128, or 96 for diffusion96)")
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--blocking", default=None, choices=["abmc", "leiden_cpm", "leiden_md"],
                   help="default: leiden_cpm for poisson128, abmc otherwise")
    p.add_argument("--gamma", type=float, default=0.5, help="Leiden CPM resolution")
    p.add_argument("--block-size", type=int, default=None, help="ABMC block size (default 8, or 32 for diffusion96)")
    p.add_argument("--tol", type=float, default=1e-8)
    p.add_argument("--maxit", type=int, default=5000)
    p.add_argument("--fp32", action="store_true", help="FP32 preconditioner (extension 1)")
    p.add_argument("--warps", type=int, default=0)
    p.add_argument("--rows", type=int, default=0)
    p.add_argument("--cpu-sample-iters", type=int, default=20)
    p.add_argument("--ref-iters", type=int, default=None,
                   help="iterations the full solve takes (scales the reference sample; default: 183 for the "
                        "default poisson128 blocking, else 176)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--nsys", type=int, default=64, help="batch64: systems")
    p.add_argument("--nrhs", type=int, default=16, help="batch64: right-hand sides per system")
    p.add_argument("--fp64-batch", action="store_true", help="batch64: FP64 preconditioner")
    p.add_argument("--no-tune", action="store_true", help="batch64: default launch shape, no autotuning")
    args = p.parse_args()
    if args.nx is None:
        args.nx = 96 if args.workload == "diffusion96" else 128
    if args.block_size is None:
        args.block_size = 32 if args.workload in ("diffusion96", "batch64") else 8
    if args.blocking is None:
        args.blocking = "leiden_cpm" if args.workload == "poisson128" else "abmc"
    if args.ref_iters is None:
        args.ref_iters = 183 if (args.blocking, args.gamma) == ("leiden_cpm", 0.5) else 176
    if args.steps < 1 or args.warmup < 0:
        raise SystemExit("steps >= 1, warmup >= 0")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch64":
        run_batch(args)
    elif args.workload == "learned":
        run_learned(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
